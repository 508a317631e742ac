// Host-side translation of a public scene description and solver configuration into the
// kernels' DevScene, with every check the C ABI applies to them.  ostrich_create and
// the allocation-free entry point both use it, so the two accept exactly the same
// scenes (apart from what needs a device allocation: the heightmap copy, which only
// ostrich_create makes).
#pragma once
#include <cstddef>
#include <cstring>

#include "ostrich.h"
#include "ostrich_scene.h"

namespace ost {
template <class Real> size_t ws_bytes(const DevScene&);
template <class Real> size_t ws_used(const DevScene&);

// Shared-memory limit of one CTA on sm_103a (the working set of one world must fit).
constexpr size_t SMEM_CTA_MAX = 227 * 1024;

// Fills s from d and cfg for element type dtype (OSTRICH_F32 / OSTRICH_F64).  The
// heightmap's device pointer is left null: the caller copies the heights.  Returns
// OSTRICH_OK, or OSTRICH_EINVAL for a description the kernels cannot represent.
inline ostrich_status build_scene(const ostrich_scene_desc* d, const ostrich_solver_cfg* cfg, int dtype,
                                  DevScene& s) {
  std::memset(&s, 0, sizeof(s));
  if (!d || !cfg) return OSTRICH_EINVAL;
  if (dtype != OSTRICH_F32 && dtype != OSTRICH_F64) return OSTRICH_EINVAL;
  if (d->n_bodies < 1 || d->n_bodies > NB_CAP || d->n_joints < 0 || d->n_joints > NJ_CAP) return OSTRICH_EINVAL;
  if (d->env != ENV_PLANE && d->env != ENV_BOX && d->env != ENV_HEIGHTMAP) return OSTRICH_EINVAL;
  if (cfg->budget < 0 || cfg->k_min < 0) return OSTRICH_EINVAL;
  s.nb = d->n_bodies; s.nj = d->n_joints; s.env = d->env;
  s.mu = d->mu; s.g = d->gravity;
  for (int i = 0; i < 5; ++i) s.box[i] = d->box[i];
  s.hn = d->hm_n; s.hsp = d->hm_spacing; s.hox = d->hm_origin[0]; s.hoy = d->hm_origin[1];
  s.nf = s.env == ENV_PLANE ? 1 : (s.env == ENV_BOX ? 4 : 8);
  // a heightmap needs at least one 2 x 2 block of cells; face ids must fit the 20-bit
  // field of a contact id
  if (s.env == ENV_HEIGHTMAP && (!d->heights || s.hn < 3 || s.hn > 724 || !(s.hsp > 0))) return OSTRICH_EINVAL;
  int slots = 0;
  for (int b = 0; b < s.nb; ++b) {
    const ostrich_body_desc& bd = d->bodies[b];
    if (!(bd.mass > 0) || !(bd.inertia[0] > 0) || !(bd.inertia[1] > 0) || !(bd.inertia[2] > 0)) return OSTRICH_EINVAL;
    s.mass[b] = bd.mass;
    for (int k = 0; k < 3; ++k) { s.inertia[b][k] = bd.inertia[k]; s.half[b][k] = bd.half_extents[k]; }
    s.radius[b] = bd.radius; s.hw[b] = bd.half_width; s.shape[b] = bd.shape;
    const int cnt = bd.shape == SHAPE_BOX ? 8 : (bd.shape == SHAPE_WHEEL ? 2 * s.nf : 0);
    if (slots + cnt > SLOT_CAP) return OSTRICH_EINVAL;
    s.slot_base[b] = slots; s.slot_count[b] = cnt;
    for (int k = 0; k < cnt; ++k) s.slot_body[slots + k] = (unsigned char)b;
    slots += cnt;
  }
  s.n_slots = slots;
  s.n_servo = 0;
  for (int j = 0; j < s.nj; ++j) {
    const ostrich_joint_desc& jd = d->joints[j];
    if (jd.parent < 0 || jd.parent >= s.nb || jd.child < 0 || jd.child >= s.nb || jd.parent == jd.child)
      return OSTRICH_EINVAL;
    s.jp[j] = jd.parent; s.jc[j] = jd.child;
    for (int k = 0; k < 3; ++k) {
      s.ap[j][k] = jd.anchor_parent[k]; s.ac[j][k] = jd.anchor_child[k];
      s.axp[j][k] = jd.axis_parent[k]; s.axc[j][k] = jd.axis_child[k];
      s.p1[j][k] = jd.perp1_parent[k]; s.p2[j][k] = jd.perp2_parent[k];
    }
    if (jd.type != JOINT_REVOLUTE && jd.type != JOINT_PRISMATIC) return OSTRICH_EINVAL;
    if (jd.servo_mode != SERVO_VELOCITY && jd.servo_mode != SERVO_POSITION) return OSTRICH_EINVAL;
    if (!(jd.kd >= 0)) return OSTRICH_EINVAL;
    s.kp[j] = jd.kp; s.kd[j] = jd.kd; s.jtype[j] = jd.type; s.smode[j] = jd.servo_mode;
    s.servo_of[j] = jd.kp > 0 ? s.n_servo++ : -1;
  }
  s.m_max = 5 * s.nj + s.n_servo + 3 * s.n_slots;
  s.n_state = 13 * s.nb + s.m_max;
  finish_scene(s);
  s.budget = cfg->budget; s.kmin = cfg->k_min; s.ls = cfg->line_search; s.pullback = cfg->pullback;
  s.tol = cfg->tol; s.delta_rel = cfg->delta_rel; s.kappa = cfg->kappa; s.eps = cfg->eps_fb; s.margin = cfg->margin;
  if (s.m_max < 7 * s.nb) return OSTRICH_EINVAL;   // the adjoint reuses row buffers for 7 values per body
  // FP32 factors lose the small eigenvalues (contact compliance kappa) of the Schur
  // matrix.  The adjoint solves once, so it refines its solution against the
  // matrix-free product (8 sweeps); the forward Newton iteration corrects an inexact
  // step by itself (without refinement it takes the same number of iterations to the
  // same residuals), so its solves are not refined.
  s.refine = 0;
  s.refine_adj = dtype == OSTRICH_F32 ? 8 : 0;
  // the direct factor by default; PCR is selected on a context (ostrich_set_linear_solver)
  s.lin = LIN_DIRECT; s.pc = PC_JACOBI; s.pcr_iters = 16; s.pcr_iters_adj = 256;
  s.pcr_rtol_adj = dtype == OSTRICH_F32 ? 1e-10 : 1e-12;
  const size_t smem = dtype == OSTRICH_F64 ? ws_bytes<double>(s) : ws_bytes<float>(s);
  const size_t used = dtype == OSTRICH_F64 ? ws_used<double>(s) : ws_used<float>(s);
  if (smem > SMEM_CTA_MAX || used > smem) return OSTRICH_EINVAL;
  return OSTRICH_OK;
}

}  // namespace ost
