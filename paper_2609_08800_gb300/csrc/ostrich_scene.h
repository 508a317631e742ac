// Device-side scene description and shared-memory layout of the Ostrich step kernels.
// Product code only (the CPU oracle has its own, independent format).
#pragma once
#include <stdint.h>

namespace ost {

constexpr int NB_CAP = 8;      // bodies per world
constexpr int NJ_CAP = 8;      // revolute joints per world
constexpr int SLOT_CAP = 64;   // contact slots per world

enum { SHAPE_NONE = 0, SHAPE_BOX = 1, SHAPE_WHEEL = 2 };
enum { ENV_PLANE = 0, ENV_BOX = 1, ENV_HEIGHTMAP = 2 };
enum { ROW_JOINT = 0, ROW_SERVO = 1, ROW_NORMAL = 2, ROW_FRIC = 3 };

// Everything a kernel needs to know about the scene and the solver settings.
// Passed by value as a kernel parameter.
struct DevScene {
  int nb, nj, n_servo, n_slots, m_max, n_state, env, nf;
  double mu, g;
  double box[5];                 // x0, x1, y0, y1, H
  int hn; double hsp, hox, hoy;  // heightmap grid
  const float* heights;          // device pointer, hn*hn, or null
  // bodies
  double mass[NB_CAP], inertia[NB_CAP][3], half[NB_CAP][3], radius[NB_CAP], hw[NB_CAP];
  int shape[NB_CAP], slot_base[NB_CAP], slot_count[NB_CAP];
  unsigned char slot_body[SLOT_CAP];
  // joints
  int jp[NJ_CAP], jc[NJ_CAP], servo_of[NJ_CAP];
  double ap[NJ_CAP][3], ac[NJ_CAP][3], axp[NJ_CAP][3], axc[NJ_CAP][3], p1[NJ_CAP][3], p2[NJ_CAP][3], kp[NJ_CAP];
  // solver settings
  int budget, kmin, ls, pullback;
  double tol, delta_rel, kappa, eps, margin;
  int refine;     // iterative-refinement sweeps after each Schur solve
  // layout caps derived from the scene
  int n_groups;   // bodies that carry contact slots (leaf blocks of the Schur matrix)
  int pg;         // largest leaf block (3 x slots of one body)
  int ss;         // separator rows (5 per joint + servos)
  int group_body[NB_CAP];
};

// Arguments of one launch of the step / adjoint kernels.
struct StepArgs {
  const void* state_in; const void* controls; void* state_out; void* impulses;
  int32_t* ids; uint32_t* status; int32_t* iters; void* tape;
  int ld, n_worlds, world0; double h;
  double* trace;   // optional diagnostic: merit of each iterate, (budget + 2) per world
};
struct AdjArgs {
  const void* tape; const void* dL_dnext; void* dL_dstate; void* dL_dcontrols;
  int ld, n_worlds, world0; double h;
};

// Tape record of one world for one step: inputs, returned iterate and the Schur factor.
// All counts in Real elements.
struct TapeLayout {
  int off_qm, off_um, off_ubar, off_u, off_lam, off_leaf, off_cpl, off_sep, total;
};

inline __host__ __device__ TapeLayout tape_layout(const DevScene& s) {
  TapeLayout t;
  int o = 0;
  t.off_qm = o; o += 7 * s.nb;
  t.off_um = o; o += 6 * s.nb;
  t.off_ubar = o; o += s.n_servo > 0 ? s.n_servo : 1;
  t.off_u = o; o += 6 * s.nb;
  t.off_lam = o; o += s.m_max;
  t.off_leaf = o; o += s.n_groups * s.pg * s.pg;
  t.off_cpl = o; o += s.n_groups * (s.ss > 0 ? s.ss : 1) * s.pg;
  t.off_sep = o; o += s.ss * s.ss;
  o = (o + 3) & ~3;   // 16-byte multiple per world for FP32
  t.total = o;
  return t;
}

}  // namespace ost
