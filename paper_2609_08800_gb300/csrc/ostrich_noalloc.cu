// ostrich_step_adjoint_noalloc: one forward step plus its adjoint without any device
// allocation, for callers that cannot call cudaMalloc -- for instance a real-time
// control loop that must not allocate once it runs, code that issues its work inside a
// stream capture, or a plugin whose host framework owns all device memory.
//
// The step's tape (the per-world record the adjoint reads back) lives in the file-scope
// array below instead of a context's cudaMalloc'd workspace.  Every GPU that loads the
// library holds this array until the process exits.
#include <cuda_runtime.h>
#include <cstring>
#include <mutex>

#include "ostrich.h"
#include "ostrich_scene.h"

namespace ost {
template <class Real> cudaError_t launch_step(const DevScene&, const StepArgs&, int, cudaStream_t);
template <class Real> cudaError_t launch_adjoint(const DevScene&, const AdjArgs&, int, cudaStream_t);
template <class Real> size_t ws_bytes(const DevScene&);
template <class Real> size_t ws_used(const DevScene&);
}  // namespace ost

static __device__ __align__(256) unsigned char g_noalloc_tape[OSTRICH_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_tape_addr[kMaxDevices] = {nullptr};

// The array's name is a host-side stand-in; its device address must be resolved per
// device, with that device current, before a kernel may use it.
cudaError_t tape_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_tape_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_tape);
    if (e != cudaSuccess) return e;
    g_tape_addr[dev] = p;
  }
  *out = g_tape_addr[dev];
  return cudaSuccess;
}

// Scene description -> kernel parameters (same rules as context creation).
bool make_scene(const ostrich_scene_desc* d, const ostrich_solver_cfg* cfg, ost::DevScene& s) {
  std::memset(&s, 0, sizeof(s));
  if (d->n_bodies < 1 || d->n_bodies > ost::NB_CAP || d->n_joints < 0 || d->n_joints > ost::NJ_CAP) return false;
  if (d->env != ost::ENV_PLANE && d->env != ost::ENV_BOX) return false;
  if (cfg->budget < 0 || cfg->k_min < 0) return false;
  s.nb = d->n_bodies; s.nj = d->n_joints; s.env = d->env; s.mu = d->mu; s.g = d->gravity;
  for (int i = 0; i < 5; ++i) s.box[i] = d->box[i];
  s.nf = s.env == ost::ENV_PLANE ? 1 : 4;
  int slots = 0;
  for (int b = 0; b < s.nb; ++b) {
    const ostrich_body_desc& bd = d->bodies[b];
    if (!(bd.mass > 0) || !(bd.inertia[0] > 0) || !(bd.inertia[1] > 0) || !(bd.inertia[2] > 0)) return false;
    s.mass[b] = bd.mass;
    for (int k = 0; k < 3; ++k) { s.inertia[b][k] = bd.inertia[k]; s.half[b][k] = bd.half_extents[k]; }
    s.radius[b] = bd.radius; s.hw[b] = bd.half_width; s.shape[b] = bd.shape;
    int cnt = bd.shape == ost::SHAPE_BOX ? 8 : (bd.shape == ost::SHAPE_WHEEL ? 2 * s.nf : 0);
    if (slots + cnt > ost::SLOT_CAP) return false;
    s.slot_base[b] = slots; s.slot_count[b] = cnt;
    for (int k = 0; k < cnt; ++k) s.slot_body[slots + k] = (unsigned char)b;
    slots += cnt;
  }
  s.n_slots = slots;
  for (int j = 0; j < s.nj; ++j) {
    const ostrich_joint_desc& jd = d->joints[j];
    if (jd.parent < 0 || jd.parent >= s.nb || jd.child < 0 || jd.child >= s.nb || jd.parent == jd.child) return false;
    s.jp[j] = jd.parent; s.jc[j] = jd.child;
    for (int k = 0; k < 3; ++k) {
      s.ap[j][k] = jd.anchor_parent[k]; s.ac[j][k] = jd.anchor_child[k];
      s.axp[j][k] = jd.axis_parent[k]; s.axc[j][k] = jd.axis_child[k];
      s.p1[j][k] = jd.perp1_parent[k]; s.p2[j][k] = jd.perp2_parent[k];
    }
    s.kp[j] = jd.kp;
    s.servo_of[j] = jd.kp > 0 ? s.n_servo++ : -1;
  }
  s.m_max = 5 * s.nj + s.n_servo + 3 * s.n_slots;
  s.n_state = 13 * s.nb + s.m_max;
  ost::finish_scene(s);
  s.budget = cfg->budget; s.kmin = cfg->k_min; s.ls = cfg->line_search; s.pullback = cfg->pullback;
  s.tol = cfg->tol; s.delta_rel = cfg->delta_rel; s.kappa = cfg->kappa; s.eps = cfg->eps_fb; s.margin = cfg->margin;
  s.refine = 0;
  s.refine_adj = 8;
  if (s.m_max < 7 * s.nb) return false;
  size_t smem = ost::ws_bytes<float>(s);
  return smem <= 227 * 1024 && ost::ws_used<float>(s) <= smem;
}

}  // namespace

extern "C" ostrich_status ostrich_step_adjoint_noalloc(const ostrich_scene_desc* scene, const ostrich_solver_cfg* cfg,
                                                       int n_worlds, int ld, const float* state_in,
                                                       const float* controls, double h, float* state_out,
                                                       const float* dL_dstate_next, float* dL_dstate,
                                                       float* dL_dcontrols, void* stream) {
  if (!scene || !cfg || !state_in || !state_out || !dL_dstate_next || !dL_dstate) return OSTRICH_EINVAL;
  if (state_in == state_out || n_worlds < 1 || (ld != 0 && ld < n_worlds) || !(h > 0)) return OSTRICH_EINVAL;
  ost::DevScene s;
  if (!make_scene(scene, cfg, s)) return OSTRICH_EINVAL;
  if (s.n_servo > 0 && !controls) return OSTRICH_EINVAL;
  ost::TapeLayout tl = ost::tape_layout(s);
  const size_t need = (size_t)n_worlds * (size_t)tl.total * sizeof(float);
  if (need > (size_t)OSTRICH_NOALLOC_SCRATCH_BYTES) return OSTRICH_EINVAL;   // beyond the fixed array
  void* tape = nullptr;
  if (tape_address(&tape) != cudaSuccess) return OSTRICH_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ost::StepArgs a;
  std::memset(&a, 0, sizeof(a));
  a.state_in = state_in; a.controls = controls; a.state_out = state_out;
  a.tape = tape; a.ld = ld ? ld : n_worlds; a.n_worlds = n_worlds; a.world0 = 0; a.h = h;
  if (ost::launch_step<float>(s, a, 64, st) != cudaSuccess) return OSTRICH_ECUDA;
  ost::AdjArgs b;
  b.tape = tape; b.dL_dnext = dL_dstate_next; b.dL_dstate = dL_dstate; b.dL_dcontrols = dL_dcontrols;
  b.ld = a.ld; b.n_worlds = n_worlds; b.world0 = 0; b.h = h;
  if (ost::launch_adjoint<float>(s, b, 64, st) != cudaSuccess) return OSTRICH_ECUDA;
  return OSTRICH_OK;
}
