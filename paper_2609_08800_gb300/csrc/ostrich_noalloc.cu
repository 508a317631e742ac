// ostrich_step_adjoint_noalloc: one forward step plus its adjoint without any device
// allocation, for callers that cannot call cudaMalloc -- for instance a real-time
// control loop that must not allocate once it runs (an allocation can block or fail at
// an arbitrary moment), or a plugin whose host framework owns all device memory and
// hands out only the buffers it manages.
//
// The step's tape (the per-world record the adjoint reads back) lives in the file-scope
// array below instead of a context's cudaMalloc'd workspace.  Every GPU that loads the
// library holds this array until the process exits.  The array's device address is
// resolved once per device and cached; after a cudaDeviceReset the cached address is
// stale, so the entry point must not be used across a device reset.
#include <cuda_runtime.h>
#include <cstring>
#include <mutex>

#include "ostrich.h"
#include "ostrich_scene.h"
#include "ostrich_scene_build.h"

namespace ost {
template <class Real> cudaError_t launch_step(const DevScene&, const StepArgs&, int, cudaStream_t);
template <class Real> cudaError_t launch_adjoint(const DevScene&, const AdjArgs&, int, cudaStream_t);
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

}  // namespace

extern "C" ostrich_status ostrich_step_adjoint_noalloc(const ostrich_scene_desc* scene, const ostrich_solver_cfg* cfg,
                                                       int n_worlds, int ld, const float* state_in,
                                                       const float* controls, double h, float* state_out,
                                                       const float* dL_dstate_next, float* dL_dstate,
                                                       float* dL_dcontrols, void* stream) {
  if (!scene || !cfg || !state_in || !state_out || !dL_dstate_next || !dL_dstate) return OSTRICH_EINVAL;
  if (state_in == state_out || n_worlds < 1 || (ld != 0 && ld < n_worlds) || !(h > 0)) return OSTRICH_EINVAL;
  // the heightmap would need a device copy of the heights: refused
  if (scene->env == OSTRICH_ENV_HEIGHTMAP) return OSTRICH_EINVAL;
  ost::DevScene s;
  if (ost::build_scene(scene, cfg, OSTRICH_F32, s) != OSTRICH_OK) return OSTRICH_EINVAL;
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

extern "C" ostrich_status ostrich_noalloc_capacity(const ostrich_scene_desc* scene, const ostrich_solver_cfg* cfg,
                                                   int32_t* max_worlds, size_t* record_bytes) {
  if (!scene || !cfg || !max_worlds) return OSTRICH_EINVAL;
  if (scene->env == OSTRICH_ENV_HEIGHTMAP) return OSTRICH_EINVAL;
  ost::DevScene s;
  if (ost::build_scene(scene, cfg, OSTRICH_F32, s) != OSTRICH_OK) return OSTRICH_EINVAL;
  const size_t rec = (size_t)ost::tape_layout(s).total * sizeof(float);
  *max_worlds = (int32_t)((size_t)OSTRICH_NOALLOC_SCRATCH_BYTES / rec);
  if (record_bytes) *record_bytes = rec;
  return OSTRICH_OK;
}
