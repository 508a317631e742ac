// C ABI of libostrich (declared in include/ostrich.h): context, tape memory,
// argument checks and kernel launches.  Every step of the path runs in the CUDA
// kernels of ostrich_kernels.cuh; this file only validates and dispatches.
#include <cuda_runtime.h>
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "ostrich.h"
#include "ostrich_scene.h"
#include "ostrich_scene_build.h"

namespace ost {
template <class Real> cudaError_t launch_step(const DevScene&, const StepArgs&, int, cudaStream_t);
template <class Real> cudaError_t launch_adjoint(const DevScene&, const AdjArgs&, int, cudaStream_t);
template <class Real> size_t adj_smem_bytes(const DevScene&, int);
}  // namespace ost

struct ostrich_ctx {
  ost::DevScene sc;
  int n_worlds = 0, ld = 0, dtype = 0, tape_slots = 0, threads = 64;
  size_t tape_world_elems = 0;
  void* tape = nullptr;
  float* d_heights = nullptr;
  std::vector<unsigned char> slot_written;
  std::vector<double> slot_h;
  double* trace = nullptr;
  int schedule = 0;
  int adj_mode = 0;                // 0: paper (frozen W), 1: exact IFT
  int32_t* krylov = nullptr;       // per-world Krylov iterations of the adjoint (GMRES of the exact mode, PCR of
                                   // the PCR solver's paper mode; the caller's device array) or null
  int32_t* d_sched = nullptr;      // persistent schedule: [queue, cost[n_worlds], order[n_worlds]]
  char err[512] = {0};
  // device memory is released with the context, on every path out of ostrich_create too
  ~ostrich_ctx() {
    if (tape) cudaFree(tape);
    if (d_heights) cudaFree(d_heights);
    if (d_sched) cudaFree(d_sched);
  }
};

static ostrich_status fail(ostrich_ctx* c, ostrich_status s, const char* msg) {
  if (c) std::snprintf(c->err, sizeof(c->err), "%s", msg);
  return s;
}

static ostrich_status cuda_fail(ostrich_ctx* c, cudaError_t e, const char* where) {
  if (c) std::snprintf(c->err, sizeof(c->err), "%s: %s", where, cudaGetErrorString(e));
  return OSTRICH_ECUDA;
}

static size_t elem_size(int dtype) { return dtype == OSTRICH_F64 ? sizeof(double) : sizeof(float); }

extern "C" {

ostrich_status ostrich_create(const ostrich_scene_desc* d, const ostrich_solver_cfg* cfg, int n_worlds, int ld,
                              int dtype, int tape_slots, ostrich_ctx** out) {
  if (!out) return OSTRICH_EINVAL;
  *out = nullptr;
  if (!d || !cfg) return OSTRICH_EINVAL;
  if (n_worlds < 1 || (ld != 0 && ld < n_worlds) || tape_slots < 0) return OSTRICH_EINVAL;
  ostrich_ctx* c = new (std::nothrow) ostrich_ctx();
  if (!c) return OSTRICH_ENOMEM;
  ost::DevScene& s = c->sc;
  ostrich_status rc = ost::build_scene(d, cfg, dtype, s);
  if (rc != OSTRICH_OK) { delete c; return rc; }
  if (s.env == ost::ENV_HEIGHTMAP) {
    // the heights stay on the device for the context's life
    size_t bytes = (size_t)s.hn * s.hn * sizeof(float);
    void* hp = nullptr;
    if (cudaMalloc(&hp, bytes) != cudaSuccess) { cudaGetLastError(); delete c; return OSTRICH_ENOMEM; }
    c->d_heights = static_cast<float*>(hp);
    if (cudaMemcpy(c->d_heights, d->heights, bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return OSTRICH_ECUDA;
    }
    s.heights = c->d_heights;
  }
  c->n_worlds = n_worlds; c->ld = ld ? ld : n_worlds; c->dtype = dtype; c->tape_slots = tape_slots;
  ost::TapeLayout tl = ost::tape_layout(s);
  c->tape_world_elems = (size_t)tl.total;
  if (tape_slots > 0) {
    size_t bytes = (size_t)tape_slots * (size_t)n_worlds * c->tape_world_elems * elem_size(dtype);
    cudaError_t e = cudaMalloc(&c->tape, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return OSTRICH_ENOMEM;
    }
  }
  c->slot_written.assign(tape_slots, 0);
  c->slot_h.assign(tape_slots, 0.0);
  *out = c;
  return OSTRICH_OK;
}

ostrich_status ostrich_layout(const ostrich_ctx* c, int32_t out[4]) {
  if (!c || !out) return OSTRICH_EINVAL;
  out[0] = c->sc.n_state; out[1] = c->sc.m_max; out[2] = c->sc.n_slots; out[3] = c->sc.n_servo;
  return OSTRICH_OK;
}

ostrich_status ostrich_set_threads(ostrich_ctx* c, int threads) {
  if (!c) return OSTRICH_EINVAL;
  if (threads != 32 && threads != 64 && threads != 128) return fail(c, OSTRICH_EINVAL, "threads must be 32, 64 or 128");
  c->threads = threads;
  return OSTRICH_OK;
}

ostrich_status ostrich_set_schedule(ostrich_ctx* c, int schedule) {
  if (!c) return OSTRICH_EINVAL;
  if (schedule != 0 && schedule != 1) return fail(c, OSTRICH_EINVAL, "schedule must be 0 or 1");
  if (schedule == 1 && !c->d_sched) {
    void* p = nullptr;
    const size_t bytes = sizeof(int32_t) * (1 + 2 * (size_t)c->n_worlds);
    if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); return fail(c, OSTRICH_ENOMEM, "schedule buffers"); }
    if (cudaMemset(p, 0, bytes) != cudaSuccess) { cudaGetLastError(); cudaFree(p); return fail(c, OSTRICH_ECUDA, "schedule buffers"); }
    c->d_sched = static_cast<int32_t*>(p);
  }
  c->schedule = schedule;
  return OSTRICH_OK;
}

static void* slot_ptr(ostrich_ctx* c, int slot) {
  return static_cast<char*>(c->tape) + (size_t)slot * c->n_worlds * c->tape_world_elems * elem_size(c->dtype);
}

ostrich_status ostrich_step(ostrich_ctx* c, const void* state_in, const void* controls, double h, void* state_out,
                            void* impulses_out, int32_t* ids, uint32_t* status, int32_t* iters, int tape_slot,
                            void* stream) {
  if (!c) return OSTRICH_EINVAL;
  if (!state_in || !state_out || state_in == state_out) return fail(c, OSTRICH_EINVAL, "state_in/state_out missing or aliased");
  if (c->sc.n_servo > 0 && !controls) return fail(c, OSTRICH_EINVAL, "controls required: the scene has servos");
  if (!(h > 0)) return fail(c, OSTRICH_EINVAL, "h must be positive");
  if (tape_slot >= c->tape_slots || tape_slot < -1) return fail(c, OSTRICH_EINVAL, "tape_slot out of range");
  ost::StepArgs a;
  a.state_in = state_in; a.controls = controls; a.state_out = state_out; a.impulses = impulses_out;
  a.ids = ids; a.status = status; a.iters = iters;
  a.tape = tape_slot >= 0 ? slot_ptr(c, tape_slot) : nullptr;
  a.ld = c->ld; a.n_worlds = c->n_worlds; a.world0 = 0; a.h = h;
  a.trace = c->trace;
  if (c->schedule == 1 && c->d_sched) {
    a.queue = c->d_sched; a.cost = c->d_sched + 1; a.order = c->d_sched + 1 + c->n_worlds;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = c->dtype == OSTRICH_F64 ? ost::launch_step<double>(c->sc, a, c->threads, st)
                                          : ost::launch_step<float>(c->sc, a, c->threads, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "ostrich_step launch");
  if (tape_slot >= 0) { c->slot_written[tape_slot] = 1; c->slot_h[tape_slot] = h; }
  return OSTRICH_OK;
}

ostrich_status ostrich_step_list(ostrich_ctx* c, const void* state_in, const void* controls, double h,
                                 void* state_out, void* impulses_out, int32_t* ids, uint32_t* status, int32_t* iters,
                                 const int32_t* worlds, const int32_t* tape_slots, int n_list, void* stream) {
  if (!c) return OSTRICH_EINVAL;
  if (!state_in || !state_out) return fail(c, OSTRICH_EINVAL, "state_in/state_out missing");
  if (c->sc.n_servo > 0 && !controls) return fail(c, OSTRICH_EINVAL, "controls required: the scene has servos");
  if (!(h > 0)) return fail(c, OSTRICH_EINVAL, "h must be positive");
  if (n_list < 0 || n_list > c->n_worlds) return fail(c, OSTRICH_EINVAL, "n_list outside [0, n_worlds]");
  if (n_list > 0 && !worlds) return fail(c, OSTRICH_EINVAL, "worlds list missing");
  if (tape_slots && !c->tape) return fail(c, OSTRICH_EINVAL, "tape slots given but the context has no tape");
  if (n_list == 0) return OSTRICH_OK;
  ost::StepArgs a;
  a.state_in = state_in; a.controls = controls; a.state_out = state_out; a.impulses = impulses_out;
  a.ids = ids; a.status = status; a.iters = iters;
  a.tape = tape_slots ? c->tape : nullptr;
  a.ld = c->ld; a.n_worlds = c->n_worlds; a.world0 = 0; a.h = h;
  a.trace = c->trace;
  a.list = worlds; a.list_slot = tape_slots; a.n_list = n_list; a.tape_slots = c->tape_slots;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = c->dtype == OSTRICH_F64 ? ost::launch_step<double>(c->sc, a, c->threads, st)
                                          : ost::launch_step<float>(c->sc, a, c->threads, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "ostrich_step_list launch");
  return OSTRICH_OK;
}

ostrich_status ostrich_adjoint_list(ostrich_ctx* c, const void* dL_dnext, double h, void* dL_dstate,
                                    void* dL_dcontrols, const int32_t* worlds, const int32_t* tape_slots, int n_list,
                                    void* stream) {
  if (!c) return OSTRICH_EINVAL;
  if (!c->tape) return fail(c, OSTRICH_ETAPE, "the context has no tape");
  if (!dL_dnext || !dL_dstate) return fail(c, OSTRICH_EINVAL, "gradient pointers missing");
  if (!(h > 0)) return fail(c, OSTRICH_EINVAL, "h must be positive");
  if (n_list < 0 || n_list > c->n_worlds) return fail(c, OSTRICH_EINVAL, "n_list outside [0, n_worlds]");
  if (n_list > 0 && (!worlds || !tape_slots)) return fail(c, OSTRICH_EINVAL, "worlds or tape_slots list missing");
  if (n_list == 0) return OSTRICH_OK;
  ost::AdjArgs a;
  a.tape = c->tape; a.dL_dnext = dL_dnext; a.dL_dstate = dL_dstate; a.dL_dcontrols = dL_dcontrols;
  a.ld = c->ld; a.n_worlds = c->n_worlds; a.world0 = 0; a.h = h;
  a.list = worlds; a.list_slot = tape_slots; a.n_list = n_list; a.tape_slots = c->tape_slots;
  a.mode = c->adj_mode; a.krylov = c->krylov;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = c->dtype == OSTRICH_F64 ? ost::launch_adjoint<double>(c->sc, a, c->threads, st)
                                          : ost::launch_adjoint<float>(c->sc, a, c->threads, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "ostrich_adjoint_list launch");
  return OSTRICH_OK;
}

ostrich_status ostrich_set_adjoint_mode(ostrich_ctx* c, int mode, int32_t* krylov_iters) {
  if (!c) return OSTRICH_EINVAL;
  if (mode != OSTRICH_ADJ_PAPER && mode != OSTRICH_ADJ_EXACT) return fail(c, OSTRICH_EINVAL, "unknown adjoint mode");
  const size_t smem = c->dtype == OSTRICH_F64 ? ost::adj_smem_bytes<double>(c->sc, mode)
                                              : ost::adj_smem_bytes<float>(c->sc, mode);
  if (smem > ost::SMEM_CTA_MAX) return fail(c, OSTRICH_EINVAL, "the exact adjoint's working set exceeds shared memory");
  c->adj_mode = mode;
  c->krylov = krylov_iters;
  return OSTRICH_OK;
}

ostrich_status ostrich_set_linear_solver(ostrich_ctx* c, int solver, int precond, int iters, int adj_iters,
                                         double adj_rtol) {
  if (!c) return OSTRICH_EINVAL;
  if (solver != OSTRICH_LIN_DIRECT && solver != OSTRICH_LIN_PCR) return fail(c, OSTRICH_EINVAL, "unknown linear solver");
  if (precond != OSTRICH_PC_JACOBI && precond != OSTRICH_PC_BLOCK) return fail(c, OSTRICH_EINVAL, "unknown preconditioner");
  if (iters < 1 || adj_iters < 1 || !(adj_rtol >= 0)) return fail(c, OSTRICH_EINVAL, "PCR counts must be >= 1");
  ost::DevScene s = c->sc;
  s.lin = solver; s.pc = precond; s.pcr_iters = iters; s.pcr_iters_adj = adj_iters;
  s.pcr_rtol_adj = adj_rtol > 0 ? adj_rtol : (c->dtype == OSTRICH_F32 ? 1e-10 : 1e-12);
  const bool f64 = c->dtype == OSTRICH_F64;
  const size_t ws = f64 ? ost::ws_bytes<double>(s) : ost::ws_bytes<float>(s);
  const size_t used = f64 ? ost::ws_used<double>(s) : ost::ws_used<float>(s);
  const size_t adj = f64 ? ost::adj_smem_bytes<double>(s, c->adj_mode) : ost::adj_smem_bytes<float>(s, c->adj_mode);
  if (ws > ost::SMEM_CTA_MAX || used > ws || adj > ost::SMEM_CTA_MAX)
    return fail(c, OSTRICH_EINVAL, "the PCR working set exceeds shared memory");
  c->sc = s;
  std::fill(c->slot_written.begin(), c->slot_written.end(), (unsigned char)0);
  return OSTRICH_OK;
}

ostrich_status ostrich_adjoint(ostrich_ctx* c, int tape_slot, const void* dL_dnext, double h, void* dL_dstate,
                               void* dL_dcontrols, void* stream) {
  return ostrich_adjoint_params(c, tape_slot, dL_dnext, h, dL_dstate, dL_dcontrols, nullptr, nullptr, nullptr, nullptr,
                                stream);
}

ostrich_status ostrich_adjoint_params(ostrich_ctx* c, int tape_slot, const void* dL_dnext, double h, void* dL_dstate,
                                      void* dL_dcontrols, void* dL_dkp, void* dL_dmass, void* dL_dinertia,
                                      void* dL_dmu, void* stream) {
  if (!c) return OSTRICH_EINVAL;
  if (tape_slot < 0 || tape_slot >= c->tape_slots) return fail(c, OSTRICH_EINVAL, "tape_slot out of range");
  if (!c->slot_written[tape_slot]) return fail(c, OSTRICH_ETAPE, "tape slot holds no recorded step");
  if (h != c->slot_h[tape_slot]) return fail(c, OSTRICH_EINVAL, "h differs from the recorded step");
  if (!dL_dnext || !dL_dstate) return fail(c, OSTRICH_EINVAL, "gradient pointers missing");
  ost::AdjArgs a;
  a.tape = slot_ptr(c, tape_slot); a.dL_dnext = dL_dnext; a.dL_dstate = dL_dstate; a.dL_dcontrols = dL_dcontrols;
  a.ld = c->ld; a.n_worlds = c->n_worlds; a.world0 = 0; a.h = h;
  a.dL_dkp = c->sc.n_servo > 0 ? dL_dkp : nullptr; a.dL_dmass = dL_dmass; a.dL_dinertia = dL_dinertia;
  a.dL_dmu = dL_dmu; a.mode = c->adj_mode; a.krylov = c->krylov;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = c->dtype == OSTRICH_F64 ? ost::launch_adjoint<double>(c->sc, a, c->threads, st)
                                          : ost::launch_adjoint<float>(c->sc, a, c->threads, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "ostrich_adjoint launch");
  return OSTRICH_OK;
}

ostrich_status ostrich_debug_trace(ostrich_ctx* c, double* merits) {
  if (!c) return OSTRICH_EINVAL;
  c->trace = merits;
  return OSTRICH_OK;
}

ostrich_status ostrich_tape_clear(ostrich_ctx* c) {
  if (!c) return OSTRICH_EINVAL;
  for (auto& v : c->slot_written) v = 0;
  return OSTRICH_OK;
}

size_t ostrich_workspace_bytes(const ostrich_ctx* c) {
  if (!c) return 0;
  return c->dtype == OSTRICH_F64 ? ost::ws_bytes<double>(c->sc) : ost::ws_bytes<float>(c->sc);
}

size_t ostrich_tape_bytes(const ostrich_ctx* c) {
  return c ? (size_t)c->n_worlds * c->tape_world_elems * elem_size(c->dtype) : 0;
}

const char* ostrich_last_error(const ostrich_ctx* c) { return c ? c->err : "null context"; }

void ostrich_destroy(ostrich_ctx* c) {
  if (!c) return;
  delete c;
}

}  // extern "C"
