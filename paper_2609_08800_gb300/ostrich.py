"""Thin Python binding of libostrich (include/ostrich.h).

Argument marshalling only: every step of the solve and the adjoint runs in the
CUDA kernels of the shared library.  PyTorch supplies device memory and the
stream.  If the library is missing or a call fails, an exception is raised; there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import scenes as S

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libostrich.so")

OSTRICH_OK, OSTRICH_EINVAL, OSTRICH_ENOMEM, OSTRICH_ECUDA, OSTRICH_ETAPE = 0, 1, 2, 3, 4
OSTRICH_F32, OSTRICH_F64 = 0, 1
ADJ_PAPER, ADJ_EXACT = 0, 1
LIN_DIRECT, LIN_PCR = 0, 1
PC_JACOBI, PC_BLOCK = 0, 1
MAX_BODIES = 8
MAX_JOINTS = 8

_d3 = ctypes.c_double * 3


class BodyDesc(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("inertia", _d3), ("shape", ctypes.c_int), ("half_extents", _d3),
                ("radius", ctypes.c_double), ("half_width", ctypes.c_double)]


class JointDesc(ctypes.Structure):
    _fields_ = [("parent", ctypes.c_int), ("child", ctypes.c_int), ("anchor_parent", _d3), ("anchor_child", _d3),
                ("axis_parent", _d3), ("axis_child", _d3), ("perp1_parent", _d3), ("perp2_parent", _d3),
                ("kp", ctypes.c_double), ("type", ctypes.c_int), ("servo_mode", ctypes.c_int), ("kd", ctypes.c_double)]


class SceneDesc(ctypes.Structure):
    _fields_ = [("n_bodies", ctypes.c_int), ("n_joints", ctypes.c_int), ("env", ctypes.c_int),
                ("mu", ctypes.c_double), ("gravity", ctypes.c_double), ("box", ctypes.c_double * 5),
                ("hm_n", ctypes.c_int), ("hm_spacing", ctypes.c_double), ("hm_origin", ctypes.c_double * 2),
                ("heights", ctypes.POINTER(ctypes.c_float)),
                ("bodies", BodyDesc * MAX_BODIES), ("joints", JointDesc * MAX_JOINTS)]


class SolverCfg(ctypes.Structure):
    _fields_ = [("budget", ctypes.c_int), ("k_min", ctypes.c_int), ("line_search", ctypes.c_int),
                ("pullback", ctypes.c_int), ("tol", ctypes.c_double), ("delta_rel", ctypes.c_double),
                ("kappa", ctypes.c_double), ("eps_fb", ctypes.c_double), ("margin", ctypes.c_double)]


_vp = ctypes.c_void_p
_lib = None


def lib():
    """Load libostrich (built in-tree by ``build()``); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libostrich is not built ({LIB_PATH} missing); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.ostrich_create.argtypes = [ctypes.POINTER(SceneDesc), ctypes.POINTER(SolverCfg), ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp)]
        L.ostrich_create.restype = ctypes.c_int
        L.ostrich_layout.argtypes = [_vp, ctypes.POINTER(ctypes.c_int32)]
        L.ostrich_set_threads.argtypes = [_vp, ctypes.c_int]
        L.ostrich_set_schedule.argtypes = [_vp, ctypes.c_int]
        L.ostrich_step.argtypes = [_vp, _vp, _vp, ctypes.c_double, _vp, _vp, _vp, _vp, _vp, ctypes.c_int, _vp]
        L.ostrich_adjoint.argtypes = [_vp, ctypes.c_int, _vp, ctypes.c_double, _vp, _vp, _vp]
        L.ostrich_adjoint_params.argtypes = [_vp, ctypes.c_int, _vp, ctypes.c_double, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
        L.ostrich_set_adjoint_mode.argtypes = [_vp, ctypes.c_int, _vp]
        L.ostrich_set_linear_solver.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_double]
        L.ostrich_set_adjoint_mode.restype = ctypes.c_int
        L.ostrich_step_list.argtypes = [_vp, _vp, _vp, ctypes.c_double, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                        ctypes.c_int, _vp]
        L.ostrich_adjoint_list.argtypes = [_vp, _vp, ctypes.c_double, _vp, _vp, _vp, _vp, ctypes.c_int, _vp]
        L.ostrich_tape_clear.argtypes = [_vp]
        L.ostrich_debug_trace.argtypes = [_vp, _vp]
        L.ostrich_debug_trace.restype = ctypes.c_int
        L.ostrich_tape_bytes.argtypes = [_vp]
        L.ostrich_tape_bytes.restype = ctypes.c_size_t
        L.ostrich_workspace_bytes.argtypes = [_vp]
        L.ostrich_workspace_bytes.restype = ctypes.c_size_t
        L.ostrich_last_error.argtypes = [_vp]
        L.ostrich_last_error.restype = ctypes.c_char_p
        L.ostrich_destroy.argtypes = [_vp]
        L.ostrich_noalloc_capacity.argtypes = [ctypes.POINTER(SceneDesc), ctypes.POINTER(SolverCfg),
                                               ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_size_t)]
        L.ostrich_step_adjoint_noalloc.argtypes = [ctypes.POINTER(SceneDesc), ctypes.POINTER(SolverCfg), ctypes.c_int,
                                                   ctypes.c_int, _vp, _vp, ctypes.c_double, _vp, _vp, _vp, _vp, _vp]
        L.ostrich_probe_ffma.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_size_t),
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _vp]
        L.ostrich_probe_ffma.restype = ctypes.c_int
        for name in ("ostrich_layout", "ostrich_set_threads", "ostrich_set_schedule", "ostrich_step", "ostrich_adjoint", "ostrich_tape_clear",
                     "ostrich_step_adjoint_noalloc", "ostrich_step_list", "ostrich_adjoint_list"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def scene_desc(scene: "S.Scene") -> SceneDesc:
    d = SceneDesc()
    d.n_bodies, d.n_joints, d.env = scene.n_bodies, len(scene.joints), scene.env.kind
    d.mu, d.gravity = scene.mu, scene.gravity
    for i, v in enumerate(scene.env.box):
        d.box[i] = v
    if scene.env.heights is not None:
        hts = np.ascontiguousarray(scene.env.heights, dtype=np.float32)
        if hts.ndim != 2 or hts.shape[0] != hts.shape[1]:
            raise ValueError("heightmap must be a square [n, n] array")
        d.hm_n = hts.shape[0]
        d.hm_spacing = scene.env.spacing
        d.hm_origin[0], d.hm_origin[1] = scene.env.origin
        d.heights = hts.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        d._heights = hts          # keeps the host array alive as long as the descriptor
    for i, b in enumerate(scene.bodies):
        bd = d.bodies[i]
        bd.mass = b.mass
        bd.inertia[:] = b.inertia
        bd.shape = b.shape
        bd.half_extents[:] = b.half_extents
        bd.radius, bd.half_width = b.radius, b.half_width
    for i, j in enumerate(scene.joints):
        jd = d.joints[i]
        jd.parent, jd.child = j.parent, j.child
        jd.anchor_parent[:] = j.anchor_parent
        jd.anchor_child[:] = j.anchor_child
        jd.axis_parent[:] = j.axis_parent
        jd.axis_child[:] = j.axis_child
        jd.perp1_parent[:] = j.perp_parent[0]
        jd.perp2_parent[:] = j.perp_parent[1]
        jd.kp = j.kp
        jd.type, jd.servo_mode, jd.kd = j.type, j.servo_mode, j.kd
    return d


def solver_cfg(cfg: "S.SolverConfig") -> SolverCfg:
    c = SolverCfg()
    c.budget, c.k_min, c.line_search, c.pullback = cfg.budget, cfg.k_min, cfg.line_search, cfg.pullback
    c.tol, c.delta_rel, c.kappa, c.eps_fb, c.margin = cfg.tol, cfg.delta_rel, cfg.kappa, cfg.eps_fb, cfg.margin
    return c


def _ptr(t):
    """Device pointer of a dense CUDA tensor.  The library reads and writes arrays as
    packed [rows, ld] (world index fastest), so a strided view would be misread: it is
    refused rather than copied (a copy would also break in-place outputs)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libostrich takes device tensors; got a host tensor")
    if not t.is_contiguous():
        raise ValueError(f"libostrich takes contiguous arrays; got shape {tuple(t.shape)} strides {t.stride()}")
    return ctypes.c_void_p(t.data_ptr())


def _checked(t, dtype, numel, what):
    """Device pointer of `t` after checking what the library assumes of it through the
    raw pointer: element type `dtype` and at least `numel` elements (a smaller array
    would be read or written past its end on the device).  Objects without a dtype --
    the column addresses of a wider array that the one-world-per-launch form passes --
    go to _ptr unchecked."""
    if t is None:
        return None
    if hasattr(t, "dtype"):
        if t.dtype != dtype:
            raise ValueError(f"{what}: expected element type {dtype}, got {t.dtype}")
        if t.numel() < numel:
            raise ValueError(f"{what}: needs at least {numel} elements, got {t.numel()} (shape {tuple(t.shape)})")
    return _ptr(t)


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


NOALLOC_SCRATCH_BYTES = 16 << 20


def ostrich_step_adjoint_noalloc(scene, cfg, n_worlds, state_in, controls, h, state_out, dL_dnext, dL_dstate,
                                 dL_dcontrols=None, ld=0, stream=None):
    """Step + adjoint with the tape in the library's fixed array (no device allocation);
    FP32 tensors [rows, ld].  Raises on a non-OK status (EINVAL beyond the array's size)."""
    import torch
    d, c = scene_desc(scene), solver_cfg(cfg)
    W, L = int(n_worlds), int(ld) or int(n_worlds)

    def arr(t, rows, what):
        return _checked(t, torch.float32, (rows - 1) * L + W if rows > 0 else 0, what)

    ns, nsv = scene.n_state, scene.n_servos
    rc = lib().ostrich_step_adjoint_noalloc(ctypes.byref(d), ctypes.byref(c), W, int(ld),
                                            arr(state_in, ns, "state_in"), arr(controls, nsv, "controls"), float(h),
                                            arr(state_out, ns, "state_out"), arr(dL_dnext, ns, "dL_dnext"),
                                            arr(dL_dstate, ns, "dL_dstate"), arr(dL_dcontrols, nsv, "dL_dcontrols"),
                                            _stream(stream))
    if rc != OSTRICH_OK:
        raise RuntimeError(f"ostrich_step_adjoint_noalloc failed with status {rc}")


def noalloc_capacity(scene, cfg=None):
    """(max worlds per ostrich_step_adjoint_noalloc call, per-world tape record in bytes)."""
    d, c = scene_desc(scene), solver_cfg(cfg or S.SolverConfig())
    mw, rb = ctypes.c_int32(), ctypes.c_size_t()
    rc = lib().ostrich_noalloc_capacity(ctypes.byref(d), ctypes.byref(c), ctypes.byref(mw), ctypes.byref(rb))
    if rc != OSTRICH_OK:
        raise ValueError(f"ostrich_noalloc_capacity refused the scene (status {rc})")
    return int(mw.value), int(rb.value)


def probe_ffma(blocks_per_sm=2, iters=40000, reps=10, stream=None):
    """Measured FP32 FFMA throughput of the current GPU (include/ostrich_probe.h):
    returns (TFLOP/s, mean kernel ms).  A measurement helper, not part of the method."""
    import torch
    n = ctypes.c_size_t()
    rc = lib().ostrich_probe_ffma(blocks_per_sm, iters, reps, None, ctypes.byref(n), None, None, None)
    if rc != 0:
        raise RuntimeError(f"ostrich_probe_ffma failed with CUDA error {rc}")
    out = torch.empty(n.value, dtype=torch.float32, device="cuda")
    tf, ms = ctypes.c_double(), ctypes.c_double()
    rc = lib().ostrich_probe_ffma(blocks_per_sm, iters, reps, _ptr(out), ctypes.byref(n), ctypes.byref(tf),
                                  ctypes.byref(ms), _stream(stream))
    if rc != 0:
        raise RuntimeError(f"ostrich_probe_ffma failed with CUDA error {rc}")
    return tf.value, ms.value


class Context:
    """One ostrich_ctx: a scene, a solver configuration, W worlds and a tape."""

    def __init__(self, scene, cfg, n_worlds, dtype="f32", tape_slots=1, ld=0, threads=None):
        import torch
        self.scene, self.cfg = scene, cfg
        self.n_worlds = int(n_worlds)
        self.dtype = torch.float64 if dtype in ("f64", torch.float64) else torch.float32
        self._desc, self._cfg = scene_desc(scene), solver_cfg(cfg)
        h = _vp()
        rc = lib().ostrich_create(ctypes.byref(self._desc), ctypes.byref(self._cfg), self.n_worlds, int(ld),
                                  OSTRICH_F64 if self.dtype == torch.float64 else OSTRICH_F32, int(tape_slots),
                                  ctypes.byref(h))
        if rc != OSTRICH_OK:
            raise RuntimeError(f"ostrich_create failed with status {rc}")
        self._h = h
        self.ld = int(ld) if ld else self.n_worlds
        out = (ctypes.c_int32 * 4)()
        lib().ostrich_layout(self._h, out)
        self.n_state, self.m_max, self.n_slots, self.n_servo = map(int, out)
        self.tape_slots = int(tape_slots)
        self.nb = scene.n_bodies
        if threads is not None:
            self.set_threads(threads)
        if getattr(cfg, "linear_solver", LIN_DIRECT) != LIN_DIRECT:
            self.set_linear_solver(cfg.linear_solver, cfg.precond, cfg.pcr_iters, cfg.pcr_iters_adj, cfg.pcr_rtol_adj)

    def _arr(self, t, rows, what):
        """A [rows, ld] array of the context's element type (the library touches element
        c * ld + w for c < rows and every world w < n_worlds)."""
        return _checked(t, self.dtype, (rows - 1) * self.ld + self.n_worlds if rows > 0 else 0, what)

    def _i32(self, t, n, what):
        import torch
        return _checked(t, torch.int32, n, what)

    def _check(self, rc, what):
        if rc != OSTRICH_OK:
            msg = lib().ostrich_last_error(self._h).decode()
            raise RuntimeError(f"{what} failed with status {rc}: {msg}")

    def set_threads(self, threads):
        self._check(lib().ostrich_set_threads(self._h, int(threads)), "ostrich_set_threads")
        self.threads = int(threads)

    def set_schedule(self, schedule):
        """0: one CTA per world; 1: persistent CTAs, heaviest worlds first."""
        self._check(lib().ostrich_set_schedule(self._h, int(schedule)), "ostrich_set_schedule")
        self.schedule = int(schedule)

    def ostrich_step(self, state_in, controls, h, state_out, impulses=None, ids=None, status=None, iters=None,
                     tape_slot=-1, stream=None):
        self._check(lib().ostrich_step(self._h, self._arr(state_in, self.n_state, "state_in"),
                                       self._arr(controls, self.n_servo, "controls"), float(h),
                                       self._arr(state_out, self.n_state, "state_out"),
                                       self._arr(impulses, self.m_max, "impulses"),
                                       self._i32(ids, (self.n_slots - 1) * self.ld + self.n_worlds if self.n_slots
                                                 else 0, "ids"),
                                       self._i32(status, self.n_worlds, "status"),
                                       self._i32(iters, self.n_worlds, "iters"), int(tape_slot),
                                       _stream(stream)), "ostrich_step")

    def ostrich_adjoint(self, tape_slot, dL_dnext, h, dL_dstate, dL_dcontrols=None, stream=None):
        self._check(lib().ostrich_adjoint(self._h, int(tape_slot), self._arr(dL_dnext, self.n_state, "dL_dnext"),
                                          float(h), self._arr(dL_dstate, self.n_state, "dL_dstate"),
                                          self._arr(dL_dcontrols, self.n_servo, "dL_dcontrols"), _stream(stream)),
                    "ostrich_adjoint")

    def ostrich_adjoint_params(self, tape_slot, dL_dnext, h, dL_dstate, dL_dcontrols=None, dL_dkp=None,
                               dL_dmass=None, dL_dinertia=None, dL_dmu=None, stream=None):
        self._check(lib().ostrich_adjoint_params(self._h, int(tape_slot), self._arr(dL_dnext, self.n_state, "dL_dnext"),
                                                 float(h), self._arr(dL_dstate, self.n_state, "dL_dstate"),
                                                 self._arr(dL_dcontrols, self.n_servo, "dL_dcontrols"),
                                                 self._arr(dL_dkp, self.n_servo, "dL_dkp"),
                                                 self._arr(dL_dmass, self.nb, "dL_dmass"),
                                                 self._arr(dL_dinertia, 3 * self.nb, "dL_dinertia"),
                                                 _checked(dL_dmu, self.dtype, self.n_worlds, "dL_dmu"), _stream(stream)),
                    "ostrich_adjoint_params")

    def set_adjoint_mode(self, mode, krylov_iters=None):
        """ADJ_PAPER (the paper's frozen-W adjoint, default) or ADJ_EXACT (the exact IFT by
        GMRES on the taped factor); krylov_iters: optional int32 device tensor [n_worlds]."""
        self._check(lib().ostrich_set_adjoint_mode(self._h, int(mode), self._i32(krylov_iters, self.n_worlds,
                                                                                 "krylov_iters")),
                    "ostrich_set_adjoint_mode")
        self.adj_mode = int(mode)

    def set_linear_solver(self, solver, precond=PC_JACOBI, iters=16, adj_iters=256, adj_rtol=0.0):
        """LIN_DIRECT (block-arrowhead factor, default) or LIN_PCR (matrix-free preconditioned
        conjugate residual, `iters` per Newton step, preconditioner PC_JACOBI or PC_BLOCK)."""
        self._check(lib().ostrich_set_linear_solver(self._h, int(solver), int(precond), int(iters), int(adj_iters),
                                                    float(adj_rtol)), "ostrich_set_linear_solver")
        self.linear_solver = int(solver)

    def ostrich_step_list(self, state_in, controls, h, state_out, worlds, tape_slots=None, impulses=None, ids=None,
                          status=None, iters=None, stream=None):
        n = int(worlds.numel())
        self._check(lib().ostrich_step_list(self._h, self._arr(state_in, self.n_state, "state_in"),
                                            self._arr(controls, self.n_servo, "controls"), float(h),
                                            self._arr(state_out, self.n_state, "state_out"),
                                            self._arr(impulses, self.m_max, "impulses"),
                                            self._i32(ids, (self.n_slots - 1) * self.ld + self.n_worlds if self.n_slots
                                                      else 0, "ids"),
                                            self._i32(status, self.n_worlds, "status"),
                                            self._i32(iters, self.n_worlds, "iters"), self._i32(worlds, n, "worlds"),
                                            self._i32(tape_slots, n, "tape_slots"), n, _stream(stream)),
                    "ostrich_step_list")

    def ostrich_adjoint_list(self, dL_dnext, h, dL_dstate, worlds, tape_slots, dL_dcontrols=None, stream=None):
        n = int(worlds.numel())
        self._check(lib().ostrich_adjoint_list(self._h, self._arr(dL_dnext, self.n_state, "dL_dnext"), float(h),
                                               self._arr(dL_dstate, self.n_state, "dL_dstate"),
                                               self._arr(dL_dcontrols, self.n_servo, "dL_dcontrols"),
                                               self._i32(worlds, n, "worlds"), self._i32(tape_slots, n, "tape_slots"),
                                               n, _stream(stream)),
                    "ostrich_adjoint_list")

    def ostrich_debug_trace(self, merits):
        import torch
        self._check(lib().ostrich_debug_trace(self._h, _checked(merits, torch.float64,
                                                                self.n_worlds * (self.cfg.budget + 2), "merits")),
                    "ostrich_debug_trace")

    def ostrich_tape_clear(self):
        self._check(lib().ostrich_tape_clear(self._h), "ostrich_tape_clear")

    def tape_bytes(self):
        return int(lib().ostrich_tape_bytes(self._h))

    def workspace_bytes(self):
        return int(lib().ostrich_workspace_bytes(self._h))

    # convenience wrappers that allocate outputs (torch tensors [rows, ld])
    def alloc_state(self):
        import torch
        return torch.zeros(self.n_state, self.ld, dtype=self.dtype, device="cuda")

    def step(self, state_in, controls, h, tape_slot=-1, stream=None):
        import torch
        dev = state_in.device
        out = torch.empty(self.n_state, self.ld, dtype=self.dtype, device=dev)
        imp = torch.empty(self.m_max, self.ld, dtype=self.dtype, device=dev)
        ids = torch.empty(max(self.n_slots, 1), self.ld, dtype=torch.int32, device=dev)
        st = torch.empty(self.ld, dtype=torch.int32, device=dev)
        it = torch.empty(self.ld, dtype=torch.int32, device=dev)
        self.ostrich_step(state_in, controls, h, out, imp, ids, st, it, tape_slot, stream)
        return dict(state=out, impulses=imp, ids=ids[:self.n_slots], status=st, iters=it)

    def adjoint(self, tape_slot, dL_dnext, h, stream=None):
        import torch
        dev = dL_dnext.device
        ds = torch.empty(self.n_state, self.ld, dtype=self.dtype, device=dev)
        du = torch.empty(max(self.n_servo, 1), self.ld, dtype=self.dtype, device=dev)
        self.ostrich_adjoint(tape_slot, dL_dnext, h, ds, du, stream)
        return ds, du[:self.n_servo]

    def adjoint_params(self, tape_slot, dL_dnext, h, stream=None, with_mu=False):
        """The adjoint plus the physical-parameter gradients: (dL/dstate, dL/dcontrols,
        dL/dk_p [n_servo, ld], dL/dm [nb, ld], dL/dI [nb, 3, ld] of the principal moments),
        and dL/dmu [n_worlds] last when with_mu."""
        import torch
        dev = dL_dnext.device
        ds = torch.empty(self.n_state, self.ld, dtype=self.dtype, device=dev)
        du = torch.empty(max(self.n_servo, 1), self.ld, dtype=self.dtype, device=dev)
        dkp = torch.empty(max(self.n_servo, 1), self.ld, dtype=self.dtype, device=dev)
        dm = torch.empty(self.nb, self.ld, dtype=self.dtype, device=dev)
        di = torch.empty(self.nb, 3, self.ld, dtype=self.dtype, device=dev)
        dmu = torch.empty(self.n_worlds, dtype=self.dtype, device=dev) if with_mu else None
        self.ostrich_adjoint_params(tape_slot, dL_dnext, h, ds, du, dkp, dm, di, dmu, stream)
        out = (ds, du[:self.n_servo], dkp[:self.n_servo], dm, di)
        return out + (dmu,) if with_mu else out

    def close(self):
        if getattr(self, "_h", None):
            lib().ostrich_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
