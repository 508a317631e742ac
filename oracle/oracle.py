"""ctypes wrapper of the FP64 CPU oracle (oracle/ostrich_oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product path.  It
packs a scene from the seeded scene module into the oracle's own flat format
and runs one world per call.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ostrich_oracle.cpp")
_LIB = os.path.join(_HERE, "libostrich_oracle.so")

ADJ_PAPER = 0
ADJ_EXACT = 1

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int32)
_up = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no FMA contraction, so its FP32 contact
    predicate rounds exactly like the CUDA one)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", _SRC, "-o", _LIB]
        subprocess.run(cmd, check=True)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.oracle_layout.argtypes = [_dp, _fp, _ip]
        L.oracle_step.argtypes = [_dp, _fp, _dp, _dp, _dp, ctypes.c_double, _dp, _dp, _ip, _up, _dp]
        L.oracle_step_adjoint.argtypes = [_dp, _fp, _dp, _dp, _dp, ctypes.c_double, _dp, ctypes.c_int,
                                          _dp, _dp, _ip, _up, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        L.oracle_adjoint_at.argtypes = [_dp, _fp, _dp, _dp, _dp, ctypes.c_double, _dp, _dp, _dp, ctypes.c_int,
                                        _dp, _dp, _dp, _dp, _dp, _dp]
        L.oracle_fb.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp]
        L.oracle_friction_W.argtypes = [ctypes.c_double] * 8
        L.oracle_friction_W.restype = ctypes.c_double
        L.oracle_rotate.argtypes = [_dp, _dp, _dp]
        L.oracle_lu_solve.argtypes = [ctypes.c_int, _dp, _dp, _dp]
        L.oracle_pcr.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int, _ip, ctypes.c_int, ctypes.c_double, _dp, _ip]
        L.oracle_contacts.argtypes = [_dp, _fp, _dp, _dp, ctypes.c_double, _ip, _ip, _dp]
        L.oracle_rows.argtypes = [_dp, _fp, _dp, _dp, _dp, ctypes.c_double, _dp, _dp, ctypes.c_int,
                                  _ip, _dp, _dp, _dp, _dp, _dp]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def pack_scene(scene):
    """Flat double array: header[14], bodies[nb*10], joints[nj*24]; heights (float32) apart."""
    env = scene.env
    hdr = [scene.n_bodies, len(scene.joints), env.kind, scene.mu, scene.gravity, *env.box,
           0 if env.heights is None else env.heights.shape[0], env.spacing, env.origin[0], env.origin[1]]
    vals = list(map(float, hdr))
    for b in scene.bodies:
        vals += [b.mass, *b.inertia, b.shape, *b.half_extents, b.radius, b.half_width]
    for j in scene.joints:
        vals += [j.parent, j.child, *j.anchor_parent, *j.anchor_child, *j.axis_parent, *j.axis_child,
                 *j.perp_parent[0], *j.perp_parent[1], j.kp, j.type, j.servo_mode, j.kd]
    p = np.ascontiguousarray(np.array(vals, dtype=np.float64))
    if env.heights is not None:
        hts = np.ascontiguousarray(env.heights.astype(np.float32).reshape(-1))
    else:
        hts = np.zeros(1, dtype=np.float32)
    return p, hts


def pack_cfg(cfg):
    return np.array([cfg.budget, cfg.k_min, cfg.tol, cfg.delta_rel, cfg.kappa, cfg.eps_fb, cfg.margin,
                     cfg.line_search, cfg.pullback, cfg.linear_solver, cfg.precond, cfg.pcr_iters,
                     cfg.pcr_iters_adj, cfg.pcr_rtol_adj if cfg.pcr_rtol_adj > 0 else 1e-12], dtype=np.float64)


class Oracle:
    """One scene + solver configuration; all arrays are one world (1-D, float64)."""

    def __init__(self, scene, cfg):
        self.scene, self.cfg = scene, cfg
        self.sp, self.hts = pack_scene(scene)
        self.cp = pack_cfg(cfg)
        out = np.zeros(4, dtype=np.int32)
        if lib().oracle_layout(_d(self.sp), self.hts.ctypes.data_as(_fp), out.ctypes.data_as(_ip)) != 0:
            raise ValueError("oracle rejected the scene")
        self.n_slots, self.m_max, self.n_state, self.n_servo = map(int, out)
        assert self.n_state == scene.n_state and self.m_max == scene.m_max

    def _state(self, state):
        state = np.ascontiguousarray(state, dtype=np.float64)
        if state.shape != (self.n_state,):
            raise ValueError(f"state of shape {state.shape}; this scene's layout has {self.n_state} entries")
        return state

    def _common(self):
        return _d(self.sp), self.hts.ctypes.data_as(_fp), _d(self.cp)

    def step(self, state, ubar, h):
        state = self._state(state)
        ubar = np.ascontiguousarray(np.atleast_1d(ubar), dtype=np.float64) if self.n_servo else np.zeros(1)
        out = np.zeros(self.n_state); imp = np.zeros(self.m_max)
        ids = np.zeros(max(self.n_slots, 1), dtype=np.int32)
        st = np.zeros(1, dtype=np.uint32); info = np.zeros(4)
        rc = lib().oracle_step(*self._common(), _d(state), _d(ubar), float(h), _d(out), _d(imp),
                               ids.ctypes.data_as(_ip), st.ctypes.data_as(_up), _d(info))
        if rc != 0:
            raise RuntimeError("oracle_step failed")
        return dict(state=out, impulses=imp, ids=ids[:self.n_slots], status=int(st[0]),
                    iters=int(info[0]), residual=float(info[1]), ret_k=int(info[2]), rows=int(info[3]))

    def step_adjoint(self, state, ubar, h, dL_dnext, mode=ADJ_PAPER):
        state = self._state(state)
        ubar = np.ascontiguousarray(np.atleast_1d(ubar), dtype=np.float64) if self.n_servo else np.zeros(1)
        g = np.ascontiguousarray(dL_dnext, dtype=np.float64)
        out = np.zeros(self.n_state); imp = np.zeros(self.m_max)
        ids = np.zeros(max(self.n_slots, 1), dtype=np.int32)
        st = np.zeros(1, dtype=np.uint32); info = np.zeros(4)
        dstate = np.zeros(self.n_state); dubar = np.zeros(max(self.n_servo, 1))
        dkp = np.zeros(max(self.n_servo, 1)); dmass = np.zeros(self.scene.n_bodies)
        dinertia = np.zeros(3 * self.scene.n_bodies)
        dmu = np.zeros(1)
        rc = lib().oracle_step_adjoint(*self._common(), _d(state), _d(ubar), float(h), _d(g), int(mode), _d(out),
                                       _d(imp), ids.ctypes.data_as(_ip), st.ctypes.data_as(_up), _d(dstate),
                                       _d(dubar), _d(info), _d(dkp), _d(dmass), _d(dinertia), _d(dmu))
        if rc != 0:
            raise RuntimeError("oracle_step_adjoint failed")
        return dict(state=out, impulses=imp, ids=ids[:self.n_slots], status=int(st[0]), iters=int(info[0]),
                    residual=float(info[1]), ret_k=int(info[2]), dstate=dstate, dubar=dubar[:self.n_servo],
                    dkp=dkp[:self.n_servo], dmass=dmass, dinertia=dinertia.reshape(-1, 3), dmu=float(dmu[0]))

    def adjoint_at(self, state, ubar, h, u, lam, dL_dnext, mode=ADJ_PAPER):
        """The adjoint of the step from `state`, taken at the given returned iterate
        (u+ [6 nb], lambda+ in the state's lambda layout [m_max]) instead of at the
        oracle's own solution."""
        state = self._state(state)
        ubar = np.ascontiguousarray(np.atleast_1d(ubar), dtype=np.float64) if self.n_servo else np.zeros(1)
        u = np.ascontiguousarray(u, dtype=np.float64)
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        if u.shape != (6 * self.scene.n_bodies,) or lam.shape != (self.m_max,):
            raise ValueError("u must have 6 nb entries and lambda m_max")
        g = np.ascontiguousarray(dL_dnext, dtype=np.float64)
        dstate = np.zeros(self.n_state); dubar = np.zeros(max(self.n_servo, 1))
        dkp = np.zeros(max(self.n_servo, 1)); dmass = np.zeros(self.scene.n_bodies)
        dinertia = np.zeros(3 * self.scene.n_bodies)
        dmu = np.zeros(1)
        rc = lib().oracle_adjoint_at(*self._common(), _d(state), _d(ubar), float(h), _d(u), _d(lam), _d(g), int(mode),
                                     _d(dstate), _d(dubar), _d(dkp), _d(dmass), _d(dinertia), _d(dmu))
        if rc != 0:
            raise RuntimeError("oracle_adjoint_at failed")
        return dict(dstate=dstate, dubar=dubar[:self.n_servo], dkp=dkp[:self.n_servo], dmass=dmass,
                    dinertia=dinertia.reshape(-1, 3), dmu=float(dmu[0]))

    def contacts(self, state, h):
        state = self._state(state)
        n = max(self.n_slots, 1)
        act = np.zeros(n, dtype=np.int32); ids = np.zeros(n, dtype=np.int32); nd = np.zeros(4 * n)
        lib().oracle_contacts(*self._common(), _d(state), float(h), act.ctypes.data_as(_ip),
                              ids.ctypes.data_as(_ip), _d(nd))
        return act[:self.n_slots], ids[:self.n_slots], nd[:4 * self.n_slots].reshape(-1, 4)

    def rows(self, state, ubar, h, u, lam, max_rows=512):
        state = self._state(state)
        ubar = np.ascontiguousarray(np.atleast_1d(ubar), dtype=np.float64) if self.n_servo else np.zeros(1)
        u = np.ascontiguousarray(u, dtype=np.float64); lam = np.ascontiguousarray(lam, dtype=np.float64)
        meta = np.zeros(4 * max_rows, dtype=np.int32)
        Jan = np.zeros(12 * max_rows); Jd = np.zeros(12 * max_rows); r = np.zeros(max_rows); C = np.zeros(max_rows)
        rdyn = np.zeros(6 * self.scene.n_bodies)
        m = lib().oracle_rows(*self._common(), _d(state), _d(ubar), float(h), _d(u), _d(lam), max_rows,
                              meta.ctypes.data_as(_ip), _d(Jan), _d(Jd), _d(r), _d(C), _d(rdyn))
        if m < 0:
            raise RuntimeError("oracle_rows failed")
        return dict(meta=meta[:4 * m].reshape(m, 4), J=Jan[:12 * m].reshape(m, 12), Jdual=Jd[:12 * m].reshape(m, 12),
                    r=r[:m], C=C[:m], rdyn=rdyn)


def fb(a, b, eps=1e-8):
    out = np.zeros(3)
    lib().oracle_fb(float(a), float(b), float(eps), _d(out))
    return out


def friction_W(vt1, vt2, ln, lf1, lf2, mu, eps=1e-8, hw=1.0):
    return lib().oracle_friction_W(vt1, vt2, ln, lf1, lf2, mu, eps, hw)


def rotate(q, v):
    q = np.ascontiguousarray(q, dtype=np.float64); v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros(3)
    lib().oracle_rotate(_d(q), _d(v), _d(out))
    return out


def lu_solve(A, b):
    A = np.ascontiguousarray(A, dtype=np.float64); b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    rc = lib().oracle_lu_solve(len(b), _d(A), _d(b), _d(x))
    if rc != 0:
        raise np.linalg.LinAlgError("singular")
    return x


def pcr(A, b, kind=0, blocks=None, iters=16, rtol=0.0):
    """Preconditioned conjugate residual on a dense SPD system (kind 0 Jacobi, 1 block
    Jacobi over the row blocks `blocks`): (x, iterations, converged)."""
    A = np.ascontiguousarray(A, dtype=np.float64); b = np.ascontiguousarray(b, dtype=np.float64)
    n = len(b)
    blk = np.ascontiguousarray(np.zeros(n) if blocks is None else blocks, dtype=np.int32)
    x = np.zeros(n); conv = np.zeros(1, dtype=np.int32)
    k = lib().oracle_pcr(n, _d(A), _d(b), int(kind), blk.ctypes.data_as(_ip), int(iters), float(rtol), _d(x),
                         conv.ctypes.data_as(_ip))
    return x, int(k), bool(conv[0])


def rollout(orc: Oracle, state, controls, h, T):
    """T forward steps; controls [T, n_servo]."""
    states = [np.asarray(state, dtype=np.float64)]
    infos = []
    for t in range(T):
        r = orc.step(states[-1], controls[t] if orc.n_servo else np.zeros(1), h)
        states.append(r["state"]); infos.append(r)
    return states, infos
