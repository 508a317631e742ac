"""Rollout autograd bookkeeping on the CPU, with an oracle-backed engine.

The CUDA engine is tested on the GPU (test_gpu_autograd.py); here the same
torch.autograd.Function drives the FP64 oracle so that the chain rule over the
horizon (direct state gradients, control gradients, checkpoint segments) is pinned
against central finite differences of the rollout itself.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2609_08800_gb300 import scenes as S
from paper_2609_08800_gb300.autograd import rollout


class OracleEngine:
    def __init__(self, scene, cfg, h, mode):
        self.orc = O.Oracle(scene, cfg)
        self.h, self.mode = h, mode
        self.tape = {}
        self.n_servo = scene.n_servos

    def step(self, s_in, a, slot):
        out = torch.empty_like(s_in)
        for w in range(s_in.shape[1]):
            aw = a[:, w].numpy() if self.n_servo else np.zeros(1)
            out[:, w] = torch.from_numpy(self.orc.step(s_in[:, w].numpy(), aw, self.h)["state"])
        if slot >= 0:
            self.tape[slot] = (s_in.clone(), a.clone())
        return out

    def adjoint(self, slot, g):
        s_in, a = self.tape[slot]
        ds = torch.empty_like(g)
        du = torch.zeros(self.n_servo, g.shape[1], dtype=g.dtype)
        for w in range(g.shape[1]):
            aw = a[:, w].numpy() if self.n_servo else np.zeros(1)
            r = self.orc.step_adjoint(s_in[:, w].numpy(), aw, self.h, g[:, w].numpy(), mode=self.mode)
            ds[:, w] = torch.from_numpy(r["dstate"])
            if self.n_servo:
                du[:, w] = torch.from_numpy(r["dubar"])
        return ds, du


def _setup(T=6, W=2):
    sc = S.robot_plane_scene()
    st = torch.from_numpy(S.robot_box_states(sc, W, seed=4, phases=False))
    ctl = torch.from_numpy(np.random.default_rng(5).uniform(1.0, 2.0, (T, sc.n_servos, W)))
    cfg = S.SolverConfig(budget=60, tol=1e-12)
    return sc, st, ctl, cfg


def _loss(traj, sc):
    nb = sc.n_bodies
    target = torch.tensor([3.0, 0.0], dtype=traj.dtype)
    pT = traj[-1, 0:2, :]
    # final position term plus a small per-step speed term (direct gradients of every state)
    return ((pT - target[:, None]) ** 2).sum() + 0.01 * (traj[:, 7 * nb:7 * nb + 2, :] ** 2).sum()


def test_checkpointed_gradient_is_bit_identical():
    sc, st, ctl, cfg = _setup()
    grads = []
    for seg in (None, 2, 4):
        eng = OracleEngine(sc, cfg, 0.1, O.ADJ_PAPER)
        s0 = st.clone().requires_grad_(True)
        u = ctl.clone().requires_grad_(True)
        _loss(rollout(s0, u, eng, segment=seg), sc).backward()
        grads.append((s0.grad.clone(), u.grad.clone()))
    for g in grads[1:]:
        assert torch.equal(g[0], grads[0][0]) and torch.equal(g[1], grads[0][1])


def test_rollout_gradient_matches_finite_differences():
    sc, st, ctl, cfg = _setup(T=5, W=1)
    eng = OracleEngine(sc, cfg, 0.1, O.ADJ_EXACT)
    s0 = st.clone().requires_grad_(True)
    u = ctl.clone().requires_grad_(True)
    _loss(rollout(s0, u, eng, segment=2), sc).backward()
    g_u = u.grad.clone()
    g_s = s0.grad.clone()

    def L(s, a):
        with torch.no_grad():
            return float(_loss(rollout(s, a, OracleEngine(sc, cfg, 0.1, O.ADJ_EXACT)), sc))

    eps = 1e-6
    for t in range(ctl.shape[0]):
        for j in range(ctl.shape[1]):
            up, um = ctl.clone(), ctl.clone()
            up[t, j, 0] += eps
            um[t, j, 0] -= eps
            fd = (L(st, up) - L(st, um)) / (2 * eps)
            assert g_u[t, j, 0].item() == pytest.approx(fd, rel=1e-5, abs=1e-7)
    for i in (0, 1, 2, 7, 35, 36):      # chassis x, y, z, a quaternion entry, chassis vx, vy
        sp, sm = st.clone(), st.clone()
        sp[i, 0] += eps
        sm[i, 0] -= eps
        fd = (L(sp, ctl) - L(sm, ctl)) / (2 * eps)
        assert g_s[i, 0].item() == pytest.approx(fd, rel=1e-5, abs=1e-7)
