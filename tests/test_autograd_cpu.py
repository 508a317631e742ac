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
from paper_2609_08800_gb300.autograd import rollout, scene_theta


class OracleEngine:
    def __init__(self, scene, cfg, h, mode):
        self.orc = O.Oracle(scene, cfg)
        self.scene = scene
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

    def adjoint_params(self, slot, g):
        s_in, a = self.tape[slot]
        ds = torch.empty_like(g)
        du = torch.zeros(self.n_servo, g.shape[1], dtype=g.dtype)
        dth = []
        for w in range(g.shape[1]):
            aw = a[:, w].numpy() if self.n_servo else np.zeros(1)
            r = self.orc.step_adjoint(s_in[:, w].numpy(), aw, self.h, g[:, w].numpy(), mode=self.mode)
            ds[:, w] = torch.from_numpy(r["dstate"])
            if self.n_servo:
                du[:, w] = torch.from_numpy(r["dubar"])
            dth.append(np.concatenate([r["dkp"], r["dmass"], r["dinertia"].ravel()]))
        return ds, du, torch.from_numpy(np.stack(dth, 1))

    def theta(self):
        return scene_theta(self.scene)


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


def _with_theta(sc, p, value):
    """A copy of the scene with parameter p (the scene_theta order) set to value."""
    import copy
    sc = copy.deepcopy(sc)
    servos = [j for j in sc.joints if j.kp > 0]
    nb = sc.n_bodies
    if p < len(servos):
        servos[p].kp = value
    elif p < len(servos) + nb:
        sc.bodies[p - len(servos)].mass = value
    else:
        q = p - len(servos) - nb
        b, k = divmod(q, 3)
        inertia = list(sc.bodies[b].inertia)
        inertia[k] = value
        sc.bodies[b].inertia = tuple(inertia)
    return sc


def test_theta_gradient_matches_finite_differences():
    """dL/dtheta of a 4-step rollout (servo gains, masses, principal moments) in the
    exact-IFT mode against central differences of the rollout itself; the FB scaling
    what, which also holds the mass properties, is left out of the gradient (a
    step-start constant), which the tolerance covers."""
    sc, st, ctl, cfg = _setup(T=4, W=1)
    # gentle wheel targets: the contacts stick, where the left-out what dependence is
    # small (with the 1-2 rad/s targets of the other tests the wheels slip and it
    # reaches a few per cent of the mass gradient)
    ctl = ctl * 0.05
    theta = scene_theta(sc).requires_grad_(True)
    eng = OracleEngine(sc, cfg, 0.1, O.ADJ_EXACT)
    _loss(rollout(st.clone(), ctl.clone(), eng, theta=theta), sc).backward()
    base = scene_theta(sc).numpy()
    fd = np.zeros_like(base)
    for p in range(base.size):
        d = 1e-4 * base[p]
        lp = float(_loss(rollout(st.clone(), ctl.clone(), OracleEngine(_with_theta(sc, p, base[p] + d), cfg, 0.1, O.ADJ_EXACT)), sc))
        lm = float(_loss(rollout(st.clone(), ctl.clone(), OracleEngine(_with_theta(sc, p, base[p] - d), cfg, 0.1, O.ADJ_EXACT)), sc))
        fd[p] = (lp - lm) / (2 * d)
    gt = theta.grad.numpy()
    ns, nb = sc.n_servos, sc.n_bodies
    for sl in (slice(0, ns), slice(ns, ns + nb), slice(ns + nb, None)):
        scale = np.abs(fd[sl]).max()
        assert scale > 0
        assert np.abs(gt[sl] - fd[sl]).max() <= 2e-4 * scale, (sl, gt[sl], fd[sl])


def test_theta_gradient_checkpointed_is_bit_identical():
    sc, st, ctl, cfg = _setup(T=4, W=2)
    grads = []
    for seg in (None, 2):
        theta = scene_theta(sc).requires_grad_(True)
        eng = OracleEngine(sc, cfg, 0.1, O.ADJ_PAPER)
        _loss(rollout(st.clone(), ctl.clone(), eng, segment=seg, theta=theta), sc).backward()
        grads.append(theta.grad.clone())
    assert torch.equal(grads[0], grads[1])


def test_theta_must_be_the_scene_parameters():
    sc, st, ctl, cfg = _setup(T=2, W=1)
    theta = scene_theta(sc) * 1.01
    with pytest.raises(ValueError):
        rollout(st.clone(), ctl.clone(), OracleEngine(sc, cfg, 0.1, O.ADJ_PAPER), theta=theta)


class CountingEngine(OracleEngine):
    """The oracle engine with the recording count the rollout's tape reuse reads, and a
    count of the steps it takes."""

    def __init__(self, *a):
        super().__init__(*a)
        self.tape_epoch = 0
        self.steps = 0

    def step(self, s_in, a, slot):
        self.steps += 1
        if slot >= 0:
            self.tape_epoch += 1
        return super().step(s_in, a, slot)


def test_checkpointed_backward_reuses_the_last_segment():
    """With checkpoints every 4 of 6 steps, the forward records steps 4-5 and the
    backward recomputes only steps 0-3 (10 steps in all), with the plain gradient."""
    sc, st, ctl, cfg = _setup()
    ref = OracleEngine(sc, cfg, 0.1, O.ADJ_PAPER)
    s0 = st.clone().requires_grad_(True)
    u = ctl.clone().requires_grad_(True)
    _loss(rollout(s0, u, ref), sc).backward()
    eng = CountingEngine(sc, cfg, 0.1, O.ADJ_PAPER)
    s1 = st.clone().requires_grad_(True)
    u1 = ctl.clone().requires_grad_(True)
    _loss(rollout(s1, u1, eng, segment=4), sc).backward()
    assert eng.steps == 6 + 4
    assert torch.equal(s1.grad, s0.grad) and torch.equal(u1.grad, u.grad)


def test_checkpointed_backward_recomputes_an_overwritten_last_segment():
    """Two rollouts on one engine, backward in either order: the second forward's
    recording overwrites the first one's last segment, so the first one's backward
    recomputes it; both gradients equal their plain ones."""
    sc, st, ctl, cfg = _setup()
    st2 = st.clone()
    st2[35] += 0.3                       # chassis vx
    plain = []
    for s in (st, st2):
        s0 = s.clone().requires_grad_(True)
        u = ctl.clone().requires_grad_(True)
        _loss(rollout(s0, u, OracleEngine(sc, cfg, 0.1, O.ADJ_PAPER)), sc).backward()
        plain.append((s0.grad, u.grad))
    eng = CountingEngine(sc, cfg, 0.1, O.ADJ_PAPER)
    ins = [(s.clone().requires_grad_(True), ctl.clone().requires_grad_(True)) for s in (st, st2)]
    losses = [_loss(rollout(s0, u, eng, segment=4), sc) for s0, u in ins]
    assert eng.steps == 12
    losses[0].backward()                 # its last segment was overwritten: recomputed
    assert eng.steps == 12 + 6
    losses[1].backward()                 # the first backward recorded since: recomputed
    assert eng.steps == 12 + 12
    for (s0, u), (gs, gu) in zip(ins, plain):
        assert torch.equal(s0.grad, gs) and torch.equal(u.grad, gu)
