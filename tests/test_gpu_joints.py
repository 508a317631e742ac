"""Prismatic joints and position-target servos (Eqs. (3), (8)) on the CUDA path.

* The servo rig (a base box on the plane carrying a cart on a prismatic joint and a wheel
  on a revolute joint, both servoed) in both servo modes, and the cart-pole (prismatic
  cart with a velocity servo, unactuated pole): one step from identical inputs against
  the oracle -- contact sets bit-exact, states and impulses, the paper-mode adjoint at
  the CUDA iterate (FP64 1e-6, FP32 1e-3) -- as the other parity tests.
* The exact adjoint on the cart-pole against the oracle's exact mode (FP64 1e-6).
* The one-step closed form of the prismatic position servo (base held by friction):
  lambda = -(v- + (s- - target)/h) / (h/m + 1/(kd + h kp)).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2609_08800_gb300 import scenes as S  # noqa: E402
from tests.test_gpu_parity import _compare  # noqa: E402

H = 0.1


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2609_08800_gb300 import ostrich as mod
    mod.lib()
    return mod


def _rig_states(sc, W, seed):
    rng = np.random.default_rng(seed)
    st = np.concatenate([S.rig_state(sc, rng.uniform(-0.2, 0.2), rng.uniform(-1.0, 1.0)) for _ in range(W)], axis=1)
    nb = sc.n_bodies
    st[7 * nb + 6] = rng.uniform(-0.5, 0.5, W)          # cart v_x
    st[7 * nb + 12 + 4] = rng.uniform(-3.0, 3.0, W)     # wheel w_y
    st[7 * nb + 2] = rng.uniform(-0.1, 0.0, W)          # base settling
    return st


def _cartpole_states(sc, W, seed):
    rng = np.random.default_rng(seed)
    return np.concatenate([S.cartpole_state(sc, rng.uniform(-0.6, 0.6), rng.uniform(-0.5, 0.5),
                                            rng.uniform(-2.0, 2.0)) for _ in range(W)], axis=1)


@pytest.mark.parametrize("mode", [S.SERVO_POSITION, S.SERVO_VELOCITY])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_rig_matches_oracle(M, mode, dtype):
    sc = S.rig_scene(mode=mode)
    W = 24
    st = _rig_states(sc, W, seed=3 + mode)
    rng = np.random.default_rng(7)
    ub = np.stack([rng.uniform(-0.2, 0.2, W), rng.uniform(-1.0, 1.0, W)]) if mode == S.SERVO_POSITION \
        else np.stack([rng.uniform(-0.5, 0.5, W), rng.uniform(-3.0, 3.0, W)])
    g = np.random.default_rng(8).normal(size=st.shape)
    g[13 * sc.n_bodies:] = 0
    if dtype == "f64":
        # a wheel at up to 3 rad/s pulled to a position target in one step can need more
        # than 40 Newton iterations at tol 1e-10: budget 80
        _compare(sc, S.SolverConfig(budget=80, tol=1e-10), M, st, ub, H, "f64", 1e-7, 1e-6, 1e-6, 0.9, grads=g)
    else:
        _compare(sc, S.SolverConfig(budget=40, tol=1e-5), M, st, ub, H, "f32", 1e-4, 1e-3, 1e-3, 0.9, grads=g,
                 oracle_cfg=S.SolverConfig(budget=60, tol=1e-9), floor=3e-4, tol_grad_exact=3e-3)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_cartpole_matches_oracle(M, dtype):
    sc = S.cartpole_scene()
    W = 24
    st = _cartpole_states(sc, W, seed=5)
    ub = np.random.default_rng(9).uniform(-1.0, 1.0, (1, W))
    g = np.random.default_rng(10).normal(size=st.shape)
    g[13 * sc.n_bodies:] = 0
    if dtype == "f64":
        _compare(sc, S.SolverConfig(budget=40, tol=1e-10), M, st, ub, 0.05, "f64", 1e-7, 1e-6, 1e-6, 0.9, grads=g)
    else:
        _compare(sc, S.SolverConfig(budget=40, tol=1e-5), M, st, ub, 0.05, "f32", 1e-4, 1e-3, 1e-3, 0.9, grads=g,
                 oracle_cfg=S.SolverConfig(budget=60, tol=1e-9), floor=3e-4, tol_grad_exact=3e-3)


def test_cartpole_exact_adjoint_matches_oracle(M):
    from tests.test_gpu_exact import _exact_vs_oracle
    sc = S.cartpole_scene()
    W = 16
    st = _cartpole_states(sc, W, seed=11)
    ub = np.random.default_rng(12).uniform(-1.0, 1.0, (1, W))
    _exact_vs_oracle(M, sc, S.SolverConfig(budget=40, tol=1e-10), st, ub, "f64", 1e-6, seed=4)


def test_cartpole_rollout_exact_gradient_matches_oracle(M):
    """A 30-step cart-pole rollout (h = 0.05) swept back with the exact adjoint on the GPU
    (FP64) against the same sweep on the oracle: dL/ds0 and dL/dcontrols to 1e-6."""
    sc = S.cartpole_scene()
    h, T = 0.05, 30
    cfg = S.SolverConfig(budget=60, k_min=4, tol=1e-12, kappa=1e-4)
    s0 = S.cartpole_state(sc, tilt=0.15, cart_v=0.1, pole_w=0.3)
    ctl = 0.8 * np.sin(np.arange(T) * 0.3)
    gT = np.random.default_rng(0).normal(size=sc.n_state)
    gT[13 * sc.n_bodies:] = 0.0
    ctx = M.Context(sc, cfg, 1, dtype="f64", tape_slots=T)
    ctx.set_adjoint_mode(M.ADJ_EXACT)
    s = torch.tensor(s0, dtype=torch.float64, device="cuda")
    states = [s]
    for t in range(T):
        states.append(ctx.step(states[-1], torch.full((1, 1), ctl[t], dtype=torch.float64, device="cuda"), h,
                               tape_slot=t)["state"])
    g = torch.tensor(gT[:, None], device="cuda")
    dctl = np.zeros(T)
    for t in reversed(range(T)):
        g, du = ctx.adjoint(t, g, h)
        dctl[t] = float(du[0, 0])
    torch.cuda.synchronize()
    orc = O.Oracle(sc, cfg)
    ost = [s0[:, 0]]
    for t in range(T):
        ost.append(orc.step(ost[-1], ctl[t:t + 1], h)["state"])
    go = gT.copy()
    dco = np.zeros(T)
    for t in reversed(range(T)):
        r = orc.step_adjoint(ost[t], ctl[t:t + 1], h, go, mode=O.ADJ_EXACT)
        go, dco[t] = r["dstate"], r["dubar"][0]
    nb13 = 13 * sc.n_bodies
    gg = g[:nb13, 0].cpu().numpy()
    assert np.abs(gg - go[:nb13]).max() <= 1e-6 * np.abs(go[:nb13]).max()
    assert np.abs(dctl - dco).max() <= 1e-6 * np.abs(dco).max()
    ctx.close()


def test_prismatic_position_servo_closed_form(M):
    sc = S.rig_scene(mode=S.SERVO_POSITION)
    cfg = S.SolverConfig(budget=60, k_min=4, tol=1e-12, kappa=0.0)
    orc = O.Oracle(sc, cfg)
    s = S.rig_state(sc)[:, 0]
    for _ in range(3):
        s = orc.step(s, np.zeros(2), H)["state"]
    nb = sc.n_bodies
    s[7] += 0.05
    s[7 * nb + 6] = 0.2
    ctx = M.Context(sc, cfg, 1, dtype="f64", tape_slots=1)
    r = ctx.step(torch.tensor(s[:, None], device="cuda"), torch.tensor([[-0.1], [0.0]], dtype=torch.float64,
                                                                        device="cuda"), H)
    out = r["state"][:, 0].cpu().numpy()
    ctx.close()
    m, kp, kd = 2.0, 50.0, 2.0
    lam = -(0.2 + (s[7] - s[0] + 0.1) / H) / (H / m + 1.0 / (kd + H * kp))
    assert out[sc.lam_index + 10] == pytest.approx(lam, rel=1e-9)
    assert out[7 * nb + 6] == pytest.approx(0.2 + H * lam / m, rel=1e-9)
