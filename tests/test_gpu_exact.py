"""The exact IFT adjoint on the GPU (OSTRICH_ADJ_EXACT) against the oracle's exact mode.

The CUDA path solves J_F^T w = [-g; 0] with the full Jacobian of the residual in
(u+, lambda+) by GMRES preconditioned with the taped paper-mode factor; the oracle forms
the same Jacobian densely with dual numbers and solves it by LU.  Both are taken at the
CUDA path's returned iterate (oracle_adjoint_at, mode exact).  Tolerances: FP64 1e-6 and
FP32 1e-3 of the largest entry (the FP32 adjoint tolerance of the parity tests); the Krylov solve
must converge in every world.  The implicit-function theorem holds at a root of the
residual: away from one the Jacobian depends on how the rows are scaled (the oracle
differentiates its merit-weighted rows, the CUDA path the Newton rows), so the worlds
compared are those whose returned iterate is a solution -- converged in FP64, an exact
residual (the oracle's residual function at the CUDA iterate) of at most 3e-4 m/s in
FP32, the FP32 floor the other parity tests use.

Pins of the exact mode beyond the oracle: the 20-step box drop (v0 from seed 0) gives dx_T/dv0 = h
through a 20-step rollout (the paper's frozen-W adjoint gives 0.69 h), and dL/dmu of a
sliding box is -g h.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2609_08800_gb300 import scenes as S  # noqa: E402

H = 0.1


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2609_08800_gb300 import ostrich as mod
    mod.lib()
    return mod


def _skid_states(sc, W, seed, steps=2):
    """Robots on the plane driven to skid (left and right wheels opposite), so that their
    rim contacts slide, then one more random step."""
    rng = np.random.default_rng(seed)
    st = S.robot_box_states(sc, W, seed=seed, phases=False)
    orc = O.Oracle(sc, S.SolverConfig(budget=60, tol=1e-10))
    ub = np.stack([np.array([1, -1, 1, -1]) * rng.uniform(1.0, 4.0) + rng.normal(scale=0.5, size=4)
                   for _ in range(W)], axis=1)
    for w in range(W):
        s = st[:, w]
        for _ in range(steps):
            s = orc.step(s, ub[:, w], H)["state"]
        st[:, w] = s
    return st, ub


def _exact_vs_oracle(M, sc, cfg, st, ub, dtype, tol, with_mu=True, seed=0, floor=3e-4):
    from tests.test_gpu_parity import _exact_residual
    W = st.shape[1]
    nb = sc.n_bodies
    tdt = torch.float64 if dtype == "f64" else torch.float32
    ctx = M.Context(sc, cfg, W, dtype=dtype, tape_slots=1)
    kry = torch.zeros(W, dtype=torch.int32, device="cuda")
    ctx.set_adjoint_mode(M.ADJ_EXACT, kry)
    s_in = torch.tensor(st, dtype=tdt, device="cuda")
    u_in = torch.tensor(ub if ub.size else np.zeros((1, W)), dtype=tdt, device="cuda")
    r = ctx.step(s_in, u_in, H, tape_slot=0)
    g = np.random.default_rng(seed + 40).normal(size=st.shape)
    g[13 * nb:] = 0
    gt = torch.tensor(g, dtype=tdt, device="cuda")
    ds, du, dkp, dm, di, dmu = ctx.adjoint_params(0, gt, H, with_mu=True)
    torch.cuda.synchronize()
    out = r["state"].double().cpu().numpy()
    s64, u64, g64 = s_in.double().cpu().numpy(), u_in.double().cpu().numpy(), gt.double().cpu().numpy()
    ds, du, dmu = ds.double().cpu().numpy(), du.double().cpu().numpy(), dmu.double().cpu().numpy()
    kry = kry.cpu().numpy()
    status = r["status"].cpu().numpy()
    ctx.close()
    orc = O.Oracle(sc, cfg)
    worst = 0.0
    n_cmp = 0
    for w in range(W):
        assert not (int(status[w]) & 2), f"world {w}: non-finite"
        assert not (int(kry[w]) >> 16), f"world {w}: GMRES did not converge ({int(kry[w]) & 0xFFFF} iterations)"
        ubw = u64[:sc.n_servos, w] if sc.n_servos else np.zeros(1)
        if dtype == "f64" and int(status[w]) & 1:
            continue                                     # not a solution: not compared
        if dtype == "f32" and _exact_residual(orc, sc, s64[:, w], ubw, H, out[:, w]) > floor:
            continue
        n_cmp += 1
        at = orc.adjoint_at(s64[:, w], ubw, H, out[7 * nb:13 * nb, w], out[13 * nb:, w], g64[:, w], mode=O.ADJ_EXACT)
        d = at["dstate"][:13 * nb]
        sc_ = np.abs(d).max()
        e = np.abs(ds[:13 * nb, w] - d).max()
        worst = max(worst, e / sc_)
        assert e <= tol * sc_, f"world {w}: dL/dstate {e} of {sc_}"
        if sc.n_servos:
            e_u = np.abs(du[:, w] - at["dubar"]).max()
            assert e_u <= tol * max(sc_, np.abs(at["dubar"]).max()), f"world {w}: dL/dcontrols {e_u}"
        if with_mu:
            assert abs(dmu[w] - at["dmu"]) <= tol * max(abs(at["dmu"]), sc_ * 1e-2), f"world {w}: dL/dmu {dmu[w]} vs {at['dmu']}"
    print(f"{dtype}: {n_cmp}/{W} converged worlds compared, worst relative error {worst:.2e}, Krylov iterations "
          f"{np.median(kry & 0xFFFF)} (median), {(kry & 0xFFFF).max()} (max)")
    assert n_cmp >= 0.75 * W


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-6), ("f32", 1e-3)])
def test_exact_adjoint_skidding_robot(M, dtype, tol):
    sc = S.robot_plane_scene()
    st, ub = _skid_states(sc, 24, seed=3)
    cfg = S.SolverConfig(budget=40, tol=1e-10 if dtype == "f64" else 1e-4)
    _exact_vs_oracle(M, sc, cfg, st, ub, dtype, tol)


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-6), ("f32", 1e-3)])
def test_exact_adjoint_robot_over_box(M, dtype, tol):
    sc = S.robot_box_scene()
    W = 32
    st = S.robot_box_states(sc, W, seed=9)
    ub = S.random_controls(sc.n_servos, W, seed=9, low=-3, high=3)
    cfg = S.SolverConfig(budget=40, tol=1e-10 if dtype == "f64" else 1e-4)
    _exact_vs_oracle(M, sc, cfg, st, ub, dtype, tol, seed=1)


def test_exact_adjoint_box_fp64(M):
    sc = S.box_drop_scene()
    W = 16
    rng = np.random.default_rng(5)
    st = np.concatenate([S.box_drop_state(sc, float(v)) for v in rng.uniform(0.0, 1.0, W)], axis=1)
    cfg = S.SolverConfig(budget=50, k_min=4, tol=1e-10, kappa=0.0)
    _exact_vs_oracle(M, sc, cfg, st, np.zeros((0, W)), "f64", 1e-6, seed=2)


def test_box_drop_rollout_gradient_is_h(M):
    """The box-drop rollout: box 0.4 x 0.4 x 0.2 m, 10 kg, dropped from 0.05 m with v0 from seed 0,
    FP64, T = 20, Newton tol 1e-10; loss x_T.  The exact adjoint swept back through the
    rollout gives dx_T/dv0 = h (the box slides h max(0, v0 - 0.3848) and stops in step
    2); the paper's frozen-W adjoint gives the landing step's sliding ratio times h."""
    sc, st = S.box_drop_inputs(0)
    cfg = S.SolverConfig(budget=50, k_min=4, tol=1e-10, kappa=0.0)
    T = 20
    grads = {}
    for mode in (M.ADJ_PAPER, M.ADJ_EXACT):
        ctx = M.Context(sc, cfg, 1, dtype="f64", tape_slots=T)
        ctx.set_adjoint_mode(mode)
        s = torch.tensor(st, dtype=torch.float64, device="cuda")
        u = torch.zeros(1, 1, dtype=torch.float64, device="cuda")
        for t in range(T):
            s = ctx.step(s, u, H, tape_slot=t)["state"]
        g = torch.zeros(sc.n_state, 1, dtype=torch.float64, device="cuda")
        g[0] = 1.0
        for t in reversed(range(T)):
            g, _ = ctx.adjoint(t, g, H)
        grads[mode] = float(g[7, 0])
        ctx.close()
    print(f"box drop dx_T/dv0: exact {grads[M.ADJ_EXACT]:.9f}, paper {grads[M.ADJ_PAPER]:.6f}")
    assert grads[M.ADJ_EXACT] == pytest.approx(H, abs=1e-6)
    assert grads[M.ADJ_PAPER] == pytest.approx(0.0686173, abs=1e-5)


def test_mu_gradient_sliding_box(M):
    """dL/dmu = -g h for a box sliding at rest load (loss v_x+), in both precisions; 0 in
    the paper's mode."""
    sc = S.box_drop_scene()
    orc = O.Oracle(sc, S.SolverConfig(budget=60, k_min=4, tol=1e-12, kappa=0.0))
    s = S.box_drop_state(sc, 0.0, gap=0.0)[:, 0]
    for _ in range(4):
        s = orc.step(s, np.zeros(1), H)["state"]
    s[7] = 2.0
    for dtype, tol in (("f64", 1e-9), ("f32", 1e-4)):
        tdt = torch.float64 if dtype == "f64" else torch.float32
        cfg = S.SolverConfig(budget=50, k_min=4, tol=1e-10 if dtype == "f64" else 1e-5, kappa=0.0)
        for mode, expect in ((M.ADJ_EXACT, -9.81 * H), (M.ADJ_PAPER, 0.0)):
            ctx = M.Context(sc, cfg, 1, dtype=dtype, tape_slots=1)
            ctx.set_adjoint_mode(mode)
            r = ctx.step(torch.tensor(s[:, None], dtype=tdt, device="cuda"), torch.zeros(1, 1, dtype=tdt, device="cuda"),
                         H, tape_slot=0)
            g = torch.zeros(sc.n_state, 1, dtype=tdt, device="cuda")
            g[7] = 1.0
            out = ctx.adjoint_params(0, g, H, with_mu=True)
            torch.cuda.synchronize()
            assert abs(float(out[-1][0]) - expect) <= tol * 10, f"{dtype} mode {mode}: {float(out[-1][0])} vs {expect}"
            ctx.close()
