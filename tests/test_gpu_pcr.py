"""The matrix-free PCR backend of the Schur solve (Sec. III-C: Eq. (12) by preconditioned
conjugate residuals; Sec. III-D: one PCR solve in the adjoint) on the CUDA path.

* Iterate parity: with PCR inner solves the Newton iterates depend on the PCR count; the
  GPU (FP64) and the oracle run the same configuration (Jacobi and block-Jacobi
  preconditioners, 16 PCR iterations per Newton step as Sec. IV-B, the best of Newton
  iterates 4-6) from identical inputs, and every world that both stop at the same
  Newton iteration with the same status is compared on its returned state (1e-7 of
  max(|x|, 1)); at least 85 % of the worlds must qualify.  Six Newton steps, not the
  paper's 16: far from convergence each inexact step amplifies rounding differences
  (a robot world with the block preconditioner reached 1.4e-5 after 16).
* Solution parity: with enough PCR iterations the step converges to the same solution
  as the direct factor; converged worlds against the oracle's dense LU step at the
  direct path's tolerances (FP64 1e-9, FP32 1e-4 / impulses 1e-3), the adjoint's PCR
  solve against the oracle's adjoint (FP64 1e-6, FP32 1e-3 at the iterate).
* The exact-mode adjoint under PCR (its GMRES preconditioner formed in the adjoint,
  nothing taped) against the oracle's exact adjoint (FP64 1e-6).
* Changing the solver discards the tape.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2609_08800_gb300 import scenes as S  # noqa: E402
from tests.test_gpu_parity import _compare, _box_states, _run_gpu  # noqa: E402

H = 0.1


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2609_08800_gb300 import ostrich as mod
    mod.lib()
    return mod


def _pcr(precond, **kw):
    return S.SolverConfig(linear_solver=S.LIN_PCR, precond=precond, **kw)


@pytest.mark.parametrize("precond", [S.PC_JACOBI, S.PC_BLOCK])
@pytest.mark.parametrize("scene", ["box", "robot"])
def test_pcr_iterates_match_oracle_fp64(M, scene, precond):
    if scene == "box":
        sc, st = _box_states(40, seed=5)
        ub = np.zeros((0, 40))
    else:
        sc = S.robot_box_scene()
        st = S.robot_box_states(sc, 40, seed=7)
        ub = S.random_controls(sc.n_servos, 40, seed=7, low=-3, high=3)
    W = st.shape[1]
    cfg = _pcr(precond, budget=6, k_min=4, tol=1e-4, pcr_iters=16)
    r = _run_gpu(M, sc, cfg, st, ub, H, "f64")
    orc = O.Oracle(sc, cfg)
    nb = sc.n_bodies
    n_cmp = 0
    for w in range(W):
        ubw = r["u_in"][:sc.n_servos, w] if sc.n_servos else np.zeros(1)
        ro = orc.step(r["s_in"][:, w], ubw, H)
        assert np.array_equal(ro["ids"], r["ids"][:, w].numpy())
        gi = int(r["iters"][w]) & 0xFFFF
        if gi != ro["iters"] or (int(r["status"][w]) & 3) != ro["status"]:
            continue
        n_cmp += 1
        x_g = r["state"][:13 * nb, w].double().numpy()
        x_o = ro["state"][:13 * nb]
        err = np.abs(x_g - x_o).max()
        assert err <= 1e-7 * max(np.abs(x_o).max(), 1.0), f"world {w}: state err {err}"
    print(f"{n_cmp}/{W} worlds compared")
    assert n_cmp >= 0.85 * W


@pytest.mark.parametrize("precond", [S.PC_JACOBI, S.PC_BLOCK])
def test_pcr_converged_robot_matches_oracle_fp64(M, precond):
    sc = S.robot_box_scene()
    W = 33
    st = S.robot_box_states(sc, W, seed=5)
    ub = S.random_controls(sc.n_servos, W, seed=5, low=-3, high=3)
    cfg = _pcr(precond, budget=40, tol=1e-9, pcr_iters=64)
    g = np.random.default_rng(6).normal(size=st.shape)
    g[13 * sc.n_bodies:] = 0
    _compare(sc, cfg, M, st, ub, H, "f64", 1e-9, 1e-7, 1e-6, 0.7, grads=g,
             oracle_cfg=S.SolverConfig(budget=40, tol=1e-9))


@pytest.mark.parametrize("precond", [S.PC_JACOBI, S.PC_BLOCK])
def test_pcr_converged_box_matches_oracle_fp32(M, precond):
    sc, st = _box_states(45, seed=2)
    cfg = _pcr(precond, budget=30, k_min=4, tol=1e-5, kappa=1e-4, pcr_iters=32)
    g = np.random.default_rng(3).normal(size=st.shape)
    g[13:] = 0
    _compare(sc, cfg, M, st, np.zeros((0, 45)), H, "f32", 1e-4, 1e-3, 1e-3, 0.9, grads=g,
             oracle_cfg=S.SolverConfig(budget=60, k_min=4, tol=1e-9, kappa=1e-4), floor=3e-4, tol_grad_exact=3e-3)


def test_pcr_converged_robot_matches_oracle_fp32(M):
    sc = S.robot_box_scene()
    W = 67
    st = S.robot_box_states(sc, W, seed=0)
    ub = S.random_controls(sc.n_servos, W, seed=0, low=-3, high=3)
    cfg = _pcr(S.PC_JACOBI, budget=40, pcr_iters=64)
    g = np.random.default_rng(10).normal(size=st.shape)
    g[13 * sc.n_bodies:] = 0
    _compare(sc, cfg, M, st, ub, H, "f32", 1e-4, 1e-3, 1e-3, 0.8, grads=g,
             oracle_cfg=S.SolverConfig(budget=60, tol=1e-8), floor=3e-4, tol_grad_exact=3e-3)


@pytest.mark.parametrize("precond", [S.PC_JACOBI, S.PC_BLOCK])
def test_pcr_terrain_matches_oracle_fp64(M, precond):
    """The mesh terrain (the large-m case PCR is meant for: 48-row wheel groups) with PCR
    inner solves and the truncated pull-back, FP64, against the oracle's direct step.
    Worlds whose Newton iteration does not reach 1e-9 within 40 iterations on either side
    (hard stick-slip steps; the direct path leaves as many) are compared on their contact
    sets only."""
    from tests.test_gpu_parity import _terrain_states
    sc = S.terrain_scene()
    W = 24
    st = _terrain_states(sc, W, 2)
    ub = S.random_controls(sc.n_servos, W, seed=2, low=-3, high=3)
    cfg = _pcr(precond, budget=40, tol=1e-9, pullback=S.PULLBACK_TRUNCATED, pcr_iters=96)
    g = np.random.default_rng(22).normal(size=st.shape)
    g[13 * sc.n_bodies:] = 0
    _compare(sc, cfg, M, st, ub, H, "f64", 1e-7, 1e-6, 1e-6, 0.6, grads=g,
             oracle_cfg=S.SolverConfig(budget=40, tol=1e-9, pullback=S.PULLBACK_TRUNCATED))


def test_pcr_exact_adjoint_matches_oracle(M):
    from tests.test_gpu_exact import _exact_vs_oracle
    sc = S.robot_box_scene()
    W = 24
    st = S.robot_box_states(sc, W, seed=2)
    ub = S.random_controls(sc.n_servos, W, seed=2, low=-3, high=3)
    _exact_vs_oracle(M, sc, _pcr(S.PC_JACOBI, budget=40, tol=1e-10, pcr_iters=64), st, ub, "f64", 1e-6, seed=3)


def test_changing_the_solver_discards_the_tape(M):
    sc, st = _box_states(4)
    ctx = M.Context(sc, S.SolverConfig(), 4, dtype="f32", tape_slots=1)
    s = torch.tensor(st, dtype=torch.float32, device="cuda")
    ctx.step(s, torch.zeros(1, 4, device="cuda"), H, tape_slot=0)
    g = torch.zeros_like(s)
    ctx.adjoint(0, g, H)
    ctx.set_linear_solver(M.LIN_PCR, M.PC_JACOBI, 16)
    with pytest.raises(RuntimeError, match="status 4"):
        ctx.adjoint(0, g, H)
    ctx.step(s, torch.zeros(1, 4, device="cuda"), H, tape_slot=0)
    ctx.adjoint(0, g, H)
    torch.cuda.synchronize()
    ctx.close()
