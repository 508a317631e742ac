"""Pins of the oracle's preconditioned conjugate residual (PCR) solver (Sec. III-C solves
Eq. (12) with it) and of the Newton step and adjoint that use it.

The iteration is pinned against what the mathematics fixes, not against the oracle:
* the k-th iterate minimises |L^T (b - A x)|_2 (P = L L^T) over the Krylov space
  K_k(P A, P b): brute force by least squares over an explicit Krylov basis, for the
  Jacobi and the block-Jacobi preconditioner;
* finite termination: n iterations on an n x n system give its solution;
* the exact preconditioner (one block holding the whole matrix, P = A^-1) converges in
  one iteration; the stopping rule stops at the first iterate with |r| <= rtol |b|.
The Newton step's fixed point does not depend on the linear solver, so a step with PCR
inner solves must reach the closed forms the direct solve reaches: the sliding box's
discrete trajectory at every h, and the paper adjoint's finite-difference agreement on
a sticking box.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2609_08800_gb300 import scenes as S


def _spd(n, seed, cond=1e3):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    ev = np.geomspace(1.0, cond, n)
    return Q @ np.diag(ev) @ Q.T, rng.normal(size=n)


def _precond(A, kind, blocks):
    n = len(A)
    if kind == S.PC_JACOBI:
        return np.diag(1.0 / np.diag(A))
    P = np.zeros_like(A)
    for b in np.unique(blocks):
        idx = np.flatnonzero(blocks == b)
        P[np.ix_(idx, idx)] = np.linalg.inv(A[np.ix_(idx, idx)])
    return P


@pytest.mark.parametrize("kind", [S.PC_JACOBI, S.PC_BLOCK])
@pytest.mark.parametrize("seed", [0, 1])
def test_pcr_iterates_minimise_the_preconditioned_residual(kind, seed):
    n = 9
    A, b = _spd(n, seed)
    blocks = np.array([0, 0, 0, 1, 1, 2, 2, 2, 2])
    P = _precond(A, kind, blocks)
    L = np.linalg.cholesky(P)
    for k in range(1, 6):
        x, its, _ = O.pcr(A, b, kind, blocks, iters=k)
        assert its == k
        # Krylov basis of K_k(P A, P b), orthonormalised for conditioning
        V = [P @ b]
        for _ in range(k - 1):
            V.append(P @ (A @ V[-1]))
        V, _ = np.linalg.qr(np.array(V).T)
        c, *_ = np.linalg.lstsq(L.T @ A @ V, L.T @ b, rcond=None)
        xbest = V @ c
        assert np.abs(x - xbest).max() <= 1e-9 * np.abs(xbest).max()


@pytest.mark.parametrize("kind", [S.PC_JACOBI, S.PC_BLOCK])
def test_pcr_finite_termination(kind):
    n = 8
    A, b = _spd(n, 3, cond=1e2)
    blocks = np.repeat(np.arange(4), 2)
    x, its, _ = O.pcr(A, b, kind, blocks, iters=n)
    ref = np.linalg.solve(A, b)
    assert np.abs(x - ref).max() <= 1e-9 * np.abs(ref).max()


def test_pcr_exact_preconditioner_and_stopping_rule():
    n = 10
    A, b = _spd(n, 4, cond=1e4)
    x, its, conv = O.pcr(A, b, S.PC_BLOCK, np.zeros(n), iters=50, rtol=1e-12)
    assert its == 1 and conv
    assert np.abs(A @ x - b).max() <= 1e-10 * np.abs(b).max()
    # Jacobi: stops at the first iterate whose residual meets the tolerance
    for rtol in (1e-2, 1e-6):
        x, its, conv = O.pcr(A, b, S.PC_JACOBI, None, iters=200, rtol=rtol)
        assert conv
        assert np.linalg.norm(b - A @ x) <= 1.001 * rtol * np.linalg.norm(b)
        xp, _, _ = O.pcr(A, b, S.PC_JACOBI, None, iters=its - 1)
        assert np.linalg.norm(b - A @ xp) > rtol * np.linalg.norm(b) * 0.999


def _pcr_cfg(precond, **kw):
    return S.SolverConfig(linear_solver=S.LIN_PCR, precond=precond, **kw)


@pytest.mark.parametrize("precond", [S.PC_JACOBI, S.PC_BLOCK])
def test_pcr_newton_reaches_the_sliding_box_closed_form(precond):
    """The discrete sliding trajectory v_{n+1} = max(0, v_n - mu g h), x_{n+1} = x_n + h v_{n+1}
    with PCR inner solves (16 iterations per Newton step, as Sec. IV-B)."""
    sc = S.box_drop_scene()
    orc = O.Oracle(sc, _pcr_cfg(precond, budget=60, k_min=4, tol=1e-10, kappa=0.0))
    v0, mu, g = 2.0, 0.8, 9.81
    for h in (0.025, 0.1):
        s = S.box_drop_state(sc, 0.0, gap=0.0)[:, 0]
        for _ in range(3):
            s = orc.step(s, np.zeros(1), h)["state"]
        x0 = s[0]
        s[7] = v0
        v, x = v0, x0
        for _ in range(int(round(0.4 / h))):
            r = orc.step(s, np.zeros(1), h)
            s = r["state"]
            v = max(0.0, v - mu * g * h)
            x = x + h * v
            assert s[7] == pytest.approx(v, abs=5e-8)
            assert s[0] == pytest.approx(x, abs=5e-8)


@pytest.mark.parametrize("precond", [S.PC_JACOBI, S.PC_BLOCK])
def test_pcr_paper_adjoint_matches_fd_on_sticking_box(precond):
    """Sec. III-D's single PCR solve in the adjoint: on a sticking box the paper's adjoint
    agrees with central differences of the step to 0.4 %, as with the direct solve."""
    sc = S.box_drop_scene()
    orc = O.Oracle(sc, _pcr_cfg(precond, budget=60, k_min=4, tol=1e-12, kappa=1e-4))
    s = S.box_drop_state(sc, 0.0, gap=0.0)[:, 0]
    for _ in range(3):
        s = orc.step(s, np.zeros(1), 0.1)["state"]
    s[7], s[8] = 0.05, 0.02
    g = np.random.default_rng(9).normal(size=sc.n_state)
    g[13:] = 0.0
    ad = orc.step_adjoint(s, np.zeros(1), 0.1, g, mode=O.ADJ_PAPER)["dstate"][:13]
    fd = np.zeros(13)
    for i in range(13):
        e = 1e-6
        sp, sm = s.copy(), s.copy()
        sp[i] += e; sm[i] -= e
        fd[i] = g @ (orc.step(sp, np.zeros(1), 0.1)["state"] - orc.step(sm, np.zeros(1), 0.1)["state"]) / (2 * e)
    assert np.abs(ad - fd).max() <= 4e-3 * np.abs(fd).max()


@pytest.mark.parametrize("precond", [S.PC_JACOBI, S.PC_BLOCK])
def test_pcr_robot_step_keeps_joint_closure(precond):
    """Eq. (3) with E = 0 at a converged robot step taken with PCR inner solves: anchors
    coincide and axles stay perpendicular to the parent's two perpendicular axes."""
    sc = S.robot_box_scene()
    st = S.robot_box_states(sc, 4, seed=0)
    orc = O.Oracle(sc, _pcr_cfg(precond, budget=80, k_min=4, tol=1e-9, kappa=1e-4, pcr_iters=48))
    nconv = 0
    for w in range(4):
        r = orc.step(st[:, w], np.full(4, 2.0), 0.1)
        if r["status"] != 0:
            continue
        nconv += 1
        out = r["state"]
        for jt in sc.joints:
            pp, Rp = out[7 * jt.parent:7 * jt.parent + 3], S._quat_to_matrix(out[7 * jt.parent + 3:7 * jt.parent + 7])
            pc, Rc = out[7 * jt.child:7 * jt.child + 3], S._quat_to_matrix(out[7 * jt.child + 3:7 * jt.child + 7])
            gap = (pp + Rp @ np.array(jt.anchor_parent)) - (pc + Rc @ np.array(jt.anchor_child))
            assert np.abs(gap).max() < 1e-8
            aw = Rc @ np.array(jt.axis_child)
            for b in jt.perp_parent:
                assert abs((Rp @ np.array(b)) @ aw) < 1e-8
    assert nconv >= 2
