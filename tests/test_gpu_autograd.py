"""Rollout autograd with the CUDA engine: checkpointed gradients (states, controls and
the scene parameters) are bit-identical to the plain ones, and the FP64 build's rollout
gradients match the oracle engine's."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2609_08800_gb300 import scenes as S  # noqa: E402


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _loss(traj, nb):
    pT = traj[-1, 0:2, :]
    return ((pT - torch.tensor([3.0, 0.0], dtype=traj.dtype, device=traj.device)[:, None]) ** 2).sum() \
        + 0.01 * (traj[:, 7 * nb:7 * nb + 2, :] ** 2).sum()


def test_checkpointing_is_bit_identical_fp32():
    _need_gpu()
    from paper_2609_08800_gb300.autograd import CudaEngine, rollout
    sc = S.robot_box_scene()
    W, T, h = 512, 20, 0.1
    st = torch.tensor(S.robot_box_states(sc, W, seed=3), dtype=torch.float32, device="cuda")
    ctl = torch.tensor(np.random.default_rng(3).uniform(-3, 3, (T, sc.n_servos, W)), dtype=torch.float32,
                       device="cuda")
    cfg = S.SolverConfig(tol=1e-4)
    out = []
    for seg, slots in ((None, T), (10, 10), (7, 7)):
        eng = CudaEngine(sc, cfg, W, h, slots)
        s0 = st.clone().requires_grad_(True)
        u = ctl.clone().requires_grad_(True)
        theta = eng.theta().requires_grad_(True)
        traj = rollout(s0, u, eng, segment=seg, theta=theta)
        _loss(traj, sc.n_bodies).backward()
        torch.cuda.synchronize()
        out.append((traj.detach().clone(), s0.grad.clone(), u.grad.clone(), theta.grad.clone()))
        eng.close()
    for o in out[1:]:
        assert torch.equal(o[0], out[0][0])
        assert torch.equal(o[1], out[0][1]) and torch.equal(o[2], out[0][2])
        assert torch.equal(o[3], out[0][3])
    assert torch.isfinite(out[0][1]).all() and torch.isfinite(out[0][3]).all()


def test_fp64_rollout_gradient_matches_oracle_engine():
    _need_gpu()
    from oracle import oracle as O
    from paper_2609_08800_gb300.autograd import CudaEngine, rollout
    from tests.test_autograd_cpu import OracleEngine
    sc = S.robot_plane_scene()
    W, T, h = 3, 5, 0.1
    st = S.robot_box_states(sc, W, seed=6, phases=False)
    ctl = np.random.default_rng(6).uniform(1.0, 2.5, (T, sc.n_servos, W))
    cfg = S.SolverConfig(budget=60, tol=1e-11)
    eng = CudaEngine(sc, cfg, W, h, T, dtype="f64")
    s0 = torch.tensor(st, dtype=torch.float64, device="cuda", requires_grad=True)
    u = torch.tensor(ctl, dtype=torch.float64, device="cuda", requires_grad=True)
    theta = eng.theta().requires_grad_(True)
    _loss(rollout(s0, u, eng, theta=theta), sc.n_bodies).backward()
    g_s, g_u, g_th = s0.grad.cpu(), u.grad.cpu(), theta.grad.clone()
    eng.close()
    oe = OracleEngine(sc, cfg, h, O.ADJ_PAPER)
    s0c = torch.tensor(st, dtype=torch.float64, requires_grad=True)
    uc = torch.tensor(ctl, dtype=torch.float64, requires_grad=True)
    thc = oe.theta().requires_grad_(True)
    _loss(rollout(s0c, uc, oe, theta=thc), sc.n_bodies).backward()
    scale = max(s0c.grad.abs().max().item(), uc.grad.abs().max().item())
    assert (g_s - s0c.grad).abs().max().item() <= 1e-6 * scale
    assert (g_u - uc.grad).abs().max().item() <= 1e-6 * scale
    ns, nb = sc.n_servos, sc.n_bodies
    for sl in (slice(0, ns), slice(ns, ns + nb), slice(ns + nb, None)):
        sc_th = thc.grad[sl].abs().max().item()
        assert (g_th[sl] - thc.grad[sl]).abs().max().item() <= 1e-6 * sc_th
