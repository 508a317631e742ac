"""Timestep sweep on the CUDA path (Sec. III-B: friction acts at the step's own h).

A box launched at v0 = 2 m/s along the plane decelerates by exactly mu g h per step until
it sticks: v_{n+1} = max(0, v_n - mu g h), x_{n+1} = x_n + h v_{n+1} (backward Euler), at
every h in 0.0125 ... 0.2 s; the stopping distance tends to the continuous v0^2/(2 mu g)
within v0 h.  The exact-mode adjoint swept back through the same rollout gives
dx_N/dv0 = h times the number of steps in which the box still slides, the derivative of
that closed form (the paper's frozen-W adjoint does not).  FP64 to 5e-8 (the oracle's
own bound on this sweep); FP32 to 5e-5.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2609_08800_gb300 import scenes as S  # noqa: E402

HS = (0.0125, 0.025, 0.05, 0.1, 0.2)


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2609_08800_gb300 import ostrich as mod
    mod.lib()
    return mod


@pytest.mark.parametrize("dtype,tol", [("f64", 5e-8), ("f32", 5e-5)])
@pytest.mark.parametrize("h", HS)
def test_sliding_box_sweep_matches_closed_form(M, dtype, tol, h):
    sc = S.box_drop_scene()
    tdt = torch.float64 if dtype == "f64" else torch.float32
    cfg = S.SolverConfig(budget=60, k_min=4, tol=1e-10 if dtype == "f64" else 1e-6, kappa=0.0)
    v0, mu, g = 2.0, 0.8, 9.81
    n = int(round(0.4 / h))
    ctx = M.Context(sc, cfg, 1, dtype=dtype, tape_slots=n)
    ctx.set_adjoint_mode(M.ADJ_EXACT)
    u = torch.zeros(1, 1, dtype=tdt, device="cuda")
    s = torch.tensor(S.box_drop_state(sc, 0.0, gap=0.0), dtype=tdt, device="cuda")
    for _ in range(3):
        s = ctx.step(s, u, h)["state"]                       # settle at rest on the plane
    s = s.clone()
    s[7] = v0
    x0 = float(s[0])
    v, x, sliding = v0, x0, 0
    for t in range(n):
        r = ctx.step(s, u, h, tape_slot=t)
        assert not (int(r["status"][0]) & 2)
        s = r["state"]
        v = max(0.0, v - mu * g * h)
        x = x + h * v
        sliding += v > 0.0
        assert float(s[7]) == pytest.approx(v, abs=tol), f"step {t}"
        assert float(s[0]) == pytest.approx(x, abs=tol), f"step {t}"
    assert v == 0.0
    assert abs((x - x0) - v0 ** 2 / (2 * mu * g)) <= v0 * h
    grad = torch.zeros(sc.n_state, 1, dtype=tdt, device="cuda")
    grad[0] = 1.0
    for t in reversed(range(n)):
        grad, _ = ctx.adjoint(t, grad, h)
    torch.cuda.synchronize()
    assert float(grad[7]) == pytest.approx(h * sliding, abs=1e-6 if dtype == "f64" else 1e-4)
    ctx.close()
