"""The allocation-free step + adjoint against the context path.

`ostrich_step_adjoint_noalloc` serves callers that cannot call cudaMalloc (a
real-time control loop that must not allocate once running, a plugin whose host
framework owns the device memory): its tape lives in a fixed library array instead of
a context's workspace.  It runs the same kernels with the same launch shape (64
threads per world, one CTA per world) as a context set to 64 threads and schedule 0,
so its results must equal that path's bit for bit, on two calls in a row (the second
call reuses the array the first one left behind).  This file is collected last so that
a run stopping at the first failure has run every other test first.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2609_08800_gb300 import scenes as S  # noqa: E402


def test_noalloc_matches_context_path_twice():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2609_08800_gb300 import ostrich as M
    sc = S.robot_box_scene()
    cfg = S.SolverConfig(tol=1e-4)
    W, h = 96, 0.1
    nb = sc.n_bodies
    st = torch.tensor(S.robot_box_states(sc, W, seed=21), dtype=torch.float32, device="cuda")
    ub = torch.tensor(S.random_controls(sc.n_servos, W, seed=21, low=-3, high=3), dtype=torch.float32, device="cuda")
    g = torch.tensor(np.random.default_rng(22).normal(size=st.shape), dtype=torch.float32, device="cuda")
    g[13 * nb:] = 0
    ctx = M.Context(sc, cfg, W, dtype="f32", tape_slots=1, threads=64)
    ctx.set_schedule(0)
    s_in = st
    for call in range(2):
        ref = ctx.step(s_in, ub, h, tape_slot=0)
        ref_ds, ref_du = ctx.adjoint(0, g, h)
        out = torch.empty_like(s_in)
        ds = torch.empty_like(s_in)
        du = torch.empty(sc.n_servos, W, dtype=torch.float32, device="cuda")
        M.ostrich_step_adjoint_noalloc(sc, cfg, W, s_in, ub, h, out, g, ds, du)
        torch.cuda.synchronize()
        assert torch.equal(out, ref["state"]), f"call {call}: state"
        assert torch.equal(ds, ref_ds), f"call {call}: dL/dstate"
        assert torch.equal(du, ref_du), f"call {call}: dL/dcontrols"
        s_in = out.clone()          # second call starts where the first ended
    ctx.close()


def test_noalloc_rejects_sizes_beyond_the_array():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2609_08800_gb300 import ostrich as M
    sc = S.robot_box_scene()
    W = 2048                        # 2048 x 10432 B > 16 MiB (at most 1608 robot worlds)
    st = torch.zeros(sc.n_state, W, dtype=torch.float32, device="cuda")
    ub = torch.zeros(sc.n_servos, W, dtype=torch.float32, device="cuda")
    with pytest.raises(RuntimeError, match="status 1"):
        M.ostrich_step_adjoint_noalloc(sc, S.SolverConfig(), W, st, ub, 0.1, torch.empty_like(st), st,
                                       torch.empty_like(st))
