"""CUDA graph per horizon chunk and the launch-shape autotuner.

A captured chunk (10 taped steps + 10 adjoints) replayed from static buffers must
give bit-identical states and gradients to the same launches issued one by one,
on two replays with different inputs.  The autotuner's choice must be one of its
candidates, be persisted, and be found again by lookup.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2609_08800_gb300 import scenes as S  # noqa: E402

H, T = 0.1, 10


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2609_08800_gb300 import ostrich
    ostrich.lib()
    return ostrich


def _inputs(sc, W, seed):
    st = torch.tensor(S.robot_box_states(sc, W, seed=seed), dtype=torch.float32, device="cuda")
    ctl = torch.tensor(np.stack([S.random_controls(sc.n_servos, W, seed=seed * 100 + t, low=-3, high=3)
                                 for t in range(T)]), dtype=torch.float32, device="cuda")
    g = torch.tensor(np.random.default_rng(seed).normal(size=st.shape), dtype=torch.float32, device="cuda")
    g[13 * sc.n_bodies:] = 0
    return st, ctl, g


def _eager(ctx, s0, ctl, gT):
    states = [s0.clone()]
    for t in range(T):
        out = torch.empty_like(s0)
        ctx.ostrich_step(states[t], ctl[t], H, out, tape_slot=t)
        states.append(out)
    g = gT.clone()
    grads, dctl = [None] * (T + 1), [None] * T
    grads[T] = g
    for t in reversed(range(T)):
        ds = torch.empty_like(g)
        du = torch.empty(ctx.n_servo, ctx.ld, dtype=g.dtype, device="cuda")
        ctx.ostrich_adjoint(t, grads[t + 1], H, ds, du)
        grads[t], dctl[t] = ds, du
    torch.cuda.synchronize()
    return torch.stack(states), torch.stack(grads), torch.stack(dctl)


def test_chunk_graph_replay_is_bit_identical(M):
    from paper_2609_08800_gb300.graphs import ChunkGraph
    sc = S.robot_box_scene()
    W = 300
    ctx = M.Context(sc, S.SolverConfig(tol=1e-4), W, dtype="f32", tape_slots=T)
    graph = ChunkGraph(ctx, T, H)
    for seed in (3, 4):
        s0, ctl, gT = _inputs(sc, W, seed)
        ref = _eager(ctx, s0, ctl, gT)
        states, grads, dctl = graph.replay(s0, ctl, gT)
        torch.cuda.synchronize()
        assert torch.equal(states, ref[0]), "states differ between graph replay and eager launches"
        assert torch.equal(grads, ref[1]), "state gradients differ"
        assert torch.equal(dctl[:, :sc.n_servos], ref[2]), "control gradients differ"
    ctx.close()


def test_autotuner_picks_persists_and_applies(M, tmp_path, monkeypatch):
    from paper_2609_08800_gb300 import tune
    monkeypatch.setenv("OSTRICH_AUTOTUNE_CACHE", str(tmp_path / "table.json"))
    sc = S.robot_box_scene()
    W = 1024
    ctx = M.Context(sc, S.SolverConfig(tol=1e-4), W, dtype="f32", tape_slots=1)
    s0, ctl, _ = _inputs(sc, W, 7)
    best, times = tune.tune(ctx, s0, ctl[0], H, reps=2)
    assert best in tune.CANDIDATES and set(times) == set(tune.CANDIDATES)
    assert times[best] == min(times.values())
    assert tune.lookup(ctx) == best
    ctx.set_threads(64 if best != 64 else 32)
    assert tune.apply(ctx) == best
    ctx.close()


def test_persistent_schedule_is_bit_identical(M):
    """The persistent, heaviest-first schedule changes only when a world runs: three
    consecutive steps (the later ones ordered by the earlier iteration counts) and their
    adjoints equal the one-CTA-per-world launch bit for bit."""
    sc = S.robot_box_scene()
    W = 1024
    outs = []
    for schedule in (0, 1):
        ctx = M.Context(sc, S.SolverConfig(tol=1e-4), W, dtype="f32", tape_slots=3)
        ctx.set_schedule(schedule)
        s0, ctl, gT = _inputs(sc, W, 9)
        states = [s0]
        iters = []
        for t in range(3):
            out = torch.empty_like(s0)
            it = torch.zeros(W, dtype=torch.int32, device="cuda")
            ctx.ostrich_step(states[t], ctl[t], H, out, iters=it, tape_slot=t)
            states.append(out)
            iters.append(it)
        g = gT.clone()
        for t in reversed(range(3)):
            ds = torch.empty_like(g)
            ctx.ostrich_adjoint(t, g, H, ds)
            g = ds
        torch.cuda.synchronize()
        outs.append((torch.stack(states), torch.stack(iters), g))
        ctx.close()
    assert torch.equal(outs[0][0], outs[1][0])
    assert torch.equal(outs[0][1], outs[1][1])
    assert torch.equal(outs[0][2], outs[1][2])
