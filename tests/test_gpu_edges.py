"""Edge cases of the CUDA path (against the oracle where a value is defined).

* one world; worlds in free flight (no active contact: only joints and servos);
* arrays with a leading dimension larger than the world count (padding untouched);
* a world with non-finite input: status bit 2 set, the other worlds unaffected and
  bit-identical to a launch without it;
* world lists with out-of-range and empty entries: skipped on the device;
* the largest contact load of the robot-over-box scene: 24 active contacts in an
  infeasible sunk pose (index sets and the non-convergence flag) and the heaviest
  feasible pose, front wheels against the obstacle face (values).
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
    from paper_2609_08800_gb300 import ostrich
    ostrich.lib()
    return ostrich


def _step(M, sc, cfg, st, ub, dtype="f64", ld=0, threads=None):
    W = st.shape[1]
    tdt = torch.float64 if dtype == "f64" else torch.float32
    ctx = M.Context(sc, cfg, W, dtype=dtype, ld=ld, tape_slots=0, threads=threads)
    L = ctx.ld
    s_in = torch.zeros(ctx.n_state, L, dtype=tdt, device="cuda")
    s_in[:, :W] = torch.tensor(st, dtype=tdt)
    u_in = torch.zeros(max(sc.n_servos, 1), L, dtype=tdt, device="cuda")
    if sc.n_servos:
        u_in[:, :W] = torch.tensor(ub, dtype=tdt)
    out = torch.full_like(s_in, 7.0)
    status = torch.zeros(L, dtype=torch.int32, device="cuda")
    ids = torch.zeros(max(ctx.n_slots, 1), L, dtype=torch.int32, device="cuda")
    ctx.ostrich_step(s_in, u_in, H, out, None, ids, status)
    torch.cuda.synchronize()
    ctx.close()
    return out.cpu(), status.cpu(), ids.cpu(), s_in.cpu()


def test_single_world_matches_oracle(M):
    sc = S.box_drop_scene()
    cfg = S.SolverConfig(budget=50, tol=1e-10, kappa=0.0)
    st = S.box_drop_state(sc, 0.7)
    out, status, ids, _ = _step(M, sc, cfg, st, np.zeros((0, 1)))
    ro = O.Oracle(sc, cfg).step(st[:, 0], np.zeros(1), H)
    assert int(status[0]) == 0 and ro["status"] == 0
    assert np.array_equal(ids[:, 0].numpy(), ro["ids"])
    np.testing.assert_allclose(out[:13, 0].numpy(), ro["state"][:13], rtol=0, atol=1e-9)


def test_free_flight_matches_oracle(M):
    """Robots high above the ground: no contact is active; the joints and servos alone."""
    sc = S.robot_box_scene()
    W = 8
    st = S.robot_box_states(sc, W, seed=12, phases=False)
    st[2:35:7] += 1.5
    ub = S.random_controls(sc.n_servos, W, seed=12, low=-4, high=4)
    cfg = S.SolverConfig(budget=40, tol=1e-10)
    out, status, ids, _ = _step(M, sc, cfg, st, ub)
    orc = O.Oracle(sc, cfg)
    nb = sc.n_bodies
    for w in range(W):
        ro = orc.step(st[:, w], ub[:, w], H)
        assert (ids[:, w].numpy() < 0).all() and (ro["ids"] < 0).all()
        assert int(status[w]) == 0
        np.testing.assert_allclose(out[:13 * nb, w].numpy(), ro["state"][:13 * nb], rtol=0, atol=1e-8)


def test_leading_dimension_padding_untouched(M):
    sc = S.robot_box_scene()
    W, L = 37, 64
    st = S.robot_box_states(sc, W, seed=13)
    ub = S.random_controls(sc.n_servos, W, seed=13, low=-3, high=3)
    cfg = S.SolverConfig()
    out, status, _, _ = _step(M, sc, cfg, st, ub, dtype="f32", ld=L)
    ref, status_ref, _, _ = _step(M, sc, cfg, st, ub, dtype="f32")
    assert torch.equal(out[:, :W], ref[:, :W])
    assert (out[:, W:] == 7.0).all()                 # padding columns keep what was there


def test_non_finite_world_is_flagged_and_isolated(M):
    sc = S.robot_box_scene()
    W = 16
    st = S.robot_box_states(sc, W, seed=14)
    ub = S.random_controls(sc.n_servos, W, seed=14, low=-3, high=3)
    bad = st.copy()
    bad[7 * sc.n_bodies + 2, 5] = np.nan             # a NaN velocity in world 5
    cfg = S.SolverConfig()
    out, status, _, _ = _step(M, sc, cfg, bad, ub, dtype="f32")
    ref, status_ref, _, _ = _step(M, sc, cfg, st, ub, dtype="f32")
    assert int(status[5]) & 3 == 3                   # not converged, non-finite
    assert not torch.isfinite(out[7 * sc.n_bodies:13 * sc.n_bodies, 5]).any()
    others = [w for w in range(W) if w != 5]
    assert torch.equal(out[:, others], ref[:, others])
    assert torch.equal(status[others], status_ref[others])
    # the NaN warm start ends the step at once: no Newton iterations, a NaN iterate
    ctx = M.Context(sc, cfg, W, dtype="f32", tape_slots=0)
    it = torch.zeros(W, dtype=torch.int32, device="cuda")
    s_in = torch.tensor(bad, dtype=torch.float32, device="cuda")
    ctx.ostrich_step(s_in, torch.tensor(ub, dtype=torch.float32, device="cuda"), H, torch.empty_like(s_in),
                     None, None, None, it)
    torch.cuda.synchronize()
    assert int(it[5]) & 0xFFFF == 0
    ctx.close()


def test_list_skips_out_of_range_entries(M):
    sc = S.robot_box_scene()
    W = 40
    ctx = M.Context(sc, S.SolverConfig(), W, dtype="f32", tape_slots=1)
    st = torch.tensor(S.robot_box_states(sc, W, seed=15), dtype=torch.float32, device="cuda")
    ub = torch.tensor(S.random_controls(sc.n_servos, W, seed=15, low=-3, high=3), dtype=torch.float32, device="cuda")
    full = torch.empty_like(st)
    ctx.ostrich_step(st, ub, H, full)
    lst = torch.tensor([3, -1, 39, 40, 1000, 7], dtype=torch.int32, device="cuda")
    slots = torch.tensor([0, 0, 5, 0, 0, -1], dtype=torch.int32, device="cuda")   # slot 5 is out of range
    out = st.clone()
    ctx.ostrich_step_list(out, ub, H, out, lst, slots)
    empty = torch.zeros(0, dtype=torch.int32, device="cuda")
    ctx.ostrich_step_list(out, ub, H, out, empty, empty)                       # nothing to do
    torch.cuda.synchronize()
    for w in (3, 39, 7):
        assert torch.equal(out[:, w], full[:, w])
    untouched = [w for w in range(W) if w not in (3, 39, 7)]
    assert torch.equal(out[:, untouched], st[:, untouched])
    ctx.close()


def test_heaviest_contact_load_matches_oracle(M):
    """Contact generation at full load: rear wheels sunk into the obstacle's near edge
    activate 24 of the 32 slots (every rim against ground, face, top and edge).  The
    pose is infeasible (the wheel centres are inside the obstacle), so neither side
    converges: the index sets must agree bit for bit and both must report it."""
    sc = S.robot_box_scene()
    W = 12
    st = np.zeros((sc.n_state, W))
    x0 = sc.env.box[0]
    rng = np.random.default_rng(16)
    for w in range(W):
        S._place_robot(st, sc, w, x0 + 0.26 + rng.uniform(0.0, 0.04), 0.0, 0.14 + rng.uniform(-0.002, 0.002),
                       rng.uniform(-0.03, 0.03))
    ub = S.random_controls(sc.n_servos, W, seed=16, low=-2, high=2)
    cfg = S.SolverConfig(budget=40, tol=1e-9)
    out, status, ids, _ = _step(M, sc, cfg, st, ub)
    orc = O.Oracle(sc, cfg)
    for w in range(W):
        ro = orc.step(st[:, w], ub[:, w], H)
        assert np.array_equal(ids[:, w].numpy(), ro["ids"])
        assert int((ro["ids"] >= 0).sum()) == 24
        assert (int(status[w]) & 1) == (ro["status"] & 1) == 1


def test_front_wheels_at_the_face_match_oracle(M):
    """The heaviest feasible load of the scene: front wheels against the obstacle face
    and on the ground, rear wheels on the ground (12 active contacts)."""
    sc = S.robot_box_scene()
    W = 12
    st = np.zeros((sc.n_state, W))
    rng = np.random.default_rng(17)
    for w in range(W):
        S._place_robot(st, sc, w, 0.58 + rng.uniform(0.0, 0.01), 0.0, S.ROBOT_CHASSIS_Z + rng.uniform(-0.003, 0.003), 0.0)
    ub = S.random_controls(sc.n_servos, W, seed=17, low=-1, high=1)
    cfg = S.SolverConfig(budget=60, tol=1e-9)
    out, status, ids, _ = _step(M, sc, cfg, st, ub)
    orc = O.Oracle(sc, cfg)
    nb = sc.n_bodies
    n_cmp = 0
    for w in range(W):
        ro = orc.step(st[:, w], ub[:, w], H)
        assert np.array_equal(ids[:, w].numpy(), ro["ids"])
        assert int((ro["ids"] >= 0).sum()) == 12
        if ro["status"] == 0 and int(status[w]) == 0:
            n_cmp += 1
            np.testing.assert_allclose(out[:13 * nb, w].numpy(), ro["state"][:13 * nb], rtol=0, atol=1e-7)
    assert n_cmp >= W - 1
