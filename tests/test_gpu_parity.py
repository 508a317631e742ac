"""CUDA path against the FP64 oracle, one step at a time from identical inputs.

Tolerances: contact index sets bit-exact; FP64 path 1e-9 relative; FP32 path
positions/velocities within 1e-4 of max(|x|, 1) per world, impulses within 1e-3 of
the step's largest impulse, adjoint gradients within 1e-3 of the largest oracle
gradient entry of the world, where the oracle's adjoint is taken at the CUDA path's
returned iterate (the paper takes A and the VJPs at the returned iterate); against
the gradient at the oracle's exact solution the FP32 path is held to 3e-3, since the
FP32 iterate itself stalls ~1e-4 m/s from the solution and moves the gradient by up
to ~1.2e-3 (measured).

The oracle runs to a tight tolerance (the exact step).  A world is compared on
values when the oracle converged and the CUDA path's returned iterate is a solution:
its exact residual, evaluated by the oracle's residual function at that iterate, is
below the FP32 floor of the scene (3e-4 m/s; FP32 states rounded from the exact
solution already sit near 1e-5, and the FP32 Newton iteration stalls around 1e-4).
Every world is compared on its contact index set.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2609_08800_gb300 import scenes as S  # noqa: E402
from tests.test_oracle_pins import hinged_boxes_scene, resting_closed_form  # noqa: E402


@pytest.fixture(scope="module")
def ostrich():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2609_08800_gb300 import ostrich as M
    M.lib()
    return M


def _run_gpu(M, scene, cfg, states, controls, h, dtype, grads=None, threads=None):
    W = states.shape[1]
    tdt = torch.float64 if dtype == "f64" else torch.float32
    ctx = M.Context(scene, cfg, W, dtype=dtype, tape_slots=1, threads=threads)
    s_in = torch.tensor(states, dtype=tdt, device="cuda")
    u_in = torch.tensor(controls if controls.size else np.zeros((1, W)), dtype=tdt, device="cuda")
    r = ctx.step(s_in, u_in, h, tape_slot=0)
    out = {k: v.cpu() for k, v in r.items()}
    if grads is not None:
        g = torch.tensor(grads, dtype=tdt, device="cuda")
        ds, du = ctx.adjoint(0, g, h)
        out["dstate"], out["dubar"] = ds.cpu(), du.cpu()
    torch.cuda.synchronize()
    out["s_in"] = s_in.double().cpu().numpy()
    out["u_in"] = u_in.double().cpu().numpy()
    ctx.close()
    return out


def _exact_residual(orc, scene, s_in, ub, h, out_state):
    """sqrt(merit) of the oracle's residual function at a given iterate (u, lambda)."""
    nb = scene.n_bodies
    u = out_state[7 * nb:13 * nb]
    lam = out_state[13 * nb:]
    rows = orc.rows(s_in, ub, h, u, lam)
    rd = rows["rdyn"].reshape(nb, 6)
    tot = float((rows["r"] ** 2).sum())
    for b in range(nb):
        R = S._quat_to_matrix(s_in[7 * b + 3:7 * b + 7])
        Iwi = R @ np.diag(1.0 / np.array(scene.bodies[b].inertia)) @ R.T
        mr = np.r_[rd[b, :3] / scene.bodies[b].mass, Iwi @ rd[b, 3:]]
        tot += float(mr @ mr)
    return np.sqrt(tot)


def _compare(scene, cfg, g, states, controls, h, dtype, tol_state, tol_imp, tol_grad, min_frac, grads=None,
             oracle_cfg=None, floor=None, threads=None, tol_grad_exact=None):
    orc = O.Oracle(scene, oracle_cfg or cfg)
    orc_cfg_run = O.Oracle(scene, cfg)
    W = states.shape[1]
    r = _run_gpu(g, scene, cfg, states, controls, h, dtype, grads, threads)
    nb = scene.n_bodies
    n_cmp = 0
    for w in range(W):
        ub = r["u_in"][:scene.n_servos, w] if scene.n_servos else np.zeros(1)
        if grads is None:
            ro = orc.step(r["s_in"][:, w], ub, h)
        else:
            ro = orc.step_adjoint(r["s_in"][:, w], ub, h, grads[:, w].astype(np.float64) if dtype == "f64"
                                  else grads[:, w].astype(np.float32).astype(np.float64))
        ids = r["ids"][:, w].numpy()
        assert np.array_equal(ro["ids"], ids), f"world {w}: contact index set"
        gs = int(r["status"][w]) & 3
        if ro["status"] != 0 or (gs & 2):
            continue
        if floor is None:
            if gs != 0:
                continue
        else:
            res = _exact_residual(orc_cfg_run, scene, r["s_in"][:, w], ub, h, r["state"][:, w].double().numpy())
            if res > floor:
                continue
        n_cmp += 1
        x_g = r["state"][:13 * nb, w].double().numpy()
        x_o = ro["state"][:13 * nb]
        err = np.abs(x_g - x_o).max()
        assert err <= tol_state * max(np.abs(x_o).max(), 1.0), f"world {w}: state err {err}"
        imp_o = ro["impulses"]
        imp_g = r["impulses"][:, w].double().numpy()
        e_imp = np.abs(imp_g - imp_o).max()
        assert e_imp <= tol_imp * max(np.abs(imp_o).max(), 1e-12), f"world {w}: impulse err {e_imp} of {np.abs(imp_o).max()}"
        if grads is not None:
            dg = r["dstate"][:13 * nb, w].double().numpy()
            du_g = r["dubar"][:, w].double().numpy() if scene.n_servos else None
            # (i) the adjoint at the returned iterate (the paper's A and VJPs at the
            # iterate the forward step returns), evaluated by the oracle at the CUDA
            # path's own iterate: the implementation of Eqs. (16)-(19), tol_grad
            gw = grads[:, w].astype(np.float64) if dtype == "f64" else grads[:, w].astype(np.float32).astype(np.float64)
            at = orc_cfg_run.adjoint_at(r["s_in"][:, w], ub, h, r["state"][7 * nb:13 * nb, w].double().numpy(),
                                        r["state"][13 * nb:, w].double().numpy(), gw)
            da = at["dstate"][:13 * nb]
            e_a = np.abs(dg - da).max()
            assert e_a <= tol_grad * np.abs(da).max(), f"world {w}: grad err at the iterate {e_a} of {np.abs(da).max()}"
            if scene.n_servos:
                e_ua = np.abs(du_g - at["dubar"]).max()
                assert e_ua <= tol_grad * max(np.abs(da).max(), np.abs(at["dubar"]).max()), f"world {w}: control grad err {e_ua}"
            # (ii) against the gradient at the oracle's exact solution: the FP32 iterate's
            # own distance from the solution adds up to ~1.2e-3 (measured), tol_grad_exact
            te = tol_grad if tol_grad_exact is None else tol_grad_exact
            do = ro["dstate"][:13 * nb]
            e_g = np.abs(dg - do).max()
            assert e_g <= te * np.abs(do).max(), f"world {w}: grad err {e_g} of {np.abs(do).max()}"
            if scene.n_servos:
                e_u = np.abs(du_g - ro["dubar"]).max()
                assert e_u <= te * max(np.abs(do).max(), np.abs(ro["dubar"]).max()), f"world {w}: control grad err {e_u}"
    print(f"compared {n_cmp}/{W} worlds on values")
    assert n_cmp >= min_frac * W, f"only {n_cmp}/{W} worlds compared"
    return n_cmp


def _box_states(n, seed=0):
    sc = S.box_drop_scene()
    rng = np.random.default_rng(seed)
    st = np.zeros((sc.n_state, n))
    for w in range(n):
        st[:, w] = S.box_drop_state(sc, rng.uniform(0, 1))[:, 0]
        st[2, w] += rng.uniform(-0.06, 0.02)
        st[8, w] = rng.uniform(-0.3, 0.3)
        ang = rng.uniform(-0.2, 0.2)
        st[3:7, w] = (np.cos(ang / 2), 0.0, 0.0, np.sin(ang / 2))
    return sc, st


def test_box_fp64_matches_oracle(ostrich):
    sc, st = _box_states(37)
    cfg = S.SolverConfig(budget=50, k_min=4, tol=1e-10, kappa=0.0)
    g = np.random.default_rng(1).normal(size=st.shape)
    g[13:] = 0
    _compare(sc, cfg, ostrich, st, np.zeros((0, 37)), 0.1, "f64", 1e-9, 1e-7, 1e-6, 0.8, grads=g)


def test_box_fp32_matches_oracle(ostrich):
    sc, st = _box_states(45, seed=2)
    cfg = S.SolverConfig(budget=30, k_min=4, tol=1e-5, kappa=1e-4)
    g = np.random.default_rng(3).normal(size=st.shape)
    g[13:] = 0
    _compare(sc, cfg, ostrich, st, np.zeros((0, 45)), 0.1, "f32", 1e-4, 1e-3, 1e-3, 0.9, grads=g,
             oracle_cfg=S.SolverConfig(budget=60, k_min=4, tol=1e-9, kappa=1e-4), floor=3e-4, tol_grad_exact=3e-3)


@pytest.mark.parametrize("seed", [0, 1])
def test_robot_box_fp32_matches_oracle(ostrich, seed):
    sc = S.robot_box_scene()
    W = 67
    st = S.robot_box_states(sc, W, seed=seed)
    ub = S.random_controls(sc.n_servos, W, seed=seed, low=-3, high=3)
    # The IFT adjoint assumes r = 0: the FP32 comparison gives the Newton loop a budget
    # of 40 so the returned iterate reaches the FP32 floor (with the paper's 16 a few
    # worlds stop short of it and their gradients differ by up to ~1e-3).
    cfg = S.SolverConfig(budget=40)
    g = np.random.default_rng(seed + 10).normal(size=st.shape)
    g[13 * sc.n_bodies:] = 0
    _compare(sc, cfg, ostrich, st, ub, 0.1, "f32", 1e-4, 1e-3, 1e-3, 0.85, grads=g,
             oracle_cfg=S.SolverConfig(budget=60, tol=1e-8), floor=3e-4, tol_grad_exact=3e-3)


@pytest.mark.parametrize("threads", [64, 32, 128])
def test_robot_box_fp64_matches_oracle(ostrich, threads):
    """The FP64 build of the same kernels against the oracle on the robot: the
    implementation itself, free of FP32 effects; at every launch shape the
    autotuner may pick."""
    sc = S.robot_box_scene()
    W = 33
    st = S.robot_box_states(sc, W, seed=5)
    ub = S.random_controls(sc.n_servos, W, seed=5, low=-3, high=3)
    cfg = S.SolverConfig(budget=40, tol=1e-9)
    g = np.random.default_rng(15).normal(size=st.shape)
    g[13 * sc.n_bodies:] = 0
    _compare(sc, cfg, ostrich, st, ub, 0.1, "f64", 1e-7, 1e-6, 1e-6, 0.8, grads=g, threads=threads)


def _terrain_states(sc, W, seed):
    """Robots over the Gaussian terrain, lowered 0-3 cm into contact range, with small
    random velocities."""
    st = S.terrain_states(sc, W, seed=seed)
    rng = np.random.default_rng(seed)
    nb = sc.n_bodies
    drop = rng.uniform(0.0, 0.03, W)
    for b in range(nb):
        st[7 * b + 2] -= drop
    st[7 * nb:7 * nb + 3] += rng.normal(scale=0.1, size=(3, W))
    return st


@pytest.mark.parametrize("seed", [0, 1])
def test_terrain_fp32_matches_oracle(ostrich, seed):
    """The mesh-terrain scene: FP32, truncated pull-back adjoint."""
    sc = S.terrain_scene()
    W = 48
    st = _terrain_states(sc, W, seed)
    ub = S.random_controls(sc.n_servos, W, seed=seed, low=-3, high=3)
    # FP32 terrain steps stall at the FP32 floor (~1e-4 m/s) above the 1e-5 tolerance, so
    # every world runs the whole budget and returns its best iterate
    cfg = S.SolverConfig(budget=40, pullback=S.PULLBACK_TRUNCATED)
    g = np.random.default_rng(seed + 20).normal(size=st.shape)
    g[13 * sc.n_bodies:] = 0
    _compare(sc, cfg, ostrich, st, ub, 0.1, "f32", 1e-4, 1e-3, 1e-3, 0.8, grads=g,
             oracle_cfg=S.SolverConfig(budget=60, tol=1e-8, pullback=S.PULLBACK_TRUNCATED), floor=3e-4,
             tol_grad_exact=3e-3)


def test_robot_box_fp64_truncated_pullback_matches_oracle(ostrich):
    """The truncated pull-back (contact geometry held fixed within the step) of the
    FP64 kernels against the oracle's."""
    sc = S.robot_box_scene()
    W = 33
    st = S.robot_box_states(sc, W, seed=8)
    ub = S.random_controls(sc.n_servos, W, seed=8, low=-3, high=3)
    cfg = S.SolverConfig(budget=40, tol=1e-9, pullback=S.PULLBACK_TRUNCATED)
    g = np.random.default_rng(18).normal(size=st.shape)
    g[13 * sc.n_bodies:] = 0
    _compare(sc, cfg, ostrich, st, ub, 0.1, "f64", 1e-7, 1e-6, 1e-6, 0.8, grads=g)


def test_terrain_fp64_matches_oracle(ostrich):
    """The FP64 build on the mesh terrain: contact search, rows, factor and the
    truncated pull-back against the oracle, free of FP32 effects."""
    sc = S.terrain_scene()
    W = 24
    st = _terrain_states(sc, W, 2)
    ub = S.random_controls(sc.n_servos, W, seed=2, low=-3, high=3)
    cfg = S.SolverConfig(budget=40, tol=1e-9, pullback=S.PULLBACK_TRUNCATED)
    g = np.random.default_rng(22).normal(size=st.shape)
    g[13 * sc.n_bodies:] = 0
    _compare(sc, cfg, ostrich, st, ub, 0.1, "f64", 1e-7, 1e-6, 1e-6, 0.7, grads=g)


def _hinged_states(sc, W, seed):
    rng = np.random.default_rng(seed)
    nb = sc.n_bodies
    st = np.zeros((sc.n_state, W))
    for w in range(W):
        z, vx = 0.1 + rng.uniform(-0.01, 0.03), rng.uniform(-0.3, 0.3)
        for b, x in enumerate((-0.21, 0.21)):
            st[7 * b:7 * b + 7, w] = (x, 0.0, z, 1.0, 0.0, 0.0, 0.0)
            st[7 * nb + 6 * b, w] = vx
            st[7 * nb + 6 * b + 2, w] = rng.uniform(-0.2, 0.1)
    return st


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_hinged_boxes_matches_oracle(ostrich, dtype):
    sc = hinged_boxes_scene()
    W = 40
    st = _hinged_states(sc, W, 4)
    ub = S.random_controls(sc.n_servos, W, seed=4, low=-2, high=2)
    g = np.random.default_rng(24).normal(size=st.shape)
    g[13 * sc.n_bodies:] = 0
    if dtype == "f64":
        cfg = S.SolverConfig(budget=60, tol=1e-9)
        _compare(sc, cfg, ostrich, st, ub, 0.1, "f64", 1e-7, 1e-6, 1e-6, 0.6, grads=g)
    else:
        cfg = S.SolverConfig(budget=40)
        _compare(sc, cfg, ostrich, st, ub, 0.1, "f32", 1e-4, 1e-3, 1e-3, 0.6, grads=g,
                 oracle_cfg=S.SolverConfig(budget=60, tol=1e-8), floor=3e-4, tol_grad_exact=3e-3)


def test_tilted_wheel_closed_form_fp64(ostrich):
    """The CUDA path's heightmap contacts, friction rows and rotation-rate map against the
    closed form of a free wheel released on a planar slope (one step from rest: rolling
    under sticking friction with the contact compliance kappa; the closed form and its
    derivation sit beside the oracle's pin of the same case).  The contact frames come
    from the oracle's FP32 contact generation, whose index set the step matches bit for
    bit; FP64 build, tangential and angular velocities to 1e-8, the sinking velocity and
    the normal force to 1e-7, friction magnitudes to 1e-6."""
    from tests.test_oracle_terrain import _tilted_wheel, tilted_wheel_closed_form
    sc, st = _tilted_wheel()
    h, kappa = 0.1, 1e-4
    cfg = S.SolverConfig(budget=60, tol=1e-12, kappa=kappa)
    r = _run_gpu(ostrich, sc, cfg, st, np.zeros((0, 1)), h, "f64")
    act, ids, nd = O.Oracle(sc, cfg).contacts(st[:, 0], h)
    assert np.array_equal(r["ids"][:, 0].numpy(), ids)
    assert int(r["status"][0]) == 0
    sl = np.nonzero(act)[0]
    t, nu, v_t, v_n, w, N, F = tilted_wheel_closed_form(sc, st, h, kappa, nd, sl)
    out = r["state"][:, 0].numpy()
    u = out[7:13]
    assert abs(u[0:3] @ t - v_t) <= 1e-8 * abs(v_t)
    assert abs(u[0:3] @ nu - v_n) <= 1e-7 * abs(v_n)
    assert abs(u[4] - w) <= 1e-8 * abs(w)
    lam = out[sc.contact_lam_index:].reshape(-1, 3)[sl]
    assert abs(lam[:, 0].sum() - N) <= 1e-7 * N
    assert np.abs(np.hypot(lam[:, 1], lam[:, 2]) - abs(F) / len(sl)).max() <= 1e-6 * abs(F)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_resting_robot_closed_form(ostrich, dtype):
    """The CUDA path against the closed form of the robot standing on the plane (equal
    rim loads, compliant sinking u_z = -kappa lambda_n, joint loads), without the oracle."""
    from tests.test_oracle_pins import resting_robot_closed_form, resting_robot_state
    sc = S.robot_plane_scene()
    h, kappa = 0.1, 1e-4
    W = 5
    st = np.repeat(resting_robot_state(sc), W, axis=1)
    tol = 1e-9 if dtype == "f64" else 2e-4
    cfg = S.SolverConfig(budget=40, tol=1e-10 if dtype == "f64" else 1e-5, kappa=kappa)
    r = _run_gpu(ostrich, sc, cfg, st, np.zeros((sc.n_servos, W)), h, dtype)
    ln, uz, lz = resting_robot_closed_form(sc, h, kappa)
    nb, nj = sc.n_bodies, len(sc.joints)
    for w in range(W):
        out = r["state"][:, w].double().numpy()
        u = out[7 * nb:13 * nb].reshape(nb, 6)
        # velocities to the Newton tolerance's order (FP64 1e-10 m/s, FP32 1e-5 m/s)
        assert np.abs(u[:, 2] - uz).max() <= (1e-9 if dtype == "f64" else 2e-5)
        assert np.abs(np.delete(u, 2, axis=1)).max() <= (1e-9 if dtype == "f64" else 2e-5)
        act = r["ids"][:, w].numpy() >= 0
        assert act.sum() == 8
        cl = out[sc.contact_lam_index:].reshape(-1, 3)
        assert np.abs(cl[act, 0] - ln).max() <= tol * ln
        assert np.abs(cl[:, 1:]).max() <= tol * ln
        jl = out[sc.lam_index:sc.lam_index + 5 * nj].reshape(nj, 5)
        assert np.abs(jl[:, 2] - np.array(lz)).max() <= tol * ln
        assert np.abs(jl[:, [0, 1, 3, 4]]).max() <= tol * ln
        assert np.abs(out[sc.lam_index + 5 * nj:sc.contact_lam_index]).max() <= tol * ln


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_param_grads_match_oracle(ostrich, dtype):
    """dL/dk_p, dL/dm and dL/dI from ostrich_adjoint_params against the oracle's adjoint at the
    CUDA path's returned iterate (Eq. (17) with xi = theta), and against the identities
    that tie them to the control and velocity gradients of the same call."""
    sc = S.robot_box_scene()
    W = 24
    st = S.robot_box_states(sc, W, seed=6)
    ub = S.random_controls(sc.n_servos, W, seed=6, low=-3, high=3)
    h = 0.1
    cfg = S.SolverConfig(budget=40, tol=1e-9 if dtype == "f64" else 1e-5)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    g = np.random.default_rng(26).normal(size=st.shape)
    g[13 * sc.n_bodies:] = 0
    ctx = ostrich.Context(sc, cfg, W, dtype=dtype, tape_slots=1)
    s_in = torch.tensor(st, dtype=tdt, device="cuda")
    u_in = torch.tensor(ub, dtype=tdt, device="cuda")
    r = ctx.step(s_in, u_in, h, tape_slot=0)
    ds, du, dkp, dm, di = ctx.adjoint_params(0, torch.tensor(g, dtype=tdt, device="cuda"), h)
    torch.cuda.synchronize()
    out = r["state"].double().cpu().numpy()
    ds, du, dkp, dm, di = (x.double().cpu().numpy() for x in (ds, du, dkp, dm, di))
    s64, u64 = s_in.double().cpu().numpy(), u_in.double().cpu().numpy()
    ctx.close()
    nb, nj = sc.n_bodies, len(sc.joints)
    orc = O.Oracle(sc, cfg)
    kp = np.array([j.kp for j in sc.joints])
    m = np.array([b.mass for b in sc.bodies])
    tol = 1e-6 if dtype == "f64" else 1e-3
    n_cmp = 0
    for w in range(W):
        if int(r["status"][w]) & 2:
            continue
        gw = g[:, w] if dtype == "f64" else g[:, w].astype(np.float32).astype(np.float64)
        at = orc.adjoint_at(s64[:, w], u64[:, w], h, out[7 * nb:13 * nb, w], out[13 * nb:, w], gw)
        scale_kp = max(np.abs(at["dkp"]).max(), 1e-12)
        scale_m = max(np.abs(at["dmass"]).max(), 1e-12)
        assert np.abs(dkp[:, w] - at["dkp"]).max() <= tol * scale_kp, f"world {w}: dL/dk_p"
        assert np.abs(dm[:, w] - at["dmass"]).max() <= tol * scale_m, f"world {w}: dL/dm"
        scale_i = max(np.abs(at["dinertia"]).max(), 1e-12)
        assert np.abs(di[:, :, w] - at["dinertia"]).max() <= tol * scale_i, f"world {w}: dL/dI"
        # identities among the outputs of the same call
        lam_c = out[sc.lam_index + 5 * nj:sc.contact_lam_index, w]
        assert np.abs(dkp[:, w] - du[:, w] * lam_c / kp ** 2).max() <= (1e-12 if dtype == "f64" else 1e-5) * scale_kp
        dv = ds[7 * nb:13 * nb, w].reshape(nb, 6)[:, :3]
        acc = out[7 * nb:13 * nb, w].reshape(nb, 6)[:, :3] - s64[7 * nb:13 * nb, w].reshape(nb, 6)[:, :3]
        acc[:, 2] -= h * sc.gravity
        assert np.abs(dm[:, w] + (dv * acc).sum(1) / m).max() <= (1e-9 if dtype == "f64" else 1e-4) * scale_m
        n_cmp += 1
    assert n_cmp >= 0.9 * W


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_resting_hinged_boxes_closed_form(ostrich, dtype):
    """The CUDA path (general separator update: each joint row couples to two contact
    groups) against the closed form of the two hinged boxes standing on the plane."""
    from tests.test_oracle_pins import hinged_resting_state
    sc = hinged_boxes_scene()
    h, kappa = 0.1, 1e-4
    W = 4
    st = np.repeat(hinged_resting_state(sc)[:, None], W, axis=1)
    tol = 1e-9 if dtype == "f64" else 1e-3
    cfg = S.SolverConfig(budget=40, tol=1e-10 if dtype == "f64" else 1e-5, kappa=kappa)
    r = _run_gpu(ostrich, sc, cfg, st, np.zeros((sc.n_servos, W)), h, dtype)
    ln, uz = resting_closed_form(sc.bodies[0].mass, 4, h, kappa)
    nb = sc.n_bodies
    for w in range(W):
        out = r["state"][:, w].double().numpy()
        u = out[7 * nb:13 * nb].reshape(nb, 6)
        # velocities to the Newton tolerance's order (FP64 1e-10 m/s; FP32 stalls near 1e-4)
        assert np.abs(u[:, 2] - uz).max() <= (1e-9 if dtype == "f64" else 1e-4)
        assert np.abs(np.delete(u, 2, axis=1)).max() <= (1e-9 if dtype == "f64" else 1e-4)
        act = r["ids"][:, w].numpy() >= 0
        assert act.sum() == 8
        cl = out[sc.contact_lam_index:].reshape(-1, 3)
        assert np.abs(cl[act, 0] - ln).max() <= tol * ln
        assert np.abs(cl[:, 1:]).max() <= tol * ln
        assert np.abs(out[sc.lam_index:sc.contact_lam_index]).max() <= tol * ln
