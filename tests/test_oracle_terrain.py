"""Oracle pins for heightmap-terrain contact generation (Sec. IV-D).

* A flat heightmap is the ground plane: every face has normal +z (to FP32 rounding)
  and offset 0, so one step of the robot on it equals the step on the plane scene
  (same contact count).
* The candidate search against brute force: for robots placed over the Gaussian
  terrain, the set of active faces of every rim equals the faces, over a 9 x 9 cell
  window, whose own deepest rim point lies on the face and passes the activation test,
  recomputed in float64 here (faces within 1e-5 of a threshold are not compared).
* Stored face planes are unit normals pointing up, with d = n . vertex.
* Converged terrain steps satisfy non-penetration, complementarity sign and the cone.
* Rows on terrain match the definition d c(q+(u))/du / h (dual numbers).
* A free wheel released on a planar slope (a tilted heightmap) follows the closed form
  of one backward-Euler step with sticking friction: rolling with the contact
  compliance kappa and the rotation-rate map of Eq. (1) on the axle direction.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2609_08800_gb300 import scenes as S


def _flat_scene(n=64, sp=0.05):
    bodies, joints = S.robot_bodies_joints()
    origin = (-(n - 1) * sp / 2, -(n - 1) * sp / 2 + 0.013)
    env = S.Env(S.ENV_HEIGHTMAP, heights=np.zeros((n, n), np.float32), spacing=sp, origin=origin)
    return S.Scene("flat", bodies, joints, env, 1.0)


def test_flat_heightmap_matches_plane():
    plane, flat = S.robot_plane_scene(mu=1.0), _flat_scene()
    cfg = S.SolverConfig(budget=60, tol=1e-9)
    st = S.robot_box_states(plane, 6, seed=3, phases=False)
    ub = S.random_controls(4, 6, seed=3, low=-3, high=3)
    op, of = O.Oracle(plane, cfg), O.Oracle(flat, cfg)
    nq = 13 * plane.n_bodies
    sf = np.zeros((flat.n_state, 6))          # same bodies, the terrain's (longer) impulse block
    sf[:nq] = st[:nq]
    for w in range(6):
        a, b = op.step(st[:, w], ub[:, w], 0.1), of.step(sf[:, w], ub[:, w], 0.1)
        assert a["status"] == 0 and b["status"] == 0
        assert (a["ids"] >= 0).sum() == (b["ids"] >= 0).sum()
        np.testing.assert_allclose(b["state"][:nq], a["state"][:nq], atol=1e-7)
    act, ids, nd = of.contacts(sf[:, 0], 0.1)
    for sl in np.nonzero(act)[0]:
        # the FP32 face normal of a flat cell is +z up to one rounding of its normalisation
        assert np.abs(nd[sl, :3] - [0.0, 0.0, 1.0]).max() <= 1.2e-7 and nd[sl, 3] == 0.0


def _rims(scene, s):
    """(body, rim, centre, axle) of every wheel rim, float64."""
    out = []
    for b, bd in enumerate(scene.bodies):
        if bd.shape != S.SHAPE_WHEEL:
            continue
        R = S._quat_to_matrix(s[7 * b + 3:7 * b + 7])
        p = s[7 * b:7 * b + 3]
        a = R @ np.array([0.0, 1.0, 0.0])
        for rim in (0, 1):
            out.append((b, rim, p + R @ np.array([0.0, bd.half_width if rim else -bd.half_width, 0.0]), a, bd.radius))
    return out


def _brute_force(scene, s, h, margin, g, win=4):
    """Active faces per rim, float64, with the ambiguous ones (within 1e-5 of a test)."""
    env = scene.env
    H = env.heights.astype(np.float64)
    n, sp, ox, oy = H.shape[0], env.spacing, env.origin[0], env.origin[1]
    res = {}
    for b, rim, c, a, r in _rims(scene, s):
        ci, cj = int((c[0] - ox) // sp), int((c[1] - oy) // sp)
        act, amb = set(), set()
        for i in range(max(ci - win, 0), min(ci + win + 1, n - 1)):
            for j in range(max(cj - win, 0), min(cj + win + 1, n - 1)):
                for t in (0, 1):
                    P = lambda ii, jj: np.array([ox + ii * sp, oy + jj * sp, H[ii, jj]])
                    A = P(i, j)
                    B, C = (P(i + 1, j), P(i + 1, j + 1)) if t == 0 else (P(i + 1, j + 1), P(i, j + 1))
                    nr = np.cross(B - A, C - A)
                    nn = nr / np.linalg.norm(nr)
                    d = nn @ A
                    perp = nn - (nn @ a) * a
                    x = c - r * perp / np.linalg.norm(perp)
                    u, v = x[0] - A[0], x[1] - A[1]
                    tests = [u, sp - u, v, sp - v, (u - v) if t == 0 else (v - u)]
                    on = min(tests) >= 0
                    pred = (nn @ x - d) + h * min(nn[2] * h * g, 0.0)
                    fid = 2 * ((n - 1) * i + j) + t
                    if min(abs(z) for z in tests) < 1e-5 or abs(pred - margin) < 1e-5:
                        amb.add(fid)
                    if on and pred < margin:
                        act.add(fid)
        res[(b, rim)] = (act, amb)
    return res


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_candidates_match_brute_force(seed):
    sc = S.terrain_scene()
    cfg = S.SolverConfig()
    orc = O.Oracle(sc, cfg)
    st = S.terrain_states(sc, 8, seed=seed)
    rng = np.random.default_rng(seed)
    h = 0.1
    n_checked = 0
    for w in range(8):
        s = st[:, w].copy()
        s[2:35:7] -= rng.uniform(0.0, 0.03)          # lower the robot into contact range
        s[35:65] = 0.0                               # at rest: the test uses zero velocity
        act, ids, nd = orc.contacts(s, h)
        got = {}
        for sl in np.nonzero(act)[0]:
            i = int(ids[sl])
            got.setdefault((i >> 24, (i >> 20) & 15), set()).add(i & 0xFFFFF)
            n_ = nd[sl, :3]
            assert abs(np.linalg.norm(n_) - 1.0) < 1e-6 and n_[2] > 0
        for key, (want, amb) in _brute_force(sc, s, h, cfg.margin, sc.gravity).items():
            g = got.get(key, set())
            assert (g - amb) == (want - amb), f"world {w} rim {key}: {sorted(g)} vs {sorted(want)}"
            n_checked += len(want)
    assert n_checked > 8


def _rough_scene(seed=7, n=96, sp=0.05):
    """Short-wavelength terrain (Gaussians of sigma 0.08-0.2 m, amplitude up to 0.15 m),
    where a tilted wheel's contact face often lies in a cell next to the first guess."""
    rng = np.random.default_rng(seed)
    size = (n - 1) * sp
    x = np.arange(n) * sp - size / 2
    X, Y = np.meshgrid(x, x, indexing="ij")
    H = np.zeros((n, n))
    for _ in range(60):
        cx, cy = rng.uniform(-size / 2, size / 2, 2)
        H += rng.uniform(0.0, 0.15) * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * rng.uniform(0.08, 0.2) ** 2))
    bodies, joints = S.robot_bodies_joints()
    env = S.Env(S.ENV_HEIGHTMAP, heights=H.astype(np.float32), spacing=sp, origin=(-size / 2, -size / 2))
    return S.Scene("rough", bodies, joints, env, 1.0)


def test_candidates_match_brute_force_rough_tilted():
    sc = _rough_scene()
    cfg = S.SolverConfig()
    orc = O.Oracle(sc, cfg)
    rng = np.random.default_rng(11)
    h = 0.1
    H = sc.env.heights
    n_checked = 0
    for w in range(40):
        s = np.zeros(sc.n_state)
        x, y = rng.uniform(-1.5, 1.5, 2)
        yaw, pitch, roll = rng.uniform(-np.pi, np.pi), rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5)
        cy, sy, cp, sp_, cr, sr = (np.cos(yaw / 2), np.sin(yaw / 2), np.cos(pitch / 2), np.sin(pitch / 2),
                                   np.cos(roll / 2), np.sin(roll / 2))
        q = np.array([cy * cp * cr + sy * sp_ * sr, cy * cp * sr - sy * sp_ * cr,
                      cy * sp_ * cr + sy * cp * sr, sy * cp * cr - cy * sp_ * sr])
        R = S._quat_to_matrix(q)
        i = int((x - sc.env.origin[0]) / sc.env.spacing)
        j = int((y - sc.env.origin[1]) / sc.env.spacing)
        z = float(H[i, j]) + S.ROBOT_WHEEL_RADIUS + rng.uniform(-0.04, 0.02)
        s[0:3], s[3:7] = (x, y, z), q
        for b, off in enumerate(S.ROBOT_WHEEL_OFFSETS, start=1):
            s[7 * b:7 * b + 3] = np.array([x, y, z]) + R @ np.array(off)
            s[7 * b + 3:7 * b + 7] = q
        act, ids, nd = orc.contacts(s, h)
        got = {}
        for sl in np.nonzero(act)[0]:
            i_ = int(ids[sl])
            got.setdefault((i_ >> 24, (i_ >> 20) & 15), set()).add(i_ & 0xFFFFF)
        for key, (want, amb) in _brute_force(sc, s, h, cfg.margin, sc.gravity).items():
            g = got.get(key, set())
            assert (g - amb) == (want - amb), f"pose {w} rim {key}: {sorted(g)} vs {sorted(want)}"
            n_checked += len(want)
    assert n_checked > 40


def test_terrain_step_invariants():
    sc = S.terrain_scene()
    cfg = S.SolverConfig(budget=60, tol=1e-9)
    orc = O.Oracle(sc, cfg)
    st = S.terrain_states(sc, 4, seed=4)
    ub = np.array([2.0, 2.0, 2.0, 2.0])
    h = 0.1
    n_ok = 0
    for w in range(4):
        s = st[:, w]
        for t in range(8):
            r = orc.step(s, ub, h)
            if r["status"] == 0:
                lam = r["state"][sc.lam_index:]
                act, ids, nd = orc.contacts(s, h)
                cl = lam[5 * len(sc.joints) + sc.n_servos:].reshape(-1, 3)
                for sl in np.nonzero(act)[0]:
                    assert cl[sl, 0] >= -1e-6
                    assert np.linalg.norm(cl[sl, 1:]) <= sc.mu * max(cl[sl, 0], 0.0) * (1 + 1e-6) + 1e-9
                inactive = np.nonzero(act == 0)[0]
                assert np.abs(cl[inactive]).max() == 0.0
                n_ok += 1
            s = r["state"]
    assert n_ok >= 16


def test_terrain_rows_match_definition():
    sc = S.terrain_scene()
    orc = O.Oracle(sc, S.SolverConfig(kappa=1e-4))
    st = S.terrain_states(sc, 3, seed=6)
    rng = np.random.default_rng(6)
    nb = sc.n_bodies
    for w in range(3):
        s = st[:, w].copy()
        s[2:35:7] -= 0.02
        u = s[7 * nb:13 * nb] + rng.normal(scale=0.5, size=6 * nb)
        lam = rng.normal(size=sc.m_max)
        rows = orc.rows(s, np.zeros(4), 0.1, u, lam)
        assert (rows["meta"][:, 0] == 2).sum() >= 1
        mask = rows["meta"][:, 0] != 1
        np.testing.assert_allclose(rows["J"][mask], rows["Jdual"][mask], rtol=1e-9, atol=1e-9)


def test_robot_resting_on_flat_heightmap_closed_form():
    """The terrain contact path against the closed form of the robot standing still: on
    a flat heightmap each rim finds one face under its lowest point, and the eight rim
    contacts share the weight as on the plane, M g / (8 + M kappa / h) each, with every
    body sinking at -kappa lambda_n."""
    from tests.test_oracle_pins import resting_robot_closed_form, resting_robot_state
    sc = _flat_scene()
    h, kappa = 0.1, 1e-4
    r = O.Oracle(sc, S.SolverConfig(budget=60, tol=1e-12, kappa=kappa)).step(
        resting_robot_state(sc)[:, 0], np.zeros(sc.n_servos), h)
    assert r["status"] == 0
    ln, uz, _ = resting_robot_closed_form(sc, h, kappa)
    nb = sc.n_bodies
    act = r["ids"] >= 0
    assert act.sum() == 8
    cl = r["state"][sc.contact_lam_index:].reshape(-1, 3)
    assert np.abs(cl[act, 0] - ln).max() <= 1e-9 * ln
    assert np.abs(cl[:, 1:]).max() <= 1e-9 * ln
    u = r["state"][7 * nb:13 * nb].reshape(nb, 6)
    assert np.abs(u[:, 2] - uz).max() <= 1e-9 * abs(uz)


def _tilted_wheel(theta=0.1, n=64, sp=0.05):
    """One free wheel (the robot's: 1 kg, r = 0.15 m, half width 0.04 m, axle along body
    y) at rest on a planar heightmap z = tan(theta) x, its rims touching the plane inside
    one triangle each (local cell coordinates (0.04, 0.005) and (0.04, 0.035))."""
    s = math.tan(theta)
    ox = oy = -(n // 2) * sp
    xs = ox + sp * np.arange(n)
    H = np.repeat((s * xs)[:, None], n, axis=1).astype(np.float32)
    bodies, _ = S.robot_bodies_joints()
    wheel = bodies[1]
    sc = S.Scene("tilted", [wheel], [], S.Env(S.ENV_HEIGHTMAP, heights=H, spacing=sp, origin=(ox, oy)), 1.0)
    xc, y1 = 0.04, 0.005                       # contact point of rim 0 (x) and its y
    nrm = np.array([-s, 0.0, 1.0]) / math.hypot(s, 1.0)
    p = np.array([xc, y1 + wheel.half_width, s * xc]) + wheel.radius * nrm
    st = np.zeros((sc.n_state, 1))
    st[0:3, 0] = p
    st[3, 0] = 1.0
    return sc, st


def tilted_wheel_closed_form(sc, st, h, kappa, nd, sl):
    """(downhill unit tangent t, unit normal, v_t, v_n, w, N, F) of one step of the wheel
    of _tilted_wheel from rest, given the active slots sl and their contact frames nd."""
    m, r, I = sc.bodies[0].mass, sc.bodies[0].radius, sc.bodies[0].inertia[1]
    nc, g = len(sl), -sc.gravity
    n = nd[sl, :3].astype(np.float64).mean(axis=0)
    cos_t = n[2] / np.linalg.norm(n)
    down = np.array([0.0, 0.0, -1.0]) - (-n[2] / (n @ n)) * n
    t = down / np.linalg.norm(down)
    sin_t = float(np.linalg.norm(down))
    cn0 = float(n @ st[0:3, 0]) - r * np.linalg.norm(n) - float(nd[sl, 3].mean())
    gamma, F, w = 1.0, 0.0, 0.0
    for _ in range(50):                    # fixed point on gamma (|h w / 2| ~ 0.02)
        F = -h * g * sin_t / (h / m + h * gamma ** 2 * r * r / I + kappa / nc)
        w = h * gamma * r * F / I
        gamma = 1.0 / (1.0 + (h * w / 2.0) ** 2)
    N = (h * m * g * cos_t - m * cn0 / h) / (h + m * kappa / nc)
    v_t = h * g * sin_t + h * F / m
    v_n = -cn0 / h - kappa * N / nc
    return t, n / np.linalg.norm(n), v_t, v_n, w, N, F


def test_wheel_on_tilted_heightmap_closed_form():
    """A free wheel released on a planar slope (Sec. III-A/B, backward Euler with sticking
    friction): one step from rest is linear in the total friction force F (along the
    downhill tangent t) and the total normal force N over the n_c contacts (one per rim):
        m v_t = h (m g sin(theta) + F),  I w = h gamma r F,  v_t + gamma r w = -kappa F / n_c
    (the friction rows: slip velocity = -kappa lambda_f, W = 0 when sticking; gamma =
    1 / (1 + (h w / 2)^2) is the rotation-rate map of Eq. (1) on the axle direction),
        m v_n = h (N - m g cos(theta)),  v_n = -c_n(q-) / h - kappa N / n_c
    (the FB normal rows at a positive multiplier: c_n(q+) / h + kappa lambda_n = 0).  The
    kappa and gamma terms move F by 2e-4 and 3e-4 of itself and kappa moves N by 5e-4;
    the pin holds the tangential and angular velocities to 1e-8 (they agree to 1e-10), the
    sinking velocity -kappa N / n_c - c_n(q-) / h to 1e-7, the per-contact friction
    magnitudes to 1e-6 and N to 1e-7 (the two faces' FP32 normals differ by a rounding,
    which splits F and N unevenly at that level)."""
    sc, st = _tilted_wheel()
    h, kappa = 0.1, 1e-4
    cfg = S.SolverConfig(budget=60, tol=1e-12, kappa=kappa)
    orc = O.Oracle(sc, cfg)
    res = orc.step(st[:, 0], np.zeros(1), h)
    assert res["status"] == 0
    act, _, nd = orc.contacts(st[:, 0], h)
    sl = np.nonzero(act)[0]
    assert sl.tolist() == [0, 8]                        # one face under each rim
    # the two faces' FP32 normals agree to a rounding (their vertices' FP32 coordinates
    # differ); the closed form takes their mean, the bounds below allow for the rest
    assert np.abs(nd[sl[0]] - nd[sl[1]]).max() <= 1e-6
    t, nu, v_t, v_n, w, N, F = tilted_wheel_closed_form(sc, st, h, kappa, nd, sl)
    nc = len(sl)
    u = res["state"][7:13]
    assert abs(u[0:3] @ t - v_t) <= 1e-8 * abs(v_t)
    assert abs(u[0:3] @ nu - v_n) <= 1e-7 * abs(v_n)
    assert abs(u[1]) <= 1e-6 * abs(v_t) and np.abs(u[[3, 5]]).max() <= 1e-6 * abs(w)
    assert abs(u[4] - w) <= 1e-8 * abs(w)
    lam = res["state"][sc.contact_lam_index:].reshape(-1, 3)[sl]
    assert abs(lam[:, 0].sum() - N) <= 1e-7 * N
    assert np.abs(np.hypot(lam[:, 1], lam[:, 2]) - abs(F) / nc).max() <= 1e-6 * abs(F)
