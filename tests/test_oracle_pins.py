"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks a closed form,
an invariant stated in the paper, a textbook special case, a library routine,
or central finite differences of the oracle's own step.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2609_08800_gb300 import scenes as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# building blocks
# --------------------------------------------------------------------------

def test_fb_complementarity():
    """Eq. (4): phi(a,b) = 0 <=> a >= 0, b >= 0, ab = 0 (eps -> 0)."""
    for a, b in [(0.0, 3.0), (2.0, 0.0), (0.0, 0.0)]:
        assert abs(O.fb(a, b, 0.0)[0]) < 1e-15
    for a, b in [(1.0, 1.0), (-1.0, 2.0), (2.0, -0.5), (-1.0, -1.0)]:
        assert abs(O.fb(a, b, 0.0)[0]) > 1e-3
    # closed form and derivatives against central differences
    a, b, eps = 0.3, -0.7, 1e-8
    phi, fa, fb_ = O.fb(a, b, eps)
    assert phi == pytest.approx(a + b - math.sqrt(a * a + b * b + eps * eps), abs=1e-15)
    d = 1e-6
    assert fa == pytest.approx((O.fb(a + d, b, eps)[0] - O.fb(a - d, b, eps)[0]) / (2 * d), rel=1e-7)
    assert fb_ == pytest.approx((O.fb(a, b + d, eps)[0] - O.fb(a, b - d, eps)[0]) / (2 * d), rel=1e-7)


def test_friction_weight_branches():
    """Sec. III-B: W -> 0 when sticking, W = v_t/(mu lambda_n) on the cone while sliding, W >= 0."""
    mu, ln = 0.8, 10.0
    assert O.friction_W(0.0, 0.0, ln, 1.0, 0.5, mu, 1e-8, 0.05) < 1e-12
    vt = 0.4
    W = O.friction_W(vt * 0.6, vt * 0.8, ln, -mu * ln * 0.6, -mu * ln * 0.8, mu, 1e-8, 0.05)
    assert W == pytest.approx(vt / (mu * ln), rel=1e-6)
    rng = np.random.default_rng(0)
    for _ in range(200):
        args = rng.normal(size=5)
        assert O.friction_W(*args, mu, 1e-8, 0.05) >= 0.0


def _rodrigues(axis, ang):
    k = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def test_rotation_matches_axis_angle():
    rng = np.random.default_rng(1)
    for _ in range(20):
        axis, ang = rng.normal(size=3), rng.uniform(-3, 3)
        k = axis / np.linalg.norm(axis)
        q = np.r_[math.cos(ang / 2), math.sin(ang / 2) * k] * rng.uniform(0.5, 2.0)   # non-unit allowed
        v = rng.normal(size=3)
        np.testing.assert_allclose(O.rotate(q, v), _rodrigues(axis, ang) @ v, atol=1e-13)


def test_dense_solve_matches_numpy():
    rng = np.random.default_rng(2)
    for n in (1, 5, 37):
        B = rng.normal(size=(n, n))
        A = B @ B.T + 0.1 * np.eye(n)
        b = rng.normal(size=n)
        np.testing.assert_allclose(O.lu_solve(A, b), np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)


# --------------------------------------------------------------------------
# closed forms of the step (Eqs. (1), (2))
# --------------------------------------------------------------------------

def _box_cfg(kappa=0.0):
    return S.SolverConfig(budget=60, k_min=4, tol=1e-11, kappa=kappa)


def test_free_flight_and_torque_free_spin():
    sc = S.box_drop_scene()
    orc = O.Oracle(sc, _box_cfg())
    s = np.zeros(sc.n_state)
    s[0:3] = (0.1, -0.2, 5.0)
    s[3:7] = (1, 0, 0, 0)
    s[7:10] = (0.3, -0.1, 0.2)
    s[10:13] = (0.0, 0.0, 1.5)       # spin about the principal z axis
    h = 0.1
    r = orc.step(s, np.zeros(1), h)
    out = r["state"]
    assert r["rows"] == 0
    v = s[7:10] + h * np.array([0, 0, -9.81])
    np.testing.assert_allclose(out[7:10], v, atol=1e-14)
    np.testing.assert_allclose(out[0:3], s[0:3] + h * v, atol=1e-14)
    np.testing.assert_allclose(out[10:13], s[10:13], atol=1e-14)      # no gyroscopic torque
    # quaternion: normalised first-order update q + h/2 (0, w) (x) q
    qz = np.array([1.0, 0.0, 0.0, 0.5 * h * 1.5])
    np.testing.assert_allclose(out[3:7], qz / np.linalg.norm(qz), atol=1e-14)


def test_box_drop_closed_form():
    gold = json.load(open(os.path.join(GOLD, "box_drop_closed_form.json")))
    sc, st = S.box_drop_inputs(0)
    v0 = st[7, 0]
    assert v0 > gold["stop_threshold_v0"]
    orc = O.Oracle(sc, _box_cfg())
    h = gold["h"]
    s = st[:, 0]
    sums = []
    for k in range(6):
        r = orc.step(s, np.zeros(1), h)
        assert r["status"] == 0 and r["residual"] < 1e-10
        imp = r["impulses"][sc.contact_row_offset:].reshape(-1, 3)
        sums.append((imp[:, 0].sum(), imp[:, 1].sum(), imp[:, 2].sum()))
        if k == 0:
            assert r["state"][9] == pytest.approx(gold["step1_uz"], abs=1e-9)
            assert r["state"][7] == pytest.approx(v0 + gold["step1_du_x_sliding"], abs=1e-9)
            assert (r["ids"] >= 0).sum() == 4
        s = r["state"]
    assert sums[0][0] == pytest.approx(gold["step1_sum_hn"], abs=1e-8)
    assert sums[0][1] == pytest.approx(-gold["mu"] * gold["step1_sum_hn"], abs=1e-8)
    assert sums[1][0] == pytest.approx(gold["step2_sum_hn"], abs=1e-8)
    for k in range(2, 6):
        assert sums[k][0] == pytest.approx(gold["rest_sum_hn"], abs=1e-8)
        assert abs(sums[k][1]) < 1e-8 and abs(sums[k][2]) < 1e-8
    np.testing.assert_allclose(s[7:13], 0.0, atol=1e-9)


def _box_rollout_x(orc, sc, v0, h, T):
    s = S.box_drop_state(sc, v0)[:, 0]
    states = [s]
    for _ in range(T):
        states.append(orc.step(states[-1], np.zeros(1), h)["state"])
    return states


def test_box_final_position_and_gradient_closed_form():
    """x_T = x0 + h max(0, v0 - 0.3848) and dx_T/dv0 = h (central differences of the
    oracle's forward rollout, hard contact)."""
    gold = json.load(open(os.path.join(GOLD, "box_drop_closed_form.json")))
    sc = S.box_drop_scene()
    orc = O.Oracle(sc, _box_cfg())
    h, T, thr = 0.1, 20, gold["stop_threshold_v0"]
    for v0 in (0.2, 0.6369616873214543, 0.9):
        xT = _box_rollout_x(orc, sc, v0, h, T)[-1][0]
        assert xT == pytest.approx(h * max(0.0, v0 - thr), abs=1e-9)
        d = 1e-5
        fd = (_box_rollout_x(orc, sc, v0 + d, h, T)[-1][0] - _box_rollout_x(orc, sc, v0 - d, h, T)[-1][0]) / (2 * d)
        assert fd == pytest.approx(h if v0 > thr else 0.0, abs=1e-7)


def test_exact_adjoint_rollout_matches_fd():
    """Exact-IFT adjoint swept over the 20-step drop (compliance 1e-4 makes the
    four-corner impulse split unique) against central differences of the rollout."""
    sc = S.box_drop_scene()
    orc = O.Oracle(sc, S.SolverConfig(budget=80, k_min=4, tol=1e-12, kappa=1e-4))
    h, T = 0.1, 20
    for v0 in (0.2, 0.6369616873214543):
        states = _box_rollout_x(orc, sc, v0, h, T)
        g = np.zeros(sc.n_state)
        g[0] = 1.0
        for t in reversed(range(T)):
            g = orc.step_adjoint(states[t], np.zeros(1), h, g, mode=O.ADJ_EXACT)["dstate"]
        d = 1e-6
        fd = (_box_rollout_x(orc, sc, v0 + d, h, T)[-1][0] - _box_rollout_x(orc, sc, v0 - d, h, T)[-1][0]) / (2 * d)
        assert g[7] == pytest.approx(fd, abs=1e-6)
        if v0 > 0.3848:
            assert g[7] == pytest.approx(h, rel=5e-3)      # h up to the O(kappa) micro-slip


def test_sliding_friction_is_timestep_consistent():
    """Sec. III-B: the converged sliding force does not depend on h (mu m g)."""
    sc = S.box_drop_scene()
    orc = O.Oracle(sc, _box_cfg())
    for h in (0.02, 0.05, 0.1, 0.2):
        s = S.box_drop_state(sc, 0.0, gap=0.0)[:, 0]
        for _ in range(3):
            s = orc.step(s, np.zeros(1), h)["state"]          # settle at rest
        s[7] = 5.0                                            # fast slide, stays sliding this step
        r = orc.step(s, np.zeros(1), h)
        imp = r["impulses"][sc.contact_row_offset:].reshape(-1, 3)
        assert imp[:, 1].sum() / h == pytest.approx(-0.8 * 10.0 * 9.81, rel=1e-8)
        assert imp[:, 0].sum() / h == pytest.approx(10.0 * 9.81, rel=1e-8)


# --------------------------------------------------------------------------
# robot: invariants at convergence (parity otherwise unpinned: no closed form)
# --------------------------------------------------------------------------

def _robot_states(n=6, seed=0):
    sc = S.robot_box_scene()
    return sc, S.robot_box_states(sc, n, seed=seed)


def _world_R(q):
    return S._quat_to_matrix(np.asarray(q))


def _qmul(a, b):
    aw, av, bw, bv = a[0], a[1:], b[0], b[1:]
    return np.r_[aw * bw - av @ bv, aw * bv + bw * av + np.cross(av, bv)]


@pytest.mark.parametrize("w", range(6))
def test_robot_step_invariants(w):
    sc, st = _robot_states()
    cfg = S.SolverConfig(budget=60, k_min=4, tol=1e-9, kappa=1e-4)
    orc = O.Oracle(sc, cfg)
    ub = np.array([2.0, 2.0, 2.0, 2.0])
    s = st[:, w]
    h = 0.1
    for _ in range(3):
        r = orc.step(s, ub, h)
        if r["status"] == 0:
            break
        s = r["state"]
    if r["status"] != 0:
        pytest.skip("step did not converge within the budget (best iterate returned)")
    out, lam = r["state"], r["state"][sc.lam_index:]
    nb = sc.n_bodies
    # joint closure (Eq. (3), E = 0): anchors coincide, axes aligned
    for j, jt in enumerate(sc.joints):
        pp, Rp = out[7 * jt.parent:7 * jt.parent + 3], _world_R(out[7 * jt.parent + 3:7 * jt.parent + 7])
        pc, Rc = out[7 * jt.child:7 * jt.child + 3], _world_R(out[7 * jt.child + 3:7 * jt.child + 7])
        gap = (pp + Rp @ np.array(jt.anchor_parent)) - (pc + Rc @ np.array(jt.anchor_child))
        assert np.abs(gap).max() < 1e-8
        aw = Rc @ np.array(jt.axis_child)
        for b in jt.perp_parent:
            assert abs((Rp @ np.array(b)) @ aw) < 1e-8
        # servo law (Eq. (8)): lambda_c = k_p (ubar - J_c u+); J_c u+ is the relative rotation
        # rate about the axle through the step's map w -> E(w) w = w / (1 + (h|w|/2)^2)
        wp = out[7 * nb + 6 * jt.parent + 3:7 * nb + 6 * jt.parent + 6]
        wc = out[7 * nb + 6 * jt.child + 3:7 * nb + 6 * jt.child + 6]
        eff = lambda w: w / (1.0 + (0.5 * h) ** 2 * (w @ w))
        # the axle is evaluated at q+ before normalisation, i.e. q- + h G(q-) u+
        qraw = s[7 * jt.parent + 3:7 * jt.parent + 7] + 0.5 * h * _qmul(np.r_[0.0, wp], s[7 * jt.parent + 3:7 * jt.parent + 7])
        rel = (_world_R(qraw) @ np.array(jt.axis_parent)) @ (eff(wc) - eff(wp))
        lc = lam[5 * len(sc.joints) + j]
        assert lc == pytest.approx(jt.kp * (ub[j] - rel), abs=1e-6 * jt.kp)
    # contacts: non-penetration, sign, complementarity, cone
    act, ids, nd = orc.contacts(st[:, w] if False else s, h)
    cl = lam[5 * len(sc.joints) + sc.n_servos:].reshape(-1, 3)
    for sl in np.nonzero(act)[0]:
        ln, lf = cl[sl, 0], cl[sl, 1:]
        assert ln >= -1e-6
        assert np.linalg.norm(lf) <= 0.9 * max(ln, 0.0) * (1 + 1e-6) + 1e-9
    inactive = np.nonzero(act == 0)[0]
    assert np.abs(cl[inactive]).max() == 0.0


def resting_robot_closed_form(sc, h, kappa, g=9.81):
    """The robot standing still on the plane, zero servo targets (Sec. III-B rows with the
    normal compliance kappa): the geometry is symmetric about the chassis centre, so its
    eight rim contacts carry equal normal forces lambda_n; the compliant normal row reads
    u_z + kappa lambda_n = 0 (the rims start exactly on the plane), and the vertical
    momentum balance M u_z = -M g h + 8 h lambda_n gives
        lambda_n = M g / (8 + M kappa / h),  u_z = -kappa lambda_n  (every body);
    each wheel's joint carries lambda_z = 2 lambda_n - m_w (g + u_z / h) on its vertical
    position row; every other velocity, friction and servo multiplier is zero."""
    M = sum(b.mass for b in sc.bodies)
    ln = M * g / (8.0 + M * kappa / h)
    uz = -kappa * ln
    lz = [2.0 * ln - sc.bodies[j.child].mass * (g + uz / h) for j in sc.joints]
    return ln, uz, lz


def resting_robot_state(sc):
    s = np.zeros((sc.n_state, 1))
    S._place_robot(s, sc, 0, 0.0, 0.0, S.ROBOT_CHASSIS_Z, 0.0)
    return s


def resting_closed_form(m, n_contacts, h, kappa, g=9.81):
    """A body of mass m standing on the plane on n_contacts symmetric contacts that start
    exactly on it (Sec. III-B with the normal compliance kappa): each carries
    lambda_n = m g / (n + m kappa / h) and the body sinks at u_z = -kappa lambda_n."""
    ln = m * g / (n_contacts + m * kappa / h)
    return ln, -kappa * ln


def hinged_boxes_scene():
    """Two boxes on the plane joined by a servoed revolute joint: both bodies carry
    contact slots, so every joint row couples to two contact groups."""
    m, a, b, c = 10.0, 0.4, 0.4, 0.2
    bodies = [S.Body(mass=m, inertia=S._box_inertia(m, a, b, c), shape=S.SHAPE_BOX,
                     half_extents=(a / 2, b / 2, c / 2)) for _ in range(2)]
    joints = [S.Joint(parent=0, child=1, anchor_parent=(0.21, 0.0, 0.0), anchor_child=(-0.21, 0.0, 0.0), kp=50.0)]
    return S.Scene("hinged_boxes", bodies, joints, S.Env(S.ENV_PLANE), 0.8)


def hinged_resting_state(sc):
    s = np.zeros(sc.n_state)
    for b, x in enumerate((-0.21, 0.21)):
        s[7 * b:7 * b + 7] = (x, 0.0, 0.1, 1.0, 0.0, 0.0, 0.0)
    return s


def test_hinged_boxes_resting_closed_form():
    """Two hinged boxes standing on the plane, zero servo target: each box rests on its
    own four corners (mirror symmetry: the joint carries nothing), so every corner holds
    m g / (4 + m kappa / h) and both boxes sink at -kappa lambda_n."""
    sc = hinged_boxes_scene()
    h, kappa = 0.1, 1e-4
    r = O.Oracle(sc, S.SolverConfig(budget=60, tol=1e-12, kappa=kappa)).step(hinged_resting_state(sc), np.zeros(1), h)
    assert r["status"] == 0
    ln, uz = resting_closed_form(sc.bodies[0].mass, 4, h, kappa)
    nb = sc.n_bodies
    out = r["state"]
    u = out[7 * nb:13 * nb].reshape(nb, 6)
    assert np.abs(u[:, 2] - uz).max() <= 1e-9 * abs(uz)
    assert np.abs(np.delete(u, 2, axis=1)).max() <= 1e-12
    act = r["ids"] >= 0
    assert act.sum() == 8
    cl = out[sc.contact_lam_index:].reshape(-1, 3)
    assert np.abs(cl[act, 0] - ln).max() <= 1e-9 * ln
    assert np.abs(cl[:, 1:]).max() <= 1e-9 * ln
    assert np.abs(out[sc.lam_index:sc.contact_lam_index]).max() <= 1e-9 * ln


def test_robot_resting_on_plane_closed_form():
    sc = S.robot_plane_scene()
    h, kappa = 0.1, 1e-4
    orc = O.Oracle(sc, S.SolverConfig(budget=60, tol=1e-12, kappa=kappa))
    r = orc.step(resting_robot_state(sc)[:, 0], np.zeros(sc.n_servos), h)
    assert r["status"] == 0
    ln, uz, lz = resting_robot_closed_form(sc, h, kappa)
    nb, nj = sc.n_bodies, len(sc.joints)
    out = r["state"]
    u = out[7 * nb:13 * nb].reshape(nb, 6)
    assert np.abs(u[:, 2] - uz).max() <= 1e-9 * abs(uz)
    assert np.abs(np.delete(u, 2, axis=1)).max() <= 1e-12
    act = r["ids"] >= 0
    assert act.sum() == 8
    cl = out[sc.contact_lam_index:].reshape(-1, 3)
    assert np.abs(cl[act, 0] - ln).max() <= 1e-9 * ln
    assert np.abs(cl[:, 1:]).max() <= 1e-9 * ln
    jl = out[sc.lam_index:sc.lam_index + 5 * nj].reshape(nj, 5)
    assert np.abs(jl[:, 2] - np.array(lz)).max() <= 1e-9 * ln
    assert np.abs(jl[:, [0, 1, 3, 4]]).max() <= 1e-9 * ln
    assert np.abs(out[sc.lam_index + 5 * nj:sc.contact_lam_index]).max() <= 1e-9 * ln
    # impulses are h lambda in the same layout
    assert r["impulses"][sc.contact_lam_index - sc.lam_index:].reshape(-1, 3)[act, 0] == pytest.approx(h * ln, rel=1e-9)


# --------------------------------------------------------------------------
# Jacobian: analytic rows equal the definition d c(q+(u))/du / h
# --------------------------------------------------------------------------

@pytest.mark.parametrize("w", range(4))
def test_row_jacobian_matches_definition(w):
    sc, st = _robot_states(n=4, seed=3)
    cfg = S.SolverConfig(kappa=1e-4)
    orc = O.Oracle(sc, cfg)
    rng = np.random.default_rng(w)
    s = st[:, w]
    nb = sc.n_bodies
    u = s[7 * nb:13 * nb] + rng.normal(scale=1.0, size=6 * nb)
    lam = rng.normal(size=sc.m_max)
    rows = orc.rows(s, np.zeros(4), 0.1, u, lam)
    assert rows["J"].shape[0] >= 24
    mask = rows["meta"][:, 0] != 1          # servo rows are not covered by the definition here
    np.testing.assert_allclose(rows["J"][mask], rows["Jdual"][mask], rtol=1e-9, atol=1e-9)


def test_box_jacobian_matches_definition():
    sc = S.box_drop_scene()
    orc = O.Oracle(sc, S.SolverConfig())
    s = S.box_drop_state(sc, 0.3, gap=0.001)[:, 0]
    s[3:7] = np.array([0.99, 0.05, -0.08, 0.1]) / np.linalg.norm([0.99, 0.05, -0.08, 0.1])
    s[2] = 0.13
    rng = np.random.default_rng(5)
    u = rng.normal(size=6)
    rows = orc.rows(s, np.zeros(1), 0.1, u, rng.normal(size=sc.m_max))
    assert rows["J"].shape[0] > 0
    np.testing.assert_allclose(rows["J"], rows["Jdual"], rtol=1e-9, atol=1e-9)


# --------------------------------------------------------------------------
# adjoint against central finite differences of the oracle's own step
# --------------------------------------------------------------------------

def _fd_grad(orc, s, ub, h, g, idx, eps=1e-6):
    out = np.zeros(len(idx))
    for k, i in enumerate(idx):
        sp, sm = s.copy(), s.copy()
        sp[i] += eps; sm[i] -= eps
        out[k] = g @ (orc.step(sp, ub, h)["state"] - orc.step(sm, ub, h)["state"]) / (2 * eps)
    return out


def _fd_ctrl(orc, s, ub, h, g, eps=1e-6):
    out = np.zeros(len(ub))
    for i in range(len(ub)):
        up, um = ub.copy(), ub.copy()
        up[i] += eps; um[i] -= eps
        out[i] = g @ (orc.step(s, up, h)["state"] - orc.step(s, um, h)["state"]) / (2 * eps)
    return out


def _resting_box(kappa):
    sc = S.box_drop_scene()
    orc = O.Oracle(sc, S.SolverConfig(budget=60, k_min=4, tol=1e-12, kappa=kappa))
    s = S.box_drop_state(sc, 0.0, gap=0.0)[:, 0]
    for _ in range(3):
        s = orc.step(s, np.zeros(1), 0.1)["state"]
    s[7], s[8] = 0.05, 0.02          # small push: the box sticks
    return sc, orc, s


def _rolling_robot(kappa):
    sc = S.robot_plane_scene()
    st = S.robot_box_states(sc, 2, seed=0, phases=False)
    orc = O.Oracle(sc, S.SolverConfig(budget=60, k_min=4, tol=1e-12, kappa=kappa))
    s, ub = st[:, 1], np.full(4, 2.0)
    for _ in range(5):
        s = orc.step(s, ub, 0.1)["state"]
    return sc, orc, s, ub


@pytest.mark.parametrize("kappa", [0.0, 1e-4])
def test_exact_adjoint_matches_fd_box(kappa):
    sc, orc, s = _resting_box(kappa)
    g = np.random.default_rng(7).normal(size=sc.n_state)
    g[13:] = 0.0
    ad = orc.step_adjoint(s, np.zeros(1), 0.1, g, mode=O.ADJ_EXACT)["dstate"][:13]
    fd = _fd_grad(orc, s, np.zeros(1), 0.1, g, range(13))
    assert np.abs(ad - fd).max() <= 1e-6 * np.abs(fd).max()


def test_exact_adjoint_matches_fd_robot():
    sc, orc, s, ub = _rolling_robot(1e-4)
    g = np.random.default_rng(8).normal(size=sc.n_state)
    g[13 * sc.n_bodies:] = 0.0
    r = orc.step_adjoint(s, ub, 0.1, g, mode=O.ADJ_EXACT)
    fd = _fd_grad(orc, s, ub, 0.1, g, range(13 * sc.n_bodies))
    assert np.abs(r["dstate"][:13 * sc.n_bodies] - fd).max() <= 1e-6 * np.abs(fd).max()
    fdu = _fd_ctrl(orc, s, ub, 0.1, g)
    assert np.abs(r["dubar"] - fdu).max() <= 1e-6 * np.abs(fdu).max()


@pytest.mark.parametrize("kappa", [0.0, 1e-4])
def test_paper_adjoint_matches_fd_on_sticking_box(kappa):
    """Sec. III-D: the paper's adjoint (forward Schur matrix, W lagged) against central
    differences on a sticking contact; the paper reports <= 0.4 % on sticking scenes."""
    sc, orc, s = _resting_box(kappa)
    g = np.random.default_rng(9).normal(size=sc.n_state)
    g[13:] = 0.0
    ad = orc.step_adjoint(s, np.zeros(1), 0.1, g, mode=O.ADJ_PAPER)["dstate"][:13]
    fd = _fd_grad(orc, s, np.zeros(1), 0.1, g, range(13))
    assert np.abs(ad - fd).max() <= 4e-3 * np.abs(fd).max()


def test_paper_adjoint_deviation_on_robot_is_bounded():
    """The paper's Newton matrix drops the geometric stiffness d(J^T lambda)/dq (it keeps M
    block diagonal); at h = 0.1 on the robot that costs a few percent against FD."""
    sc, orc, s, ub = _rolling_robot(1e-4)
    g = np.random.default_rng(10).normal(size=sc.n_state)
    g[13 * sc.n_bodies:] = 0.0
    r = orc.step_adjoint(s, ub, 0.1, g, mode=O.ADJ_PAPER)
    fd = _fd_grad(orc, s, ub, 0.1, g, range(13 * sc.n_bodies))
    assert np.abs(r["dstate"][:13 * sc.n_bodies] - fd).max() <= 0.1 * np.abs(fd).max()


def test_truncated_pullback_differs_only_in_contact_terms():
    """Sec. IV-D: truncation holds contact geometry fixed; with no contacts it is exact."""
    sc = S.box_drop_scene()
    cfg_f = S.SolverConfig(budget=60, tol=1e-12, pullback=S.PULLBACK_FULL)
    cfg_t = S.SolverConfig(budget=60, tol=1e-12, pullback=S.PULLBACK_TRUNCATED)
    s = S.box_drop_state(sc, 0.3, gap=3.0)[:, 0]
    s[10:13] = (0.2, -0.4, 0.9)
    g = np.random.default_rng(11).normal(size=sc.n_state)
    a = O.Oracle(sc, cfg_f).step_adjoint(s, np.zeros(1), 0.1, g)["dstate"]
    b = O.Oracle(sc, cfg_t).step_adjoint(s, np.zeros(1), 0.1, g)["dstate"]
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)
    sc2, orc2, s2 = _resting_box(1e-4)
    a = O.Oracle(sc2, S.SolverConfig(budget=60, tol=1e-12, kappa=1e-4)).step_adjoint(s2, np.zeros(1), 0.1, g)
    b = O.Oracle(sc2, S.SolverConfig(budget=60, tol=1e-12, kappa=1e-4, pullback=1)).step_adjoint(s2, np.zeros(1), 0.1, g)
    assert np.abs(a["dstate"] - b["dstate"]).max() > 1e-6        # contact terms do change


# --------------------------------------------------------------------------
# contact predicate: hand-placed cases
# --------------------------------------------------------------------------

def test_box_corner_activation():
    sc = S.box_drop_scene()
    orc = O.Oracle(sc, S.SolverConfig())
    h = 0.1
    s = S.box_drop_state(sc, 0.0, gap=0.0)[:, 0]
    s[2] = 0.1 + 0.019 + h * h * 9.81          # margin - 1 mm + one step at the predicted h g speed
    act, ids, _ = orc.contacts(s, h)
    assert list(act) == [1, 1, 1, 1, 0, 0, 0, 0]
    s[2] = 0.1 + 0.021 + h * h * 9.81
    act, _, _ = orc.contacts(s, h)
    assert act.sum() == 0
    s[9] = -1.0                                                     # approaching at 1 m/s
    act, _, _ = orc.contacts(s, h)
    assert list(act[:4]) == [1, 1, 1, 1]
    assert list(ids[:4]) == [(0 << 24) | (k << 20) for k in range(4)]


def _robot_at(x, z=None, scene=None):
    sc = scene or S.robot_box_scene()
    s = np.zeros((sc.n_state, 1))
    S._place_robot(s, sc, 0, x, 0.0, S.ROBOT_CHASSIS_Z if z is None else z, 0.0)
    return sc, s[:, 0]


def test_wheel_features_on_box_scene():
    sc, s = _robot_at(0.0)
    orc = O.Oracle(sc, S.SolverConfig())
    act, ids, nd = orc.contacts(s, 0.1)
    # flat ground: each wheel touches the ground with both rims (feature 0), nothing else
    assert act.sum() == 8
    assert all((ids[act > 0] & 0xFFFFF) == 0)
    # front wheels against the face: ground + near face (feature 2) on both rims
    sc, s = _robot_at(1.0 - 0.25 - 0.15 - 0.005)
    act, ids, nd = orc.contacts(s, 0.1)
    feats = sorted(set(int(i) & 0xF for i in ids[act > 0]))
    assert feats == [0, 2]
    front = [int(i) for i in ids[act > 0] if (int(i) >> 24) in (1, 2)]
    assert sum((i & 0xF) == 2 for i in front) == 4
    for sl in np.nonzero(act)[0]:
        if ids[sl] & 0xF == 2:
            np.testing.assert_allclose(nd[sl], [-1, 0, 0, -1.0], atol=1e-7)
    # robot on top: top face only
    sc, s = _robot_at(1.5, z=S.ROBOT_CHASSIS_Z + 0.15)
    act, ids, nd = orc.contacts(s, 0.1)
    assert act.sum() == 8 and all((ids[act > 0] & 0xF) == 1)
    # front wheels just past the back edge: edge feature with normal toward the rim centre
    sc, s = _robot_at(2.0 - 0.25 + 0.03, z=S.ROBOT_CHASSIS_Z + 0.15)
    act, ids, nd = orc.contacts(s, 0.1)
    edge = [sl for sl in np.nonzero(act)[0] if ids[sl] & 0xF == 3]
    assert len(edge) == 4
    for sl in edge:
        n = nd[sl, :3]
        assert n[0] > 0 and n[2] > 0 and abs(np.linalg.norm(n) - 1) < 1e-6


def test_adjoint_at_own_solution_equals_step_adjoint():
    """The adjoint taken at a supplied iterate reproduces the step's own adjoint when
    given the step's returned iterate (the same A, the same VJPs)."""
    sc, st = _robot_states(n=3, seed=9)
    orc = O.Oracle(sc, S.SolverConfig(budget=40, tol=1e-9))
    nb = sc.n_bodies
    g = np.random.default_rng(4).normal(size=sc.n_state)
    g[13 * nb:] = 0
    ub = np.array([1.0, -2.0, 2.5, 0.5])
    for w in range(3):
        r = orc.step_adjoint(st[:, w], ub, 0.1, g)
        a = orc.adjoint_at(st[:, w], ub, 0.1, r["state"][7 * nb:13 * nb], r["state"][13 * nb:], g)
        np.testing.assert_array_equal(a["dstate"], r["dstate"])
        np.testing.assert_array_equal(a["dubar"], r["dubar"])


# --------------------------------------------------------------------------
# Physical-parameter gradients (Eq. (17) with xi = theta): servo gains, body masses
# --------------------------------------------------------------------------

def _param_case():
    """The robot standing on the plane with small servo targets (the wheels start to roll
    and the contacts stick) and a random cotangent on the next poses and velocities."""
    sc = S.robot_plane_scene()
    s0 = resting_robot_state(sc)[:, 0]
    ub = np.array([0.05, -0.03, 0.04, 0.02])
    rng = np.random.default_rng(7)
    g = np.zeros(sc.n_state)
    g[:13 * sc.n_bodies] = rng.normal(size=13 * sc.n_bodies)
    return sc, s0, ub, g


def _loss_of(scene, cfg, s0, ub, h, g):
    r = O.Oracle(scene, cfg).step(s0, ub, h)
    assert r["status"] == 0
    nb = scene.n_bodies
    return g[:13 * nb] @ r["state"][:13 * nb]


def test_param_grads_exact_match_central_differences():
    """Exact-IFT mode: dL/dk_p and dL/dm_b against central differences of the loss through
    the converged step (the contact set is fixed at q-, so the step is smooth in theta)."""
    import copy
    sc, s0, ub, g = _param_case()
    h, cfg = 0.1, S.SolverConfig(budget=60, tol=1e-12)
    r = O.Oracle(sc, cfg).step_adjoint(s0, ub, h, g, mode=O.ADJ_EXACT)
    fd_kp, fd_m = [], []
    for j in range(len(sc.joints)):
        d = 1e-4 * sc.joints[j].kp
        sp, sm = copy.deepcopy(sc), copy.deepcopy(sc)
        sp.joints[j].kp += d
        sm.joints[j].kp -= d
        fd_kp.append((_loss_of(sp, cfg, s0, ub, h, g) - _loss_of(sm, cfg, s0, ub, h, g)) / (2 * d))
    for b in range(sc.n_bodies):
        d = 1e-3 * sc.bodies[b].mass
        sp, sm = copy.deepcopy(sc), copy.deepcopy(sc)
        sp.bodies[b].mass += d
        sm.bodies[b].mass -= d
        fd_m.append((_loss_of(sp, cfg, s0, ub, h, g) - _loss_of(sm, cfg, s0, ub, h, g)) / (2 * d))
    fd_kp, fd_m = np.array(fd_kp), np.array(fd_m)
    assert np.abs(fd_kp).max() > 1e-5 and np.abs(fd_m).max() > 1e-4       # not a trivial zero
    assert np.abs(r["dkp"] - fd_kp).max() <= 1e-5 * np.abs(fd_kp).max()
    # the masses also enter the step through the FB scaling what = J M^-1 J^T (normal rows,
    # friction cone margin), a step-start constant that the parameter gradient leaves
    # out; against the differences that omission measures 3e-5 of the largest entry
    assert np.abs(r["dmass"] - fd_m).max() <= 1e-4 * np.abs(fd_m).max()


@pytest.mark.parametrize("mode", [0, 1])
def test_param_grads_identities(mode):
    """In both adjoint modes the parameter gradients are the same adjoint vector
    contracted with other partials of the same rows, so they follow from the gradients
    the dual-number VJP returns:  dL/dk_p = dL/dubar * lambda_c / k_p^2 (servo row
    v + lambda_c/k_p - ubar) and dL/dm_b = -(dL/dv-_b . (v+ - v- - h g e_z)) / m_b (linear
    rows of Eq. (10), whose only v- dependence is -m_b v-)."""
    sc, s0, ub, g = _param_case()
    h = 0.1
    r = O.Oracle(sc, S.SolverConfig(budget=60, tol=1e-12)).step_adjoint(s0, ub, h, g, mode=mode)
    nb, nj = sc.n_bodies, len(sc.joints)
    lam_c = r["state"][sc.lam_index + 5 * nj:sc.contact_lam_index]
    kp = np.array([j.kp for j in sc.joints])
    assert r["dkp"] == pytest.approx(r["dubar"] * lam_c / kp ** 2, rel=1e-12, abs=1e-18)
    dv = r["dstate"][7 * nb:13 * nb].reshape(nb, 6)[:, :3]
    vp = r["state"][7 * nb:13 * nb].reshape(nb, 6)[:, :3]
    vm = s0[7 * nb:13 * nb].reshape(nb, 6)[:, :3]
    m = np.array([b.mass for b in sc.bodies])
    acc = vp - vm
    acc[:, 2] -= h * sc.gravity
    assert r["dmass"] == pytest.approx(-(dv * acc).sum(1) / m, rel=1e-9, abs=1e-15)


def test_inertia_grads_exact_match_central_differences():
    """Exact-IFT mode: dL/dI_k (body-frame principal moments) against central differences
    through the converged step, with every body spinning (~1 rad/s) so the gyroscopic
    part h w- x (I_w w-) of Eq. (10) carries weight.  The moments also enter the FB
    scaling what of the rim contacts (lever arm off the normal), a step-start constant the
    gradient leaves out: 8e-6 of the largest entry here."""
    import copy
    sc, s0, ub, g = _param_case()
    nb = sc.n_bodies
    s0 = s0.copy()
    rng = np.random.default_rng(11)
    for b in range(nb):
        s0[7 * nb + 6 * b + 3:7 * nb + 6 * b + 6] = rng.normal(scale=1.0, size=3)
    h, cfg = 0.1, S.SolverConfig(budget=60, tol=1e-12)
    r = O.Oracle(sc, cfg).step_adjoint(s0, ub, h, g, mode=O.ADJ_EXACT)
    assert r["status"] == 0
    fd = np.zeros((nb, 3))
    for b in range(nb):
        for k in range(3):
            inertia = list(sc.bodies[b].inertia)
            d = 1e-3 * inertia[k]
            sp, sm = copy.deepcopy(sc), copy.deepcopy(sc)
            sp.bodies[b].inertia = tuple(v + (d if i == k else 0.0) for i, v in enumerate(inertia))
            sm.bodies[b].inertia = tuple(v - (d if i == k else 0.0) for i, v in enumerate(inertia))
            fd[b, k] = (_loss_of(sp, cfg, s0, ub, h, g) - _loss_of(sm, cfg, s0, ub, h, g)) / (2 * d)
    assert np.abs(fd).max() > 1e-2
    assert np.abs(r["dinertia"] - fd).max() <= 5e-5 * np.abs(fd).max()


def test_sliding_box_trajectory_matches_discrete_closed_form_at_every_h():
    """Timestep sweep (Sec. III-B, friction at the step's own h): a box launched at
    v0 = 2 m/s along the plane decelerates by exactly mu g h per step until it sticks,
    v_{n+1} = max(0, v_n - mu g h), x_{n+1} = x_n + h v_{n+1} (backward Euler), at every h;
    the stopping distance tends to the continuous v0^2 / (2 mu g) as h -> 0, within v0 h."""
    sc = S.box_drop_scene()
    orc = O.Oracle(sc, S.SolverConfig(budget=60, k_min=4, tol=1e-10, kappa=0.0))
    v0, mu, g = 2.0, 0.8, 9.81
    for h in (0.0125, 0.025, 0.05, 0.1, 0.2):
        s = S.box_drop_state(sc, 0.0, gap=0.0)[:, 0]
        for _ in range(3):
            s = orc.step(s, np.zeros(1), h)["state"]          # settle at rest on the plane
        x0 = s[0]
        s[7] = v0
        v, x = v0, x0
        for _ in range(int(round(0.4 / h))):
            r = orc.step(s, np.zeros(1), h)
            assert r["status"] & 2 == 0
            s = r["state"]
            v = max(0.0, v - mu * g * h)
            x = x + h * v
            # at h = 0.0125 the frozen-W iteration stalls at residuals of 1e-9 to 1e-6 m/s in
            # the slow-sliding steps (any budget); the returned iterates stay within 1.5e-8
            assert s[7] == pytest.approx(v, abs=5e-8)
            assert s[0] == pytest.approx(x, abs=5e-8)
        assert v == 0.0                                       # stopped within 0.4 s
        assert abs((x - x0) - v0 ** 2 / (2 * mu * g)) <= v0 * h


# --------------------------------------------------------------------------
# paper-mode (frozen W) adjoint on a sliding contact; truncated pull-back
# --------------------------------------------------------------------------

def _corner_what(b, k):
    """J_n M^-1 J_n^T of bottom corner k of a flat box on z = 0, from its geometry."""
    hx, hy, hz = b.half_extents
    rho = np.array([hx if k & 1 else -hx, hy if k & 2 else -hy, hz if k & 4 else -hz])
    rn = np.cross(rho, [0.0, 0.0, 1.0])
    return 1.0 / b.mass + rn @ (rn / np.array(b.inertia))


def _paper_sliding_ratio(sc, h, v_plus, lam_n, act, kappa=0.0):
    """Closed form of dv+/dv- for a flat box sliding on a plane under the paper's frozen W
    (Sec. III-B, III-D): each sliding corner i linearises to dv + (W_i + rho_i + kappa) dlam_f = 0,
    with W_i = v+/(mu lam_n,i) (the sliding branch) and rho_i = h what_i (the radial term of
    W's |lambda_f| dependence, which the paper keeps); the normal rows hold pitch and roll,
    so m dv+ = m dv- + h sum dlam_f gives 1 / (1 + (h/m) sum_i 1/(W_i + rho_i + kappa))."""
    b = sc.bodies[0]
    tot = 0.0
    for k in range(8):
        if act[k]:
            tot += 1.0 / (v_plus / (sc.mu * lam_n[k]) + h * _corner_what(b, k) + kappa)
    return 1.0 / (1.0 + h / b.mass * tot)


@pytest.mark.parametrize("v", [0.9, 1.5, 3.0])
def test_paper_adjoint_on_sliding_box_closed_form(v):
    """A flat box resting on the plane, pushed to slide (v+ = v- - mu g h > 0): the paper's
    adjoint gives dv+/dv- = 1/(1 + (h/m) sum_i 1/(W_i + h what_i)) (frozen-W linearisation),
    the exact IFT gives 1 (the slide loses mu g h whatever v- is)."""
    sc = S.box_drop_scene()
    h = 0.1
    orc = O.Oracle(sc, _box_cfg())
    s = S.box_drop_state(sc, 0.0, gap=0.0)[:, 0]
    for _ in range(4):
        s = orc.step(s, np.zeros(1), h)["state"]
    s[7] = v
    g = np.zeros(sc.n_state)
    g[7] = 1.0
    rp = orc.step_adjoint(s, np.zeros(1), h, g, mode=O.ADJ_PAPER)
    re = orc.step_adjoint(s, np.zeros(1), h, g, mode=O.ADJ_EXACT)
    v_plus = rp["state"][7]
    assert v_plus == pytest.approx(v - 0.8 * 9.81 * h, abs=1e-9)
    lam = rp["state"][sc.lam_index:].reshape(-1, 3)
    act = rp["ids"] >= 0
    assert act.sum() == 4
    ratio = _paper_sliding_ratio(sc, h, v_plus, lam[:, 0], act)
    assert rp["dstate"][7] == pytest.approx(ratio, rel=1e-5)
    assert ratio < 0.9                                    # a real bias, not a rounding effect
    assert re["dstate"][7] == pytest.approx(1.0, abs=1e-9)


def test_paper_adjoint_box_drop_bias():
    """The box-drop rollout (v0 from seed 0, T = 20): the exact gradient dx_T/dv0 is h; the
    paper's frozen-W adjoint gives h times the landing step's sliding ratio (the box stops
    in step 2, where sticking makes both modes agree), a bias of about -31 %."""
    sc, st = S.box_drop_inputs(0)
    h, T = 0.1, 20
    orc = O.Oracle(sc, S.SolverConfig(budget=50, k_min=4, tol=1e-10, kappa=0.0))
    states = [st[:, 0]]
    for _ in range(T):
        states.append(orc.step(states[-1], np.zeros(1), h)["state"])
    grads = {}
    for mode in (O.ADJ_PAPER, O.ADJ_EXACT):
        g = np.zeros(sc.n_state)
        g[0] = 1.0
        for t in reversed(range(T)):
            g = orc.step_adjoint(states[t], np.zeros(1), h, g, mode=mode)["dstate"]
        grads[mode] = g[7]
    r1 = orc.step(states[0], np.zeros(1), h)
    lam = r1["state"][sc.lam_index:].reshape(-1, 3)
    ratio = _paper_sliding_ratio(sc, h, r1["state"][7], lam[:, 0], r1["ids"] >= 0)
    print(f"box drop dx_T/dv0: exact {grads[O.ADJ_EXACT]:.6f}, paper {grads[O.ADJ_PAPER]:.6f} "
          f"(bias {grads[O.ADJ_PAPER] / h - 1:+.4f})")
    assert grads[O.ADJ_EXACT] == pytest.approx(h, abs=1e-9)
    assert grads[O.ADJ_PAPER] == pytest.approx(h * ratio, rel=1e-5)
    assert -0.35 < grads[O.ADJ_PAPER] / h - 1 < -0.25


def _box_at_compliant_rest(sc, h, kappa, g0=9.81):
    """A flat box at rest on the plane at the depth its compliance gives (each of the four
    bottom corners carries m g / 4 and sits kappa h m g / 4 below the plane), warm-started
    with those impulses: the step returns u+ = 0 and the same impulses."""
    b = sc.bodies[0]
    s = np.zeros(sc.n_state)
    s[2] = b.half_extents[2] - h * kappa * b.mass * g0 / 4.0
    s[3] = 1.0
    lam = np.zeros((sc.n_slots, 3))
    lam[:4, 0] = b.mass * g0 / 4.0                   # slots 0-3: the bottom corners (k & 4 == 0)
    s[sc.lam_index:] = lam.ravel()
    return s


def _damping(sc, h, delta_rel=1e-6):
    """delta = delta_rel mean diag(h J M^-1 J^T) over the 12 rows of the four bottom corners
    of the flat box (normal z, tangents x and y), from the geometry."""
    b = sc.bodies[0]
    hx, hy, hz = b.half_extents
    I = np.array(b.inertia)
    d = []
    for k in range(4):
        rho = np.array([hx if k & 1 else -hx, hy if k & 2 else -hy, -hz])
        for e in np.eye(3)[[2, 0, 1]]:
            a = np.cross(rho, e)
            d.append(h * (1.0 / b.mass + a @ (a / I)))
    return delta_rel * float(np.mean(d))


@pytest.mark.parametrize("kappa", [0.0, 1e-4])
@pytest.mark.parametrize("pullback", [S.PULLBACK_FULL, S.PULLBACK_TRUNCATED])
def test_resting_box_height_gradient_closed_form(kappa, pullback):
    """Sec. IV-D truncated pull-back (and the full one): a box at rest on the plane, loss
    z+.  Raising the box by dz makes the step lower it again through the normal rows; with
    the compliance C = kappa + delta the paper's linearised rows give
    dz+/dz- = C m / (4 h + C m) and dz+/dvz- = h C m / (4 h + C m) (0 for a rigid contact).
    Dropping the contact point's first-order rigid motion from the truncated rows would
    give dz+/dz- = 1 instead."""
    sc = S.box_drop_scene()
    h = 0.1
    cfg = S.SolverConfig(budget=60, k_min=4, tol=1e-12, kappa=kappa, pullback=pullback)
    orc = O.Oracle(sc, cfg)
    s = _box_at_compliant_rest(sc, h, kappa)
    g = np.zeros(sc.n_state)
    g[2] = 1.0
    r = orc.step_adjoint(s, np.zeros(1), h, g)
    assert abs(r["state"][9]) < 1e-12 and r["state"][2] == pytest.approx(s[2], abs=1e-12)
    C = kappa + _damping(sc, h)
    m = sc.bodies[0].mass
    assert r["dstate"][2] == pytest.approx(C * m / (4 * h + C * m), rel=1e-6)
    assert r["dstate"][9] == pytest.approx(h * C * m / (4 * h + C * m), rel=1e-6)
    assert r["dstate"][0] == pytest.approx(0.0, abs=1e-12) and r["dstate"][1] == pytest.approx(0.0, abs=1e-12)


@pytest.mark.parametrize("kappa", [0.0, 1e-4])
def test_truncated_minus_full_is_the_lever_arm_term(kappa):
    """What truncation drops, by hand: for a box at rest on the plane (u+ = 0, lambda_f = 0,
    each bottom corner carrying Lambda/4 = m g/4), the full pull-back differentiates the
    force term -h lambda_n (R rho_i x n) . w_omega of each normal row through R(q-); the
    truncated one holds the lever arm.  Summed over the corners (sum rho_i = -4 hz e_z) the
    difference is d/dq [h Lambda hz ((R e_z)_y w_x - (R e_z)_x w_y)] at R = I, i.e.
    -2 h Lambda hz (w_x, w_y) in the (qx, qy) entries and zero elsewhere, with
    w_omega = -I^-1 dL/domega- (the shared adjoint at omega- = 0)."""
    sc = S.box_drop_scene()
    h = 0.1
    s = _box_at_compliant_rest(sc, h, kappa)
    g = np.random.default_rng(3).normal(size=sc.n_state)
    g[13:] = 0.0
    out = {}
    for pb in (S.PULLBACK_FULL, S.PULLBACK_TRUNCATED):
        orc = O.Oracle(sc, S.SolverConfig(budget=60, k_min=4, tol=1e-12, kappa=kappa, pullback=pb))
        out[pb] = orc.step_adjoint(s, np.zeros(1), h, g)["dstate"]
    d = out[S.PULLBACK_FULL][:13] - out[S.PULLBACK_TRUNCATED][:13]
    b = sc.bodies[0]
    w = -out[S.PULLBACK_FULL][10:13] / np.array(b.inertia)
    lam_tot, hz = b.mass * 9.81, b.half_extents[2]
    expect = np.zeros(13)
    expect[4] = -2.0 * h * lam_tot * hz * w[0]
    expect[5] = -2.0 * h * lam_tot * hz * w[1]
    assert np.abs(expect[4:6]).min() > 1e-7                 # the case exercises the term
    np.testing.assert_allclose(d, expect, rtol=1e-6, atol=1e-9 * np.abs(expect).max())


# --------------------------------------------------------------------------
# friction-coefficient gradient (Eq. (17) with xi = mu)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("v", [1.5, 3.0])
def test_mu_gradient_sliding_box_closed_form(v):
    """A flat box sliding at rest load loses mu g h of speed per step (Sec. III-B,
    timestep-consistent sliding force), so dv+/dmu = -g h exactly; the exact adjoint gives
    it, the paper's frozen W gives 0."""
    sc = S.box_drop_scene()
    h = 0.1
    orc = O.Oracle(sc, _box_cfg())
    s = S.box_drop_state(sc, 0.0, gap=0.0)[:, 0]
    for _ in range(4):
        s = orc.step(s, np.zeros(1), h)["state"]
    s[7] = v
    g = np.zeros(sc.n_state)
    g[7] = 1.0
    assert orc.step_adjoint(s, np.zeros(1), h, g, mode=O.ADJ_EXACT)["dmu"] == pytest.approx(-9.81 * h, rel=1e-7)
    assert orc.step_adjoint(s, np.zeros(1), h, g, mode=O.ADJ_PAPER)["dmu"] == 0.0


def test_mu_gradient_landing_step_closed_form():
    """The box drop's landing step: the box lands (u_z+ = -0.5 m/s) while sliding, the friction
    impulse is mu m (g h - 0.5), so dv_x+/dmu = -(g h - 0.5)."""
    gold = json.load(open(os.path.join(GOLD, "box_drop_closed_form.json")))
    sc, st = S.box_drop_inputs(0)
    g = np.zeros(sc.n_state)
    g[7] = 1.0
    r = O.Oracle(sc, _box_cfg()).step_adjoint(st[:, 0], np.zeros(1), gold["h"], g, mode=O.ADJ_EXACT)
    assert r["dmu"] == pytest.approx(gold["step1_du_x_sliding"] / gold["mu"], rel=1e-7)


def test_mu_gradient_matches_central_differences_on_robot():
    """The exact adjoint's dL/dmu against central differences of the converged step in mu,
    on a skid-steering robot (left wheels forward, right wheels backward) whose eight rim
    contacts all slide; the paper-mode gradient is zero there."""
    import dataclasses
    sc = S.robot_plane_scene()
    h = 0.1
    cfg = S.SolverConfig(budget=60, k_min=4, tol=1e-12, kappa=1e-4)
    orc = O.Oracle(sc, cfg)
    ub = np.array([3.0, -3.0, 3.0, -3.0])
    s = S.robot_box_states(sc, 2, seed=0, phases=False)[:, 1]
    for _ in range(2):
        s = orc.step(s, ub, h)["state"]
    gvec = np.random.default_rng(12).normal(size=sc.n_state)
    gvec[13 * sc.n_bodies:] = 0.0
    r = orc.step_adjoint(s, ub, h, gvec, mode=O.ADJ_EXACT)
    lam = r["state"][sc.contact_lam_index:].reshape(-1, 3)
    act = r["ids"] >= 0
    assert act.sum() == 8 and (np.hypot(lam[act, 1], lam[act, 2]) > 0.99 * sc.mu * lam[act, 0]).all()
    eps = 1e-5
    lp = gvec @ O.Oracle(dataclasses.replace(sc, mu=sc.mu + eps), cfg).step(s, ub, h)["state"]
    lm = gvec @ O.Oracle(dataclasses.replace(sc, mu=sc.mu - eps), cfg).step(s, ub, h)["state"]
    fd = (lp - lm) / (2 * eps)
    assert abs(fd) > 0.1
    assert r["dmu"] == pytest.approx(fd, rel=1e-6)
    assert orc.step_adjoint(s, ub, h, gvec, mode=O.ADJ_PAPER)["dmu"] == 0.0


# --------------------------------------------------------------------------
# servo modes (Eq. (8)) and the prismatic joint: the rig and the cart-pole
# --------------------------------------------------------------------------

def _rig(mode, kd=2.0, kp=50.0, kappa=0.0):
    sc = S.rig_scene(mode=mode, kp=kp, kd=kd)
    orc = O.Oracle(sc, S.SolverConfig(budget=60, k_min=4, tol=1e-12, kappa=kappa))
    s = S.rig_state(sc)[:, 0]
    tgt = np.zeros(2) if mode == S.SERVO_POSITION else np.zeros(2)
    for _ in range(3):
        s = orc.step(s, tgt, 0.1)["state"]           # settle on the plane
    return sc, orc, s


@pytest.mark.parametrize("mode", [S.SERVO_POSITION, S.SERVO_VELOCITY])
def test_prismatic_servo_one_step_closed_form(mode):
    """Eq. (8) on a prismatic joint: the cart (m = 2 kg) slides on a base held by static
    friction, so the servo row J_c u + alpha lambda + b_c = 0 and m dv = h lambda give
    lambda = -(v- + b_c) / (h/m + alpha): position target b_c = (s- - sbar)/h with
    alpha = 1/(kd + h kp); velocity target b_c = -ubar with alpha = 1/kp."""
    h, m, kp, kd = 0.1, 2.0, 50.0, 2.0
    sc, orc, s = _rig(mode)
    nb = sc.n_bodies
    s = s.copy()
    s[7] += 0.05                                      # cart 5 cm along the rail
    s[7 * nb + 6] = 0.2                               # moving at 0.2 m/s
    target = -0.1 if mode == S.SERVO_POSITION else 1.0
    r = orc.step(s, np.array([target, 0.0]), h)
    assert r["status"] == 0
    slide = s[7] - s[0]
    if mode == S.SERVO_POSITION:
        alpha, bc = 1.0 / (kd + h * kp), (slide - target) / h
    else:
        alpha, bc = 1.0 / kp, -target
    lam = -(0.2 + bc) / (h / m + alpha)
    assert r["state"][sc.lam_index + 10] == pytest.approx(lam, rel=1e-9)
    assert r["state"][7 * nb + 6] == pytest.approx(0.2 + h * lam / m, rel=1e-9)
    assert abs(r["state"][7 * nb]) < 1e-12            # the base does not move


def test_revolute_position_servo_one_step_closed_form():
    """Eq. (8), position target, on a wheel turning about its own axle (I = m r^2 / 2):
    the servo row measures the rotation rate of the quaternion update, v = c w with
    c = 1 / (1 + (h w / 2)^2) (the map E of Eq. (1)), and the torque is c lambda, so
    c w + alpha lambda + (theta- - thetabar)/h = 0 with I w = h c lambda; solved here by
    fixed-point iteration on w."""
    h, kp, kd = 0.1, 50.0, 2.0
    sc, orc, s = _rig(S.SERVO_POSITION)
    nb = sc.n_bodies
    tbar = 0.3
    r = orc.step(s, np.array([0.0, tbar]), h)
    I = 0.5 * 1.0 * 0.15 ** 2
    alpha = 1.0 / (kd + h * kp)
    w = 0.0
    for _ in range(200):
        c = 1.0 / (1.0 + (h * w / 2) ** 2)
        lam = (tbar / h) / (h * c * c / I + alpha)
        w = h * c * lam / I
    assert r["state"][sc.lam_index + 11] == pytest.approx(lam, rel=1e-9)
    assert r["state"][7 * nb + 12 + 4] == pytest.approx(w, rel=1e-9)


def test_position_servos_settle_at_their_targets():
    """Implicit PD servos (Eq. (8)) are stable at any gain: both joints reach their targets
    and the servo forces vanish."""
    sc, orc, s = _rig(S.SERVO_POSITION, kp=500.0, kd=5.0)
    tgt = np.array([0.12, -0.7])
    for _ in range(80):
        s = orc.step(s, tgt, 0.1)["state"]
    assert s[7] - s[0] == pytest.approx(0.12, abs=1e-7)
    q = s[17:21]
    assert 2.0 * np.arctan2(q[2], q[0]) == pytest.approx(-0.7, abs=1e-7)
    assert np.abs(s[sc.lam_index + 10:sc.lam_index + 12]).max() < 1e-5


def test_prismatic_row_jacobian_matches_definition():
    """The analytic Jacobian of the prismatic rows (two perpendicular-translation rows, two
    axis-alignment rows, the twist lock) equals the definition d c(q+(u))/du / h, on the
    cart-pole with random velocities."""
    sc = S.cartpole_scene()
    orc = O.Oracle(sc, S.SolverConfig())
    s = S.cartpole_state(sc, tilt=0.3, cart_v=0.4, pole_w=-1.0)[:, 0]
    rng = np.random.default_rng(21)
    u = rng.normal(scale=0.5, size=6 * sc.n_bodies)
    rows = orc.rows(s, np.zeros(1), 0.1, u, np.zeros(sc.m_max))
    jr = rows["meta"][:, 0] == 0
    assert jr.sum() == 10
    np.testing.assert_allclose(rows["J"][jr], rows["Jdual"][jr], rtol=1e-9, atol=1e-9)


def _cartpole_rollout(orc, sc, s0, ctl, h, T):
    states = [s0]
    for t in range(T):
        states.append(orc.step(states[-1], ctl[t:t + 1], h)["state"])
    return states


def test_cartpole_exact_adjoint_matches_fd():
    """Sec. III-D's finite-difference validation on the cart-pole (the paper reports its
    adjoint within 1.6 % over up to 50 steps): the exact adjoint swept back through a
    30-step rollout matches central differences of the rollout in every initial-state
    coordinate and in the cart-velocity targets to 1e-6.  The paper's frozen-W adjoint
    here also drops the joints' geometric stiffness d(J^T lambda)/du, which carries the
    swinging pole; its deviation is printed and recorded, not held to the paper's
    1.6 %.  The base's four coplanar corners make the contact split indeterminate
    without compliance, so kappa = 1e-4 (as the box's FD pins).  The pole starts
    0.15 rad from upright and falls past the horizontal within the horizon."""
    sc = S.cartpole_scene()
    h, T = 0.05, 30
    cfg = S.SolverConfig(budget=60, k_min=4, tol=1e-12, kappa=1e-4)
    orc = O.Oracle(sc, cfg)
    nb = sc.n_bodies
    s0 = S.cartpole_state(sc, tilt=0.15, cart_v=0.1, pole_w=0.3)[:, 0]
    for _ in range(2):                                # base settles on the plane
        s0 = orc.step(s0, np.zeros(1), h)["state"]
    ctl = 0.8 * np.sin(np.arange(T) * 0.3)
    states = _cartpole_rollout(orc, sc, s0, ctl, h, T)
    gT = np.random.default_rng(0).normal(size=sc.n_state)
    gT[13 * nb:] = 0.0
    out = {}
    for mode in (O.ADJ_EXACT, O.ADJ_PAPER):
        g = gT.copy()
        dctl = np.zeros(T)
        for t in reversed(range(T)):
            r = orc.step_adjoint(states[t], ctl[t:t + 1], h, g, mode=mode)
            g, dctl[t] = r["dstate"], r["dubar"][0]
        out[mode] = (g[:13 * nb], dctl)
    eps = 1e-6
    fd_s = np.zeros(13 * nb)
    for i in range(13 * nb):
        e = np.zeros(sc.n_state)
        e[i] = eps
        fd_s[i] = (gT @ _cartpole_rollout(orc, sc, s0 + e, ctl, h, T)[-1]
                   - gT @ _cartpole_rollout(orc, sc, s0 - e, ctl, h, T)[-1]) / (2 * eps)
    ts = [0, 10, 20, 29]
    fd_c = []
    for t in ts:
        e = np.zeros(T)
        e[t] = eps
        fd_c.append((gT @ _cartpole_rollout(orc, sc, s0, ctl + e, h, T)[-1]
                     - gT @ _cartpole_rollout(orc, sc, s0, ctl - e, h, T)[-1]) / (2 * eps))
    fd_c = np.array(fd_c)
    gx, cx = out[O.ADJ_EXACT]
    assert np.abs(gx - fd_s).max() <= 1e-6 * np.abs(fd_s).max()
    assert np.abs(cx[ts] - fd_c).max() <= 1e-6 * np.abs(fd_c).max()
    gp, cp = out[O.ADJ_PAPER]
    dev = max(np.abs(gp - fd_s).max() / np.abs(fd_s).max(), np.abs(cp[ts] - fd_c).max() / np.abs(fd_c).max())
    print(f"cart-pole, {T} steps: paper-mode adjoint deviates {100 * dev:.1f} % from central differences "
          f"(largest entry), the exact adjoint {np.abs(gx - fd_s).max() / np.abs(fd_s).max():.1e}")


def test_position_target_gradient_matches_fd():
    """dL/dthetabar of the position-servo rig through the exact adjoint (the servo row's
    b_c = (x(q-) - target)/h gives dL/dtarget = -w_c/h) against central differences over
    a 10-step rollout (compliant contacts: the base's four coplanar corners need kappa > 0
    for a unique, differentiable impulse split)."""
    sc, orc, s = _rig(S.SERVO_POSITION, kappa=1e-4)
    h, T = 0.1, 10
    tgt = np.array([0.05, 0.4])

    def run(tg):
        st = [s]
        for _ in range(T):
            st.append(orc.step(st[-1], tg, h)["state"])
        return st

    st = run(tgt)
    g = np.zeros(sc.n_state)
    g[7], g[14 + 5] = 1.0, 2.0                       # cart x and a wheel quaternion entry
    dt = np.zeros(2)
    for t in reversed(range(T)):
        r = orc.step_adjoint(st[t], tgt, h, g, mode=O.ADJ_EXACT)
        g, dt = r["dstate"], dt + r["dubar"]
    eps = 1e-6
    for k in range(2):
        e = np.zeros(2)
        e[k] = eps
        fd = (run(tgt + e)[-1][[7, 19]] @ [1.0, 2.0] - run(tgt - e)[-1][[7, 19]] @ [1.0, 2.0]) / (2 * eps)
        assert dt[k] == pytest.approx(fd, rel=1e-6, abs=1e-9)
