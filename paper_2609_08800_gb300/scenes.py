"""Seeded synthetic scenes and inputs for the Ostrich per-step solve.

This module is the one place that both the CUDA path and the FP64 oracle take
their inputs from.  It holds scene *data* (masses, inertias, dimensions,
obstacle and terrain geometry, initial states, controls) and the state-layout
convention, and none of the solver's arithmetic: no residual, Jacobian,
contact predicate or Newton step lives here.

The scenes stand in for the paper's workloads (Sec. IV):
  * ``box_drop``   -- one rigid box dropped onto a plane (4 corner contacts),
  * ``robot_box``  -- a four-wheeled robot (chassis + 4 wheel cylinders on
                      revolute joints with velocity servos, Sec. III-B control
                      constraints) driving over a box obstacle,
  * ``terrain``    -- the same robot on a triangle-mesh heightmap (Sec. IV-D).
The paper's real robot model, pallet dataset and terrain seeds are not
available; these are synthetic substitutes with the same structure.

State layout (one world, the CUDA path stores it structure-of-arrays with the
world index fastest, i.e. component ``c`` of world ``w`` at ``c*ld + w``):
    [q: 7 per body (px,py,pz, qw,qx,qy,qz)]
    [u: 6 per body (vx,vy,vz, wx,wy,wz), angular velocity in the world frame]
    [lambda: 5 per joint (3 anchor rows + 2 axis rows)]
    [lambda: 1 per servo joint]
    [lambda: 3 per contact slot (normal, tangent 1, tangent 2)]
Contact slots are fixed per body: 8 per box (its corners), and for a wheel
2 rims x F features, F = 1 on a plane, 4 on the box-obstacle scene
(ground, top, near face, near top edge), 8 on a heightmap (triangles).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

SHAPE_NONE = 0
SHAPE_BOX = 1
SHAPE_WHEEL = 2

ENV_PLANE = 0
ENV_BOX = 1
ENV_HEIGHTMAP = 2

PULLBACK_FULL = 0
PULLBACK_TRUNCATED = 1

# status bits written per world by the step
STATUS_NOT_CONVERGED = 1
STATUS_NONFINITE = 2
STATUS_CONTACT_OVERFLOW = 4


@dataclasses.dataclass
class Body:
    mass: float
    inertia: tuple            # body-frame principal moments (Ixx, Iyy, Izz)
    shape: int = SHAPE_NONE
    half_extents: tuple = (0.0, 0.0, 0.0)   # box
    radius: float = 0.0                     # wheel cylinder radius
    half_width: float = 0.0                 # wheel half width along body y


JOINT_REVOLUTE = 0
JOINT_PRISMATIC = 1
SERVO_VELOCITY = 0
SERVO_POSITION = 1


@dataclasses.dataclass
class Joint:
    """Joint between two bodies.  Revolute: rotation about ``axis_parent`` (parent
    frame) = ``axis_child`` (child frame) through the anchors.  Prismatic: translation
    of the child's anchor along ``axis_parent`` with the orientations locked.
    ``perp_parent`` are two unit vectors orthogonal to ``axis_parent`` (parent frame)
    used by the alignment rows; the same coordinates name the child's reference
    direction.  ``kp`` > 0 adds a servo row on the joint coordinate: a target velocity
    (``servo_mode`` SERVO_VELOCITY, compliance 1/kp) or a target position
    (SERVO_POSITION, compliance 1/(kd + h kp))."""
    parent: int
    child: int
    anchor_parent: tuple
    anchor_child: tuple
    axis_parent: tuple = (0.0, 1.0, 0.0)
    axis_child: tuple = (0.0, 1.0, 0.0)
    perp_parent: tuple = ((1.0, 0.0, 0.0), (0.0, 0.0, 1.0))
    kp: float = 0.0
    type: int = JOINT_REVOLUTE
    servo_mode: int = SERVO_VELOCITY
    kd: float = 0.0


@dataclasses.dataclass
class Env:
    kind: int = ENV_PLANE
    # box obstacle [x0,x1] x [y0,y1] x [0,H]
    box: tuple = (0.0, 0.0, 0.0, 0.0, 0.0)
    # heightmap: heights[i, j] at (origin_x + i*spacing, origin_y + j*spacing)
    heights: Optional[np.ndarray] = None
    spacing: float = 0.0
    origin: tuple = (0.0, 0.0)


LIN_DIRECT, LIN_PCR = 0, 1
PC_JACOBI, PC_BLOCK = 0, 1


@dataclasses.dataclass
class SolverConfig:
    budget: int = 16          # Newton iterations per step (Sec. IV-B: 16)
    k_min: int = 4            # best-iterate floor (Sec. III-C)
    tol: float = 1e-5         # stop when sqrt(merit) < tol (m/s)
    delta_rel: float = 1e-6   # step damping, relative to mean diag(h J M^-1 J^T)
    kappa: float = 1e-4       # contact compliance added to normal/friction rows (s/kg)
    eps_fb: float = 1e-8      # Fischer-Burmeister smoothing (Sec. III-D)
    margin: float = 0.02      # contact activation margin (m)
    line_search: int = 0      # 0: full steps + best iterate (Sec. III-C); 1: backtracking alpha in {1,1/2,1/4,1/8}
    pullback: int = PULLBACK_FULL
    # Schur solve of Eq. (12): LIN_DIRECT (block-arrowhead Cholesky factor) or LIN_PCR
    # (matrix-free preconditioned conjugate residual, the paper's solver)
    linear_solver: int = 0
    precond: int = 0          # PCR preconditioner: PC_JACOBI or PC_BLOCK
    pcr_iters: int = 16       # PCR iterations per Newton step (Sec. IV-B: 16)
    pcr_iters_adj: int = 256  # at most this many PCR iterations in the adjoint's solve
    pcr_rtol_adj: float = 0.0  # adjoint PCR stops at |r| <= rtol |b|; 0: 1e-10 (FP32), 1e-12 (FP64)


@dataclasses.dataclass
class Scene:
    name: str
    bodies: List[Body]
    joints: List[Joint]
    env: Env
    mu: float
    gravity: float = -9.81

    # ---- layout helpers (conventions, not solver arithmetic) ----
    @property
    def n_bodies(self) -> int:
        return len(self.bodies)

    @property
    def n_servos(self) -> int:
        return sum(1 for j in self.joints if j.kp > 0)

    def features_per_rim(self) -> int:
        return {ENV_PLANE: 1, ENV_BOX: 4, ENV_HEIGHTMAP: 8}[self.env.kind]

    def slots_of_body(self, b: int) -> int:
        s = self.bodies[b].shape
        if s == SHAPE_BOX:
            return 8
        if s == SHAPE_WHEEL:
            return 2 * self.features_per_rim()
        return 0

    @property
    def n_slots(self) -> int:
        return sum(self.slots_of_body(b) for b in range(self.n_bodies))

    @property
    def m_max(self) -> int:
        return 5 * len(self.joints) + self.n_servos + 3 * self.n_slots

    @property
    def n_state(self) -> int:
        return 13 * self.n_bodies + self.m_max

    def q_index(self, b: int) -> int:
        return 7 * b

    def u_index(self, b: int) -> int:
        return 7 * self.n_bodies + 6 * b

    @property
    def lam_index(self) -> int:
        return 13 * self.n_bodies

    @property
    def contact_lam_index(self) -> int:
        return self.lam_index + 5 * len(self.joints) + self.n_servos

    @property
    def contact_row_offset(self) -> int:
        """Offset of the first contact row inside the lambda / impulse block."""
        return 5 * len(self.joints) + self.n_servos


# ---------------------------------------------------------------------------
# scene builders
# ---------------------------------------------------------------------------

def _box_inertia(m, a, b, c):
    return (m * (b * b + c * c) / 12.0, m * (a * a + c * c) / 12.0, m * (a * a + b * b) / 12.0)


def _cyl_inertia_y(m, r, w):
    # cylinder with its axis along body y
    ixx = m * (3.0 * r * r + w * w) / 12.0
    return (ixx, 0.5 * m * r * r, ixx)


def box_drop_scene(mu: float = 0.8) -> Scene:
    """Box 0.4 x 0.4 x 0.2 m, 10 kg, on the plane z = 0."""
    m, a, b, c = 10.0, 0.4, 0.4, 0.2
    body = Body(mass=m, inertia=_box_inertia(m, a, b, c), shape=SHAPE_BOX,
                half_extents=(a / 2, b / 2, c / 2))
    return Scene("box_drop", [body], [], Env(ENV_PLANE), mu)


ROBOT_WHEEL_OFFSETS = ((0.25, 0.25, 0.0), (0.25, -0.25, 0.0), (-0.25, 0.25, 0.0), (-0.25, -0.25, 0.0))
ROBOT_WHEEL_RADIUS = 0.15
ROBOT_CHASSIS_Z = 0.15   # chassis centre height with the wheels resting on z = 0


def robot_bodies_joints(kp: float = 50.0):
    chassis = Body(mass=20.0, inertia=_box_inertia(20.0, 0.6, 0.4, 0.15), shape=SHAPE_NONE,
                   half_extents=(0.3, 0.2, 0.075))
    bodies = [chassis]
    joints = []
    for i, off in enumerate(ROBOT_WHEEL_OFFSETS):
        bodies.append(Body(mass=1.0, inertia=_cyl_inertia_y(1.0, ROBOT_WHEEL_RADIUS, 0.08),
                           shape=SHAPE_WHEEL, radius=ROBOT_WHEEL_RADIUS, half_width=0.04))
        joints.append(Joint(parent=0, child=i + 1, anchor_parent=off, anchor_child=(0.0, 0.0, 0.0), kp=kp))
    return bodies, joints


BOX_OBSTACLE = (1.0, 2.0, -1.0, 1.0, 0.15)   # x0, x1, y0, y1, height


def robot_box_scene(mu: float = 0.9, box=BOX_OBSTACLE) -> Scene:
    bodies, joints = robot_bodies_joints()
    return Scene("robot_box", bodies, joints, Env(ENV_BOX, box=tuple(box)), mu)


def robot_plane_scene(mu: float = 0.9) -> Scene:
    bodies, joints = robot_bodies_joints()
    return Scene("robot_plane", bodies, joints, Env(ENV_PLANE), mu)


def heightmap(n: int = 256, spacing: float = 0.05, n_gauss: int = 40, seed: int = 0):
    """Sum of Gaussians: amplitude U[0,0.2] m, sigma U[0.3,1.5] m, centres uniform."""
    rng = np.random.default_rng(seed)
    size = (n - 1) * spacing
    origin = (-0.5 * size, -0.5 * size)
    amp = rng.uniform(0.0, 0.2, n_gauss)
    sig = rng.uniform(0.3, 1.5, n_gauss)
    cx = rng.uniform(origin[0], origin[0] + size, n_gauss)
    cy = rng.uniform(origin[1], origin[1] + size, n_gauss)
    xs = origin[0] + spacing * np.arange(n)
    ys = origin[1] + spacing * np.arange(n)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    H = np.zeros((n, n))
    for k in range(n_gauss):
        H += amp[k] * np.exp(-((X - cx[k]) ** 2 + (Y - cy[k]) ** 2) / (2.0 * sig[k] ** 2))
    # heights are stored in FP32: the contact predicate reads them in FP32 on both sides
    return H.astype(np.float32), spacing, origin


def terrain_scene(mu: float = 1.0, n: int = 256, spacing: float = 0.05, seed: int = 0) -> Scene:
    bodies, joints = robot_bodies_joints()
    H, sp, origin = heightmap(n, spacing, seed=seed)
    return Scene("terrain", bodies, joints, Env(ENV_HEIGHTMAP, heights=H, spacing=sp, origin=origin), mu)


CART_BASE = (1.0, 0.3, 0.1)      # base box (rail) extents, resting on the plane


def rig_scene(mode: int = SERVO_POSITION, kp: float = 50.0, kd: float = 2.0, mu: float = 1.0) -> Scene:
    """Servo test rig: a 1000 kg base box standing on the plane carries a 2 kg cart on a
    prismatic joint along x and a 1 kg wheel cylinder on a revolute joint about y through
    the wheel's centre; both joints have a servo of the given mode.  With the base held by
    static friction each servo drives a single free coordinate."""
    bx, by, bz = CART_BASE
    base = Body(mass=1000.0, inertia=_box_inertia(1000.0, bx, by, bz), shape=SHAPE_BOX,
                half_extents=(bx / 2, by / 2, bz / 2))
    cart = Body(mass=2.0, inertia=_box_inertia(2.0, 0.2, 0.2, 0.1), shape=SHAPE_NONE)
    wheel = Body(mass=1.0, inertia=_cyl_inertia_y(1.0, 0.15, 0.08), shape=SHAPE_NONE)
    joints = [Joint(parent=0, child=1, anchor_parent=(0.0, 0.0, 0.15), anchor_child=(0.0, 0.0, 0.0),
                    axis_parent=(1.0, 0.0, 0.0), axis_child=(1.0, 0.0, 0.0),
                    perp_parent=((0.0, 1.0, 0.0), (0.0, 0.0, 1.0)), kp=kp, type=JOINT_PRISMATIC,
                    servo_mode=mode, kd=kd),
              Joint(parent=0, child=2, anchor_parent=(0.3, 0.3, 0.1), anchor_child=(0.0, 0.0, 0.0), kp=kp,
                    servo_mode=mode, kd=kd)]
    return Scene("rig", [base, cart, wheel], joints, Env(ENV_PLANE), mu)


def rig_state(scene: Scene, slide: float = 0.0, angle: float = 0.0) -> np.ndarray:
    """The rig at rest: base on the plane, the cart displaced by `slide` along the rail,
    the wheel turned by `angle` about its axle."""
    s = np.zeros((scene.n_state, 1))
    bz = CART_BASE[2]
    s[0:7, 0] = (0.0, 0.0, bz / 2, 1.0, 0.0, 0.0, 0.0)
    s[7:14, 0] = (slide, 0.0, bz / 2 + 0.15, 1.0, 0.0, 0.0, 0.0)
    s[14:21, 0] = (0.3, 0.3, bz / 2 + 0.1, math.cos(angle / 2), 0.0, math.sin(angle / 2), 0.0)
    return s


def cartpole_scene(kp: float = 20.0, mu: float = 1.0) -> Scene:
    """Cart-pole: a 1000 kg base box standing on the plane is the rail; a 1 kg cart slides
    on it along x (prismatic joint with a velocity servo, the control) and carries a
    0.5 m, 0.2 kg pole on a revolute joint about y at the cart's centre (unactuated)."""
    bx, by, bz = CART_BASE
    base = Body(mass=1000.0, inertia=_box_inertia(1000.0, bx, by, bz), shape=SHAPE_BOX,
                half_extents=(bx / 2, by / 2, bz / 2))
    cart = Body(mass=1.0, inertia=_box_inertia(1.0, 0.2, 0.2, 0.1), shape=SHAPE_NONE)
    L = 0.5
    pole = Body(mass=0.2, inertia=_box_inertia(0.2, 0.02, 0.02, L), shape=SHAPE_NONE)
    joints = [Joint(parent=0, child=1, anchor_parent=(0.0, 0.0, 0.15), anchor_child=(0.0, 0.0, 0.0),
                    axis_parent=(1.0, 0.0, 0.0), axis_child=(1.0, 0.0, 0.0),
                    perp_parent=((0.0, 1.0, 0.0), (0.0, 0.0, 1.0)), kp=kp, type=JOINT_PRISMATIC),
              Joint(parent=1, child=2, anchor_parent=(0.0, 0.0, 0.0), anchor_child=(0.0, 0.0, -L / 2))]
    return Scene("cartpole", [base, cart, pole], joints, Env(ENV_PLANE), mu)


def cartpole_state(scene: Scene, tilt: float = 0.2, cart_v: float = 0.0, pole_w: float = 0.0) -> np.ndarray:
    """Base on the plane, cart at the rail's centre, the pole tilted by `tilt` about y
    (through the hinge), with cart velocity `cart_v` and pole angular velocity `pole_w`."""
    s = np.zeros((scene.n_state, 1))
    bz = CART_BASE[2]
    L = 0.5
    zc = bz / 2 + 0.15
    s[0:7, 0] = (0.0, 0.0, bz / 2, 1.0, 0.0, 0.0, 0.0)
    s[7:14, 0] = (0.0, 0.0, zc, 1.0, 0.0, 0.0, 0.0)
    c = np.array([math.sin(tilt) * L / 2, 0.0, zc + math.cos(tilt) * L / 2])
    s[14:21, 0] = (*c, math.cos(tilt / 2), 0.0, math.sin(tilt / 2), 0.0)
    nb = scene.n_bodies
    s[7 * nb + 6, 0] = cart_v                      # cart v_x
    # the pole turns about the hinge: v = w x (c - hinge), w = (0, pole_w, 0)
    s[7 * nb + 12: 7 * nb + 15, 0] = np.cross([0.0, pole_w, 0.0], c - np.array([0.0, 0.0, zc]))
    s[7 * nb + 12, 0] += cart_v
    s[7 * nb + 16, 0] = pole_w
    return s


# ---------------------------------------------------------------------------
# initial states (one world per column: array [n_state, W], float64)
# ---------------------------------------------------------------------------

def _yaw_quat(psi):
    return (math.cos(0.5 * psi), 0.0, 0.0, math.sin(0.5 * psi))


def box_drop_state(scene: Scene, v0x: float, gap: float = 0.05) -> np.ndarray:
    s = np.zeros((scene.n_state, 1))
    hz = scene.bodies[0].half_extents[2]
    s[0:3, 0] = (0.0, 0.0, hz + gap)
    s[3:7, 0] = (1.0, 0.0, 0.0, 0.0)
    s[7, 0] = v0x
    return s


def box_drop_inputs(seed: int = 0):
    """Config: box dropped from 0.05 m with a seeded initial velocity v0x ~ U[0,1]."""
    scene = box_drop_scene()
    v0x = float(np.random.default_rng(seed).uniform(0.0, 1.0))
    return scene, box_drop_state(scene, v0x)


def _place_robot(s, scene, w, x, y, z, psi, pitch=0.0):
    # yaw psi about z then pitch about the chassis y axis
    cy, sy = math.cos(0.5 * psi), math.sin(0.5 * psi)
    cp, sp = math.cos(0.5 * pitch), math.sin(0.5 * pitch)
    # q = q_yaw * q_pitch
    qw = cy * cp
    qx = -sy * sp
    qy = cy * sp
    qz = sy * cp
    q = np.array([qw, qx, qy, qz])
    R = _quat_to_matrix(q)
    s[0:3, w] = (x, y, z)
    s[3:7, w] = q
    for i, off in enumerate(ROBOT_WHEEL_OFFSETS):
        b = i + 1
        pw = np.array([x, y, z]) + R @ np.array(off)
        s[7 * b:7 * b + 3, w] = pw
        s[7 * b + 3:7 * b + 7, w] = q


def _quat_to_matrix(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def robot_box_states(scene: Scene, n_worlds: int, seed: int = 0, phases: bool = True) -> np.ndarray:
    """Robots spread over the flat approach, the obstacle face and the obstacle top.

    Phase per world (when ``phases``): 50% flat with x ~ U[-0.6, 0.3],
    25% with the front wheels touching the obstacle face, 25% on the top.
    Yaw ~ U[-0.3, 0.3] everywhere."""
    rng = np.random.default_rng(seed)
    s = np.zeros((scene.n_state, n_worlds))
    x0, x1, y0, y1, H = scene.env.box if scene.env.kind == ENV_BOX else (1.0, 2.0, -1, 1, 0.15)
    r = ROBOT_WHEEL_RADIUS
    for w in range(n_worlds):
        psi = rng.uniform(-0.3, 0.3)
        u = rng.uniform()
        if not phases or u < 0.5:
            _place_robot(s, scene, w, rng.uniform(-0.6, 0.3), 0.0, ROBOT_CHASSIS_Z, psi)
        elif u < 0.75:
            # front wheel rims just touch the face: chassis x so that x_wheel + r ~ x0
            reach = 0.25 * math.cos(psi) + 0.25 * abs(math.sin(psi)) + r
            _place_robot(s, scene, w, x0 - reach - rng.uniform(0.0, 0.01), 0.0, ROBOT_CHASSIS_Z, 0.0)
        else:
            _place_robot(s, scene, w, rng.uniform(x0 + 0.45, x1 - 0.45), 0.0, ROBOT_CHASSIS_Z + H, psi)
    return s


def terrain_states(scene: Scene, n_worlds: int, seed: int = 0) -> np.ndarray:
    """Robots dropped level onto the heightmap, 1 cm above the highest terrain
    point under their wheels, at uniform positions in the central 6 x 6 m."""
    rng = np.random.default_rng(seed)
    env = scene.env
    H = env.heights.astype(np.float64)
    n = H.shape[0]
    s = np.zeros((scene.n_state, n_worlds))
    for w in range(n_worlds):
        x, y = rng.uniform(-3.0, 3.0, 2)
        psi = rng.uniform(-math.pi, math.pi)
        top = -1e9
        for off in ROBOT_WHEEL_OFFSETS:
            wx = x + math.cos(psi) * off[0] - math.sin(psi) * off[1]
            wy = y + math.sin(psi) * off[0] + math.cos(psi) * off[1]
            i0 = int((wx - env.origin[0]) / env.spacing)
            j0 = int((wy - env.origin[1]) / env.spacing)
            patch = H[max(i0 - 4, 0):min(i0 + 5, n), max(j0 - 4, 0):min(j0 + 5, n)]
            top = max(top, float(patch.max()))
        _place_robot(s, scene, w, x, y, top + ROBOT_WHEEL_RADIUS + 0.01, psi)
    return s


def spline_knots(n_worlds: int, n_wheels: int = 4, n_knots: int = 8, seed: int = 0,
                 low: float = -5.0, high: float = 5.0) -> np.ndarray:
    """Wheel-velocity spline knots, uniform in [low, high] rad/s: [n_worlds, n_wheels, n_knots]."""
    return np.random.default_rng(seed).uniform(low, high, (n_worlds, n_wheels, n_knots))


def random_controls(n_servos: int, n_worlds: int, seed: int = 0, low=-5.0, high=5.0) -> np.ndarray:
    """Per-servo target velocities [n_servos, W] for single-step tests."""
    return np.random.default_rng(seed).uniform(low, high, (n_servos, n_worlds))
