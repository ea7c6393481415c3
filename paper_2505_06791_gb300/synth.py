"""Seeded synthetic workloads: arms, collision spheres, obstacle scenes, motion endpoints.

This module only draws inputs. It holds none of the method's arithmetic (no kinematics,
no projection, no collision test); both the CUDA path and the FP64 oracle consume what it
returns. Every floating-point value it returns is rounded to FP32 first (stored in float64
arrays), so the GPU (which computes in FP32) and the oracle (which promotes to FP64) see
bit-identical inputs.

Shapes follow the paper's workloads (cpRRTC, Sec. V): redundant 7-DOF arms carrying
collision spheres, cuboid/sphere/capsule obstacles in front of the base, straight-line
motion segments between joint configurations.

Array conventions (shared with the C-ABI structs and the oracle):
  joints   (dof, 7)  {type (0 revolute, 1 prismatic), d, a, alpha, theta0, lo, hi}
                     standard DH: T_k = Rz(theta0 + q) Tz(d) Tx(a) Rx(alpha)   (revolute)
                                  T_k = Rz(theta0) Tz(d + q) Tx(a) Rx(alpha)   (prismatic)
  ee       (3,)      end-effector point in the last joint frame
  spheres  (S, 5)    {frame, x, y, z, r}; frame 0 = base, frame k = after joint k
  obs_sph  (n, 4)    {x, y, z, r}
  obs_box  (n, 15)   {cx, cy, cz, hx, hy, hz, R00..R22}; world = c + R @ local
  obs_cap  (n, 7)    {p0x, p0y, p0z, p1x, p1y, p1z, r}
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Obstacle region: a 1.2 m cube in front of the base (base at the origin, +x forward).
CUBE_LO = np.array([0.1, -0.6, 0.0])
CUBE_HI = np.array([1.3, 0.6, 1.2])

ALPHA_7 = [-math.pi / 2, math.pi / 2, -math.pi / 2, math.pi / 2, -math.pi / 2, math.pi / 2, 0.0]
SPHERES_PER_BODY_7 = [8, 8, 9, 9, 9, 8, 8]          # 59 spheres on bodies 1..7
SPHERES_PER_BODY_8 = [15, 15, 15, 15, 15, 15, 15, 15]  # 120 spheres on bodies 1..8


def f32(x):
    """Round to the nearest FP32 value, keep float64 storage."""
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


@dataclass
class Robot:
    joints: np.ndarray          # (dof, 7)
    ee: np.ndarray              # (3,)
    spheres: np.ndarray         # (S, 5)

    @property
    def dof(self) -> int:
        return int(self.joints.shape[0])

    @property
    def lo(self) -> np.ndarray:
        return self.joints[:, 5]

    @property
    def hi(self) -> np.ndarray:
        return self.joints[:, 6]


@dataclass
class Scene:
    sph: np.ndarray = field(default_factory=lambda: np.zeros((0, 4)))
    box: np.ndarray = field(default_factory=lambda: np.zeros((0, 15)))
    cap: np.ndarray = field(default_factory=lambda: np.zeros((0, 7)))

    @property
    def n(self) -> int:
        return len(self.sph) + len(self.box) + len(self.cap)


def _body_spheres(rng, frame: int, length: float, count: int) -> list:
    """`count` spheres spread along the body segment [0,0,0] -> [0,0,length] of `frame`."""
    out = []
    for j in range(count):
        t = (j + 0.5) / count
        x, y = rng.uniform(-0.02, 0.02, 2)
        r = rng.uniform(0.03, 0.08)
        out.append([frame, x, y, t * length, r])
    return out


def make_arm7(seed: int = 1, limit: float = 2.8) -> Robot:
    """7-DOF revolute DH arm, alternating twists, body lengths U[0.08, 0.38] m, 59 spheres.

    Joint 1 turns about the world z axis (frame 0 = world). Body k (k = 1..7) spans
    [0,0,0] -> [0,0,d_{k+1}] in frame k (the tool length for body 7).
    """
    rng = np.random.default_rng(seed)
    d = rng.uniform(0.08, 0.38, 7)
    tool = rng.uniform(0.08, 0.20)
    joints = np.zeros((7, 7))
    for k in range(7):
        joints[k] = [0, d[k], 0.0, ALPHA_7[k], 0.0, -limit, limit]
    sph = []
    for body in range(1, 8):
        length = d[body] if body < 7 else tool
        sph += _body_spheres(rng, body, length, SPHERES_PER_BODY_7[body - 1])
    return Robot(f32(joints), f32([0.0, 0.0, tool]), f32(np.array(sph)))


def make_arm6(seed: int = 1) -> Robot:
    """The 7-DOF arm without its last joint (spheres of body 7 move to body 6's tip)."""
    r7 = make_arm7(seed)
    joints = r7.joints[:6].copy()
    sph = r7.spheres.copy()
    tip = r7.joints[6, 1]
    sph = sph[sph[:, 0] <= 6]
    ee = f32([0.0, 0.0, tip])
    return Robot(joints, ee, sph)


def make_arm8(seed: int = 1, limit: float = 2.8) -> Robot:
    """8-DOF: a prismatic vertical torso (0..0.4 m) carrying the 7-DOF arm, 120 spheres."""
    rng = np.random.default_rng(seed + 7919)
    r7 = make_arm7(seed, limit)
    joints = np.zeros((8, 7))
    joints[0] = [1, 0.0, 0.0, 0.0, 0.0, 0.0, 0.4]
    joints[1:] = r7.joints
    d = joints[:, 1]
    tool = r7.ee[2]
    sph = []
    for body in range(1, 9):
        length = d[body] if body < 8 else tool
        sph += _body_spheres(rng, body, length, SPHERES_PER_BODY_8[body - 1])
    return Robot(f32(joints), f32(r7.ee), f32(np.array(sph)))


def _random_rotation(rng) -> np.ndarray:
    """Uniform random rotation from a normalised Gaussian quaternion."""
    w, x, y, z = rng.normal(size=4)
    n = math.sqrt(w * w + x * x + y * y + z * z)
    w, x, y, z = w / n, x / n, y / n, z / n
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def _unit(rng) -> np.ndarray:
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def make_scene(seed: int, n_sph: int = 16, n_box: int = 0, n_cap: int = 0,
               sph_r=(0.05, 0.15), box_side=(0.05, 0.3), cap_len=(0.1, 0.4),
               cap_r=(0.02, 0.08), lo=CUBE_LO, hi=CUBE_HI) -> Scene:
    """Obstacles with centres uniform in the box [lo, hi]."""
    rng = np.random.default_rng(seed)
    sph = np.zeros((n_sph, 4))
    for i in range(n_sph):
        sph[i, :3] = rng.uniform(lo, hi)
        sph[i, 3] = rng.uniform(*sph_r)
    box = np.zeros((n_box, 15))
    for i in range(n_box):
        box[i, :3] = rng.uniform(lo, hi)
        box[i, 3:6] = rng.uniform(*box_side, 3) / 2
        box[i, 6:] = _random_rotation(rng).reshape(-1)
    cap = np.zeros((n_cap, 7))
    for i in range(n_cap):
        c = rng.uniform(lo, hi)
        u = _unit(rng) * rng.uniform(*cap_len) / 2
        cap[i, :3] = c - u
        cap[i, 3:6] = c + u
        cap[i, 6] = rng.uniform(*cap_r)
    return Scene(f32(sph), f32(box), f32(cap))


# Planning workspace around the arm, and the keep-out cylinder around its base (robot
# mount): obstacle centres are drawn outside it.
WORK_LO = np.array([-1.5, -1.5, 0.0])
WORK_HI = np.array([1.5, 1.5, 1.8])
BASE_KEEPOUT = 0.35


def make_planning_scene(seed: int, n_sph: int = 100, n_box: int = 60, n_cap: int = 40,
                        lo=WORK_LO, hi=WORK_HI, keepout: float = BASE_KEEPOUT,
                        scale: float = 1.0) -> Scene:
    """Mixed obstacles for one planning problem: centres uniform in the workspace box,
    redrawn while within `keepout` (m, horizontal) of the base axis. `scale` multiplies every
    obstacle size (sphere radius, box sides, capsule length and radius)."""
    rng = np.random.default_rng(seed)
    sc = make_scene(int(rng.integers(1 << 31)), n_sph, n_box, n_cap, lo=lo, hi=hi,
                    sph_r=(0.05 * scale, 0.15 * scale), box_side=(0.05 * scale, 0.3 * scale),
                    cap_len=(0.1 * scale, 0.4 * scale), cap_r=(0.02 * scale, 0.08 * scale))

    def centre_ok(c):
        return math.hypot(c[0], c[1]) >= keepout

    def redraw(arr, centre_fn, move):
        for i in range(len(arr)):
            while not centre_ok(centre_fn(arr[i])):
                move(arr, i, rng.uniform(lo, hi) - centre_fn(arr[i]))

    def mv_sph(a, i, d):
        a[i, :3] += d

    def mv_box(a, i, d):
        a[i, :3] += d

    def mv_cap(a, i, d):
        a[i, :3] += d
        a[i, 3:6] += d

    sph, box, cap = sc.sph.copy(), sc.box.copy(), sc.cap.copy()
    redraw(sph, lambda r: r[:3], mv_sph)
    redraw(box, lambda r: r[:3], mv_box)
    redraw(cap, lambda r: (r[:3] + r[3:6]) / 2, mv_cap)
    return Scene(f32(sph), f32(box), f32(cap))


def make_subdivided_boxes(seed: int, n_boxes: int = 24, split: int = 1) -> Scene:
    """Axis-aligned boxes with sides U[0.1, 0.4] m, centres uniform in the obstacle cube; each
    box is cut into `split` equal boxes (split = 10: ten slabs along x; 100: a 10 x 10 grid
    in x and y), so the occupied volume stays the same while the primitive count grows (the
    density scaling of Sec. V-A)."""
    rng = np.random.default_rng(seed)
    nx, ny = {1: (1, 1), 10: (10, 1), 100: (10, 10)}[split]
    rows = []
    for _ in range(n_boxes):
        c = rng.uniform(CUBE_LO, CUBE_HI)
        h = rng.uniform(0.1, 0.4, 3) / 2
        for i in range(nx):
            for j in range(ny):
                hx, hy = h[0] / nx, h[1] / ny
                cx = c[0] - h[0] + (2 * i + 1) * hx
                cy = c[1] - h[1] + (2 * j + 1) * hy
                rows.append([cx, cy, c[2], hx, hy, h[2], 1, 0, 0, 0, 1, 0, 0, 0, 1])
    return Scene(box=f32(np.array(rows)))


def make_mixed_scene(seed: int, n_sph: int = 100, n_box: int = 60, n_cap: int = 40) -> Scene:
    """Mixed primitives: spheres r U[0.05,0.15], oriented boxes with sides U[0.05,0.3],
    capsules with length U[0.1,0.4] and radius U[0.02,0.08]."""
    return make_scene(seed, n_sph, n_box, n_cap)


def make_box_surface_cloud(seed: int, n_boxes: int = 12, n_points: int = 4096,
                           radius: float = 0.02) -> Scene:
    """Point-cloud-like sphere obstacles: points uniform (area-weighted) on the surfaces of
    random yawed boxes with sides U[0.1, 0.4] in the obstacle cube."""
    rng = np.random.default_rng(seed)
    boxes = []
    for _ in range(n_boxes):
        c = rng.uniform(CUBE_LO, CUBE_HI)
        h = rng.uniform(0.1, 0.4, 3) / 2
        yaw = rng.uniform(-math.pi, math.pi)
        cy, sy = math.cos(yaw), math.sin(yaw)
        R = np.array([[cy, -sy, 0], [sy, cy, 0], [0, 0, 1.0]])
        boxes.append((c, h, R))
    # face areas: 2 faces per axis
    areas = []
    for c, h, R in boxes:
        a = [4 * h[1] * h[2], 4 * h[0] * h[2], 4 * h[0] * h[1]]
        areas += [a[0], a[0], a[1], a[1], a[2], a[2]]
    areas = np.array(areas)
    face = rng.choice(len(areas), size=n_points, p=areas / areas.sum())
    pts = np.zeros((n_points, 4))
    for i, f in enumerate(face):
        c, h, R = boxes[f // 6]
        axis, sign = (f % 6) // 2, (1.0 if f % 2 == 0 else -1.0)
        local = rng.uniform(-h, h)
        local[axis] = sign * h[axis]
        pts[i, :3] = c + R @ local
        pts[i, 3] = radius
    return Scene(sph=f32(pts))


def uniform_configs(robot: Robot, n: int, seed: int) -> np.ndarray:
    """n configurations uniform within the joint limits, (n, dof), FP32-representable."""
    rng = np.random.default_rng(seed)
    return f32(rng.uniform(robot.lo, robot.hi, size=(n, robot.dof)))


def nearby_configs(robot: Robot, q: np.ndarray, step: float, seed: int) -> np.ndarray:
    """For each row of q, a configuration at L2 distance `step` in a uniform random
    direction, clipped to the limits (short motions like RRT-Connect steering)."""
    rng = np.random.default_rng(seed)
    d = rng.normal(size=q.shape)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return f32(np.clip(q + step * d, robot.lo, robot.hi))


# Constraint presets (type codes shared with the C-ABI and the oracle).
C_NONE, C_ROLL_PITCH, C_Z_PLANE, C_LINE, C_ORIENT_PLANE, C_ORIENT_LINE = 0, 1, 2, 3, 4, 5


@dataclass
class Constraint:
    type: int = C_ROLL_PITCH
    target: float = 0.0        # plane (C_Z_PLANE, C_ORIENT_PLANE) or line (C_LINE, C_ORIENT_LINE) height
    tol_task: float = 1e-4     # ||E_task||_inf threshold
    c_sm: float = 2.0          # tau_step = max(c_sm * ||q1-q0||_inf / (W-1), tau_floor)
    tau_floor: float = 1e-3
    tol_sm: float = 1e-4       # max_k E_sm,k threshold
    alpha: float = 1.0         # step size
    lam: float = 1e-3          # damping of the pseudoinverse
    max_iters: int = 20
    line_y: float = 0.0        # y of the line {y = line_y, z = target} (parallel to x)
    yaw: float = 0.0           # end-effector yaw of the fixed orientation


def line(y0: float = 0.0, z0: float = 0.6, max_iters: int = 20) -> Constraint:
    """End-effector point on the line {y = y0, z = z0}."""
    return Constraint(type=C_LINE, target=z0, line_y=y0, max_iters=max_iters)


def orient_plane(yaw: float = 0.0, z0: float = 0.6, max_iters: int = 20) -> Constraint:
    """Fixed end-effector orientation (roll = pitch = 0, yaw) on the plane z = z0."""
    return Constraint(type=C_ORIENT_PLANE, target=z0, yaw=yaw, max_iters=max_iters)


def orient_line(yaw: float = 0.0, y0: float = 0.0, z0: float = 0.6,
                max_iters: int = 20) -> Constraint:
    """Fixed end-effector orientation on the line {y = y0, z = z0}."""
    return Constraint(type=C_ORIENT_LINE, target=z0, line_y=y0, yaw=yaw, max_iters=max_iters)


def roll_pitch(max_iters: int = 20) -> Constraint:
    return Constraint(type=C_ROLL_PITCH, max_iters=max_iters)


def z_plane(z0: float = 0.9, max_iters: int = 20) -> Constraint:
    return Constraint(type=C_Z_PLANE, target=z0, max_iters=max_iters)


def no_constraint() -> Constraint:
    return Constraint(type=C_NONE)


def make_batch_mix(n: int, seed: int, max_obstacles: int = 5000):
    """Uneven batch: each problem draws a robot (6-, 7- or 8-DOF arm), a constraint (none,
    roll-pitch, z-plane at 0.9 m), W in {16, 32, 64} and an obstacle count log-uniform in
    [10, max_obstacles], split 50/30/20 into spheres, boxes and capsules. Above 200
    obstacles every obstacle is shrunk by (200 / count)^(1/3), keeping the occupied volume
    (like splitting each primitive into smaller ones). Returns robots, constraints, problems
    [(robot, constraint, scene, W)] and scenes (scene p belongs to problem p)."""
    rng = np.random.default_rng(seed)
    robots = [make_arm6(1), make_arm7(1), make_arm8(1)]
    constraints = [no_constraint(), roll_pitch(), z_plane(0.9)]
    problems, scenes = [], []
    for p in range(n):
        r = int(rng.integers(3))
        c = int(rng.integers(3))
        W = (16, 32, 64)[int(rng.integers(3))]
        count = int(round(math.exp(rng.uniform(math.log(10), math.log(max_obstacles)))))
        ns, nb = int(round(0.5 * count)), int(round(0.3 * count))
        nc = max(0, count - ns - nb)
        scale = min(1.0, (200.0 / count) ** (1.0 / 3.0))
        scenes.append(make_planning_scene(seed * 100_003 + p, ns, nb, nc, scale=scale))
        problems.append((r, c, p, W))
    return robots, constraints, problems, scenes


def self_pairs_gap(robot: Robot, gap: int = 2) -> np.ndarray:
    """Self-collision frame pairs: spheres of frames a and b are tested against each other
    when |a - b| >= gap (adjacent links, which touch at their joint, are left out)."""
    n = robot.dof + 1
    a = np.arange(n)
    return (np.abs(a[:, None] - a[None, :]) >= gap).astype(np.uint8)
