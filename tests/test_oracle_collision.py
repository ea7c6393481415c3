"""Pins of the oracle's collision checks (Sec. IV) against brute force, dense sampling of
each primitive and hand-placed contacts."""
import numpy as np
import pytest

from paper_2505_06791_gb300 import synth as S
from tests import indep


def test_sphere_clearance_brute_force(oracle_mod):
    rng = np.random.default_rng(0)
    P = rng.uniform(-1, 1, (5, 3))
    R = rng.uniform(0.01, 0.2, 5)
    O = np.c_[rng.uniform(-1, 1, (5, 3)), rng.uniform(0.01, 0.2, 5)]
    D = np.sqrt(((P[:, None, :] - O[None, :, :3]) ** 2).sum(-1)) - R[:, None] - O[None, :, 3]
    for i in range(5):
        for j in range(5):
            assert abs(oracle_mod.Oracle.clear_sphere(P[i], R[i], O[j]) - D[i, j]) < 1e-15


def _box(rng):
    c = rng.uniform(-0.2, 0.2, 3)
    h = rng.uniform(0.05, 0.2, 3)
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    from scipy.spatial.transform import Rotation as Rot
    R = Rot.from_quat(q).as_matrix()
    return np.r_[c, h, R.reshape(-1)], c, h, R


def test_box_clearance_dense_sampling(oracle_mod):
    rng = np.random.default_rng(1)
    g = np.linspace(-1, 1, 41)
    grid = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    for _ in range(6):
        b, c, h, R = _box(rng)
        pts = c + (grid * h) @ R.T       # dense samples of the solid box
        spacing = np.linalg.norm(2 * h / 40)
        for _ in range(5):
            p = rng.uniform(-0.8, 0.8, 3)
            r = 0.03
            ref = np.sqrt(((pts - p) ** 2).sum(-1)).min() - r
            v = oracle_mod.Oracle.clear_box(p, r, b)
            local = R.T @ (p - c)
            if np.all(np.abs(local) <= h):
                assert v < -r + 1e-15
            else:
                assert ref - spacing <= v <= ref + 1e-12


def test_box_clearance_hand_cases(oracle_mod):
    b = np.r_[[0, 0, 0], [0.1, 0.2, 0.3], np.eye(3).reshape(-1)]
    C = oracle_mod.Oracle
    assert abs(C.clear_box([0.5, 0, 0], 0.1, b) - 0.3) < 1e-15
    assert abs(C.clear_box([0.0, 0.0, 0.0], 0.05, b) - (-0.1 - 0.05)) < 1e-15
    assert abs(C.clear_box([0.4, 0.6, 0], 0.0, b) - 0.5) < 1e-15  # corner region, 3-4-5


def test_capsule_clearance_dense_sampling(oracle_mod):
    rng = np.random.default_rng(2)
    t = np.linspace(0, 1, 20001)[:, None]
    for _ in range(20):
        p0, p1 = rng.uniform(-0.5, 0.5, (2, 3))
        rc = rng.uniform(0.01, 0.1)
        seg = p0 + t * (p1 - p0)
        p = rng.uniform(-1, 1, 3)
        r = rng.uniform(0.01, 0.1)
        ref = np.sqrt(((seg - p) ** 2).sum(-1)).min() - r - rc
        v = oracle_mod.Oracle.clear_capsule(p, r, np.r_[p0, p1, rc])
        assert ref - np.linalg.norm(p1 - p0) / 20000 <= v <= ref + 1e-12


def test_config_clearance_brute_force(oracle_mod):
    rb = S.make_arm7(1)
    sc = S.make_mixed_scene(5, 6, 4, 3)
    orc = oracle_mod.Oracle(rb, sc)
    for q in S.uniform_configs(rb, 4, 3):
        C = indep.sphere_centres(rb.joints, rb.ee, rb.spheres, q)
        best = np.inf
        for (x, y, z), r in zip(C, rb.spheres[:, 4]):
            p = np.array([x, y, z])
            for o in sc.sph:
                best = min(best, np.linalg.norm(p - o[:3]) - r - o[3])
            for bx in sc.box:
                best = min(best, oracle_mod.Oracle.clear_box(p, r, bx))
            for cp in sc.cap:
                best = min(best, oracle_mod.Oracle.clear_capsule(p, r, cp))
        assert abs(orc.config_clearance(q) - best) < 1e-13


def _one_sphere_robot():
    rb = S.make_arm7(1)
    return S.Robot(rb.joints, rb.ee, rb.spheres[-1:].copy())


@pytest.mark.parametrize("offset,expect_first", [(-2e-5, 9), (2e-5, 10)])
def test_validate_first_collision_index_and_strict_contact(oracle_mod, offset, expect_first):
    """An obstacle placed just ahead of waypoint 9's tool sphere, 2e-5 m inside / outside
    contact: waypoint 9 collides or not, and the first colliding waypoint is the one brute
    force finds (the sweep continues into the obstacle)."""
    rb = _one_sphere_robot()
    q0 = np.zeros(7)
    q0[1] = 0.8
    q1 = q0.copy()
    q1[0] = 1.2
    W = 32
    xi = np.asarray(np.linspace(0, 1, W)[:, None] * (q1 - q0) + q0)
    # the motion is on the FP32 grid: the oracle promotes FP32 inputs
    q0f, q1f = np.float32(q0), np.float32(q1)
    xi = q0f.astype(np.float64) + (np.arange(W)[:, None] / (W - 1)) * (
        q1f.astype(np.float64) - q0f.astype(np.float64))
    c9 = indep.sphere_centres(rb.joints, rb.ee, rb.spheres, xi[9])[0]
    c8 = indep.sphere_centres(rb.joints, rb.ee, rb.spheres, xi[8])[0]
    r = rb.spheres[0, 4]
    # obstacle on the far side of waypoint 9 along the direction of travel
    u = (c9 - c8) / np.linalg.norm(c9 - c8)
    rho = 0.05
    centre = c9 + u * (r + rho + offset)
    sc = S.Scene(sph=np.array([[*centre, rho]]))
    orc = oracle_mod.Oracle(rb, sc, S.no_constraint())
    out = orc.validate(q0f[None], q1f[None], W)
    clear = [np.linalg.norm(indep.sphere_centres(rb.joints, rb.ee, rb.spheres, x)[0] - centre)
             - r - rho for x in xi]
    first = next((i for i, v in enumerate(clear) if v < 0), -1)
    assert first == expect_first
    assert out["status"][0] == 2
    assert out["first_fail"][0] == first
    assert abs(out["cc_margin"][0] - min(abs(v) for v in clear[: (first + 1 if first >= 0 else W)])) < 1e-12


@pytest.mark.parametrize("ctype", [1, 2, 4])
def test_segment_check_against_independent_pieces(oracle_mod, ctype):
    """The segment judge used on warm-started segments and planner paths: its largest task
    error (waypoints 1..W-1, independent forward kinematics and Euler angles), its largest
    per-joint step excess over tau, and its smallest clearance (brute force over every
    robot sphere, every obstacle sphere and every waypoint, waypoint 0 included)."""
    rb = S.make_arm7(1)
    c = {1: S.roll_pitch(), 2: S.z_plane(0.9), 4: S.orient_plane(0.5, 0.6)}[ctype]
    sc = S.make_scene(300 + ctype, n_sph=30)
    orc = oracle_mod.Oracle(rb, sc, c)
    rng = np.random.default_rng(310 + ctype)
    q0 = S.uniform_configs(rb, 5, 320 + ctype)
    q1 = S.nearby_configs(rb, q0, 0.4, 330 + ctype)
    for a, b in zip(q0, q1):
        W = 9
        xi = oracle_mod.interpolate(a, b, W) + rng.normal(scale=0.01, size=(W, rb.dof))
        tau = 0.02
        mt, ms, mc = orc.check_segment(xi, tau)
        errs = []
        for i in range(1, W):
            e = indep.task_error(rb.joints, rb.ee, xi[i], c.type, c.target, c.line_y, c.yaw)
            if ctype == 4:  # the yaw row up to its wrap at +-pi
                e[2] = min(abs(e[2]), abs(abs(e[2]) - 2 * np.pi))
            errs.append(np.abs(e).max())
        assert abs(mt - max(errs)) < 1e-12
        assert abs(ms - (np.abs(np.diff(xi, axis=0)) - tau).max()) < 1e-15
        clear = np.inf
        for q in xi:
            C = indep.sphere_centres(rb.joints, rb.ee, rb.spheres, q)
            D = np.sqrt(((C[:, None, :] - sc.sph[None, :, :3]) ** 2).sum(-1))
            clear = min(clear, (D - rb.spheres[:, 4][:, None] - sc.sph[None, :, 3]).min())
        assert abs(mc - clear) < 1e-12


@pytest.mark.parametrize("ctype", [0, 1])
def test_validate_is_projection_then_first_collision(oracle_mod, ctype):
    """The batched validation composes the two stages as Sec. III orders them: Alg. 1 on the
    interpolated segment (its verdict, failing waypoint and iterations), then, for projected
    segments, the smallest waypoint index whose robot spheres overlap an obstacle, found here
    by brute force on independent forward kinematics (waypoint 0 included; with the planner's
    flag it is skipped). Host threads change nothing."""
    rb = S.make_arm7(1)
    c = S.roll_pitch() if ctype == 1 else S.no_constraint()
    sc = S.make_scene(400 + ctype, n_sph=40)
    orc = oracle_mod.Oracle(rb, sc, c)
    starts = []
    for q in S.uniform_configs(rb, 200, 410 + ctype):
        ok, qp, _, _ = orc.project_config(q, max_iters=60)
        if ok or ctype == 0:
            starts.append(qp if ok else q)
        if len(starts) == 24:
            break
    q0 = S.f32(np.array(starts))
    q1 = np.vstack([S.nearby_configs(rb, q0[:12], 0.3, 420 + ctype),
                    S.uniform_configs(rb, 12, 430 + ctype)])
    W = 16
    out = orc.validate(q0, q1, W, n_threads=1)
    par = orc.validate(q0, q1, W, n_threads=5)
    for k in ("status", "first_fail", "iters", "q"):
        assert np.array_equal(out[k], par[k]), k
    skip = orc.validate(q0, q1, W, cc_skip_first=True)
    seen = set()
    for m in range(len(q0)):
        xi = oracle_mod.interpolate(q0[m], q1[m], W)
        if ctype == 1:
            r = orc.project_motion(xi, oracle_mod.tau_step(c, q0[m], q1[m], W))
            if not r["ok"]:
                assert out["status"][m] == 1 and out["first_fail"][m] == r["first_fail"]
                assert out["iters"][m] == r["iters"]
                seen.add(1)
                continue
            xi = r["xi"]
            assert out["iters"][m] == r["iters"]
        assert np.abs(out["q"][m] - xi).max() == 0
        first = -1
        for i in range(W):
            C = indep.sphere_centres(rb.joints, rb.ee, rb.spheres, xi[i])
            D = np.sqrt(((C[:, None, :] - sc.sph[None, :, :3]) ** 2).sum(-1))
            if (D - rb.spheres[:, 4][:, None] - sc.sph[None, :, 3]).min() < 0:
                first = i
                break
        assert out["status"][m] == (2 if first >= 0 else 0)
        assert out["first_fail"][m] == first
        seen.add(out["status"][m])
        if first == 0:  # the planner's form skips waypoint 0 (a tree node)
            assert skip["first_fail"][m] != 0
        else:
            assert skip["first_fail"][m] == first and skip["status"][m] == out["status"][m]
    assert 0 in seen and 2 in seen and (ctype == 0 or 1 in seen)


def test_config_clearance_is_the_minimum_over_every_pair(oracle_mod):
    """A configuration's clearance is the smallest clearance of any (robot sphere, obstacle)
    pair over spheres, boxes and capsules: independent forward kinematics for the sphere
    centres, and the per-primitive clearances pinned above."""
    rb = S.make_arm7(1)
    sc = S.make_scene(501, n_sph=6, n_box=5, n_cap=5)
    orc = oracle_mod.Oracle(rb, sc)
    O = oracle_mod.Oracle
    for q in S.uniform_configs(rb, 6, 502):
        C = indep.sphere_centres(rb.joints, rb.ee, rb.spheres, q)
        best = np.inf
        for c, r in zip(C, rb.spheres[:, 4]):
            for o in sc.sph:
                best = min(best, O.clear_sphere(c, r, o))
            for b in sc.box:
                best = min(best, O.clear_box(c, r, b))
            for cp in sc.cap:
                best = min(best, O.clear_capsule(c, r, cp))
        assert abs(orc.config_clearance(q) - best) < 1e-12
