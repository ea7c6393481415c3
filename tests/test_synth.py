"""The seeded input generators draw what the workload recipe says: robot tables with the
stated DOF, joint types, limits and sphere counts, obstacles of the stated counts, sizes and
regions, boxes subdivided at constant occupied volume, endpoints inside the joint limits,
the uneven batch's mix, and every value FP32-representable and reproducible from its seed.
"""
import math

import numpy as np
import pytest

from paper_2505_06791_gb300 import synth as S


def is_f32(a):
    a = np.asarray(a, np.float64)
    return np.array_equal(a, a.astype(np.float32).astype(np.float64))


def sphere_bodies(rb):
    """Body length of each sphere's frame: the next joint's offset d, the tool for the last."""
    d = rb.joints[:, 1]
    lengths = np.append(d[1:], rb.ee[2])
    return lengths[rb.spheres[:, 0].astype(int) - 1]


@pytest.mark.parametrize("make, dof, n_sph", [(S.make_arm6, 6, None), (S.make_arm7, 7, 59),
                                              (S.make_arm8, 8, 120)])
def test_robot_tables(make, dof, n_sph):
    rb = make(1)
    assert rb.dof == dof and rb.joints.shape == (dof, 7) and rb.ee.shape == (3,)
    assert is_f32(rb.joints) and is_f32(rb.ee) and is_f32(rb.spheres)
    if n_sph is not None:
        assert len(rb.spheres) == n_sph
    fr = rb.spheres[:, 0]
    assert np.array_equal(fr, np.sort(fr)) and fr.min() >= 1 and fr.max() <= dof
    assert np.all((rb.spheres[:, 4] >= S.f32(0.03)) & (rb.spheres[:, 4] <= S.f32(0.08)))
    assert np.all(np.abs(rb.spheres[:, 1:3]) <= S.f32(0.02))
    # spheres lie along their body segment [0, 0, 0] -> [0, 0, length]
    z, L = rb.spheres[:, 3], sphere_bodies(rb)
    assert np.all((z > 0) & (z < L))
    rev = rb.joints[:, 0] == 0
    assert np.allclose(rb.joints[rev, 5], -2.8, atol=1e-6)
    assert np.allclose(rb.joints[rev, 6], 2.8, atol=1e-6)
    arm = rb.joints[rev]
    assert np.all(arm[:, 2] == 0) and np.all(arm[:, 4] == 0)  # a = 0, theta0 = 0
    # twists alternate -pi/2, +pi/2 from the base; the 7-DOF chain's last is 0
    alpha = arm[:, 3]
    assert np.allclose(alpha[:6], [(-1) ** (k + 1) * math.pi / 2 for k in range(6)], atol=1e-6)
    if len(alpha) == 7:
        assert alpha[6] == 0


def test_arm_family_shares_the_seven_dof_chain():
    r6, r7, r8 = S.make_arm6(1), S.make_arm7(1), S.make_arm8(1)
    assert np.array_equal(r6.joints, r7.joints[:6])
    assert np.array_equal(r8.joints[1:], r7.joints)
    assert r8.joints[0, 0] == 1 and r8.joints[0, 5] == 0 and r8.joints[0, 6] == S.f32(0.4)
    assert np.all(r7.joints[:, 0] == 0)
    ds = r7.joints[:, 1]
    assert np.all((ds >= S.f32(0.08)) & (ds <= S.f32(0.38)))
    assert S.f32(0.08) <= r7.ee[2] <= S.f32(0.20) and r7.ee[0] == 0 and r7.ee[1] == 0
    assert np.all(r6.spheres[:, 0] <= 6)


@pytest.mark.parametrize("fn, args", [
    (S.make_arm7, (3,)), (S.make_scene, (5, 16, 4, 4)), (S.make_planning_scene, (6,)),
    (S.make_subdivided_boxes, (7, 24, 10)), (S.make_box_surface_cloud, (8, 12, 256)),
])
def test_same_seed_same_input(fn, args):
    a, b = fn(*args), fn(*args)
    c = fn(args[0] + 1, *args[1:])
    fa = [getattr(a, k) for k in vars(a)]
    fb = [getattr(b, k) for k in vars(b)]
    fc = [getattr(c, k) for k in vars(c)]
    assert all(np.array_equal(x, y) for x, y in zip(fa, fb))
    assert not all(np.array_equal(x, y) for x, y in zip(fa, fc) if x.size)


def test_obstacle_scene_sizes_and_region():
    sc = S.make_scene(11, 200, 150, 120)
    assert sc.sph.shape == (200, 4) and sc.box.shape == (150, 15) and sc.cap.shape == (120, 7)
    assert is_f32(sc.sph) and is_f32(sc.box) and is_f32(sc.cap)
    lo, hi = S.f32(S.CUBE_LO), S.f32(S.CUBE_HI)
    assert np.all((sc.sph[:, :3] >= lo) & (sc.sph[:, :3] <= hi))
    assert np.all((sc.sph[:, 3] >= S.f32(0.05)) & (sc.sph[:, 3] <= S.f32(0.15)))
    assert np.all((sc.box[:, :3] >= lo) & (sc.box[:, :3] <= hi))
    assert np.all((sc.box[:, 3:6] >= S.f32(0.025)) & (sc.box[:, 3:6] <= S.f32(0.15)))
    for row in sc.box:
        R = row[6:].reshape(3, 3)
        assert np.abs(R @ R.T - np.eye(3)).max() < 1e-6 and np.linalg.det(R) > 0
    mid = (sc.cap[:, :3] + sc.cap[:, 3:6]) / 2
    length = np.linalg.norm(sc.cap[:, 3:6] - sc.cap[:, :3], axis=1)
    assert np.all((mid >= lo - 1e-6) & (mid <= hi + 1e-6))
    assert np.all((length >= 0.1 - 1e-6) & (length <= 0.4 + 1e-6))
    assert np.all((sc.cap[:, 6] >= S.f32(0.02)) & (sc.cap[:, 6] <= S.f32(0.08)))
    # uniform centres: each half of the cube along x holds about half of them
    frac = np.mean(sc.sph[:, 0] < (lo[0] + hi[0]) / 2)
    assert 0.35 < frac < 0.65


def test_planning_scene_keeps_the_base_clear():
    sc = S.make_planning_scene(12)
    assert (len(sc.sph), len(sc.box), len(sc.cap)) == (100, 60, 40)
    lo, hi = S.WORK_LO - 1e-6, S.WORK_HI + 1e-6
    for centres in (sc.sph[:, :3], sc.box[:, :3], (sc.cap[:, :3] + sc.cap[:, 3:6]) / 2):
        assert np.all(np.hypot(centres[:, 0], centres[:, 1]) >= S.BASE_KEEPOUT - 1e-6)
        assert np.all((centres >= lo) & (centres <= hi))
    small = S.make_planning_scene(12, scale=0.5)
    assert np.all(small.sph[:, 3] <= S.f32(0.075)) and np.all(small.box[:, 3:6] <= 0.075 + 1e-6)


def test_subdivided_boxes_keep_the_occupied_volume():
    """Cutting each box into 10 or 100 equal pieces changes the primitive count only: the
    pieces are axis-aligned, disjoint, and fill their parent box exactly."""
    scenes = {s: S.make_subdivided_boxes(21, 24, s) for s in (1, 10, 100)}
    for s, sc in scenes.items():
        assert sc.box.shape == (24 * s, 15) and len(sc.sph) == 0 and len(sc.cap) == 0
        assert np.all(sc.box[:, 6:] == np.eye(3).reshape(-1))
    parent = scenes[1].box
    vol = lambda b: 8 * np.prod(b[:, 3:6], axis=1)
    for s in (10, 100):
        pieces = scenes[s].box.reshape(24, s, 15)
        for p in range(24):
            lo_p, hi_p = parent[p, :3] - parent[p, 3:6], parent[p, :3] + parent[p, 3:6]
            lo_c = pieces[p, :, :3] - pieces[p, :, 3:6]
            hi_c = pieces[p, :, :3] + pieces[p, :, 3:6]
            assert np.all(lo_c >= lo_p - 1e-6) and np.all(hi_c <= hi_p + 1e-6)
            assert abs(vol(pieces[p]).sum() - vol(parent[p:p + 1])[0]) < 1e-6 * vol(parent[p:p + 1])[0] + 1e-12
            # pairwise disjoint interiors: on some axis the intervals do not overlap
            ov = np.minimum(hi_c[:, None], hi_c[None]) - np.maximum(lo_c[:, None], lo_c[None])
            inside = np.all(ov > 1e-6, axis=2)
            np.fill_diagonal(inside, False)
            assert not inside.any()
    sides = 2 * parent[:, 3:6]
    assert np.all((sides >= S.f32(0.1) - 1e-6) & (sides <= S.f32(0.4) + 1e-6))


def test_box_surface_cloud():
    sc = S.make_box_surface_cloud(31)
    assert sc.sph.shape == (4096, 4) and len(sc.box) == 0 and len(sc.cap) == 0
    assert np.all(sc.sph[:, 3] == S.f32(0.02))
    # every point lies on a box surface near the cube (half-diagonal of a 0.4 m box)
    reach = 0.2 * math.sqrt(3) + 1e-6
    assert np.all(sc.sph[:, :3] >= S.CUBE_LO - reach) and np.all(sc.sph[:, :3] <= S.CUBE_HI + reach)
    # the boxes are only yawed, so their top and bottom faces are horizontal: the points
    # drawn on them share one of 24 heights (about a third of the area)
    _, cnt = np.unique(sc.sph[:, 2], return_counts=True)
    assert np.sort(cnt)[-24:].sum() > 0.15 * len(sc.sph)


def test_endpoints_within_limits():
    rb = S.make_arm8(1)
    q = S.uniform_configs(rb, 4000, 41)
    assert q.shape == (4000, 8) and is_f32(q)
    assert np.all((q >= rb.lo) & (q <= rb.hi))
    span = rb.hi - rb.lo
    assert np.all(q.min(axis=0) < rb.lo + 0.01 * span) and np.all(q.max(axis=0) > rb.hi - 0.01 * span)
    q1 = S.nearby_configs(rb, q, 0.3, 42)
    assert is_f32(q1) and np.all((q1 >= rb.lo) & (q1 <= rb.hi))
    step = np.linalg.norm(q1 - q, axis=1)
    assert np.all(step <= 0.3 + 1e-5)
    inner = np.all((q1 > rb.lo) & (q1 < rb.hi), axis=1)
    assert inner.mean() > 0.5
    assert np.allclose(step[inner], 0.3, atol=1e-5)


def test_uneven_batch_mix():
    robots, cons, problems, scenes = S.make_batch_mix(300, 51)
    assert [r.dof for r in robots] == [6, 7, 8]
    assert [c.type for c in cons] == [S.C_NONE, S.C_ROLL_PITCH, S.C_Z_PLANE]
    assert len(problems) == len(scenes) == 300
    counts = []
    for (r, c, p, W), sc in zip(problems, scenes):
        assert r in (0, 1, 2) and c in (0, 1, 2) and W in (16, 32, 64)
        n = sc.n
        assert 10 <= n <= 5000
        assert abs(len(sc.sph) - 0.5 * n) <= 1 and abs(len(sc.box) - 0.3 * n) <= 1
        scale = min(1.0, (200.0 / n) ** (1.0 / 3.0))
        assert np.all(sc.sph[:, 3] <= 0.15 * scale + 1e-6)
        counts.append(n)
    logs = np.log(counts)
    # log-uniform in [10, 5000]: about a third below exp(mid-third boundary)
    edge = math.log(10) + (math.log(5000) - math.log(10)) / 3
    assert 0.2 < np.mean(logs < edge) < 0.45
    for col, k in ((0, 3), (1, 3), (3, 3)):
        vals = [pr[col] for pr in problems]
        assert len(set(vals)) == k


def test_self_pairs_and_constraint_presets():
    rb = S.make_arm7(1)
    m = S.self_pairs_gap(rb, 2)
    assert m.shape == (8, 8) and m.dtype == np.uint8
    assert np.array_equal(m, m.T) and not np.diag(m).any()
    assert not any(m[a, a + 1] for a in range(7)) and m[0, 2] and m[0, 7]
    c = S.line(0.1, 0.6)
    assert (c.type, c.target, c.line_y) == (S.C_LINE, 0.6, 0.1)
    c = S.orient_plane(0.5, 0.6)
    assert (c.type, c.target, c.yaw) == (S.C_ORIENT_PLANE, 0.6, 0.5)
    c = S.orient_line(-0.4, 0.1, 0.6)
    assert (c.type, c.target, c.line_y, c.yaw) == (S.C_ORIENT_LINE, 0.6, 0.1, -0.4)
    assert S.z_plane().target == 0.9 and S.roll_pitch().type == S.C_ROLL_PITCH
