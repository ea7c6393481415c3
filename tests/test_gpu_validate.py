"""GPU parity of cprrtc_validate / cprrtc_project_configs (through the C ABI) with the
FP64 oracle on identical seeded inputs."""
import numpy as np
import pytest

from paper_2505_06791_gb300 import synth as S
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_06791_gb300 import build
    build.build()
    return torch


def make_ctx(robot, scene, constraint):
    from paper_2505_06791_gb300.capi import Context
    ctx = Context(0)
    ctx.set_robot(robot)
    ctx.set_obstacles(scene)
    ctx.set_constraint(constraint)
    return ctx


def manifold_starts(orc, robot, n, seed):
    out = []
    for q in S.uniform_configs(robot, 3 * n + 20, seed):
        ok, qp, _, _ = orc.project_config(q, max_iters=60)
        if ok:
            out.append(qp)
        if len(out) == n:
            break
    assert len(out) == n
    return S.f32(np.array(out))


def run_case(torch, oracle_mod, robot, scene, c, q0, q1, W, min_exact=0.8, fail_drift=False):
    ctx = make_ctx(robot, scene, c)
    dq0 = torch.from_numpy(q0.astype(np.float32)).cuda()
    dq1 = torch.from_numpy(q1.astype(np.float32)).cuda()
    out = ctx.validate(dq0, dq1, W)
    torch.cuda.synchronize()
    runs = parity.oracle_runs(oracle_mod.Oracle(robot, scene, c), c, q0, q1, W)
    stats, bad = parity.compare(out, runs, fail_drift=fail_drift)
    ctx.close()
    assert not bad, (stats, bad[:10])
    assert stats["exact"] >= min_exact * stats["n"], stats
    return stats, out, runs[0]


def test_validation_256_motions_full_size_roll_pitch(torch_cuda, oracle_mod):
    """7-DOF arm, 59 spheres, 16 obstacle spheres, 256 motions x 32 waypoints, roll/pitch."""
    rb = S.make_arm7(1)
    sc = S.make_scene(1001, n_sph=16)
    c = S.roll_pitch()
    orc = oracle_mod.Oracle(rb, sc, c)
    q0 = manifold_starts(orc, rb, 256, 1002)
    q1 = S.uniform_configs(rb, 256, 1003)
    stats, out, o = run_case(torch_cuda, oracle_mod, rb, sc, c, q0, q1, 32)
    st = parity.to_np(out["status"])
    assert set(np.unique(st)) <= {0, 1, 2}
    print(stats, np.bincount(st, minlength=3))


def test_short_motions_mixed_obstacles(torch_cuda, oracle_mod):
    """Planner-like 0.3 rad motions among 100 spheres, 60 boxes, 40 capsules."""
    rb = S.make_arm7(1)
    sc = S.make_mixed_scene(2001)
    c = S.roll_pitch()
    orc = oracle_mod.Oracle(rb, sc, c)
    q0 = manifold_starts(orc, rb, 200, 2002)
    q1 = S.nearby_configs(rb, q0, 0.3, 2003)
    stats, out, o = run_case(torch_cuda, oracle_mod, rb, sc, c, q0, q1, 32)
    print(stats, np.bincount(parity.to_np(out["status"]), minlength=3))


@pytest.mark.parametrize("W", [2, 7, 31, 32, 33, 64])
def test_no_constraint_collision_parity(torch_cuda, oracle_mod, W):
    """Projection bypassed: interpolation + FK + CC on all three primitive kinds, with
    ragged waypoint counts around the warp width."""
    rb = S.make_arm7(2)
    sc = S.make_mixed_scene(3001, 20, 12, 8)
    c = S.no_constraint()
    q0 = S.uniform_configs(rb, 150, 3002)
    q1 = np.concatenate([S.nearby_configs(rb, q0[:75], 0.4, 3003), S.uniform_configs(rb, 75, 3004)])
    stats, out, o = run_case(torch_cuda, oracle_mod, rb, sc, c, q0, q1, W, min_exact=0.95)
    gq = parity.to_np(out["q"]).astype(np.float64)
    assert np.abs(gq - o["q"]).max() < 1e-6
    assert (parity.to_np(out["iters"]) == 0).all()


def test_z_plane_eight_dof_long_segments(torch_cuda, oracle_mod):
    """8-DOF arm on a prismatic torso, 120 spheres, z-plane constraint, W = 64 (two
    waypoints per lane)."""
    rb = S.make_arm8(3)
    sc = S.make_scene(4001, n_sph=64, sph_r=(0.02, 0.02))
    c = S.z_plane(0.9)
    orc = oracle_mod.Oracle(rb, sc, c)
    q0 = manifold_starts(orc, rb, 96, 4002)
    q1 = np.concatenate([S.nearby_configs(rb, q0[:48], 0.5, 4003), S.uniform_configs(rb, 48, 4004)])
    stats, out, o = run_case(torch_cuda, oracle_mod, rb, sc, c, q0, q1, 64)
    print(stats)


@pytest.mark.parametrize("W", [40, 64])
def test_roll_pitch_long_segments(torch_cuda, oracle_mod, W):
    """Roll–pitch motions of 40 and 64 waypoints (two per lane) among mixed obstacles match
    the oracle under the parity protocol, with first colliding waypoints on both sides of
    32, and turning early exit off changes nothing."""
    rb = S.make_arm7(1)
    sc = S.make_mixed_scene(4101, 40, 20, 12)
    c = S.roll_pitch()
    orc = oracle_mod.Oracle(rb, sc, c)
    q0 = manifold_starts(orc, rb, 96, 4102)
    q1 = np.concatenate([S.nearby_configs(rb, q0[:64], 0.6, 4103), S.uniform_configs(rb, 32, 4104)])
    stats, out, o = run_case(torch_cuda, oracle_mod, rb, sc, c, q0, q1, W)
    st = parity.to_np(out["status"])
    ff = parity.to_np(out["first_fail"])
    assert (st == 2).sum() >= 10 and (st == 0).sum() >= 5, np.bincount(st, minlength=3)
    # collisions in both of a lane's waypoint slots
    hit = ff[st == 2]
    assert (hit < 32).any() and (hit >= 32).any(), hit
    ctx = make_ctx(rb, sc, c)
    dq0 = torch_cuda.from_numpy(q0.astype(np.float32)).cuda()
    dq1 = torch_cuda.from_numpy(q1.astype(np.float32)).cuda()
    a = {k: parity.to_np(v).copy() for k, v in ctx.validate(dq0, dq1, W).items()}
    ctx.set_early_exit(False)
    b = {k: parity.to_np(v).copy() for k, v in ctx.validate(dq0, dq1, W).items()}
    ctx.close()
    for k in ("status", "first_fail", "iters", "q"):
        assert np.array_equal(a[k], b[k]), k


def test_six_dof_arm_and_tiny_robot(torch_cuda, oracle_mod):
    rb = S.make_arm6(4)
    sc = S.make_mixed_scene(5001, 10, 5, 5)
    c = S.roll_pitch()
    orc = oracle_mod.Oracle(rb, sc, c)
    q0 = manifold_starts(orc, rb, 64, 5002)
    q1 = S.nearby_configs(rb, q0, 0.3, 5003)
    run_case(torch_cuda, oracle_mod, rb, sc, c, q0, q1, 16, min_exact=0.6)
    one = S.Robot(rb.joints, rb.ee, rb.spheres[:1].copy())
    run_case(torch_cuda, oracle_mod, one, sc, S.no_constraint(), q0, q1, 5, min_exact=0.9)


def test_host_and_device_pointers_agree(torch_cuda, oracle_mod):
    rb = S.make_arm7(1)
    sc = S.make_mixed_scene(6001, 30, 10, 10)
    c = S.roll_pitch()
    orc = oracle_mod.Oracle(rb, sc, c)
    q0 = manifold_starts(orc, rb, 40, 6002)
    q1 = S.nearby_configs(rb, q0, 0.3, 6003)
    ctx = make_ctx(rb, sc, c)
    host = ctx.validate(q0.astype(np.float32), q1.astype(np.float32), 32)
    dev = ctx.validate(torch_cuda.from_numpy(q0.astype(np.float32)).cuda(),
                       torch_cuda.from_numpy(q1.astype(np.float32)).cuda(), 32)
    for k in host:
        assert np.array_equal(host[k], parity.to_np(dev[k])), k
    ctx.close()


def test_edge_cases_and_errors(torch_cuda, oracle_mod):
    from paper_2505_06791_gb300 import capi
    rb = S.make_arm7(1)
    ctx = capi.Context(0)
    q = np.zeros((3, 7), np.float32)
    with pytest.raises(capi.CprrtcError) as e:
        ctx.validate(q, q, 32)
    assert e.value.code == capi.E_NOT_CONFIGURED
    ctx.set_robot(rb)
    ctx.set_constraint(S.no_constraint())
    out = ctx.validate(q[:0], q[:0], 32)                    # n = 0: no-op
    assert len(out["status"]) == 0
    out = ctx.validate(q, q, 8)                             # no obstacles at all
    assert (out["status"] == 0).all() and (out["first_fail"] == -1).all()
    for W, code in ((1, capi.E_INVALID_ARG), (65, capi.E_UNSUPPORTED)):
        with pytest.raises(capi.CprrtcError) as e:
            ctx.validate(q, q, W)
        assert e.value.code == code
    bad = S.Constraint(max_iters=0)
    with pytest.raises(capi.CprrtcError):
        ctx.set_constraint(bad)
    ctx.close()


def test_project_configs_parity(torch_cuda, oracle_mod):
    rb = S.make_arm7(1)
    c = S.roll_pitch()
    orc = oracle_mod.Oracle(rb, constraint=c)
    q = S.uniform_configs(rb, 300, 7001)
    ctx = make_ctx(rb, S.Scene(), c)
    out = ctx.project_configs(torch_cuda.from_numpy(q.astype(np.float32)).cuda(), 60)
    gq, gok = parity.to_np(out["q"]), parity.to_np(out["ok"])
    agree = 0
    for i in range(len(q)):
        ok, qp, it, res = orc.project_config(q[i], max_iters=60)
        if ok and gok[i]:
            if np.abs(gq[i] - qp).max() < 1e-4:
                agree += 1
        elif ok == bool(gok[i]):
            agree += 1
    assert agree >= 0.95 * len(q)
    ctx.close()


def test_work_counters_match_outputs(torch_cuda, oracle_mod):
    """The executed-work counters agree with what the outputs imply: every motion that
    reaches collision checking costs one swept-bound chain per waypoint plus at most one
    more in the fused pass (50 obstacles fit one candidate list), tests every obstacle chunk
    against every swept frame bound, and Alg. 1 needs no more than iterations x (W - 1)
    updates."""
    rb = S.make_arm7(1)
    sc = S.make_mixed_scene(8001, 30, 10, 10)
    c = S.roll_pitch()
    orc = oracle_mod.Oracle(rb, sc, c)
    q0 = manifold_starts(orc, rb, 64, 8002)
    q1 = S.nearby_configs(rb, q0, 0.3, 8003)
    ctx = make_ctx(rb, sc, c)
    ctx.work_counters(reset=True)
    out = ctx.validate(torch_cuda.from_numpy(q0.astype(np.float32)).cuda(),
                       torch_cuda.from_numpy(q1.astype(np.float32)).cuda(), 32)
    cnt = ctx.work_counters()
    st, it = (parity.to_np(out[k]).astype(np.int64) for k in ("status", "iters"))
    reached = int((st != 1).sum())
    nb = len(np.unique(rb.spheres[:, 0]))
    assert 0 < cnt[0] <= (it * 31).sum()
    assert 32 * reached <= cnt[1] <= 2 * 32 * reached
    # chunk boxes: 8 obstacles of one kind each
    n_chunks = sum(-(-len(x) // 8) for x in (sc.sph, sc.box, sc.cap))
    assert cnt[3:].sum() >= reached * nb * n_chunks
    assert cnt[2] >= 32 * reached * nb
    ctx.close()


def test_culling_layouts_and_degenerate_primitives(torch_cuda, oracle_mod):
    """Collision parity over obstacle layouts that stress the culling: each kind alone,
    partial chunks of 8 at every kind boundary, more than 32 chunks of one kind, and
    degenerate primitives (zero-radius spheres, zero-extent boxes, zero-length capsules)."""
    rb = S.make_arm7(1)
    c = S.no_constraint()
    q0 = S.uniform_configs(rb, 48, 9100)
    q1 = S.nearby_configs(rb, q0, 0.3, 9101)
    layouts = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (9, 1, 17), (8, 8, 8), (33, 0, 7),
               (0, 257, 0), (300, 20, 1)]
    for k, (a, b, cc) in enumerate(layouts):
        sc = S.make_scene(9200 + k, a, b, cc, sph_r=(0.02, 0.08), box_side=(0.02, 0.2),
                          cap_len=(0.05, 0.3), cap_r=(0.01, 0.05))
        stats, _, _ = run_case(torch_cuda, oracle_mod, rb, sc, c, q0, q1, 32)
        print((a, b, cc), stats)
    # degenerate primitives in the arm's workspace
    rng = np.random.default_rng(9300)
    sph = np.zeros((40, 4))
    sph[:, :3] = rng.uniform(S.CUBE_LO, S.CUBE_HI, (40, 3))
    box = np.zeros((40, 15))
    box[:, :3] = rng.uniform(S.CUBE_LO, S.CUBE_HI, (40, 3))
    box[:, 6:] = np.eye(3).reshape(-1)
    box[::2, 3:6] = rng.uniform(0.0, 0.1, (20, 3)) * (rng.random((20, 3)) < 0.5)
    cap = np.zeros((40, 7))
    cap[:, :3] = rng.uniform(S.CUBE_LO, S.CUBE_HI, (40, 3))
    cap[:, 3:6] = cap[:, :3]
    cap[:, 6] = rng.uniform(0.0, 0.05, 40)
    sc = S.Scene(S.f32(sph), S.f32(box), S.f32(cap))
    stats, out, _ = run_case(torch_cuda, oracle_mod, rb, sc, c, q0, q1, 32)
    print("degenerate", stats)


def test_candidate_list_overflow(torch_cuda, oracle_mod):
    """Thousands of small spheres packed around each motion but clear of the arm: more
    obstacles touch a motion's swept frame bounds than one candidate list holds (512), so
    listing and checking alternate (seen in the chain counter: more than two chains per
    waypoint), and the obstacle stream does not fit shared memory. Every motion is free by
    construction; the verdicts match the oracle's."""
    spatial = pytest.importorskip("scipy.spatial")
    rb = S.make_arm7(1)
    c = S.no_constraint()
    W = 32
    q0 = S.uniform_configs(rb, 16, 9401)
    q1 = S.nearby_configs(rb, q0, 0.3, 9402)
    orc = oracle_mod.Oracle(rb, S.Scene(), c)
    centres = np.concatenate([orc.sphere_centres(x) for a, b in zip(q0, q1)
                              for x in oracle_mod.interpolate(a, b, W)])
    rng = np.random.default_rng(9403)
    r_obs, clear = 0.005, rb.spheres[:, 4].max() + 0.005 + 0.01
    pts = centres[rng.integers(0, len(centres), 120_000)]
    d = rng.normal(size=pts.shape)
    pts = pts + d / np.linalg.norm(d, axis=1, keepdims=True) * rng.uniform(0.1, 0.35, (len(pts), 1))
    near, _ = spatial.cKDTree(centres).query(pts)
    keep = pts[near > clear]
    sph = np.concatenate([keep, np.full((len(keep), 1), r_obs)], axis=1)
    sc = S.Scene(S.f32(sph), np.zeros((0, 15)), np.zeros((0, 7)))
    ctx = make_ctx(rb, sc, c)
    ctx.work_counters(reset=True)
    out = ctx.validate(torch_cuda.from_numpy(q0.astype(np.float32)).cuda(),
                       torch_cuda.from_numpy(q1.astype(np.float32)).cuda(), W)
    torch_cuda.cuda.synchronize()
    chains = int(ctx.work_counters()[1])
    ctx.close()
    runs = parity.oracle_runs(oracle_mod.Oracle(rb, sc, c), c, q0, q1, W, n_threads=8)
    stats, bad = parity.compare(out, runs)
    assert not bad, (stats, bad[:10])
    assert (parity.to_np(out["status"]) == 0).all()
    assert chains > 2 * (W - 1) * len(q0), chains
    print(len(keep), "obstacles", stats, chains)


def test_fp32_peak_measurement(torch_cuda):
    """The FMA-chain measurement lands near the nominal FP32 rate (SMs x 128 x 2 x clock),
    below it by no more than clock and issue losses, and not above it by more than the
    clock's rounding."""
    from paper_2505_06791_gb300.capi import Context
    ctx = Context(0)
    t = ctx.measure_fp32_peak()
    sm = torch_cuda.cuda.get_device_properties(0).multi_processor_count
    nominal = sm * 128 * 2 * 2.2e9 / 1e12  # above any SM clock of this GPU
    assert 0.3 * nominal < t < 1.05 * nominal, (t, nominal)
    print("fp32 peak", t, "TFLOP/s")
    ctx.close()


NEW_CONSTRAINTS = {3: lambda: S.line(0.1, 0.6), 4: lambda: S.orient_plane(0.5, 0.6),
                   5: lambda: S.orient_line(-0.4, 0.1, 0.6)}


@pytest.mark.parametrize("ctype", [3, 4, 5])
def test_line_and_fixed_orientation_parity(torch_cuda, oracle_mod, ctype):
    """The paper's other constraint variants (Sec. V-B: a line; a fixed orientation with a
    plane or a line; 2, 4 and 5 task rows, Cholesky-solved damped steps): strict parity with
    the oracle on planner-like 0.3 rad motions; on long motions, which mostly fail to
    project, the give-up waypoint of a failing projection may drift with four or five task
    rows (ill-conditioned damped system), for at most 5 % of the motions."""
    rb = S.make_arm7(1)
    sc = S.make_mixed_scene(9500 + ctype, 40, 20, 10)
    c = NEW_CONSTRAINTS[ctype]()
    orc = oracle_mod.Oracle(rb, sc, c)
    q0 = manifold_starts(orc, rb, 96, 9510 + ctype)
    short = S.nearby_configs(rb, q0, 0.3, 9520 + ctype)
    far = S.uniform_configs(rb, 96, 9530 + ctype)
    for q1, drift in ((short, False), (far, ctype >= 4)):
        stats, out, _ = run_case(torch_cuda, oracle_mod, rb, sc, c, q0, q1, 32, min_exact=0.7,
                                 fail_drift=drift)
        assert stats["fail_drift"] <= 0.05 * stats["n"], stats
        print(ctype, stats, np.bincount(parity.to_np(out["status"]), minlength=3))


@pytest.mark.parametrize("ctype", [3, 4, 5])
def test_line_and_fixed_orientation_single_config_projection(torch_cuda, oracle_mod, ctype):
    """cprrtc_project_configs for the new constraints, from uniform configurations (up to 60
    damped steps): the oracle's success verdict on at least 90 %, every GPU success on the
    manifold, and converged points within 1e-4 of the oracle's for the line (two rows). With
    four or five rows the steps drift along the null space, differently in FP32 and FP64,
    over tens of iterations: the two land on different points of the manifold."""
    rb = S.make_arm7(1)
    c = NEW_CONSTRAINTS[ctype]()
    orc = oracle_mod.Oracle(rb, constraint=c)
    q = S.uniform_configs(rb, 300, 9600 + ctype)
    ctx = make_ctx(rb, S.Scene(), c)
    out = ctx.project_configs(torch_cuda.from_numpy(q.astype(np.float32)).cuda(), 60)
    gq, gok = parity.to_np(out["q"]), parity.to_np(out["ok"])
    verdict, both, close = 0, 0, 0
    for i in range(len(q)):
        ok, qp, it, res = orc.project_config(q[i], max_iters=60)
        verdict += ok == bool(gok[i])
        if gok[i]:
            e, _ = orc.task(gq[i].astype(np.float64))
            assert np.abs(e).max() < 2 * c.tol_task
        if ok and gok[i]:
            both += 1
            close += np.abs(gq[i] - qp).max() < 1e-4
    assert verdict >= 0.9 * len(q), verdict
    if ctype == 3:
        assert close >= 0.95 * both, (close, both)
    print(ctype, "verdicts", verdict, "both projected", both, "within 1e-4", close)
    ctx.close()


def test_early_exit_ablation_gives_identical_outputs(torch_cuda, oracle_mod):
    """With early termination switched off every waypoint meets every candidate obstacle:
    more primitive tests, the same outputs (status, first colliding waypoint, waypoints), on
    sparse and subdivided (dense) box scenes and on mixed primitives."""
    rb, c = S.make_arm7(1), S.roll_pitch()
    orc = oracle_mod.Oracle(rb, constraint=c)
    q0 = manifold_starts(orc, rb, 128, 9800)
    q1 = S.nearby_configs(rb, q0, 0.3, 9801)
    far = S.uniform_configs(rb, 128, 9802)
    for sc in (S.make_subdivided_boxes(41, 24, 1), S.make_subdivided_boxes(41, 24, 100),
               S.make_mixed_scene(9803)):
        ctx = make_ctx(rb, sc, c)
        for end in (q1, far):
            d0 = torch_cuda.from_numpy(q0.astype(np.float32)).cuda()
            d1 = torch_cuda.from_numpy(end.astype(np.float32)).cuda()
            res = {}
            for early in (True, False):
                ctx.set_early_exit(early)
                ctx.work_counters(reset=True)
                out = {k: parity.to_np(v) for k, v in ctx.validate(d0, d1, 32).items()}
                res[early] = (out, ctx.work_counters())
            for k in ("status", "first_fail", "q", "iters"):
                assert np.array_equal(res[True][0][k], res[False][0][k]), k
            tests_on, tests_off = res[True][1][3:].sum(), res[False][1][3:].sum()
            assert tests_off >= tests_on
            if (res[True][0]["status"] == 2).any():
                assert tests_off > tests_on
        ctx.close()


def test_sequential_projection_parity(torch_cuda, oracle_mod):
    """The naive baseline's sequential projection (cpRRTC-Naive, Sec. V) on the GPU against
    the oracle's: the same verdict and failing waypoint, projected waypoints within 1e-4, the
    same total number of damped steps, on short and long roll-pitch motions (at least 95 %:
    FP32 and FP64 may take a threshold decision differently); collision verdicts of the
    projected motions agree with the oracle's clearances."""
    rb, c = S.make_arm7(1), S.roll_pitch()
    sc = S.make_mixed_scene(9900, 30, 10, 10)
    orc = oracle_mod.Oracle(rb, sc, c)
    q0 = manifold_starts(orc, rb, 96, 9901)
    W = 32
    for q1 in (S.nearby_configs(rb, q0, 0.3, 9902), S.uniform_configs(rb, 96, 9903)):
        ctx = make_ctx(rb, sc, c)
        ctx.set_projection(True)
        out = {k: parity.to_np(v) for k, v in ctx.validate(
            torch_cuda.from_numpy(q0.astype(np.float32)).cuda(),
            torch_cuda.from_numpy(q1.astype(np.float32)).cuda(), W).items()}
        ctx.close()
        agree = 0
        for m in range(len(q0)):
            xi = oracle_mod.interpolate(S.f32(q0[m]), S.f32(q1[m]), W)
            tau = oracle_mod.tau_step(c, S.f32(q0[m]), S.f32(q1[m]), W)
            ok, xo, ff, tot = orc.project_motion_sequential(xi, tau)
            g_ok = out["status"][m] != 1
            same = ok == g_ok and int(out["iters"][m]) == min(tot, 255)
            if same and not ok:
                same = int(out["first_fail"][m]) == ff
            if same and ok:
                same = np.abs(out["q"][m].astype(np.float64) - xo).max() < 1e-4
                if same:  # collision verdict on the GPU's own waypoints
                    cl = np.array([orc.config_clearance(x) for x in out["q"][m]])
                    hit = np.nonzero(cl < 0)[0]
                    ref_ff = int(hit[0]) if len(hit) else -1
                    if np.abs(cl).min() > 1e-5:
                        assert int(out["first_fail"][m]) == ref_ff, (m, ref_ff, out["first_fail"][m])
            agree += same
        assert agree >= 0.95 * len(q0), agree
        print("sequential agreement", agree, "of", len(q0),
              np.bincount(out["status"], minlength=3))


@pytest.mark.parametrize("constrained", [False, True])
def test_self_collision_parity(torch_cuda, oracle_mod, constrained):
    """Self-collision (spheres of frames two or more apart) after the obstacle check: status
    and first colliding waypoint under the parity protocol against the oracle, whose
    clearance then includes the robot's own sphere pairs; switching it off restores the
    plain outputs."""
    rb = S.make_arm7(1)
    pairs = S.self_pairs_gap(rb, 2)
    sc = S.make_mixed_scene(9990, 20, 10, 10)
    c = S.roll_pitch() if constrained else S.no_constraint()
    orc = oracle_mod.Oracle(rb, sc, c, self_pairs=pairs)
    q0 = manifold_starts(oracle_mod.Oracle(rb, sc, c), rb, 128, 9991) if constrained \
        else S.uniform_configs(rb, 128, 9991)
    q1 = S.uniform_configs(rb, 128, 9992)
    ctx = make_ctx(rb, sc, c)
    d0 = torch_cuda.from_numpy(q0.astype(np.float32)).cuda()
    d1 = torch_cuda.from_numpy(q1.astype(np.float32)).cuda()
    plain = {k: parity.to_np(v) for k, v in ctx.validate(d0, d1, 32).items()}
    ctx.set_self_collision(pairs)
    out = ctx.validate(d0, d1, 32)
    torch_cuda.cuda.synchronize()
    runs = parity.oracle_runs(orc, c, q0, q1, 32)
    stats, bad = parity.compare(out, runs)
    assert not bad, (stats, bad[:10])
    got = {k: parity.to_np(v) for k, v in out.items()}
    changed = (got["status"] != plain["status"]) | (got["first_fail"] != plain["first_fail"])
    assert changed.sum() >= 5, changed.sum()  # the folding arm hits itself
    # the planner runs with it (its paths are re-validated with the pairs in test_gpu_plan);
    # the binding refuses arrays of another element type instead of passing their bytes on
    with pytest.raises(TypeError):
        ctx.plan(q0[:2], q1[:2], ctx.plan_params(use_scene_batch=False))
    ctx.plan(q0[:2].astype(np.float32), q1[:2].astype(np.float32),
             ctx.plan_params(use_scene_batch=False, max_rounds=20))
    ctx.set_self_collision(None)
    again = {k: parity.to_np(v) for k, v in ctx.validate(d0, d1, 32).items()}
    for k in ("status", "first_fail", "q"):
        assert np.array_equal(again[k], plain[k]), k
    print(stats, "self-collision changed", int(changed.sum()), "motions")
    ctx.close()


@pytest.mark.parametrize("ctype", [3, 4, 5])
def test_new_constraints_on_the_prismatic_arm(torch_cuda, oracle_mod, ctype):
    """The generic task columns of a prismatic joint (linear velocity along its axis, no
    angular part): parity on the 8-DOF arm's planner-like motions."""
    rb = S.make_arm8(1)
    c = NEW_CONSTRAINTS[ctype]()
    sc = S.make_mixed_scene(9970 + ctype, 30, 10, 10)
    orc = oracle_mod.Oracle(rb, sc, c)
    q0 = manifold_starts(orc, rb, 64, 9975 + ctype)
    q1 = S.nearby_configs(rb, q0, 0.3, 9980 + ctype)
    stats, out, _ = run_case(torch_cuda, oracle_mod, rb, sc, c, q0, q1, 32, min_exact=0.7)
    print(ctype, stats)
