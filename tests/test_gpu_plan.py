"""GPU RRT-Connect (cprrtc_plan) through the C ABI: every returned path is re-validated by
the FP64 oracle, runs are deterministic for a seed, and the device Philox4x32-10 matches the
oracle's bit for bit."""
import os

import numpy as np
import pytest

from paper_2505_06791_gb300 import synth as S
from tests import problems as PB

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_06791_gb300 import build
    build.build()
    return torch


def ctx_for(robot, constraint):
    from paper_2505_06791_gb300.capi import Context
    ctx = Context(0)
    ctx.set_robot(robot)
    ctx.set_constraint(constraint)
    return ctx


def test_philox_matches_oracle(torch_cuda, oracle_mod):
    ctx = ctx_for(S.make_arm7(1), S.roll_pitch())
    gold = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    for line in open(gold):
        f = line.split()
        ctr = np.array([[int(x, 16) for x in f[2:6]]], np.uint32)
        key = [int(x, 16) for x in f[6:8]]
        assert ctx.philox(key[0], key[1], ctr)[0].tolist() == [int(x, 16) for x in f[8:12]]
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2**32, size=(100_000, 4), dtype=np.uint64).astype(np.uint32)
    out = ctx.philox(12345, 678, ctr)
    for i in range(0, 100_000, 997):
        assert out[i].tolist() == oracle_mod.philox4x32_10(ctr[i].tolist(), [12345, 678])
    ctx.close()


def run_plan(torch, ctx, scenes, start, goal, params):
    if scenes is not None:
        ctx.set_scene_batch(scenes)
    s = torch.from_numpy(start.astype(np.float32)).cuda()
    g = torch.from_numpy(goal.astype(np.float32)).cuda()
    out = ctx.plan(s, g, params)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}


def test_plan_roll_pitch_paths_are_valid_and_deterministic(torch_cuda, oracle_mod):
    rb, c = S.make_arm7(1), S.roll_pitch()
    scenes, start, goal = PB.planning_problems(oracle_mod, rb, c, 12, 900)
    ctx = ctx_for(rb, c)
    prm = ctx.plan_params(range_=0.3, W=32, max_rounds=600, workers=8, seed=7)
    out = run_plan(torch_cuda, ctx, scenes, start, goal, prm)
    again = run_plan(torch_cuda, ctx, None, start, goal, prm)
    PB.assert_same_plans(out, again)
    L = out["path_len"]
    assert (L >= 0).all()
    checked, issues = PB.check_paths(oracle_mod, rb, c, scenes, start, goal, out, 32, 0.3)
    assert not issues, issues[:10]
    # the oracle's planner, same problems and seed (trees differ with FP32 vs FP64 decisions)
    import concurrent.futures as cf

    def oracle_solves(p):
        r = oracle_mod.Oracle(rb, scenes[p], c).plan(
            start[p:p + 1], goal[p:p + 1], range_=0.3, W=32, max_rounds=600, n_workers=8,
            max_nodes=2048, max_connect=32, seed=7, first_problem=p)
        return int(r["path_len"][0] > 0)

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        solved_ref = sum(ex.map(oracle_solves, range(len(scenes))))
    print("gpu solved", int((L > 0).sum()), "oracle solved", solved_ref, "checked", checked)
    assert checked == int((L > 0).sum())
    assert (L > 0).sum() >= max(1, solved_ref // 2)
    assert (out["waypoints"] % 32 == 0).all() and (out["waypoints"] > 0).all()
    assert (out["plan_ms"] > 0).all()
    ctx.close()


@pytest.mark.parametrize("cons", ["none", "roll_pitch"])
def test_plan_follows_the_oracle_planner(torch_cuda, oracle_mod, cons):
    """The GPU planner and the FP64 oracle's planner run the same search (R18, R19): on 24
    problems among 36 mixed obstacles each, problem p planned by the oracle alone with its
    batch index, they take the same number of rounds and return paths of the same length
    whose nodes agree within the parity protocol's 1e-4 (rad), except where an FP32 decision
    (a clearance at contact, a near-tie of nearest nodes, a projection at a threshold) went
    the other way than in FP64 and the two searches parted; that may happen in a few
    problems (measured: 24 of 24 unconstrained, 23 of 24 roll–pitch, nodes within 7e-6)."""
    import concurrent.futures as cf
    rb = S.make_arm7(1)
    c = S.no_constraint() if cons == "none" else S.roll_pitch()
    n = 24
    scenes, start, goal = PB.planning_problems(oracle_mod, rb, c, n, 1700, counts=(20, 10, 6))
    ctx = ctx_for(rb, c)
    prm = ctx.plan_params(range_=0.3, W=16, max_rounds=300, workers=8, max_nodes=2048,
                          max_connect=32, seed=11)
    out = run_plan(torch_cuda, ctx, scenes, start, goal, prm)
    ctx.close()

    def oracle_plan(p):
        return oracle_mod.Oracle(rb, scenes[p], c).plan(
            start[p:p + 1], goal[p:p + 1], range_=0.3, W=16, max_rounds=300, n_workers=8,
            max_nodes=2048, max_connect=32, seed=11, first_problem=p)

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        ref = list(ex.map(oracle_plan, range(n)))
    same, solved = 0, 0
    for p, r in enumerate(ref):
        L = int(out["path_len"][p])
        if L != int(r["path_len"][0]) or int(out["rounds"][p]) != int(r["rounds"][0]):
            continue
        same += 1
        assert int(out["waypoints"][p]) == int(r["waypoints"][0]), p
        if L > 0:
            solved += 1
            assert np.abs(out["path"][p, :L] - r["path"][0, :L]).max() < 1e-4, p
    print(cons, "same search", same, "of", n, "solved among them", solved)
    assert same >= 20 and solved >= 15, (same, solved)


def test_plan_unconstrained_shared_scene(torch_cuda, oracle_mod):
    rb, c = S.make_arm7(2), S.no_constraint()
    scenes, start, goal = PB.planning_problems(oracle_mod, rb, c, 1, 950, counts=(40, 20, 10))
    n = 6
    start = np.repeat(start, n, 0)
    goal = np.repeat(goal, n, 0)
    ctx = ctx_for(rb, c)
    ctx.set_obstacles(scenes[0])
    prm = ctx.plan_params(range_=0.4, W=16, max_rounds=600, workers=4, seed=3,
                          use_scene_batch=False)
    out = run_plan(torch_cuda, ctx, None, start, goal, prm)
    assert (out["path_len"] > 0).sum() >= 1
    checked, issues = PB.check_paths(oracle_mod, rb, c, [scenes[0]] * n, start, goal, out, 16, 0.4)
    assert not issues, issues[:10]
    ctx.close()


def test_plan_z_plane_eight_dof_w64(torch_cuda, oracle_mod):
    rb, c = S.make_arm8(3), S.z_plane(0.9)
    scenes, start, goal = PB.planning_problems(oracle_mod, rb, c, 4, 970, counts=(30, 15, 10))
    ctx = ctx_for(rb, c)
    prm = ctx.plan_params(range_=0.3, W=64, max_rounds=400, workers=4, seed=11, max_path=600)
    out = run_plan(torch_cuda, ctx, scenes, start, goal, prm)
    checked, issues = PB.check_paths(oracle_mod, rb, c, scenes, start, goal, out, 64, 0.3)
    assert not issues, issues[:10]
    print("z-plane solved", checked)
    ctx.close()


def test_plan_argument_errors(torch_cuda, oracle_mod):
    from paper_2505_06791_gb300 import capi
    rb, c = S.make_arm7(1), S.roll_pitch()
    ctx = ctx_for(rb, c)
    q = np.zeros((2, 7), np.float32)
    with pytest.raises(capi.CprrtcError) as e:
        ctx.plan(q, q, ctx.plan_params(use_scene_batch=True))   # no scene batch set
    assert e.value.code == capi.E_NOT_CONFIGURED
    ctx.set_scene_batch([S.Scene(), S.Scene()])
    for bad in (dict(W=1), dict(W=65), dict(workers=0), dict(workers=17), dict(max_path=1),
                dict(max_nodes=1), dict(range_=0.0)):
        with pytest.raises(capi.CprrtcError) as e:
            ctx.plan(q, q, ctx.plan_params(**bad))
        assert e.value.code == capi.E_INVALID_ARG, bad
    # W = 64 (two waypoints per lane) takes fewer than 16 workers: a clear refusal, not a
    # failed launch
    with pytest.raises(capi.CprrtcError) as e:
        ctx.plan(q, q, ctx.plan_params(W=64, workers=16))
    assert e.value.code == capi.E_UNSUPPORTED
    # start == goal in an empty scene, unconstrained: connects in the first round
    ctx.set_constraint(S.no_constraint())
    out = ctx.plan(q, q, ctx.plan_params(W=8, workers=2))
    assert (out["path_len"] >= 2).all()
    ctx.close()


def test_plan_time_budget_and_allocation_failure(torch_cuda, oracle_mod):
    """A per-problem time budget stops problems early (fewer rounds, no path unless they
    connected); a tree allocation beyond device memory is reported as E_OOM, not a fault."""
    from paper_2505_06791_gb300.capi import CprrtcError
    torch = torch_cuda
    rb, c = S.make_arm7(1), S.roll_pitch()
    scenes, start, goal = PB.planning_problems(oracle_mod, rb, c, 8, 950)
    ctx = ctx_for(rb, c)
    free = ctx.plan_params(range_=0.05, W=32, max_rounds=4000, workers=8, seed=3)
    capped = ctx.plan_params(range_=0.05, W=32, max_rounds=4000, workers=8, seed=3,
                             time_budget_ms=0.5)
    a = run_plan(torch, ctx, scenes, start, goal, free)
    b = run_plan(torch, ctx, None, start, goal, capped)
    assert (b["rounds"] <= a["rounds"]).all()
    assert (b["rounds"] < a["rounds"]).any()
    stopped = b["rounds"] < a["rounds"]
    assert (b["path_len"][stopped] == 0).all()
    same = ~stopped
    assert np.array_equal(a["path_len"][same], b["path_len"][same])
    # 2 trees x 2^27 nodes x 64 waypoints x 7 joints x 4 bytes of edges: 481 GB
    huge = ctx.plan_params(range_=0.3, W=64, max_rounds=10, workers=8, max_nodes=1 << 27,
                           seed=1, use_scene_batch=False)
    with pytest.raises(CprrtcError) as err:
        run_plan(torch, ctx, None, start[:1], goal[:1], huge)
    assert err.value.code == -4  # CPRRTC_E_OOM
    # the context stays usable after the failed allocation
    again = run_plan(torch, ctx, scenes, start, goal, free)
    for k in ("path_len", "rounds", "waypoints"):
        assert np.array_equal(again[k], a[k]), k
    bad = ctx.plan_params(range_=0.3, time_budget_ms=-1.0, use_scene_batch=False)
    with pytest.raises(CprrtcError) as err:
        run_plan(torch, ctx, None, start[:1], goal[:1], bad)
    assert err.value.code == -1  # CPRRTC_E_INVALID_ARG
    ctx.close()


@pytest.mark.parametrize("ctype", [3, 4, 5])
def test_plan_line_and_fixed_orientation(torch_cuda, oracle_mod, ctype):
    """The planner under the new constraints: every returned path is re-validated by the
    oracle (on the manifold, continuous, collision-free) and runs are deterministic. With
    the orientation fixed only one or two joints' worth of freedom is left, so those
    problems get sparser scenes and more rounds."""
    rb = S.make_arm7(1)
    c = {3: S.line(0.1, 0.6), 4: S.orient_plane(0.5, 0.6), 5: S.orient_line(-0.4, 0.1, 0.6)}[ctype]
    scenes, start, goal = PB.planning_problems(oracle_mod, rb, c, 8, 9700 + ctype,
                                               counts=(40, 20, 10) if ctype == 3 else (6, 3, 3))
    ctx = ctx_for(rb, c)
    prm = ctx.plan_params(range_=0.3, W=32, max_rounds=400 if ctype == 3 else 2000,
                          workers=8, max_nodes=4096, seed=5)
    out = run_plan(torch_cuda, ctx, scenes, start, goal, prm)
    again = run_plan(torch_cuda, ctx, None, start, goal, prm)
    PB.assert_same_plans(out, again)
    checked, issues = PB.check_paths(oracle_mod, rb, c, scenes, start, goal, out, 32, 0.3)
    assert not issues, issues[:10]
    assert checked >= 1, "no path to check"
    # the oracle's planner on the same problems (each alone with its index): the same search
    # where no FP32 decision of the four- and five-row damped solves went the other way
    import concurrent.futures as cf

    def oracle_plan(p):
        return oracle_mod.Oracle(rb, scenes[p], c).plan(
            start[p:p + 1], goal[p:p + 1], range_=0.3, W=32, max_rounds=prm.max_rounds,
            n_workers=8, max_nodes=4096, max_connect=32, seed=5, first_problem=p)

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        ref = list(ex.map(oracle_plan, range(8)))
    same = sum(int(out["path_len"][p]) == int(r["path_len"][0]) and
               int(out["rounds"][p]) == int(r["rounds"][0]) for p, r in enumerate(ref))
    print(ctype, "solved", checked, "of 8; same search as the oracle's", same, "of 8")
    assert same >= 6, same  # measured 8 of 8 for each of the three constraints
    ctx.close()


def test_plan_with_sequential_projection(torch_cuda, oracle_mod):
    """The naive baseline's planner (sequential projection, Sec. V): paths re-validated by
    the oracle; modes it does not support are refused."""
    from paper_2505_06791_gb300.capi import CprrtcError, E_UNSUPPORTED
    rb, c = S.make_arm7(1), S.roll_pitch()
    scenes, start, goal = PB.planning_problems(oracle_mod, rb, c, 8, 9950, counts=(40, 20, 10))
    ctx = ctx_for(rb, c)
    ctx.set_projection(True)
    prm = ctx.plan_params(range_=0.3, W=32, max_rounds=400, workers=8, seed=6)
    out = run_plan(torch_cuda, ctx, scenes, start, goal, prm)
    checked, issues = PB.check_paths(oracle_mod, rb, c, scenes, start, goal, out, 32, 0.3)
    assert not issues, issues[:10]
    assert checked >= 1
    # the oracle's planner with the same sequential projection runs the same search
    import concurrent.futures as cf

    def oracle_plan(p):
        return oracle_mod.Oracle(rb, scenes[p], c).plan(
            start[p:p + 1], goal[p:p + 1], range_=0.3, W=32, max_rounds=400, n_workers=8,
            max_nodes=2048, max_connect=32, seed=6, first_problem=p, sequential=True)

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        ref = list(ex.map(oracle_plan, range(8)))
    same = sum(int(out["path_len"][p]) == int(r["path_len"][0]) and
               int(out["rounds"][p]) == int(r["rounds"][0]) for p, r in enumerate(ref))
    print("sequential search as the oracle's:", same, "of 8")
    assert same >= 6, same  # measured 8 of 8
    with pytest.raises(CprrtcError) as e:
        run_plan(torch_cuda, ctx, None, start, goal, ctx.plan_params(W=64, seed=6))
    assert e.value.code == E_UNSUPPORTED
    print("sequential planner solved", checked, "of 8")
    ctx.close()


def test_plan_learned_form_paths_are_valid(torch_cuda, oracle_mod):
    """The planner's learned form (extend motions warm-started by the network, trained here on
    oracle projections; plain Alg. 1 as judge and fallback): every returned path is
    re-validated by the oracle, runs are deterministic, the network was evaluated on extend
    motions and some warm-started segments were accepted; and it refuses to run without a
    network for the robot."""
    from paper_2505_06791_gb300 import capi
    torch = torch_cuda
    rb, c = S.make_arm7(1), S.roll_pitch()
    scenes, start, goal = PB.planning_problems(oracle_mod, rb, c, 12, 1900)
    ctx = ctx_for(rb, c)
    prm = ctx.plan_params(range_=0.3, W=32, max_rounds=500, workers=8, seed=13)
    ctx.set_plan_warm_start(5)
    ctx.set_scene_batch(scenes)
    with pytest.raises(capi.CprrtcError) as e:   # no network yet
        run_plan(torch, ctx, None, start, goal, prm)
    assert e.value.code == capi.E_NOT_CONFIGURED
    orc = oracle_mod.Oracle(rb, None, c)
    q = S.uniform_configs(rb, 40000, 1901).astype(np.float32)
    ok, qp, _ = orc.project_configs(q, 60, n_threads=os.cpu_count() or 4)
    ctx.mlp_init(3)
    ctx.mlp_train(torch.from_numpy(q[ok]).cuda(), torch.from_numpy(qp[ok].astype(np.float32)).cuda(),
                  batch=512, epochs=15, lr=1e-3, seed=4)
    ctx.work_counters(reset=True)
    out = run_plan(torch, ctx, None, start, goal, prm)
    cnt = ctx.work_counters(reset=True)
    again = run_plan(torch, ctx, None, start, goal, prm)
    PB.assert_same_plans(out, again, keys=("path_len", "path", "path_edges", "rounds", "waypoints", "work"))
    assert cnt[6] > 0 and 0 < cnt[7] <= cnt[6], cnt
    checked, issues = PB.check_paths(oracle_mod, rb, c, scenes, start, goal, out, 32, 0.3)
    assert not issues, issues[:10]
    assert checked == int((out["path_len"] > 0).sum()) >= 1
    ctx.set_plan_warm_start(0)
    plain = run_plan(torch, ctx, None, start, goal, prm)
    print("learned solved", checked, "plain solved", int((plain["path_len"] > 0).sum()),
          "warm tried", int(cnt[6]), "accepted", int(cnt[7]))
    # the learned form is for roll-pitch and z-plane with the parallel projection
    ctx.set_plan_warm_start(5)
    ctx.set_constraint(S.no_constraint())
    with pytest.raises(capi.CprrtcError) as e:
        run_plan(torch, ctx, None, start, goal, prm)
    assert e.value.code == capi.E_UNSUPPORTED
    with pytest.raises(capi.CprrtcError) as e:
        ctx.set_plan_warm_start(21)
    assert e.value.code == capi.E_INVALID_ARG
    ctx.close()


def test_plan_with_self_collision(torch_cuda, oracle_mod):
    """Self-collision inside the planners: with frame pairs two or more apart named, every
    path cprrtc_plan returns is free of the robot's own spheres too (oracle re-validation
    with the same pairs), and so is every path of the uneven batch whose table robot has the
    pairs; the batch of one robot plans exactly as cprrtc_plan."""
    torch = torch_cuda
    rb, c = S.make_arm7(1), S.roll_pitch()
    pairs = S.self_pairs_gap(rb, 2)
    n = 10
    scenes, start, goal = PB.planning_problems(oracle_mod, rb, c, n, 2100, counts=(40, 20, 10),
                                               self_pairs=pairs)
    ctx = ctx_for(rb, c)
    prm = ctx.plan_params(range_=0.3, W=32, max_rounds=400, workers=8, seed=17)
    ctx.set_self_collision(pairs)
    out = run_plan(torch, ctx, scenes, start, goal, prm)
    checked, issues = PB.check_paths(oracle_mod, rb, c, scenes, start, goal, out, 32, 0.3,
                                     self_pairs=pairs)
    assert not issues, issues[:10]
    assert checked >= 1
    # and the oracle's planner with the same pairs runs the same search (R30)
    import concurrent.futures as cf

    def oracle_plan(p):
        return oracle_mod.Oracle(rb, scenes[p], c, self_pairs=pairs).plan(
            start[p:p + 1], goal[p:p + 1], range_=0.3, W=32, max_rounds=400, n_workers=8,
            max_nodes=2048, max_connect=32, seed=17, first_problem=p)

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        ref = list(ex.map(oracle_plan, range(n)))
    same = sum(int(out["path_len"][p]) == int(r["path_len"][0]) and
               int(out["rounds"][p]) == int(r["rounds"][0]) for p, r in enumerate(ref))
    print("self-aware search as the oracle's:", same, "of", n)
    assert same >= n - 2, same
    # without the pairs the same problems may give paths through the robot itself
    ctx.set_self_collision(None)
    plain = run_plan(torch, ctx, None, start, goal, prm)
    _, plain_issues = PB.check_paths(oracle_mod, rb, c, scenes, start, goal, plain, 32, 0.3,
                                     self_pairs=pairs)
    print("self-aware solved", checked, "plain paths crossing the robot",
          len({i[0] for i in plain_issues}))
    # the uneven batch with the table robot's pairs: the same plans
    ctx.set_robot_table([rb])
    ctx.set_constraint_table([c])
    ctx.set_table_self_collision(0, pairs)
    s8 = torch.zeros((n, 8), device="cuda")
    g8 = torch.zeros((n, 8), device="cuda")
    s8[:, :7] = torch.from_numpy(start.astype(np.float32)).cuda()
    g8[:, :7] = torch.from_numpy(goal.astype(np.float32)).cuda()
    ob = ctx.plan_batch([(0, 0, p, 32) for p in range(n)], s8, g8, prm, edges=True)
    torch.cuda.synchronize()
    ob = {k: (v.cpu().numpy() if v is not None else None) for k, v in ob.items()}
    for k in ("path_len", "rounds", "waypoints", "work"):
        assert np.array_equal(ob[k], out[k]), k
    ctx.close()


def test_plan_rejects_tree_sizes_whose_byte_count_would_wrap(torch_cuda):
    """n * 2 * max_nodes * W * dof * 4 = 2^22 * 2^31 * 64 * 8 * 4 = 2^64 wraps to 0 in 64-bit
    arithmetic: cprrtc_plan must still see that the trees cannot be allocated (E_OOM) and
    launch nothing, whatever the schedule."""
    from paper_2505_06791_gb300 import capi
    torch = torch_cuda
    ctx = ctx_for(S.make_arm8(1), S.z_plane())
    ctx.set_obstacles(S.make_scene(3, n_sph=4))
    s = torch.zeros((4, 8), dtype=torch.float32, device="cuda")
    path_len = torch.zeros(4, dtype=torch.int32, device="cuda")
    path = torch.zeros((4, 4, 8), dtype=torch.float32, device="cuda")
    for first in (200, 0):
        ctx.set_plan_slicing(first)
        for n, max_nodes, workers in ((1 << 22, 1 << 30, 8), (1 << 30, 1 << 30, 8),
                                      (2_000_000_000, 1 << 20, 1)):
            prm = ctx.plan_params(range_=0.3, W=64, max_rounds=1, workers=workers,
                                  max_nodes=max_nodes, max_path=4, seed=1, use_scene_batch=False)
            rc = capi.cprrtc_plan(ctx.h, s, s, n, prm, path_len, path, None, None, None, None,
                                  None)
            assert rc == capi.E_OOM, (n, max_nodes, rc)
    torch.cuda.synchronize()
    assert int(path_len.abs().sum()) == 0  # nothing ran
    ctx.close()
