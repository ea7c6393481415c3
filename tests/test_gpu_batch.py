"""Persistent batches of uneven planning problems (cprrtc_plan_batch), their CUDA-graph
capture and the autotuner, through the C ABI."""
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


def to_np(out):
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}


def test_homogeneous_batch_equals_plan(torch_cuda, oracle_mod):
    """A batch whose problems share robot, constraint and W plans exactly as cprrtc_plan."""
    from paper_2505_06791_gb300.capi import Context
    torch = torch_cuda
    rb, c = S.make_arm7(1), S.roll_pitch()
    scenes, start, goal = PB.planning_problems(oracle_mod, rb, c, 10, 1900)
    stream = torch.cuda.Stream()
    ctx = Context(0, stream.cuda_stream)
    ctx.set_robot(rb)
    ctx.set_constraint(c)
    ctx.set_scene_batch(scenes)
    ctx.set_robot_table([rb])
    ctx.set_constraint_table([c])
    prm = ctx.plan_params(range_=0.3, W=32, max_rounds=300, workers=8, seed=9)
    with torch.cuda.stream(stream):
        s = torch.from_numpy(start.astype(np.float32)).cuda()
        g = torch.from_numpy(goal.astype(np.float32)).cuda()
        ref = to_np(ctx.plan(s, g, prm))
        s8 = torch.zeros((10, 8), device="cuda")
        g8 = torch.zeros((10, 8), device="cuda")
        s8[:, :7] = s
        g8[:, :7] = g
        probs = [(0, 0, p, 32) for p in range(10)]
        out = to_np(ctx.plan_batch(probs, s8, g8, prm, edges=True))
    stream.synchronize()
    for k in ("path_len", "rounds", "waypoints", "work"):
        assert np.array_equal(out[k], ref[k]), k
    for p in range(10):
        n = int(ref["path_len"][p])
        if n > 0:
            assert np.array_equal(out["path"][p, :n, :7], ref["path"][p, :n])
            assert np.array_equal(out["path_edges"][p, :n - 1, :32, :7],
                                  ref["path_edges"][p, :n - 1])
    ctx.close()


def test_mixed_batch_paths_graph_and_tuning(torch_cuda, oracle_mod):
    """Mixed robots, constraints, W and obstacle counts: every path is re-validated by the
    oracle; repeated runs, a CUDA-graph replay and an autotuned launch shape all give the
    same results."""
    from paper_2505_06791_gb300.capi import Context
    torch = torch_cuda
    robots, cons, probs, scenes = S.make_batch_mix(18, 77, max_obstacles=400)
    start, goal = PB.batch_start_goal(oracle_mod, robots, cons, probs, scenes, 31)
    stream = torch.cuda.Stream()
    ctx = Context(0, stream.cuda_stream)
    ctx.set_robot_table(robots)
    ctx.set_constraint_table(cons)
    ctx.set_scene_batch(scenes)
    prm = ctx.plan_params(range_=0.3, max_rounds=400, workers=8, seed=3, max_path=400)
    max_W = max(p[3] for p in probs)
    with torch.cuda.stream(stream):
        s = torch.from_numpy(start.astype(np.float32)).cuda()
        g = torch.from_numpy(goal.astype(np.float32)).cuda()
        first = to_np(ctx.plan_batch(probs, s, g, prm, edges=True))
        second = to_np(ctx.plan_batch(probs, s, g, prm, edges=True))
        span_direct = ctx.batch_spans(len(probs))
        out = ctx.alloc_batch_outputs(len(probs), prm, max_W, s, edges=True)
        ctx.batch_capture(probs, s, g, prm, out)
        ctx.batch_replay()
        ctx.batch_replay()
        span_replay = ctx.batch_spans(len(probs))
    stream.synchronize()
    replay = to_np(out)
    # each problem's span on the global timer is the time its plan_ms reports, for the last
    # direct run and for the last replay
    for sp, res in ((span_direct, second), (span_replay, replay)):
        assert (sp[:, 0] > 0).all() and (sp[:, 1] >= sp[:, 0]).all()
        np.testing.assert_allclose((sp[:, 1] - sp[:, 0]) / 1e6, res["plan_ms"], rtol=1e-5, atol=1e-5)
    assert not np.array_equal(span_direct, span_replay)
    from paper_2505_06791_gb300.capi import CprrtcError, E_INVALID_ARG
    with pytest.raises(CprrtcError) as e:
        ctx.batch_spans(len(probs) + 1)
    assert e.value.code == E_INVALID_ARG
    keys = ("path_len", "path", "path_edges", "rounds", "waypoints", "work")
    dofs = [robots[pr[0]].dof for pr in probs]
    Ws = [pr[3] for pr in probs]
    PB.assert_same_plans(first, second, keys, dofs, Ws)
    PB.assert_same_plans(first, replay, keys, dofs, Ws)
    checked, issues = PB.check_batch_paths(oracle_mod, robots, cons, probs, scenes, start, goal,
                                           first, 0.3)
    assert not issues, issues[:10]
    assert checked >= 3, checked
    with torch.cuda.stream(stream):
        tuned = ctx.autotune_batch(probs, s, g, prm, trial_rounds=5)
        again = to_np(ctx.plan_batch(probs, s, g, prm, tuning=tuned, edges=True))
    stream.synchronize()
    # with warp pairs chosen, the collision-work counts depend on timing; Alg. 1's do not
    PB.assert_same_plans(first, again, keys[:-1], dofs, Ws)
    assert np.array_equal(first["work"][:, 0], again["work"][:, 0])
    ctx.close()


def test_warp_pairs_plan_as_one_warp(torch_cuda, oracle_mod):
    """Every class planned with a warp pair per worker gives the paths, edges, rounds and
    waypoints of the one-warp kernels: problems of 33..64 waypoints split by waypoints (one
    per lane, Alg. 1 in step over both warps, each checking its own waypoints), with W = 33
    (a pair whose second warp holds one waypoint), 47 and 64; problems of 16 and 32 waypoints
    split by obstacles (both warps project, each checks half of the obstacle chunks); and
    each class's two heaviest problems on pairs while the rest keep one warp. Every
    constraint, self-collision pairs on one robot; the long problems' paths pass the oracle's
    re-validation."""
    from paper_2505_06791_gb300.capi import Context, default_tuning as _tuning
    torch = torch_cuda
    robots, cons, probs, scenes = S.make_batch_mix(30, 4242, max_obstacles=1500)
    probs = [(r, c, sc, (33, 47, 64)[p % 3] if W == 64 else W)
             for p, (r, c, sc, W) in enumerate(probs)]
    assert sum(W > 32 for *_, W in probs) >= 6
    start, goal = PB.batch_start_goal(oracle_mod, robots, cons, probs, scenes, 57)
    stream = torch.cuda.Stream()
    ctx = Context(0, stream.cuda_stream)
    ctx.set_robot_table(robots)
    ctx.set_constraint_table(cons)
    ctx.set_scene_batch(scenes)
    ctx.set_table_self_collision(2, S.self_pairs_gap(robots[2], 3))
    prm = ctx.plan_params(range_=0.3, max_rounds=300, workers=8, seed=17, max_path=300)
    keys = ("path_len", "path", "path_edges", "rounds", "waypoints")
    dofs = [robots[pr[0]].dof for pr in probs]
    Ws = [pr[3] for pr in probs]
    with torch.cuda.stream(stream):
        s = torch.from_numpy(start.astype(np.float32)).cuda()
        g = torch.from_numpy(goal.astype(np.float32)).cuda()
        one = to_np(ctx.plan_batch(probs, s, g, prm, tuning=_tuning(1), edges=True))
        pair = to_np(ctx.plan_batch(probs, s, g, prm, tuning=_tuning(2), edges=True))
        pair2 = to_np(ctx.plan_batch(probs, s, g, prm, tuning=_tuning(2), edges=True))
        # each class's 2 heaviest problems on warp pairs, the others on one warp
        mixed = to_np(ctx.plan_batch(probs, s, g, prm, tuning=_tuning(1, 2), edges=True))
    stream.synchronize()
    PB.assert_same_plans(one, pair, keys, dofs, Ws)
    PB.assert_same_plans(one, pair2, keys, dofs, Ws)
    PB.assert_same_plans(one, mixed, keys, dofs, Ws)
    assert np.array_equal(one["work"][:, 0], pair["work"][:, 0])  # Alg. 1 updates
    long_solved = [p for p, (*_, W) in enumerate(probs) if W > 32 and one["path_len"][p] > 0]
    assert len(long_solved) >= 2, long_solved
    checked, issues = PB.check_batch_paths(oracle_mod, robots, cons, probs, scenes, start, goal,
                                           pair, 0.3, sample=set(long_solved))
    assert not issues, issues[:10]
    assert checked == len(long_solved)
    ctx.close()


def test_batch_argument_errors(torch_cuda):
    from paper_2505_06791_gb300 import capi
    ctx = capi.Context(0)
    prm = ctx.plan_params()
    q = np.zeros((1, 8), np.float32)
    with pytest.raises(capi.CprrtcError) as e:
        ctx.plan_batch([(0, 0, 0, 32)], q, q, prm)
    assert e.value.code == capi.E_NOT_CONFIGURED
    with pytest.raises(capi.CprrtcError) as e:
        ctx.batch_spans(1)  # no batch has run
    assert e.value.code == capi.E_NOT_CONFIGURED
    ctx.set_robot_table([S.make_arm7(1)])
    ctx.set_constraint_table([S.no_constraint()])
    ctx.set_scene_batch([S.Scene()])
    for bad in ([(1, 0, 0, 32)], [(0, 1, 0, 32)], [(0, 0, 1, 32)], [(0, 0, 0, 1)],
                [(0, 0, 0, 65)]):
        with pytest.raises(capi.CprrtcError) as e:
            ctx.plan_batch(bad, q, q, prm)
        assert e.value.code == capi.E_INVALID_ARG, bad
    with pytest.raises(capi.CprrtcError):
        ctx.batch_replay()
    out = ctx.plan_batch([(0, 0, 0, 16)], q, q, prm)
    assert out["path_len"][0] >= 2      # start == goal, empty scene, no constraint
    ctx.close()


def test_batch_learned_form_equals_plan(torch_cuda, oracle_mod):
    """The uneven batch's learned form: with the context's network (trained here on oracle
    projections) adopted for its (robot, constraint) pair, a batch of one robot plans exactly
    as cprrtc_plan's learned form; its paths are re-validated by the oracle; a pair without a
    network plans as without the learned form; adopting for another dof is refused."""
    import os
    from paper_2505_06791_gb300.capi import Context, CprrtcError, E_NOT_CONFIGURED
    torch = torch_cuda
    rb, c = S.make_arm7(1), S.roll_pitch()
    n = 8
    scenes, start, goal = PB.planning_problems(oracle_mod, rb, c, n, 2300)
    ctx = Context(0)
    ctx.set_robot(rb)
    ctx.set_constraint(c)
    ctx.set_scene_batch(scenes)
    orc = oracle_mod.Oracle(rb, None, c)
    q = S.uniform_configs(rb, 30000, 2301).astype(np.float32)
    ok, qp, _ = orc.project_configs(q, 60, n_threads=os.cpu_count() or 4)
    ctx.mlp_init(5)
    ctx.mlp_train(torch.from_numpy(q[ok]).cuda(), torch.from_numpy(qp[ok].astype(np.float32)).cuda(),
                  batch=512, epochs=10, lr=1e-3, seed=6)
    ctx.set_robot_table([rb, S.make_arm6(1)])
    ctx.set_constraint_table([c])
    with pytest.raises(CprrtcError) as e:   # the network is for 7 joints, robot 1 has 6
        ctx.batch_adopt_network(1, 0)
    assert e.value.code == E_NOT_CONFIGURED
    prm = ctx.plan_params(range_=0.3, W=32, max_rounds=300, workers=8, seed=19)
    s = torch.from_numpy(start.astype(np.float32)).cuda()
    g = torch.from_numpy(goal.astype(np.float32)).cuda()
    s8 = torch.zeros((n, 8), device="cuda")
    g8 = torch.zeros((n, 8), device="cuda")
    s8[:, :7] = s
    g8[:, :7] = g
    probs = [(0, 0, p, 32) for p in range(n)]
    ctx.set_plan_warm_start(5)
    plain_batch = to_np(ctx.plan_batch(probs, s8, g8, prm, edges=True))  # no network adopted yet
    ctx.batch_adopt_network(0, 0)
    ctx.work_counters(reset=True)
    learned_batch = to_np(ctx.plan_batch(probs, s8, g8, prm, edges=True))
    cnt = ctx.work_counters(reset=True)
    learned_plan = to_np(ctx.plan(s, g, prm))
    # warp pairs asked for in the tuning: the learned form has none and keeps one warp
    from paper_2505_06791_gb300.capi import default_tuning
    learned_paired = to_np(ctx.plan_batch(probs, s8, g8, prm, tuning=default_tuning(2, 4), edges=True))
    torch.cuda.synchronize()
    assert cnt[6] > 0 and cnt[7] > 0, cnt
    for k in ("path_len", "rounds", "waypoints", "work"):
        assert np.array_equal(learned_batch[k], learned_plan[k]), k
        assert np.array_equal(learned_paired[k], learned_batch[k]), k
    ctx.set_plan_warm_start(0)
    plain_plan = to_np(ctx.plan(s, g, prm))
    for k in ("path_len", "rounds", "waypoints", "work"):
        assert np.array_equal(plain_batch[k], plain_plan[k]), k
    out = {"path_len": learned_batch["path_len"], "path": learned_batch["path"][:, :, :7],
           "path_edges": learned_batch["path_edges"][:, :, :32, :7]}
    checked, issues = PB.check_paths(oracle_mod, rb, c, scenes, start, goal, out, 32, 0.3)
    assert not issues, issues[:10]
    assert checked >= 1
    ctx.close()


def test_batch_parts_edge_cases(torch_cuda, oracle_mod):
    """Launch shapes at their edges plan as the default: warp pairs asked for with 12
    workers (no room for pairs: one warp per motion, on problems of up to 32 waypoints, the
    ones 12 warps fit), more heavy problems on pairs than a class holds (the whole class on
    pairs), one heavy problem per class, and pairs on a batch of one class."""
    from paper_2505_06791_gb300.capi import Context, default_tuning
    torch = torch_cuda
    robots, cons, probs, scenes = S.make_batch_mix(16, 9191, max_obstacles=300)
    start, goal = PB.batch_start_goal(oracle_mod, robots, cons, probs, scenes, 23)
    ctx = Context(0)
    ctx.set_robot_table(robots)
    ctx.set_constraint_table(cons)
    ctx.set_scene_batch(scenes)
    keys = ("path_len", "path", "rounds", "waypoints")
    s = torch.from_numpy(start.astype(np.float32)).cuda()
    g = torch.from_numpy(goal.astype(np.float32)).cuda()

    def run(sel, workers, tuning):
        prm = ctx.plan_params(range_=0.3, max_rounds=150, workers=workers, seed=4, max_path=200)
        return to_np(ctx.plan_batch([probs[i] for i in sel], s[sel], g[sel], prm, tuning=tuning))

    short = [i for i, p in enumerate(probs) if p[3] <= 32]
    cls0 = [i for i, p in enumerate(probs)
            if (cons[p[1]].type, p[3] > 32) == (cons[probs[0][1]].type, probs[0][3] > 32)]
    assert len(short) >= 4 and len(cls0) >= 2
    for sel, workers in ((short, 12), (list(range(len(probs))), 8), (cls0, 8)):
        dofs = [robots[probs[i][0]].dof for i in sel]
        ref = run(sel, workers, default_tuning())
        for t in (default_tuning(2), default_tuning(1, 1000), default_tuning(1, 1)):
            got = run(sel, workers, t)
            PB.assert_same_plans(ref, got, keys, dofs)
            if workers == 12:  # one warp per motion throughout: the work counts agree too
                assert np.array_equal(ref["work"], got["work"])
    ctx.close()


def test_mixed_batch_follows_the_oracle_planner(torch_cuda, oracle_mod):
    """Every problem of a mixed batch (6/7/8 DOF, three constraints, W 16/32/64, up to 400
    obstacles) runs the search of the oracle's planner with its own robot, constraint, scene,
    W and batch index: the same rounds, path length and waypoints and nodes within 1e-4 on
    most problems; a problem may part where an FP32 decision differs from FP64."""
    import concurrent.futures as cf
    import os
    from paper_2505_06791_gb300.capi import Context
    torch = torch_cuda
    robots, cons, probs, scenes = S.make_batch_mix(18, 5151, max_obstacles=400)
    start, goal = PB.batch_start_goal(oracle_mod, robots, cons, probs, scenes, 53)
    ctx = Context(0)
    ctx.set_robot_table(robots)
    ctx.set_constraint_table(cons)
    ctx.set_scene_batch(scenes)
    prm = ctx.plan_params(range_=0.3, max_rounds=150, workers=8, max_nodes=2048, max_connect=32,
                          seed=29, max_path=300)
    s = torch.from_numpy(start.astype(np.float32)).cuda()
    g = torch.from_numpy(goal.astype(np.float32)).cuda()
    out = to_np(ctx.plan_batch(probs, s, g, prm))
    ctx.close()

    def oracle_plan(p):
        r, c, sc, W = probs[p]
        dof = robots[r].dof
        return oracle_mod.Oracle(robots[r], scenes[sc], cons[c]).plan(
            start[p:p + 1, :dof], goal[p:p + 1, :dof], range_=0.3, W=W, max_rounds=150, n_workers=8,
            max_nodes=2048, max_connect=32, seed=29, max_path=300, first_problem=p)

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        ref = list(ex.map(oracle_plan, range(len(probs))))
    same = 0
    for p, r in enumerate(ref):
        L, dof = int(out["path_len"][p]), robots[probs[p][0]].dof
        if L != int(r["path_len"][0]) or int(out["rounds"][p]) != int(r["rounds"][0]):
            continue
        same += 1
        assert int(out["waypoints"][p]) == int(r["waypoints"][0]), p
        if L > 0:
            assert np.abs(out["path"][p, :L, :dof] - r["path"][0, :L]).max() < 1e-4, p
    print("same search", same, "of", len(probs))
    assert same >= len(probs) - 3, same
