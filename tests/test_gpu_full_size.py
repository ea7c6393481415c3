"""Parity at the benchmarks' full sizes, in the launch configurations bench.py times: the
planner on 1000 problems, the uneven batch on 512 problems with up to 5000 obstacles, and
the GEMM-form check on 4096 motions x 64 waypoints. Inputs come from the oracle (start,
goal and motion starts are oracle projections); the oracle then checks sampled outputs one
by one (paths re-validated, motions compared with the parity protocol)."""
import concurrent.futures as cf
import os

import numpy as np
import pytest

from paper_2505_06791_gb300 import synth as S
from tests import parity
from tests import problems as PB

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_06791_gb300 import build
    build.build()
    return torch


def pool_map(fn, items):
    with cf.ThreadPoolExecutor(max_workers=THREADS) as ex:
        return list(ex.map(fn, items))


def to_np(d):
    return {k: (v.detach().cpu().numpy() if hasattr(v, "detach") else v) for k, v in d.items()
            if v is not None}


def test_full_planner_1000_problems_full_size(torch_cuda, oracle_mod):
    """1000 problems of 200 mixed obstacles, range 0.3, W = 32, 8 workers, 1000 rounds (the
    headline launch): deterministic; 40 sampled solved paths re-validated by the oracle; 16
    sampled problems run the oracle planner's search."""
    from paper_2505_06791_gb300.capi import Context
    torch = torch_cuda
    rb, c = S.make_arm7(1), S.roll_pitch(20)
    chunks = pool_map(lambda k: PB.planning_problems(oracle_mod, rb, c, 50, 5_000_000 + 1000 * k),
                      range(20))
    scenes = [sc for ch in chunks for sc in ch[0]]
    start = np.concatenate([ch[1] for ch in chunks])
    goal = np.concatenate([ch[2] for ch in chunks])
    n = len(scenes)
    assert n == 1000
    ctx = Context(0)
    ctx.set_robot(rb)
    ctx.set_constraint(c)
    ctx.set_scene_batch(scenes)
    prm = ctx.plan_params(range_=0.3, W=32, max_rounds=1000, workers=8, max_nodes=2048,
                          max_connect=32, max_path=512, seed=11)
    s = torch.from_numpy(start.astype(np.float32)).cuda()
    g = torch.from_numpy(goal.astype(np.float32)).cuda()
    out = to_np(ctx.plan(s, g, prm))
    again = to_np(ctx.plan(s, g, prm))
    torch.cuda.synchronize()
    for k in ("path_len", "rounds", "waypoints"):
        assert np.array_equal(out[k], again[k]), k
    L = out["path_len"]
    solved = np.nonzero(L > 0)[0]
    assert len(solved) > 0.3 * n, len(solved)
    assert (out["waypoints"] % 32 == 0).all()
    sample = np.random.default_rng(5).choice(solved, 40, replace=False)
    checked, issues = PB.check_paths(oracle_mod, rb, c, scenes, start, goal, out, 32, 0.3,
                                     problems=sorted(int(p) for p in sample))
    assert checked == 40 and not issues, issues[:10]
    # the oracle's planner on 16 sampled problems, each alone with its batch index: the same
    # search (rounds, path length, waypoints, nodes within 1e-4) unless an FP32 decision went
    # the other way than in FP64 over the up to 8000 motions of its 1000 rounds
    pick = sorted(int(p) for p in np.random.default_rng(6).choice(n, 16, replace=False))

    def oracle_plan(p):
        return oracle_mod.Oracle(rb, scenes[p], c).plan(
            start[p:p + 1], goal[p:p + 1], range_=0.3, W=32, max_rounds=1000, n_workers=8,
            max_nodes=2048, max_connect=32, seed=11, first_problem=p)

    same = 0
    for p, r in zip(pick, pool_map(oracle_plan, pick)):
        Lp = int(L[p])
        if Lp != int(r["path_len"][0]) or int(out["rounds"][p]) != int(r["rounds"][0]):
            continue
        same += 1
        assert int(out["waypoints"][p]) == int(r["waypoints"][0]), p
        if Lp > 0:
            assert np.abs(out["path"][p, :Lp] - r["path"][0, :Lp]).max() < 1e-4, p
    print("same search as the oracle planner:", same, "of", len(pick))
    assert same >= 13, same  # measured 16 of 16
    ctx.close()


def test_uneven_batch_512_problems_full_size(torch_cuda, oracle_mod):
    """512 problems, DOF 6/7/8, 10..5000 obstacles, three constraints, W 16/32/64, one graph
    replay: the replay equals a direct launch; 24 sampled solved paths re-validated."""
    from paper_2505_06791_gb300.capi import Context
    torch = torch_cuda
    robots, cons, probs, scenes = S.make_batch_mix(512, 5)
    parts = pool_map(lambda k: PB.batch_start_goal(oracle_mod, robots, cons, probs[k::16],
                                                    scenes, 900 + k), range(16))
    start = np.zeros((512, 8), np.float32)
    goal = np.zeros((512, 8), np.float32)
    for k in range(16):
        start[k::16], goal[k::16] = parts[k]
    stream = torch.cuda.Stream()
    ctx = Context(0, stream.cuda_stream)
    ctx.set_robot_table(robots)
    ctx.set_constraint_table(cons)
    ctx.set_scene_batch(scenes)
    prm = ctx.plan_params(range_=0.3, max_rounds=1000, workers=8, max_nodes=2048, max_connect=32,
                          max_path=512, seed=5)
    max_W = max(p[3] for p in probs)
    with torch.cuda.stream(stream):
        s = torch.from_numpy(start).cuda()
        gl = torch.from_numpy(goal).cuda()
        direct = to_np(ctx.plan_batch(probs, s, gl, prm, edges=True))
        out = ctx.alloc_batch_outputs(len(probs), prm, max_W, s, edges=True)
        ctx.batch_capture(probs, s, gl, prm, out)
        ctx.batch_replay()
    stream.synchronize()
    replay = to_np(out)
    PB.assert_same_plans(direct, replay, dofs=[robots[pr[0]].dof for pr in probs])
    L = direct["path_len"]
    solved = np.nonzero(L > 0)[0]
    assert len(solved) > 0.3 * len(probs), len(solved)
    # sample across the obstacle-count range: 16 at random and the 8 heaviest solved
    n_obs = np.array([len(scenes[p[2]].sph) + len(scenes[p[2]].box) + len(scenes[p[2]].cap)
                      for p in probs])
    heavy = solved[np.argsort(-n_obs[solved])[:8]]
    rand = np.random.default_rng(3).choice(np.setdiff1d(solved, heavy), 16, replace=False)
    sample = set(int(p) for p in np.concatenate([heavy, rand]))
    checked, issues = PB.check_batch_paths(oracle_mod, robots, cons, probs, scenes, start, goal,
                                           direct, 0.3, sample=sample)
    assert checked == len(sample) and not issues, issues[:10]
    print("solved", len(solved), "heaviest checked", int(n_obs[heavy].max()))
    ctx.close()


def test_gemm_form_4096_point_cloud_full_size(torch_cuda, oracle_mod):
    """4096 motions x 64 waypoints on the 4096-point cloud: TF32 and BF16 GEMM forms equal
    the exact check on every motion; the exact check is compared with the oracle on 24
    sampled motions (parity protocol)."""
    from paper_2505_06791_gb300.capi import Context
    torch = torch_cuda
    rb, sc, c = S.make_arm8(1), S.make_box_surface_cloud(3), S.z_plane(0.9)
    orc = oracle_mod.Oracle(rb, sc, c)
    q0 = []
    k = 0
    while len(q0) < 4096:
        q = S.uniform_configs(rb, 8192, 70_000 + k).astype(np.float32)
        ok, qp, _ = orc.project_configs(q, 60, n_threads=THREADS)
        q0.extend(qp[ok])
        k += 1
    q0 = S.f32(np.array(q0[:4096])).astype(np.float32)
    q1 = S.uniform_configs(rb, 4096, 80_000).astype(np.float32)
    ctx = Context(0)
    ctx.set_robot(rb)
    ctx.set_obstacles(sc)
    ctx.set_constraint(c)
    d0, d1 = torch.from_numpy(q0).cuda(), torch.from_numpy(q1).cuda()
    res = {}
    for name, mode in (("exact", 0), ("tf32", 1), ("bf16", 2)):
        ctx.set_cc_mode(mode, 0.005)
        res[name] = to_np(ctx.validate(d0, d1, 64))
    torch.cuda.synchronize()
    ex = res["exact"]
    assert (ex["status"] == 2).sum() > 300
    for name in ("tf32", "bf16"):
        for key in ("status", "first_fail", "q"):
            np.testing.assert_array_equal(res[name][key], ex[key], err_msg=f"{name} {key}")
    # oracle parity of the exact check on sampled colliding and valid motions
    rng = np.random.default_rng(9)
    coll = np.nonzero(ex["status"] == 2)[0]
    free = np.nonzero(ex["status"] == 0)[0]
    pick = np.concatenate([rng.choice(coll, 16, replace=False),
                           rng.choice(free, min(8, len(free)), replace=False)])
    runs = parity.oracle_runs(orc, c, q0[pick], q1[pick], 64, n_threads=THREADS)
    sub = {k: v[pick] for k, v in ex.items()}
    stats, bad = parity.compare(sub, runs)
    assert not bad, (stats, bad[:5])
    ctx.close()


def test_validation_65536_motions_full_size(torch_cuda, oracle_mod):
    """The configuration-1 distribution at the throughput sweep's largest size, 65536
    motions x 32 waypoints (roll-pitch, 16 obstacle spheres), where every warp of the
    persistent validation kernel takes motion after motion: 200 sampled motions (projection
    failures, collisions and valid ones) match the oracle under the parity protocol, and the
    outcome counts are those of a run with the motions in reverse order (no state carried
    from one motion to the next)."""
    from paper_2505_06791_gb300.capi import Context
    torch = torch_cuda
    rb, sc, c = S.make_arm7(1), S.make_scene(1001, n_sph=16), S.roll_pitch()
    orc = oracle_mod.Oracle(rb, sc, c)
    n = 65536
    q0 = []
    k = 0
    while len(q0) < n:
        q = S.uniform_configs(rb, 32768, 90_000 + k).astype(np.float32)
        ok, qp, _ = orc.project_configs(q, 60, n_threads=THREADS)
        q0.extend(qp[ok])
        k += 1
    q0 = S.f32(np.array(q0[:n])).astype(np.float32)
    q1 = S.uniform_configs(rb, n, 91_000).astype(np.float32)
    ctx = Context(0)
    ctx.set_robot(rb)
    ctx.set_obstacles(sc)
    ctx.set_constraint(c)
    d0, d1 = torch.from_numpy(q0).cuda(), torch.from_numpy(q1).cuda()
    out = to_np(ctx.validate(d0, d1, 32))
    rev = to_np(ctx.validate(d0.flip(0).contiguous(), d1.flip(0).contiguous(), 32))
    torch.cuda.synchronize()
    ctx.close()
    for key in ("status", "first_fail", "iters", "q"):
        np.testing.assert_array_equal(rev[key][::-1], out[key], err_msg=key)
    st = out["status"]
    rng = np.random.default_rng(12)
    pick = np.concatenate([rng.choice(np.nonzero(st == v)[0], m, replace=False)
                           for v, m in ((0, min(40, int((st == 0).sum()))), (1, 80), (2, 80))])
    runs = parity.oracle_runs(orc, c, q0[pick], q1[pick], 32, n_threads=THREADS)
    stats, bad = parity.compare({k_: v[pick] for k_, v in out.items()}, runs)
    assert not bad, (stats, bad[:5])
    assert stats["exact"] >= 0.8 * stats["n"], stats
