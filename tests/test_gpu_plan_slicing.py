"""The planner's time-sliced schedule (cprrtc_set_plan_slicing) through the C ABI: persistent
CTAs hand unsolved problems to a queue between slices of rounds, and every output but the
plan times is that of one CTA per problem planned in one stretch, bit for bit, whatever the
slice lengths (the rounds, Philox counters and tree appends do not depend on which CTA runs
a round)."""
import numpy as np
import pytest

from paper_2505_06791_gb300 import synth as S
from tests import problems as PB

pytestmark = pytest.mark.gpu

KEYS = ("path_len", "path", "path_edges", "rounds", "waypoints", "work")


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


def run(torch, ctx, start, goal, prm, device=True):
    if not device:
        out = ctx.plan(start, goal, prm)
        return {k: np.asarray(v) for k, v in out.items() if v is not None}
    s = torch.from_numpy(start).cuda()
    g = torch.from_numpy(goal).cuda()
    out = ctx.plan(s, g, prm)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items() if v is not None}


@pytest.fixture(scope="module")
def problems(oracle_mod):
    """40 cluttered roll-pitch problems, each repeated 16 times: 640 problems (about twice
    the CTAs a GB300 holds at once), each copy with its own Philox stream (problem index)."""
    rb, c = S.make_arm7(1), S.roll_pitch()
    scenes, start, goal = PB.planning_problems(oracle_mod, rb, c, 40, 4100, counts=(30, 15, 10))
    reps = 16
    tile = lambda x: np.ascontiguousarray(np.tile(x, (reps, 1)), dtype=np.float32)  # noqa: E731
    return rb, c, scenes * reps, tile(start), tile(goal)


def test_sliced_schedule_plans_as_one_cta_per_problem(torch_cuda, problems):
    rb, c, scenes, start, goal = problems
    ctx = ctx_for(rb, c)
    ctx.set_scene_batch(scenes)
    prm = ctx.plan_params(range_=0.3, W=32, max_rounds=90, workers=8, seed=5,
                          use_scene_batch=True)
    ctx.set_plan_slicing(0)
    ref = run(torch_cuda, ctx, start, goal, prm)
    L = ref["path_len"]
    # the workload spans every case of the schedule: problems solved in their first slice,
    # in a later one, and problems that reach max_rounds
    print("solved", int((L > 0).sum()), "of", len(L), "rounds > 5:", int((ref["rounds"] > 5).sum()))
    assert (L > 0).any() and (L == 0).any()
    assert (ref["rounds"] > 5).sum() >= 400
    for first, sl in [(3, 2), (1, 1), (17, 5), (200, 50), (89, 1), (90, 7)]:
        ctx.set_plan_slicing(first, sl)
        out = run(torch_cuda, ctx, start, goal, prm)
        PB.assert_same_plans(ref, out, keys=KEYS)
        assert (out["plan_ms"] > 0).all(), (first, sl)
    # host arrays: the call is synchronous and reads the queue's status
    ctx.set_plan_slicing(2, 3)
    host = run(torch_cuda, ctx, start, goal, prm, device=False)
    PB.assert_same_plans(ref, host, keys=KEYS)
    ctx.close()


def test_sliced_schedule_shared_scene_and_small_batch(torch_cuda, problems, oracle_mod):
    """One scene for every problem (staged once per CTA), and the schedule's defaults on a
    batch that fits the GPU at once (no hand-over: each problem stays with its CTA)."""
    rb, c, scenes, start, goal = problems
    ctx = ctx_for(rb, c)
    ctx.set_obstacles(scenes[0])
    prm = ctx.plan_params(range_=0.3, W=32, max_rounds=70, workers=8, seed=9,
                          use_scene_batch=False)
    ctx.set_plan_slicing(0)
    ref = run(torch_cuda, ctx, start, goal, prm)
    ctx.set_plan_slicing(4, 3)
    PB.assert_same_plans(ref, run(torch_cuda, ctx, start, goal, prm), keys=KEYS)
    small = slice(0, 100)
    ctx.set_plan_slicing(0)
    ref_s = run(torch_cuda, ctx, start[small], goal[small], prm)
    ctx.set_plan_slicing(200, 50)
    PB.assert_same_plans(ref_s, run(torch_cuda, ctx, start[small], goal[small], prm), keys=KEYS)
    # sliced paths are valid paths: the oracle re-validates those of the problems whose start
    # and goal were drawn for this scene (copies of problem 0)
    out = run(torch_cuda, ctx, start, goal, prm)
    checked, issues = PB.check_paths(oracle_mod, rb, c, [scenes[0]] * len(start), start, goal,
                                     out, 32, 0.3, problems=range(0, 640, 40))
    assert not issues, issues[:5]
    ctx.close()


def test_slicing_arguments(torch_cuda):
    from paper_2505_06791_gb300.capi import CprrtcError
    ctx = ctx_for(S.make_arm7(1), S.roll_pitch())
    for bad in [(-1, 5), (3, 0), (3, -2)]:
        with pytest.raises(CprrtcError) as err:
            ctx.set_plan_slicing(*bad)
        assert err.value.code == -1  # CPRRTC_E_INVALID_ARG
    ctx.set_plan_slicing(0, 0)  # one CTA per problem: slice ignored
    ctx.close()


@pytest.mark.parametrize("form", ["sequential", "w64_z_plane", "self_collision", "learned"])
def test_sliced_schedule_in_every_planner_form(torch_cuda, oracle_mod, form):
    """The other instantiations of the planner kernel under hand-overs: the naive baseline's
    sequential projection, two waypoints per lane (W = 64, 8-DOF, z-plane, 4 workers), the
    robot's self-collision pairs, and the learned form (a network warm-starting extend
    motions): 400 problems (more than the GPU holds at once) in slices of 3 then 2 rounds plan
    exactly as one CTA per problem."""
    if form == "w64_z_plane":
        rb, c, W, workers = S.make_arm8(3), S.z_plane(0.9), 64, 4
    else:
        rb, c, W, workers = S.make_arm7(1), S.roll_pitch(), 32, 8
    pairs = S.self_pairs_gap(rb, 2) if form == "self_collision" else None
    base_sc, base_s, base_g = PB.planning_problems(oracle_mod, rb, c, 20, 5300,
                                                   counts=(30, 15, 10), self_pairs=pairs)
    reps = 20
    tile = lambda x: np.ascontiguousarray(np.tile(x, (reps, 1)), dtype=np.float32)  # noqa: E731
    scenes, start, goal = base_sc * reps, tile(base_s), tile(base_g)
    ctx = ctx_for(rb, c)
    ctx.set_scene_batch(scenes)
    if form == "sequential":
        ctx.set_projection(True)
    if pairs is not None:
        ctx.set_self_collision(pairs)
    if form == "learned":
        ctx.mlp_init(3)
        ctx.set_plan_warm_start(5)
    prm = ctx.plan_params(range_=0.3, W=W, max_rounds=40, workers=workers, seed=21,
                          use_scene_batch=True, max_path=600)
    ctx.set_plan_slicing(0)
    ref = run(torch_cuda, ctx, start, goal, prm)
    ctx.set_plan_slicing(3, 2)
    out = run(torch_cuda, ctx, start, goal, prm)
    PB.assert_same_plans(ref, out, keys=KEYS)
    print(form, "problems past their first slice:", int((ref["rounds"] > 3).sum()))
    assert (ref["rounds"] > 3).sum() > 304  # more than the GPU holds at once: hand-overs
    ctx.close()
