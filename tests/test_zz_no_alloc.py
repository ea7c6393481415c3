"""cprrtc_plan_static: planning for callers that must not allocate device memory while they
run (a control loop that cannot absorb cudaMalloc's latency and implicit synchronisation, or
a process whose device memory is all held by another allocator). Its trees live in the
library's fixed 16 MiB device array; its results must be those of cprrtc_plan.

This file is collected last on purpose: a failure here leaves every other test already run.
"""
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


def _to_np(out):
    return {k: v.cpu().numpy() for k, v in out.items() if v is not None}


def _plan_static(capi, ctx, s, g, n, prm):
    out = ctx.alloc_plan_outputs(n, prm, s)
    rc = capi.cprrtc_plan_static(ctx.h, s, g, n, prm, out["path_len"], out["path"],
                                 out["path_edges"], out["rounds"], out["waypoints"],
                                 out["plan_ms"], out["work"])
    assert rc == capi.OK, capi.lib().cprrtc_last_error(ctx.h)
    return out


def _same_results(torch, got, ref, n):
    torch.cuda.synchronize()
    got, ref = _to_np(got), _to_np(ref)
    for k in ("path_len", "rounds", "waypoints", "work"):
        assert np.array_equal(got[k], ref[k]), k
    for p in range(n):
        m = int(ref["path_len"][p])
        if m > 0:
            assert np.allclose(got["path"][p, :m], ref["path"][p, :m], rtol=0, atol=1e-6)
            assert np.allclose(got["path_edges"][p, :m - 1], ref["path_edges"][p, :m - 1],
                               rtol=0, atol=1e-6)
    return got


def test_plan_static_matches_plan_on_two_calls_in_a_row(torch_cuda, oracle_mod):
    from paper_2505_06791_gb300 import capi
    torch = torch_cuda
    rb, c = S.make_arm7(1), S.roll_pitch()
    scenes, start, goal = PB.planning_problems(oracle_mod, rb, c, 4, 4321)
    ctx = capi.Context(0)
    ctx.set_robot(rb)
    ctx.set_constraint(c)
    ctx.set_scene_batch(scenes)
    prm = ctx.plan_params(range_=0.3, W=32, max_rounds=300, workers=8, max_nodes=512,
                          max_connect=32, max_path=256, seed=5)
    s = torch.from_numpy(start.astype(np.float32)).cuda()
    g = torch.from_numpy(goal.astype(np.float32)).cuda()
    ctx.work_counters(reset=True)
    ref = ctx.plan(s, g, prm)
    torch.cuda.synchronize()
    w_plan = ctx.work_counters(reset=True)
    for call in range(2):
        got = _same_results(torch, _plan_static(capi, ctx, s, g, 4, prm), ref, 4)
        # its executed work reaches the context's counters exactly as cprrtc_plan's does
        assert np.array_equal(ctx.work_counters(reset=True), w_plan), call
    assert (got["path_len"] > 0).any()

    # a smaller call of another shape after the larger one: fewer problems, other scenes,
    # seed, waypoints, workers and tree size, so the array's leftovers from the calls above
    # lie where this call's trees now are; its results must still be cprrtc_plan's
    scenes2, start2, goal2 = PB.planning_problems(oracle_mod, rb, c, 2, 977)
    ctx.set_scene_batch(scenes2)
    prm2 = ctx.plan_params(range_=0.25, W=16, max_rounds=200, workers=4, max_nodes=200,
                           max_connect=16, max_path=128, seed=11)
    s2 = torch.from_numpy(start2.astype(np.float32)).cuda()
    g2 = torch.from_numpy(goal2.astype(np.float32)).cuda()
    ref2 = ctx.plan(s2, g2, prm2)
    _same_results(torch, _plan_static(capi, ctx, s2, g2, 2, prm2), ref2, 2)

    # beyond the fixed array: a clear capacity error, nothing launched
    ctx.set_scene_batch(scenes)
    big = ctx.plan_params(range_=0.3, W=32, max_rounds=10, workers=8, max_nodes=8192, seed=5)
    out = ctx.alloc_plan_outputs(4, big, s)
    rc = capi.cprrtc_plan_static(ctx.h, s, g, 4, big, out["path_len"], out["path"], None,
                                 None, None, None, None)
    assert rc == capi.E_CAPACITY
    assert b"fixed array" in capi.lib().cprrtc_last_error(ctx.h)
    # host memory would need staging buffers: refused
    host_len = np.zeros(4, np.int32)
    host_path = np.zeros((4, prm.max_path, 7), np.float32)
    rc = capi.cprrtc_plan_static(ctx.h, s, g, 4, prm, host_len, host_path, None, None, None,
                                 None, None)
    assert rc == capi.E_INVALID_ARG
    ctx.close()


def test_plan_static_rejects_sizes_whose_byte_count_would_wrap(torch_cuda):
    """n * 2 * max_nodes * W * dof * 4 = 2^22 * 2^31 * 64 * 8 * 4 = 2^64 wraps to 0 in 64-bit
    arithmetic; the call must still see that it does not fit and launch nothing."""
    from paper_2505_06791_gb300 import capi
    torch = torch_cuda
    rb = S.make_arm8(1)
    ctx = capi.Context(0)
    ctx.set_robot(rb)
    ctx.set_obstacles(S.make_scene(3, n_sph=4))
    ctx.set_constraint(S.z_plane())
    s = torch.zeros((4, 8), dtype=torch.float32, device="cuda")
    path_len = torch.zeros(4, dtype=torch.int32, device="cuda")
    path = torch.zeros((4, 4, 8), dtype=torch.float32, device="cuda")
    for n, max_nodes, workers in ((1 << 22, 1 << 30, 8), (1 << 30, 1 << 30, 8),
                                  (2_000_000_000, 2, 1), (1, 2_000_000_000, 1)):
        prm = ctx.plan_params(range_=0.3, W=64, max_rounds=1, workers=workers,
                              max_nodes=max_nodes, max_path=4, seed=1, use_scene_batch=False)
        rc = capi.cprrtc_plan_static(ctx.h, s, s, n, prm, path_len, path, None, None, None,
                                     None, None)
        assert rc == capi.E_CAPACITY, (n, max_nodes, rc)
    torch.cuda.synchronize()
    assert int(path_len.abs().sum()) == 0  # nothing ran
    ctx.close()
