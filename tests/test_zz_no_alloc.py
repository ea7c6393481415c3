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
    ref = ctx.plan(s, g, prm)
    torch.cuda.synchronize()
    ref = {k: v.cpu().numpy() for k, v in ref.items()}
    for _ in range(2):
        out = ctx.alloc_plan_outputs(4, prm, s)
        rc = capi.cprrtc_plan_static(ctx.h, s, g, 4, prm, out["path_len"], out["path"],
                                     out["path_edges"], out["rounds"], out["waypoints"],
                                     out["plan_ms"], out["work"])
        assert rc == capi.OK, capi.lib().cprrtc_last_error(ctx.h)
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy() for k, v in out.items()}
        for k in ("path_len", "rounds", "waypoints", "work"):
            assert np.array_equal(got[k], ref[k]), k
        for p in range(4):
            n = int(ref["path_len"][p])
            if n > 0:
                assert np.allclose(got["path"][p, :n], ref["path"][p, :n], rtol=0, atol=1e-6)
                assert np.allclose(got["path_edges"][p, :n - 1], ref["path_edges"][p, :n - 1],
                                   rtol=0, atol=1e-6)
    # beyond the fixed array: a clear capacity error, nothing launched
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
