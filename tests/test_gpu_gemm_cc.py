"""GPU checks of the GEMM-form collision check (tcgen05 TF32 / BF16 contraction with an
exact FP32 recheck): its outputs must equal the exact kernel's on every motion, with and
without a guard band, on the point-cloud scene of the 8-DOF arm."""
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


def setup_ctx(rb, sc, c):
    from paper_2505_06791_gb300.capi import Context
    ctx = Context(0)
    ctx.set_robot(rb)
    ctx.set_obstacles(sc)
    ctx.set_constraint(c)
    return ctx


def motions(torch, ctx, rb, n, seed):
    """Starts on the manifold (library projection; inputs only), ends uniform for half the
    motions and nearby for the other half."""
    q = torch.from_numpy(S.uniform_configs(rb, 6 * n, seed).astype(np.float32)).cuda()
    r = ctx.project_configs(q, 60)
    q0 = r["q"][r["ok"].bool()][:n].contiguous()
    assert q0.shape[0] == n
    q1 = torch.from_numpy(S.uniform_configs(rb, n, seed + 1).astype(np.float32)).cuda()
    g = torch.Generator(device="cpu").manual_seed(seed)
    near = (q0[n // 2:] + (torch.rand((n - n // 2, rb.dof), generator=g) * 0.6 - 0.3).cuda())
    lo = torch.tensor(rb.lo, dtype=torch.float32).cuda()
    hi = torch.tensor(rb.hi, dtype=torch.float32).cuda()
    q1[n // 2:] = torch.maximum(torch.minimum(near, hi), lo)
    return q0, q1.contiguous()


def run_modes(torch, ctx, q0, q1, W, guard):
    out = {}
    for name, mode in (("exact", 0), ("tf32", 1), ("bf16", 2)):
        ctx.set_cc_mode(mode, guard)
        o = ctx.validate(q0, q1, W)
        torch.cuda.synchronize()
        out[name] = {k: parity.to_np(v) for k, v in o.items()}
        out[name]["stats"] = ctx.cc_stats(reset=True)
    ctx.set_cc_mode(0)
    return out


@pytest.mark.parametrize("guard", [0.005, 0.0])
def test_gemm_cc_identical_to_exact(torch_cuda, guard):
    torch = torch_cuda
    rb, sc, c = S.make_arm8(1), S.make_box_surface_cloud(3), S.z_plane(0.9)
    ctx = setup_ctx(rb, sc, c)
    q0, q1 = motions(torch, ctx, rb, 512, 300)
    res = run_modes(torch, ctx, q0, q1, 64, guard)
    ex = res["exact"]
    n_coll = int((ex["status"] == 2).sum())
    assert n_coll > 50, n_coll  # the check has collisions to find
    for name in ("tf32", "bf16"):
        r = res[name]
        np.testing.assert_array_equal(r["status"], ex["status"], err_msg=name)
        np.testing.assert_array_equal(r["first_fail"], ex["first_fail"], err_msg=name)
        np.testing.assert_array_equal(r["q"], ex["q"], err_msg=name)
        bound, rechecks = r["stats"]
        assert 0 < bound < 5e-3, (name, bound)
        assert rechecks > 0
        print(name, "E", bound, "rechecks", rechecks, "collisions", n_coll)
    ctx.close()


def test_gemm_cc_ragged_obstacles_and_wide_motions(torch_cuda):
    """Obstacle count not a multiple of the 256-column tile, W = 16 and W = 33."""
    torch = torch_cuda
    rb, c = S.make_arm8(1), S.z_plane(0.9)
    sc = S.make_box_surface_cloud(5, n_boxes=4, n_points=1000)
    ctx = setup_ctx(rb, sc, c)
    q0, q1 = motions(torch, ctx, rb, 128, 900)
    for W in (16, 33):
        res = run_modes(torch, ctx, q0, q1, W, 0.005)
        for name in ("tf32", "bf16"):
            np.testing.assert_array_equal(res[name]["status"], res["exact"]["status"])
            np.testing.assert_array_equal(res[name]["first_fail"], res["exact"]["first_fail"])
    ctx.close()


def test_gemm_cc_streams_large_obstacle_sets(torch_cuda):
    """8192 obstacles: the TF32 image (512 KB) and the BF16 image (256 KB) stream through the
    ring instead of staying resident."""
    torch = torch_cuda
    rb, c = S.make_arm8(1), S.z_plane(0.9)
    sc = S.make_box_surface_cloud(7, n_boxes=12, n_points=8192)
    ctx = setup_ctx(rb, sc, c)
    q0, q1 = motions(torch, ctx, rb, 128, 1200)
    res = run_modes(torch, ctx, q0, q1, 32, 0.005)
    for name in ("tf32", "bf16"):
        np.testing.assert_array_equal(res[name]["status"], res["exact"]["status"])
        np.testing.assert_array_equal(res[name]["first_fail"], res["exact"]["first_fail"])
    ctx.close()


def test_gemm_cc_rejects_boxes(torch_cuda):
    from paper_2505_06791_gb300.capi import CprrtcError
    torch = torch_cuda
    rb, c = S.make_arm7(1), S.roll_pitch(20)
    sc = S.make_planning_scene(11)
    ctx = setup_ctx(rb, sc, c)
    ctx.set_cc_mode(2)
    q = torch.from_numpy(S.uniform_configs(rb, 4, 1).astype(np.float32)).cuda()
    with pytest.raises(CprrtcError):
        ctx.validate(q, q, 8)
    ctx.close()
