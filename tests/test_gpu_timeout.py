"""Failure detection in the tensor-core kernels, tested without a GPU fault: every wait in
the GEMM-form collision check and in the warm-start network's fused inference is bounded in
time. With the limit set very short (cprrtc_set_wait_limit), the waits of an ordinary call
run out; the kernel must then give up cleanly (abort flag, its copies and MMAs drained,
tensor memory freed), the call must report it (E_TIMEOUT, or the plain-Alg. 1 fallback of
the warm-started validation), and the same context must give correct results on the next
call with the default limit."""
import numpy as np
import pytest

from paper_2505_06791_gb300 import synth as S

pytestmark = pytest.mark.gpu

SHORT = 1e-6  # seconds: far below any wait of these kernels on a real input


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_06791_gb300 import build
    build.build()
    return torch


def _ctx(rb, sc, c):
    from paper_2505_06791_gb300.capi import Context
    ctx = Context(0)
    ctx.set_robot(rb)
    ctx.set_obstacles(sc)
    ctx.set_constraint(c)
    return ctx


def _host(out):
    return {k: np.array(v, copy=True) for k, v in out.items()}


@pytest.mark.parametrize("n_points", [4096, 8192], ids=["resident", "streamed"])
def test_gemm_cc_wait_limit_expires_then_recovers(torch_cuda, n_points):
    from paper_2505_06791_gb300.capi import CprrtcError, E_TIMEOUT
    rb, c = S.make_arm8(1), S.z_plane(0.9)
    sc = S.make_box_surface_cloud(3, n_boxes=12, n_points=n_points)
    ctx = _ctx(rb, sc, c)
    n, W = 256, 64
    q = S.uniform_configs(rb, 6 * n, 41).astype(np.float32)
    r = ctx.project_configs(q, 60)
    q0 = np.ascontiguousarray(r["q"][r["ok"].astype(bool)][:n])
    assert q0.shape[0] == n
    q1 = np.clip(q0 + np.random.default_rng(5).uniform(-0.3, 0.3, q0.shape), rb.lo,
                 rb.hi).astype(np.float32)
    ctx.set_cc_mode(0)
    exact = _host(ctx.validate(q0, q1, W))
    assert (exact["status"] != 1).sum() > n // 2  # most motions reach the collision check
    for mode in (1, 2):  # TF32, BF16
        ctx.set_cc_mode(mode)
        ref = _host(ctx.validate(q0, q1, W))
        for k in ("status", "first_fail", "q"):
            np.testing.assert_array_equal(ref[k], exact[k], err_msg=k)
        ctx.set_wait_limit(SHORT)
        with pytest.raises(CprrtcError) as ei:
            ctx.validate(q0, q1, W)   # host arrays: synchronous, the flag is read
        assert ei.value.code == E_TIMEOUT
        ctx.set_wait_limit(0.0)
        again = _host(ctx.validate(q0, q1, W))
        for k in ("status", "first_fail", "q"):
            np.testing.assert_array_equal(again[k], exact[k], err_msg=(mode, k))
    ctx.close()


def test_fused_inference_wait_limit_expires_then_recovers(torch_cuda, oracle_mod):
    from paper_2505_06791_gb300.capi import CprrtcError, E_TIMEOUT
    rb, sc, c = S.make_arm7(1), S.make_scene(1001, n_sph=16), S.roll_pitch(20)
    ctx = _ctx(rb, sc, c)
    ctx.mlp_init(9)
    q = S.uniform_configs(rb, 3000, 77).astype(np.float32)
    ref = np.array(ctx.mlp_infer(q), copy=True)
    ctx.set_wait_limit(SHORT)
    with pytest.raises(CprrtcError) as ei:
        ctx.mlp_infer(q)
    assert ei.value.code == E_TIMEOUT
    # the warm-started validation falls back to plain Alg. 1 for every motion
    orc = oracle_mod.Oracle(rb, sc, c)
    q0 = np.stack([x for ok, x, _, _ in (orc.project_config(y, 60) for y in
                                          S.uniform_configs(rb, 400, 78)) if ok][:128])
    q0 = q0.astype(np.float32)
    q1 = S.uniform_configs(rb, len(q0), 79).astype(np.float32)
    W = 32
    ws = _host(ctx.validate_ws(q0, q1, W, refine_iters=5))
    assert not ws["warm"].any()
    ctx.set_wait_limit(0.0)
    plain = _host(ctx.validate(q0, q1, W))
    for k in ("status", "first_fail", "q"):
        np.testing.assert_array_equal(ws[k], plain[k], err_msg=k)
    # the same context, default limit: the inference is back and unchanged
    np.testing.assert_array_equal(np.array(ctx.mlp_infer(q), copy=True), ref)
    ctx.close()

