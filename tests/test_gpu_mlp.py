"""GPU checks of the learned warm start: the network's forward pass and gradient (BF16
tensor-core kernels) against the FP64 oracle on weights and data the test draws itself,
training on oracle-projected pairs, and cprrtc_validate_ws, whose answers are judged by
the plain projection's acceptance tests and the oracle's collision check."""
import os

import numpy as np
import pytest

from paper_2505_06791_gb300 import synth as S
from tests import mlp_bounds as MB
from tests import parity

pytestmark = pytest.mark.gpu

DOF, H = 7, 256
# Per-element tolerance: C standard deviations of the probabilistic rounding model of
# tests/mlp_bounds.py (BF16: u = 2^-8 per stored value, FP32 sums; the FP32 checking mode:
# u = 2^-24 everywhere). On a CPU emulation of the BF16 arithmetic the largest error is
# about 2 sigma (tests/test_oracle_mlp.py), so C = 8 leaves a factor of 4.
C_SIGMA = 8.0
# The FP32 checking mode must also agree to 1e-4 relative: against each element's
# magnitude scale (sum of |terms|) everywhere, and against the element itself wherever
# cancellation is mild (|value| >= 0.1 x its magnitude scale).
REL_FP32 = 1e-4


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_06791_gb300 import build
    build.build()
    return torch


@pytest.fixture(scope="module")
def setup():
    rb = S.make_arm7(1)
    sc = S.make_scene(1001, n_sph=16)
    c = S.roll_pitch(20)
    return rb, sc, c


def make_ctx(rb, sc, c):
    from paper_2505_06791_gb300.capi import Context
    ctx = Context(0)
    ctx.set_robot(rb)
    ctx.set_obstacles(sc)
    ctx.set_constraint(c)
    return ctx


def bf16(x):
    """Round FP32 values to the nearest BF16 (ties to even), returned as float64."""
    a = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((a + 0x7FFF + ((a >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def random_params(oracle_mod, seed, out_scale=1.0):
    """He-scaled FP32 weights and small biases in the compact layout."""
    rng = np.random.default_rng(seed)
    dims = [(H, DOF), (H, H), (H, H), (DOF, H)]
    parts, weight_mask = [], []
    for l, (o, i) in enumerate(dims):
        s = np.sqrt(2.0 / i) * (out_scale if l == 3 else 1.0)
        parts += [rng.normal(0, s, o * i), rng.normal(0, 0.05, o)]
        weight_mask += [np.ones(o * i, bool), np.zeros(o, bool)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == oracle_mod.mlp_param_count(DOF, H)
    return p, np.concatenate(weight_mask)


def oracle_view(p32, wmask):
    """What the GPU computes with: BF16 weights, FP32 biases."""
    p = p32.astype(np.float64)
    p[wmask] = bf16(p32[wmask])
    return p


def check_elementwise(got, want, sigma, what, extra=0.0):
    """Every element within C_SIGMA * sigma (+ extra); reports the worst element."""
    got, want = np.ravel(got), np.ravel(want)
    tol = np.ravel(C_SIGMA * np.asarray(sigma) + extra)
    ratio = np.abs(got - want) / np.maximum(tol, 1e-300)
    k = int(np.argmax(ratio))
    assert ratio[k] <= 1.0, (what, k, float(got[k]), float(want[k]), float(tol[k]))
    return float(ratio.max())


def check_rel_fp32(got, want, mag, what):
    """The FP32 mode's 1e-4 relative agreement (see REL_FP32)."""
    got, want, mag = np.ravel(got), np.ravel(want), np.ravel(mag)
    d = np.abs(got - want)
    assert np.all(d <= REL_FP32 * mag + 1e-30), (what, float(np.max(d / np.maximum(mag, 1e-300))))
    mild = np.abs(want) >= 0.1 * mag
    assert np.all(d[mild] <= REL_FP32 * np.abs(want[mild])), what


def test_param_roundtrip_and_init(torch_cuda, oracle_mod, setup):
    ctx = make_ctx(*setup)
    ctx.mlp_init(7)
    a = ctx.mlp_get_params()
    ctx.mlp_init(7)
    np.testing.assert_array_equal(ctx.mlp_get_params(), a)
    ctx.mlp_init(8)
    assert not np.array_equal(ctx.mlp_get_params(), a)
    assert a.size == oracle_mod.mlp_param_count(DOF, H) == ctx.mlp_param_count()
    w2 = a[H * DOF + H: H * DOF + H + H * H]
    assert abs(w2.std() - np.sqrt(2.0 / H)) < 0.05 * np.sqrt(2.0 / H)
    p, _ = random_params(oracle_mod, 1)
    ctx.mlp_set_params(p)
    np.testing.assert_array_equal(ctx.mlp_get_params(), p)
    ctx.close()


@pytest.mark.parametrize("fp32", [False, True], ids=["bf16", "fp32"])
@pytest.mark.parametrize("rows", [1, 65, 1000])
def test_forward_matches_oracle(torch_cuda, oracle_mod, setup, rows, fp32):
    """Every element of the correction (the fused tensor-core kernel in BF16; the unfused
    FP32 forward pass in the checking mode) against the FP64 oracle on the weights the GPU
    uses, within its per-element tolerance; the FP32 mode also to 1e-4 relative."""
    ctx = make_ctx(*setup)
    ctx.mlp_set_precision(fp32)
    ctx.mlp_init(0)
    p, wmask = random_params(oracle_mod, 10 + rows, out_scale=0.3)
    ctx.mlp_set_params(p)
    rb = setup[0]
    q = S.uniform_configs(rb, rows, 500 + rows).astype(np.float32)
    got = ctx.mlp_infer(torch_cuda.from_numpy(q).cuda()).cpu().numpy().astype(np.float64)
    pv = p.astype(np.float64) if fp32 else oracle_view(p, wmask)
    want = oracle_mod.mlp_forward(pv, q.astype(np.float64), DOF, H)
    ev = MB.evaluate(pv, q)
    if fp32:
        fs = MB.forward_sigma(ev, MB.U_FP32)
    else:  # tensor-core accumulation: not necessarily round-to-nearest, widened 2x
        fs = MB.forward_sigma(ev, MB.U_BF16, acc_factor=2.0)
    # q_out = q + correction is one FP32 addition; got - q is exact in FP64
    extra = 2 * MB.U_FP32 * np.abs(q.astype(np.float64) + want)
    worst = check_elementwise(got - q, want, fs["y"], "correction", extra)
    if fp32:
        ymag = np.abs(ev["h"][2]) @ np.abs(ev["layers"][3][0]).T + np.abs(ev["layers"][3][1])
        check_rel_fp32(got - q, want, ymag + np.abs(q), "correction")
    print(f"rows {rows} {'fp32' if fp32 else 'bf16'}: worst |err| / tolerance {worst:.3f}")
    ctx.close()


@pytest.mark.parametrize("fp32", [False, True], ids=["bf16", "fp32"])
def test_gradient_matches_oracle(torch_cuda, oracle_mod, setup, fp32):
    """Every element of every gradient tensor (W and b of all four layers) and the loss
    against the FP64 oracle within the per-element tolerance; the FP32 checking mode also
    to 1e-4 relative."""
    rb = setup[0]
    ctx = make_ctx(*setup)
    ctx.mlp_set_precision(fp32)
    ctx.mlp_init(0)
    p, wmask = random_params(oracle_mod, 3, out_scale=0.3)
    ctx.mlp_set_params(p)
    rows = 777   # ragged against the 64-row tiles
    rng = np.random.default_rng(4)
    q = S.uniform_configs(rb, rows, 41).astype(np.float32)
    t = (q + rng.normal(0, 0.3, q.shape)).astype(np.float32)
    loss, g = ctx.mlp_grad(torch_cuda.from_numpy(q).cuda(), torch_cuda.from_numpy(t).cuda())
    pv = p.astype(np.float64) if fp32 else oracle_view(p, wmask)
    l_ref, g_ref = oracle_mod.mlp_loss_grad(pv, q, t, DOF, H, n_threads=8)
    ev = MB.evaluate(pv, q, t)
    u = MB.U_FP32 if fp32 else MB.U_BF16
    fs = MB.forward_sigma(ev, u)
    gs = MB.gradient_sigma(ev, fs, u)
    # the loss: sum_r 0.5 |y - T|^2 / R moves by sum (y - T) e_y / R; FP32 partial sums
    r = (ev["y"] - ev["T"]) / rows
    s_loss = np.sqrt(np.sum(r ** 2 * fs["y"] ** 2))
    assert abs(loss - l_ref) <= C_SIGMA * s_loss + 2 * rows * DOF * MB.U_FP32 * l_ref, (loss, l_ref)
    g = g.astype(np.float64)
    mag = MB.gradient_magnitude(ev)
    off, worst = 0, 0.0
    for l, (o, i) in enumerate([(H, DOF), (H, H), (H, H), (DOF, H)]):
        for name, size in (("W", o * i), ("b", o)):
            sl = slice(off, off + size)
            worst = max(worst, check_elementwise(g[sl], g_ref[sl], gs[sl], f"{name}{l + 1}"))
            if fp32:
                check_rel_fp32(g[sl], g_ref[sl], mag[sl], f"{name}{l + 1}")
            off += size
    assert off == g.size
    print(f"{'fp32' if fp32 else 'bf16'} gradient: worst |err| / tolerance {worst:.3f}")
    ctx.close()


def oracle_pairs(oracle_mod, rb, sc, c, n, seed):
    """Uniform configurations and their oracle projections (successful ones)."""
    orc = oracle_mod.Oracle(rb, sc, c)
    q = S.uniform_configs(rb, n, seed).astype(np.float32)
    ok, qp, _ = orc.project_configs(q, 60, n_threads=16)
    return q[ok], qp[ok].astype(np.float32)


@pytest.fixture(scope="module")
def trained(torch_cuda, oracle_mod, setup):
    rb, sc, c = setup
    q, t = oracle_pairs(oracle_mod, rb, sc, c, 60000, 11)
    qh, th = oracle_pairs(oracle_mod, rb, sc, c, 4000, 12)
    ctx = make_ctx(rb, sc, c)
    ctx.mlp_init(3)
    p0 = ctx.mlp_get_params()
    dq, dt = torch_cuda.from_numpy(q).cuda(), torch_cuda.from_numpy(t).cuda()
    losses = ctx.mlp_train(dq, dt, batch=512, epochs=30, lr=1e-3, seed=5)
    return dict(ctx=ctx, p0=p0, losses=losses, held=(qh, th), n_train=len(q))


def test_training_reduces_loss(oracle_mod, trained):
    ctx, losses = trained["ctx"], trained["losses"]
    assert np.all(np.isfinite(losses))
    # uniform configurations -> projections is a hard, partly discontinuous map (the
    # projection can land on either side of a branch): the loss falls by about half
    assert losses[-1] < 0.7 * losses[0], losses
    # held-out loss of the trained parameters, evaluated by the oracle in FP64
    qh, th = trained["held"]
    l0, _ = oracle_mod.mlp_loss_grad(trained["p0"], qh, th, DOF, H, n_threads=8, grad=False)
    l1, _ = oracle_mod.mlp_loss_grad(ctx.mlp_get_params(), qh, th, DOF, H, n_threads=8,
                                     grad=False)
    zero = 0.5 * np.mean(np.sum((th.astype(np.float64) - qh) ** 2, axis=1))
    assert l1 < 0.7 * zero and l1 < 0.7 * l0, (l0, l1, zero)


def first_colliding(orc, seg):
    """(first colliding waypoint or -1, deciding clearance) of a segment, FP64."""
    cl = np.array([orc.config_clearance(x) for x in seg])
    hit = np.nonzero(cl < 0)[0]
    if len(hit):
        return int(hit[0]), float(min(abs(cl[hit[0]]), np.abs(cl[: hit[0]]).min()
                                      if hit[0] else np.inf))
    return -1, float(np.abs(cl).min())


def test_validate_ws_judged_by_plain_projection(torch_cuda, oracle_mod, setup, trained):
    """Warm-started segments satisfy Alg. 1's acceptance tests (oracle re-check) and their
    collision verdicts match the oracle; fallen-back motions are the plain method's
    results; and the network pays: fewer iterations, no lost successes."""
    torch = torch_cuda
    rb, sc, c = setup
    ctx = trained["ctx"]
    orc = oracle_mod.Oracle(rb, sc, c)
    n, W = 256, 32
    q0 = np.stack([orc.project_config(q, 60)[1]
                   for q in S.uniform_configs(rb, 3 * n, 71)
                   if orc.project_config(q, 60)[0]][:n])
    q0 = S.f32(q0).astype(np.float32)
    q1 = S.uniform_configs(rb, n, 72).astype(np.float32)
    # planner-like short motions too: q1 near q0 on the manifold side
    rng = np.random.default_rng(73)
    q1[n // 2:] = np.clip(q0[n // 2:] + rng.uniform(-0.3, 0.3, (n - n // 2, DOF)),
                          rb.lo, rb.hi).astype(np.float32)
    d0, d1 = torch.from_numpy(q0).cuda(), torch.from_numpy(q1).cuda()
    plain = {k: parity.to_np(v) for k, v in ctx.validate(d0, d1, W).items()}
    ws = {k: parity.to_np(v) for k, v in ctx.validate_ws(d0, d1, W, refine_iters=5).items()}
    used = ws["warm"].astype(bool)
    fb = ~used
    # fallback: the plain method's answer, plus the refine iterations spent first
    np.testing.assert_array_equal(ws["status"][fb], plain["status"][fb])
    np.testing.assert_array_equal(ws["first_fail"][fb], plain["first_fail"][fb])
    np.testing.assert_array_equal(ws["q"][fb], plain["q"][fb])
    extra = ws["iters"][fb].astype(int) - plain["iters"][fb].astype(int)
    assert set(np.unique(extra)) <= {0, 5}, np.unique(extra)
    # warm-started and accepted: judge with the oracle
    checked = 0
    for m in np.nonzero(used)[0]:
        assert ws["status"][m] != 1 and ws["iters"][m] <= 5
        seg = ws["q"][m].astype(np.float64)
        assert np.array_equal(seg[0], q0[m].astype(np.float64))
        tau = oracle_mod.tau_step(c, q0[m], q1[m], W)
        max_task, step_excess, _ = orc.check_segment(seg, tau)
        assert max_task < c.tol_task + parity.DELTA, (m, max_task)
        assert step_excess < c.tol_sm + parity.DELTA, (m, step_excess)
        ff, margin = first_colliding(orc, seg)
        if margin > parity.CONTACT_MARGIN:
            assert ff == ws["first_fail"][m], (m, ff, ws["first_fail"][m], margin)
            assert (ws["status"][m] == 2) == (ff >= 0)
            checked += 1
    assert used.sum() >= n // 10, used.sum()
    assert checked >= 0.9 * used.sum()
    # gain: no motion the plain method projects is lost, and iterations drop
    plain_ok = plain["status"] != 1
    ws_ok = ws["status"] != 1
    assert np.all(ws_ok[plain_ok])
    assert ws_ok.sum() >= plain_ok.sum()
    it_plain = plain["iters"].astype(float)[plain_ok].mean()
    it_ws = ws["iters"].astype(float)[plain_ok].mean()
    print(f"warm used {used.mean():.2f}; projected plain {plain_ok.sum()} warm {ws_ok.sum()}; "
          f"mean iters (plain-projected motions) plain {it_plain:.2f} warm {it_ws:.2f}")
    assert ws_ok.sum() > plain_ok.sum() or it_ws < it_plain


def test_validate_ws_full_size(torch_cuda, oracle_mod, setup, trained):
    """16384 motions x 32 waypoints (the configuration-4 launch, roll-pitch): fallen-back
    motions equal the plain method's results; 200 sampled warm-started motions are judged by
    the oracle; no motion the plain method projects is lost."""
    torch = torch_cuda
    rb, sc, c = setup
    ctx = trained["ctx"]
    orc = oracle_mod.Oracle(rb, sc, c)
    n, W = 16384, 32
    threads = os.cpu_count() or 4
    q0, k = [], 0
    while len(q0) < n:
        q = S.uniform_configs(rb, 2 * n, 90_000 + k).astype(np.float32)
        ok, qp, _ = orc.project_configs(q, 60, n_threads=threads)
        q0.extend(qp[ok])
        k += 1
    q0 = S.f32(np.array(q0[:n])).astype(np.float32)
    q1 = S.uniform_configs(rb, n, 91_000).astype(np.float32)
    d0, d1 = torch.from_numpy(q0).cuda(), torch.from_numpy(q1).cuda()
    plain = {k_: parity.to_np(v) for k_, v in ctx.validate(d0, d1, W).items()}
    ws = {k_: parity.to_np(v) for k_, v in ctx.validate_ws(d0, d1, W, refine_iters=5).items()}
    used = ws["warm"].astype(bool)
    fb = ~used
    for key in ("status", "first_fail", "q"):
        np.testing.assert_array_equal(ws[key][fb], plain[key][fb], err_msg=key)
    plain_ok, ws_ok = plain["status"] != 1, ws["status"] != 1
    assert np.all(ws_ok[plain_ok]) and ws_ok.sum() > plain_ok.sum()
    rng = np.random.default_rng(17)
    for m in rng.choice(np.nonzero(used)[0], min(200, int(used.sum())), replace=False):
        seg = ws["q"][m].astype(np.float64)
        tau = oracle_mod.tau_step(c, q0[m], q1[m], W)
        max_task, step_excess, _ = orc.check_segment(seg, tau)
        assert max_task < c.tol_task + parity.DELTA and step_excess < c.tol_sm + parity.DELTA, m
        ff, margin = first_colliding(orc, seg)
        if margin > parity.CONTACT_MARGIN:
            assert ff == ws["first_fail"][m], (m, ff, ws["first_fail"][m])
    print("full size: plain projected", int(plain_ok.sum()), "warm", int(ws_ok.sum()),
          "warm used", int(used.sum()))


def test_checkpoint_roundtrip_and_corruption(torch_cuda, oracle_mod, setup, tmp_path):
    """Save / load restores parameters, Adam moments and step exactly (continued training
    from the loaded state equals continued training from the saved one); the file's CRC-32
    agrees with zlib's; a flipped byte, a wrong robot and a truncated file are rejected."""
    import zlib
    from paper_2505_06791_gb300.capi import Context, CprrtcError
    torch = torch_cuda
    rb, sc, c = setup
    ctx = make_ctx(rb, sc, c)
    ctx.mlp_init(4)
    rng = np.random.default_rng(8)
    q = S.uniform_configs(rb, 2048, 44).astype(np.float32)
    t = (q + rng.normal(0, 0.2, q.shape)).astype(np.float32)
    dq, dt = torch.from_numpy(q).cuda(), torch.from_numpy(t).cuda()
    ctx.mlp_train(dq, dt, batch=256, epochs=2, lr=1e-3, seed=1)
    path = str(tmp_path / "net.ckpt")
    ctx.mlp_save(path)
    blob = open(path, "rb").read()
    assert blob[:8] == b"CPRMLP01"
    assert int.from_bytes(blob[-4:], "little") == zlib.crc32(blob[:-4])
    saved = ctx.mlp_get_params()
    # a single-batch epoch is deterministic (one gradient, no split across batches)
    ref = ctx.mlp_train(dq[:256], dt[:256], batch=256, epochs=1, lr=1e-3, seed=2)
    after_ref = ctx.mlp_get_params()
    other = make_ctx(rb, sc, c)
    other.mlp_load(path)
    np.testing.assert_array_equal(other.mlp_get_params(), saved)
    got = other.mlp_train(dq[:256], dt[:256], batch=256, epochs=1, lr=1e-3, seed=2)
    np.testing.assert_allclose(got, ref, rtol=1e-5)
    np.testing.assert_allclose(other.mlp_get_params(), after_ref, rtol=1e-4, atol=1e-6)
    bad = bytearray(blob)
    bad[100] ^= 0x40
    open(path, "wb").write(bytes(bad))
    with pytest.raises(CprrtcError):
        other.mlp_load(path)
    open(path, "wb").write(blob[:-10])
    with pytest.raises(CprrtcError):
        other.mlp_load(path)
    open(path, "wb").write(blob)
    six = make_ctx(S.make_arm6(1), sc, S.roll_pitch(20))
    with pytest.raises(CprrtcError):
        six.mlp_load(path)
    for x in (ctx, other, six):
        x.close()
