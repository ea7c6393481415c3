"""Pins of the oracle's warm-start network (FP64 forward pass and reverse-mode gradient).

The network has no counterpart in the paper; its definition is the one the library states:
x = q / pi, three GELU layers (gelu(z) = z Phi(z)), a linear output predicting the
correction t - q, loss (1/rows) sum 0.5 |f(q) - (t - q)|^2, parameters per layer as
W [out][in] then b [out]. Each pin below fails on a plausible slip: a transposed weight,
a dropped 1/pi, the tanh approximation of GELU, a wrong sign or scale in the loss, a
missing GELU derivative factor.
"""
import numpy as np
import pytest
from scipy.stats import norm

from paper_2505_06791_gb300 import synth as S


def gelu_ref(x):
    """GELU from scipy's normal CDF."""
    return x * norm.cdf(x)


def layer_slices(dof, H):
    """(W slice, b slice, shape) per layer of the compact layout."""
    dims = [(H, dof), (H, H), (H, H), (dof, H)]
    out, off = [], 0
    for o, i in dims:
        out.append((slice(off, off + o * i), slice(off + o * i, off + o * i + o), (o, i)))
        off += o * i + o
    return out


def test_param_count(oracle_mod):
    assert oracle_mod.mlp_param_count(7, 256) == 256 * 7 + 256 + 2 * (256 * 256 + 256) + 7 * 256 + 7
    assert oracle_mod.mlp_param_count(7, 256) == 135431
    assert oracle_mod.mlp_param_count(3, 5) == 5 * 3 + 5 + 2 * 30 + 3 * 5 + 3


def test_forward_single_path_closed_form(oracle_mod):
    """A network that routes one input through one unit per layer computes
    y4 = -gelu(2 gelu(gelu(q5))) + b4[4]; every other output is its bias."""
    dof, H = 7, 8
    p = np.zeros(oracle_mod.mlp_param_count(dof, H))
    L = layer_slices(dof, H)
    W = [np.zeros(shape) for _, _, shape in L]
    W[0][3, 5] = np.pi          # unit 3 = gelu(q5)  (input is q / pi)
    W[1][6, 3] = 1.0            # unit 6 = gelu(gelu(q5))
    W[2][1, 6] = 2.0            # unit 1 = gelu(2 gelu(gelu(q5)))
    W[3][4, 1] = -1.0
    b4 = np.arange(dof) * 0.01 - 0.03
    for (ws, bs, shape), w in zip(L, W):
        p[ws] = w.ravel()
    p[L[3][1]] = b4
    q = np.random.default_rng(3).uniform(-2.8, 2.8, (64, dof))
    y = oracle_mod.mlp_forward(p, q, dof, H)
    expect = np.tile(b4, (64, 1))
    expect[:, 4] += -gelu_ref(2 * gelu_ref(gelu_ref(q[:, 5])))
    np.testing.assert_allclose(y, expect, rtol=1e-13, atol=1e-14)


def test_hidden_bias_and_exact_gelu(oracle_mod):
    """Zero weights: every hidden unit is gelu(b); the output is W4 gelu(b3) + b4. GELU is
    the exact z Phi(z) (the tanh form differs by ~1e-4 at z = 1.5)."""
    dof, H = 3, 4
    p = np.zeros(oracle_mod.mlp_param_count(dof, H))
    L = layer_slices(dof, H)
    b3 = np.array([1.5, -0.7, 0.2, 2.5])
    p[L[2][1]] = b3
    W4 = np.array([[1.0, 0, 0, 0], [0, 1.0, 0, 0], [0, 0, 0, 1.0]])
    p[L[3][0]] = W4.ravel()
    y = oracle_mod.mlp_forward(p, np.zeros((1, dof)), dof, H)[0]
    np.testing.assert_allclose(y, W4 @ gelu_ref(b3), rtol=1e-14)
    tanh_form = 0.5 * 1.5 * (1 + np.tanh(np.sqrt(2 / np.pi) * (1.5 + 0.044715 * 1.5 ** 3)))
    assert abs(y[0] - tanh_form) > 1e-5


def test_loss_of_zero_network(oracle_mod):
    """A zero network predicts no correction: loss = mean_r 0.5 |t_r - q_r|^2, and the
    output-bias gradient is -mean_r (t_r - q_r)."""
    dof, H = 7, 8
    rng = np.random.default_rng(5)
    q = rng.uniform(-2, 2, (40, dof))
    t = q + rng.normal(0, 0.2, (40, dof))
    p = np.zeros(oracle_mod.mlp_param_count(dof, H))
    loss, g = oracle_mod.mlp_loss_grad(p, q, t, dof, H)
    assert loss == pytest.approx(0.5 * np.mean(np.sum((t - q) ** 2, axis=1)), rel=1e-13)
    L = layer_slices(dof, H)
    np.testing.assert_allclose(g[L[3][1]], -np.mean(t - q, axis=0), rtol=1e-12, atol=1e-15)
    # zero hidden weights -> zero gradient for W1..W3 (no signal flows back through W4 = 0)
    assert np.all(g[: L[3][0].start] == 0)


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_central_differences(oracle_mod, seed):
    """Reverse-mode gradient of a 7 -> 8 -> 8 -> 8 -> 7 network against central finite
    differences of the loss, every parameter."""
    dof, H = 7, 8
    rng = np.random.default_rng(seed)
    n = oracle_mod.mlp_param_count(dof, H)
    p = rng.normal(0, 0.6, n)
    q = rng.uniform(-2.8, 2.8, (6, dof))
    t = q + rng.normal(0, 0.3, (6, dof))
    _, g = oracle_mod.mlp_loss_grad(p, q, t, dof, H)
    eps = 1e-6
    fd = np.empty(n)
    for i in range(n):
        e = np.zeros(n)
        e[i] = eps
        lp, _ = oracle_mod.mlp_loss_grad(p + e, q, t, dof, H, grad=False)
        lm, _ = oracle_mod.mlp_loss_grad(p - e, q, t, dof, H, grad=False)
        fd[i] = (lp - lm) / (2 * eps)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-8)


def test_gradient_threads_agree(oracle_mod):
    """Row-parallel accumulation gives the single-thread sums (up to rounding order)."""
    dof, H = 7, 16
    rng = np.random.default_rng(9)
    p = rng.normal(0, 0.3, oracle_mod.mlp_param_count(dof, H))
    q = rng.uniform(-2.8, 2.8, (257, dof))
    t = q + rng.normal(0, 0.1, q.shape)
    l1, g1 = oracle_mod.mlp_loss_grad(p, q, t, dof, H, n_threads=1)
    l8, g8 = oracle_mod.mlp_loss_grad(p, q, t, dof, H, n_threads=8)
    assert l8 == pytest.approx(l1, rel=1e-12)
    np.testing.assert_allclose(g8, g1, rtol=1e-10, atol=1e-14)


def test_batch_projection_matches_single(oracle_mod):
    rb = S.make_arm7(1)
    orc = oracle_mod.Oracle(rb, S.make_scene(1001, n_sph=16), S.roll_pitch(20))
    q = S.f32(S.uniform_configs(rb, 33, 77))
    ok, out, res = orc.project_configs(q, 60, n_threads=4)
    for k in range(len(q)):
        ok1, q1, _, r1 = orc.project_config(q[k], max_iters=60)
        assert ok1 == ok[k]
        np.testing.assert_array_equal(out[k], q1)
        assert res[k] == r1
    assert ok.mean() > 0.5


def _bound_case(seed, rows, out_scale=0.3):
    rng = np.random.default_rng(seed)
    dims = [(256, 7), (256, 256), (256, 256), (7, 256)]
    parts = []
    for l, (o, i) in enumerate(dims):
        s = np.sqrt(2.0 / i) * (out_scale if l == 3 else 1.0)
        parts += [rng.normal(0, s, o * i), rng.normal(0, 0.05, o)]
    p = np.concatenate(parts).astype(np.float32).astype(np.float64)
    rb = S.make_arm7(1)
    q = S.uniform_configs(rb, rows, seed + 1).astype(np.float32)
    t = (q + rng.normal(0, 0.3, q.shape)).astype(np.float32)
    return p, q, t


def test_bound_helper_evaluation_is_the_oracle(oracle_mod):
    """The FP64 re-evaluation the GPU tests size their tolerances with (tests/mlp_bounds.py)
    computes the oracle's network: same corrections, loss and gradient."""
    from tests import mlp_bounds as MB
    p, q, t = _bound_case(5, 97)
    ev = MB.evaluate(p, q, t)
    np.testing.assert_allclose(ev["y"], oracle_mod.mlp_forward(p, q.astype(np.float64), 7, 256),
                               rtol=1e-12, atol=1e-14)
    loss, g = oracle_mod.mlp_loss_grad(p, q, t, 7, 256)
    assert abs(ev["loss"] - loss) <= 1e-12 * loss
    np.testing.assert_allclose(ev["grad"], g, rtol=1e-10, atol=1e-16)


def test_bf16_tolerances_hold_for_emulated_bf16_arithmetic():
    """The per-element tolerances (C = 8 standard deviations of the probabilistic rounding
    model) hold for a CPU emulation of the GPU's BF16 arithmetic (BF16 storage of inputs,
    activations and back-propagated signals; FP32 sums), for every element of the
    correction and of every gradient tensor; and they are tight enough to catch a wrong
    element: each is a small fraction of the element's magnitude scale, and the emulated
    errors reach a sizeable part of them (the model is neither loose nor optimistic)."""
    from tests import mlp_bounds as MB
    p, q, t = _bound_case(7, 301)
    p16 = p.copy()
    # the GPU works with BF16 weights (biases FP32); so does the evaluation it is compared to
    for (ws, _, _) in layer_slices(7, 256):
        p16[ws] = MB.bf16_round(p[ws])
    ev = MB.evaluate(p16, q, t)
    fs = MB.forward_sigma(ev, MB.U_BF16, acc_factor=2.0)
    gs = MB.gradient_sigma(ev, fs, MB.U_BF16)
    y_em, g_em = MB.emulate_bf16(p16, q, t)
    ry = np.abs(y_em - ev["y"]) / fs["y"]
    rg = np.abs(g_em - ev["grad"]) / gs
    assert ry.max() < 8.0 and rg.max() < 8.0, (ry.max(), rg.max())
    assert ry.max() > 1.0 and rg.max() > 1.0, (ry.max(), rg.max())
    mag = MB.gradient_magnitude(ev)
    used = mag > 0
    assert np.max(8.0 * gs[used] / mag[used]) < 0.05
    ymag = np.abs(ev["h"][2]) @ np.abs(ev["layers"][3][0]).T + np.abs(ev["layers"][3][1])
    assert np.max(8.0 * fs["y"] / ymag) < 0.05
