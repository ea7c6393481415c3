"""Per-element error bounds for the warm-start network's forward pass and gradient.

The network (dof -> 256 -> 256 -> 256 -> dof, GELU, inputs q / pi, output = correction) is
re-evaluated here in FP64 with every intermediate kept: pre-activations z_l, activations
h_l, the back-propagated signals D_l = dL/dz_l and the parameter gradients. That
evaluation is pinned to the oracle's (`oracle.mlp_forward`, `oracle.mlp_loss_grad`) by a
CPU test; it serves only to size tolerances, never as the parity reference.

Error model: probabilistic rounding error analysis (Higham and Mary, "A New Approach to
Probabilistic Rounding Error Analysis", SIAM J. Sci. Comput. 41(5), 2019): each rounding
to storage precision u_st contributes an independent, mean-zero error of size at most
u_st |x|, each accumulation step one of at most u_acc times the magnitude of the sum, and
errors travel through the layers as variances: Var(sum_k W_jk e_k) = sum_k W_jk^2 Var(e_k),
through gelu with gelu'(z)^2, into gelu'(z) with gelu''(z)^2. The tolerance of an element
is C sigma (C = 8 in the tests). A worst-case bound that carries |errors| through |W| is
sound but useless here: a 256-wide layer of He-scaled weights multiplies it by about 20
while the actual error grows by about 1.4, so after three layers it exceeds the values.
The CPU test checks the model against an emulation of the GPU's BF16 arithmetic.
Unit roundoffs: BF16 (8 significant bits) 2^-8, FP32 2^-24.
"""
import numpy as np
from scipy.special import ndtr

U_BF16 = 2.0 ** -8
U_FP32 = 2.0 ** -24
GELU_EVAL = 1e-6  # the GPU's GELU and GELU' (A&S 7.1.28 in FP32), absolute, per unit |z|


def unpack(p, dof, H=256):
    """Compact parameter vector -> [(W, b)] for the four layers (W [out][in])."""
    dims = [(H, dof), (H, H), (H, H), (dof, H)]
    out, o = [], 0
    for (r, c) in dims:
        W = np.asarray(p[o:o + r * c], np.float64).reshape(r, c)
        o += r * c
        b = np.asarray(p[o:o + r], np.float64)
        o += r
        out.append((W, b))
    assert o == len(p)
    return out


def gelu(z):
    return z * ndtr(z)


def gelu_d(z):
    return ndtr(z) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def evaluate(p, q, t=None, dof=7, H=256):
    """FP64 forward (and, with targets t, the loss gradient) keeping every intermediate."""
    L = unpack(p, dof, H)
    q = np.asarray(q, np.float64)
    x = q / np.pi
    a, zs, hs = x, [], []
    for l in range(3):
        z = a @ L[l][0].T + L[l][1]
        zs.append(z)
        a = gelu(z)
        hs.append(a)
    y = a @ L[3][0].T + L[3][1]
    r = dict(x=x, z=zs, h=hs, y=y, layers=L)
    if t is None:
        return r
    R = q.shape[0]
    T = np.asarray(t, np.float64) - q
    r["T"] = T
    r["loss"] = 0.5 * np.sum((y - T) ** 2) / R
    D = (y - T) / R
    Ds = [None, None, None, D]
    for l in (2, 1, 0):
        Ds[l] = (Ds[l + 1] @ L[l + 1][0]) * gelu_d(zs[l])
    acts = [x] + hs
    grads = []
    for l in range(4):
        grads.append(Ds[l].T @ acts[l])
        grads.append(Ds[l].sum(axis=0))
    r["D"] = Ds
    r["grad"] = np.concatenate([g.ravel() for g in grads])
    return r


def gelu_dd(z):
    return np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi) * (2.0 - z * z)


def forward_sigma(ev, u_st, u_acc=U_FP32, acc_factor=1.0):
    """Per-element standard deviations of the GPU's error in the correction y and in each
    layer's z and h (as dicts of arrays).

    u_st: storage precision of the input and the activations (BF16, or FP32 in the checking
    mode); u_acc: the accumulation precision; acc_factor widens the accumulation term for
    hardware whose accumulation is not IEEE round-to-nearest (the tensor cores)."""
    L = ev["layers"]
    x = ev["x"]
    # x = q * fp32(1/pi) in FP32, then stored: two FP32 roundings and the storage rounding
    var = ((u_st + 2 * U_FP32) * x) ** 2
    v_z, v_h = [], []
    a = x
    for l in range(4):
        W, b = L[l]
        K = W.shape[1]
        mag = np.abs(a) @ np.abs(W).T + np.abs(b)
        vz = var @ (W * W).T + (K + 1) * (acc_factor * u_acc * mag) ** 2
        if l == 3:
            return dict(y=np.sqrt(vz), vz=v_z, vh=v_h)
        z, h = ev["z"][l], ev["h"][l]
        v_z.append(vz)
        var = (gelu_d(z) ** 2 * vz + (GELU_EVAL * z) ** 2 + ((u_st + 4 * U_FP32) * h) ** 2)
        v_h.append(var)
        a = h


def gradient_sigma(ev, fs, u_st, u_acc=U_FP32):
    """Per-element standard deviations of the GPU's gradient error (compact layout), given
    forward_sigma's fs.

    D_3 = (y - T) / R is formed in FP32 (T = t - q in FP32) and stored (u_st); each
    D_{l-1} = (D_l W_l) * gelu'(z_{l-1}) takes the GEMM's accumulation error, the error of
    D_l through W_l^2, the error of z_{l-1} through gelu'' and the storage rounding. Weight
    gradients sum over the rows (split-K, FP32 atomics), bias gradients likewise."""
    L = ev["layers"]
    R = ev["x"].shape[0]
    D = ev["D"]
    acts = [ev["x"]] + ev["h"]
    v_acts = [((u_st + 2 * U_FP32) * ev["x"]) ** 2] + fs["vh"]
    vD = [None] * 4
    vD[3] = ((fs["y"] / R) ** 2 + (U_FP32 * ev["T"] / R) ** 2
             + ((u_st + 2 * U_FP32) * D[3]) ** 2)
    for l in (2, 1, 0):
        W = L[l + 1][0]
        K = W.shape[0]
        G = D[l + 1] @ W
        vG = vD[l + 1] @ (W * W) + (K + 1) * (u_acc * (np.abs(D[l + 1]) @ np.abs(W))) ** 2
        z = ev["z"][l]
        vD[l] = (vG * gelu_d(z) ** 2 + G ** 2 * (gelu_dd(z) ** 2 * fs["vz"][l] + GELU_EVAL ** 2)
                 + ((u_st + 2 * U_FP32) * D[l]) ** 2)
    out = []
    for l in range(4):
        A, vA, Dl = acts[l], v_acts[l], D[l]
        mag = np.abs(Dl).T @ np.abs(A)
        out.append(np.sqrt(vD[l].T @ (A * A) + (Dl * Dl).T @ vA + (R + 8) * (u_acc * mag) ** 2))
        out.append(np.sqrt(vD[l].sum(axis=0) + (R + 8) * (u_acc * np.abs(Dl).sum(axis=0)) ** 2))
    return np.concatenate([g.ravel() for g in out])


def gradient_magnitude(ev):
    """sum over rows of |D_l| |a_{l-1}| per weight (and sum |D_l| per bias): the scale a
    relative error of a sum with cancellation is measured against."""
    acts = [ev["x"]] + ev["h"]
    out = []
    for l in range(4):
        out.append(np.abs(ev["D"][l]).T @ np.abs(acts[l]))
        out.append(np.abs(ev["D"][l]).sum(axis=0))
    return np.concatenate([g.ravel() for g in out])


def bf16_round(x):
    """Round to the nearest BF16 (ties to even), as float64."""
    a = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((a + 0x7FFF + ((a >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def emulate_bf16(p, q, t, dof=7, H=256):
    """A CPU stand-in for the GPU's BF16 arithmetic (BF16 storage of inputs, activations and
    back-propagated signals, FP32 products and sums), used to check on the CPU that the
    bounds above hold for arithmetic of that kind."""
    f32 = np.float32
    L = [(W.astype(f32), b.astype(f32)) for (W, b) in unpack(p, dof, H)]
    q32 = np.asarray(q, f32)
    x = bf16_round(q32 * f32(1.0 / np.pi)).astype(f32)
    a, zs, hs = x, [], []
    for l in range(3):
        z = (a @ L[l][0].T + L[l][1]).astype(f32)
        zs.append(z)
        a = bf16_round(gelu(z.astype(np.float64)).astype(f32)).astype(f32)
        hs.append(a)
    y = (a @ L[3][0].T + L[3][1]).astype(f32)
    R = q32.shape[0]
    T = (np.asarray(t, f32) - q32).astype(f32)
    D = bf16_round(((y - T) / f32(R)).astype(f32)).astype(f32)
    Ds = [None, None, None, D]
    for l in (2, 1, 0):
        G = (Ds[l + 1] @ L[l + 1][0]).astype(f32)
        Ds[l] = bf16_round((G * gelu_d(zs[l].astype(np.float64)).astype(f32)).astype(f32)).astype(f32)
    acts = [x] + hs
    grads = []
    for l in range(4):
        grads.append((Ds[l].T @ acts[l]).astype(f32))
        grads.append(Ds[l].sum(axis=0, dtype=f32))
    return y.astype(np.float64), np.concatenate([g.ravel() for g in grads]).astype(np.float64)
