"""Plain FP64 reference of the learned fan initializer -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import this
module; it shares no code with the CUDA library.

The initializer is a small multilayer perceptron that maps a Gaussian's parameters to
per-vertex corrections of its fan, standing in for part of the fine-tuning of Sec. 3
("Fine-tuning", "Optimization and Pruning": vertex positions and opacities are
optimised after the conversion).  Readings:

* Input (15 features + a constant 1 = 16): log-scales (3), the normalised quaternion
  (w, x, y, z) (4), opacity (1), the degree-0 SH coefficients (3), the scales sorted in
  descending order and divided by the largest (3), and log(s_min / s_mid) (1).
* Layers 16 -> 128 -> 128 -> 2(K+1) with exact GELU, 0.5 x (1 + erf(x / sqrt 2)), after
  the two hidden layers; the constant input is the only bias.  Outputs are the radial
  corrections dr_0..dr_K then the log-opacity corrections do_0..do_K of the fan: boundary
  vertex i sits at m + (1 + dr_i)(cos t_i a + sin t_i b) and vertex k's opacity is
  clamp(alpha_k exp(do_k), 0, 1) (the centre keeps its position; dr_0 is unused).
* BF16 network, FP32 accumulation: the inputs, the weights and the activations that feed
  a product (h1, h2 in the forward; dy, dz2, dz1 in the backward) are rounded to
  bfloat16 (round to nearest even, via binary32); sums are exact here (FP64).
  round_bf16=False gives the plain FP64 network (used to pin the gradients by finite
  differences).
* Loss for training pairs: mean squared error over the 2(K+1) outputs of every row.
"""
from __future__ import annotations

import math

import numpy as np

from scipy.special import erf as _erf

HIDDEN = 128
N_IN = 16


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), through binary32; returns FP64."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(f)
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def features(means, log_scales, quats, opacity, sh_dc) -> np.ndarray:
    """N x 16 inputs (FP64, not yet rounded); sh_dc: N x 3 degree-0 coefficients."""
    ls = np.asarray(log_scales, np.float64)
    q = np.asarray(quats, np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    s = np.sort(np.exp(ls), axis=1)[:, ::-1]          # descending
    n = ls.shape[0]
    X = np.empty((n, N_IN))
    X[:, 0:3] = ls
    X[:, 3:7] = q
    X[:, 7] = np.asarray(opacity, np.float64)
    X[:, 8:11] = np.asarray(sh_dc, np.float64)
    X[:, 11:14] = s / s[:, :1]
    X[:, 14] = np.log(s[:, 2] / s[:, 1])
    X[:, 15] = 1.0
    return X


def scene_features(scene) -> np.ndarray:
    sh = scene.sh_f32()
    return features(scene.means, scene.log_scales, scene.quats, scene.opacity, sh[:, 0, :])


def forward(X, W1, W2, W3, round_bf16=True):
    """Returns (y, cache).  X: n x 16; W1: 16 x 128; W2: 128 x 128; W3: 128 x n_out."""
    r = bf16_round if round_bf16 else (lambda a: np.asarray(a, np.float64))
    x = r(X)
    w1, w2, w3 = r(W1), r(W2), r(W3)
    z1 = x @ w1
    h1 = r(gelu(z1))
    z2 = h1 @ w2
    h2 = r(gelu(z2))
    y = h2 @ w3
    return y, {"x": x, "w1": w1, "w2": w2, "w3": w3, "z1": z1, "h1": h1, "z2": z2, "h2": h2, "r": r}


def mse_grad(y, target):
    """Mean squared error over all outputs and its gradient dL/dy."""
    d = y - target
    return float(np.mean(d * d)), 2.0 * d / d.size


def backward(cache, dy):
    """Gradients of the weights (FP64, from the cache's rounded operands)."""
    r = cache["r"]
    dyr = r(dy)
    dW3 = cache["h2"].T @ dyr
    dz2 = r((dyr @ cache["w3"].T) * gelu_grad(cache["z2"]))
    dW2 = cache["h1"].T @ dz2
    dz1 = r((dz2 @ cache["w2"].T) * gelu_grad(cache["z1"]))
    dW1 = cache["x"].T @ dz1
    return dW1, dW2, dW3


def adam(params, grads, m, v, step, lr, betas=(0.9, 0.999), eps=1e-8):
    """In-place Adam over lists of FP64 arrays (the same update rule as the fans')."""
    b1, b2 = betas
    bc1, bc2 = 1.0 - b1 ** step, 1.0 - b2 ** step
    for p, g, mm, vv in zip(params, grads, m, v):
        mm *= b1
        mm += (1.0 - b1) * g
        vv *= b2
        vv += (1.0 - b2) * g * g
        p -= lr * (mm / bc1) / (np.sqrt(vv / bc2) + eps)


def init_weights(n_out, seed=0):
    """He-style random hidden layers and a zero output layer (a zero network leaves the
    plain conversion unchanged)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W1 = rng.normal(0.0, math.sqrt(2.0 / N_IN), (N_IN, HIDDEN))
    W2 = rng.normal(0.0, math.sqrt(2.0 / HIDDEN), (HIDDEN, HIDDEN))
    W3 = np.zeros((HIDDEN, n_out))
    return W1, W2, W3


def corrections_from_finetune(xyz0, a0, xyz1, a1, K):
    """Training targets from one fine-tune: per fan, dr_i = the radial component of the
    moved boundary offset relative to the original offset, minus 1, and
    do_k = log(alpha_after / alpha_before) (0 where the original opacity is 0)."""
    n = xyz0.shape[0] // (K + 1)
    X0 = xyz0.reshape(n, K + 1, 3)
    X1 = xyz1.reshape(n, K + 1, 3)
    off0 = X0[:, 1:, :] - X0[:, :1, :]
    off1 = X1[:, 1:, :] - X0[:, :1, :]
    nn = np.einsum("nkc,nkc->nk", off0, off0)
    dr = np.zeros((n, K + 1))
    dr[:, 1:] = np.where(nn > 0, np.einsum("nkc,nkc->nk", off1, off0) / np.where(nn > 0, nn, 1.0) - 1.0, 0.0)
    A0 = a0.reshape(n, K + 1)
    A1 = a1.reshape(n, K + 1)
    ok = (A0 > 0) & (A1 > 0)
    do = np.where(ok, np.log(np.where(ok, A1, 1.0) / np.where(ok, A0, 1.0)), 0.0)
    return np.concatenate([dr, do], axis=1)
