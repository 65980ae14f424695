"""Plain FP64 reference of the fine-tuning loss -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import this
module; it shares no code with the CUDA library.

Sec. 3 "Loss Function" (Eq. 3): a weighted combination of the L1 loss and SSIM with
lambda = 0.6, taken as in 3DGS.  Readings:

* The SSIM term enters as (1 - lambda)(1 - SSIM): the equation as printed adds SSIM
  itself, which a minimiser would drive down, while the text says the loss follows 3DGS,
  whose loss is (1 - lambda) L1 + lambda (1 - SSIM) with the weights the other way round;
  the paper's lambda = 0.6 weighs L1.
* SSIM as in 3DGS: per colour channel, local statistics under an 11 x 11 Gaussian window
  (sigma 1.5, weights normalised to sum 1) with zero padding outside the image,
  C1 = 0.01^2, C2 = 0.03^2 (data range 1), the SSIM map averaged over all pixels and the
  three channels.  Only RGB enters; the alpha channel gets no gradient.
* L1 = mean |C - C*| over the three channels (as oracle.l1_loss_grad).

Local statistics at pixel q (w the window, sums over the window around q; pixels outside
the image count as 0):  mu_x = sum w x, mu_y = sum w y, s_xx = sum w x^2 - mu_x^2,
s_yy = sum w y^2 - mu_y^2, s_xy = sum w x y - mu_x mu_y, and
SSIM(q) = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_xx + s_yy + C2)).

Gradient with respect to the rendered image x (y, the target, is fixed): with the raw
moments m1 = sum w x, m2 = sum w x^2, m11 = sum w x y at q, SSIM(q) depends on x only
through them, so
  d SSIM_mean / d x_p = (1/N) sum_q w(q - p) [dS_q/dm1 + 2 x_p dS_q/dm2 + y_p dS_q/dm11],
  dS/dm2 = dS/ds_xx,  dS/dm11 = dS/ds_xy,
  dS/dm1 = dS/dmu_x - 2 mu_x dS/ds_xx - mu_y dS/ds_xy,
with, writing A = 2 mu_x mu_y + C1, B = 2 s_xy + C2, C = mu_x^2 + mu_y^2 + C1,
D = s_xx + s_yy + C2 and S = AB/(CD):
  dS/dmu_x = 2 mu_y B / (C D) - 2 mu_x S / C,  dS/ds_xx = -S / D,  dS/ds_xy = 2 A / (C D).
The sum over q runs over the pixels of the image (the SSIM map has one entry per pixel).
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage

WINDOW = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2
LAMBDA = 0.6


def gaussian_window(size: int = WINDOW, sigma: float = SIGMA) -> np.ndarray:
    """2D window: outer product of the normalised 1D Gaussian (sums to 1)."""
    t = np.arange(size) - size // 2
    g = np.exp(-(t * t) / (2.0 * sigma * sigma))
    g /= g.sum()
    return np.outer(g, g)


def _wsum(img: np.ndarray, w: np.ndarray) -> np.ndarray:
    """sum_{d} w(d) img(q + d) at every q, zero outside the image (a library correlation)."""
    return ndimage.correlate(img, w, mode="constant", cval=0.0)


def ssim_map(x: np.ndarray, y: np.ndarray):
    """Per-pixel, per-channel SSIM of H x W x 3 images (FP64), and the local statistics."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    w = gaussian_window()
    S = np.empty(x.shape)
    stats = []
    for ch in range(x.shape[2]):
        a, b = x[..., ch], y[..., ch]
        mx, my = _wsum(a, w), _wsum(b, w)
        sxx = _wsum(a * a, w) - mx * mx
        syy = _wsum(b * b, w) - my * my
        sxy = _wsum(a * b, w) - mx * my
        A = 2 * mx * my + C1
        B = 2 * sxy + C2
        Cc = mx * mx + my * my + C1
        D = sxx + syy + C2
        S[..., ch] = A * B / (Cc * D)
        stats.append((mx, my, sxx, syy, sxy, A, B, Cc, D))
    return S, stats


def ssim(x, y) -> float:
    S, _ = ssim_map(x, y)
    return float(S.mean())


def ssim_grad(x, y) -> np.ndarray:
    """d SSIM_mean / d x (H x W x 3), by the moment chain rule in the module docstring."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    S, stats = ssim_map(x, y)
    N = S.size
    w = gaussian_window()
    g = np.empty(x.shape)
    for ch in range(x.shape[2]):
        mx, my, sxx, syy, sxy, A, B, Cc, D = stats[ch]
        s = S[..., ch]
        d_mux = 2 * my * B / (Cc * D) - 2 * mx * s / Cc
        d_sxx = -s / D
        d_sxy = 2 * A / (Cc * D)
        g1 = d_mux - 2 * mx * d_sxx - my * d_sxy
        g2 = d_sxx
        g3 = d_sxy
        # sum_q w(q - p) G(q): the window is symmetric, so this is the same correlation
        g[..., ch] = (_wsum(g1, w) + 2 * x[..., ch] * _wsum(g2, w) + y[..., ch] * _wsum(g3, w)) / N
    return g


def fine_tune_loss(x, y, lam: float = LAMBDA):
    """Eq. 3 as read here: lam * L1 + (1 - lam)(1 - SSIM), on the RGB channels of
    H x W x 3 (or x 4, alpha ignored) images.  Returns (loss, dL/dx over RGB)."""
    x = np.asarray(x, np.float64)[..., :3]
    y = np.asarray(y, np.float64)[..., :3]
    d = x - y
    l1 = np.abs(d).sum() / d.size
    s = ssim(x, y)
    grad = lam * np.sign(d) / d.size - (1.0 - lam) * ssim_grad(x, y)
    return float(lam * l1 + (1.0 - lam) * (1.0 - s)), grad
