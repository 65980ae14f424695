"""Pins of the FP64 fine-tuning loss oracle (oracle/loss.py): Eq. 3 read as
lambda L1 + (1 - lambda)(1 - SSIM), SSIM with an 11 x 11 Gaussian window (sigma 1.5),
zero padding, C1 = 0.01^2, C2 = 0.03^2."""
import math

import numpy as np
import pytest

import oracle
from oracle import loss as OL


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def test_window_is_the_normalised_gaussian():
    w = OL.gaussian_window()
    assert w.shape == (11, 11)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w, w.T) and np.allclose(w, w[::-1, ::-1])
    g = [math.exp(-(t * t) / (2 * 1.5 * 1.5)) for t in range(-5, 6)]
    z = sum(g)
    assert abs(w[5, 5] - (1.0 / z) ** 2) < 1e-15
    assert abs(w[5, 0] - g[0] / z / z) < 1e-15


def test_ssim_of_an_image_with_itself_is_one():
    x = _rng(1).random((23, 17, 3))
    S, _ = OL.ssim_map(x, x)
    assert np.abs(S - 1.0).max() < 1e-12
    loss, grad = OL.fine_tune_loss(x, x)
    assert abs(loss) < 1e-12
    assert np.abs(grad).max() < 1e-12


def test_constant_images_interior_closed_form():
    a, b = 0.3, 0.7
    x = np.full((20, 21, 3), a)
    y = np.full((20, 21, 3), b)
    S, _ = OL.ssim_map(x, y)
    inner = S[5:-5, 5:-5]
    want = (2 * a * b + OL.C1) / (a * a + b * b + OL.C1)
    assert np.abs(inner - want).max() < 1e-11   # E[x^2] - mu^2 rounds at ~1e-16, against C2 = 9e-4
    # at the border the zero padding lowers the local means: no longer the closed form
    assert abs(S[0, 0, 0] - want) > 1e-3


def test_brute_force_window_sums_with_zero_padding():
    rng = _rng(2)
    x = rng.random((9, 7, 1))
    y = rng.random((9, 7, 1))
    w = OL.gaussian_window()
    H, W = 9, 7
    want = np.zeros((H, W))
    for i in range(H):
        for j in range(W):
            m = {"x": 0.0, "y": 0.0, "xx": 0.0, "yy": 0.0, "xy": 0.0}
            for di in range(-5, 6):
                for dj in range(-5, 6):
                    ii, jj = i + di, j + dj
                    if 0 <= ii < H and 0 <= jj < W:
                        wt = w[di + 5, dj + 5]
                        a, b = x[ii, jj, 0], y[ii, jj, 0]
                        m["x"] += wt * a
                        m["y"] += wt * b
                        m["xx"] += wt * a * a
                        m["yy"] += wt * b * b
                        m["xy"] += wt * a * b
            sxx = m["xx"] - m["x"] ** 2
            syy = m["yy"] - m["y"] ** 2
            sxy = m["xy"] - m["x"] * m["y"]
            want[i, j] = ((2 * m["x"] * m["y"] + OL.C1) * (2 * sxy + OL.C2) /
                          ((m["x"] ** 2 + m["y"] ** 2 + OL.C1) * (sxx + syy + OL.C2)))
    S, _ = OL.ssim_map(x, y)
    assert np.abs(S[..., 0] - want).max() < 1e-13


@pytest.mark.parametrize("shape", [(13, 12, 3), (4, 19, 3)])
def test_ssim_gradient_matches_finite_differences(shape):
    rng = _rng(3)
    x = rng.random(shape)
    y = np.clip(x + rng.normal(0, 0.2, shape), 0, 1)
    g = OL.ssim_grad(x, y)
    h = 1e-6
    for idx in [(0, 0, 0), (shape[0] - 1, shape[1] - 1, 2), (shape[0] // 2, shape[1] // 2, 1), (1, shape[1] - 2, 0)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (OL.ssim(xp, y) - OL.ssim(xm, y)) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-7 * abs(g).max() + 1e-6 * abs(fd), (idx, fd, g[idx])


def test_lambda_one_is_the_l1_oracle():
    rng = _rng(4)
    x = rng.random((11, 14, 3))
    y = rng.random((11, 14, 3))
    loss, grad = OL.fine_tune_loss(x, y, lam=1.0)
    l1, g1 = oracle.l1_loss_grad(x, y)
    assert abs(loss - l1) < 1e-15
    assert np.abs(grad - g1).max() < 1e-15


def test_full_loss_gradient_matches_finite_differences():
    rng = _rng(5)
    x = rng.random((10, 9, 4))
    y = rng.random((10, 9, 4))
    loss, g = OL.fine_tune_loss(x, y)
    assert 0.0 < loss < 2.0
    h = 1e-7
    for idx in [(0, 0, 0), (5, 4, 1), (9, 8, 2), (3, 7, 0)]:
        assert abs(x[idx] - y[idx]) > 1e-3   # away from the kink of |x - y|
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (OL.fine_tune_loss(xp, y)[0] - OL.fine_tune_loss(xm, y)[0]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * abs(g).max(), (idx, fd, g[idx])
    assert g.shape == (10, 9, 3)   # alpha gets no gradient: only RGB is returned
