"""GPU parity of the full fine-tuning loss (ms_fine_tune_loss: Eq. 3 read as
lambda L1 + (1 - lambda)(1 - SSIM)) against the FP64 oracle (oracle/loss.py).

Tolerances, from the arithmetic: each local moment is an FP32 sum of 121 window terms
(relative rounding <= 121 * 2^-24 = 7e-6 of the summed magnitudes, ~1e-6 absolute for
values in [0, 1]); a variance E[x^2] - mu^2 carries that absolute error against a
denominator D >= C2 = 9e-4.  With the per-tile shift, flat regions are exact and
textured ones lose little; windows made mostly of zero padding (a 1 x 1 image: the
padding becomes -r after the shift) come closest, 5e-5 relative measured on the loss of
a 1 x 1 image.  The loss is checked to 2e-4 relative (a wrong window, constant or
padding rule moves it by 1e-2 or more).  Gradient entries
are sums of ~121 products of such factors, divided by N = 3HW: checked elementwise to
1e-4 of the largest entry (measured at most 4.2e-6 on these images)."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import loss as OL  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_07754_gb300._lib as L
    L.lib()


import paper_2502_07754_gb300 as ms  # noqa: E402
from paper_2502_07754_gb300 import _lib  # noqa: E402


def _images(H, W, seed):
    """A render-like image (smooth shading, texture, a flat bright region) and a target
    that differs by noise and a slight shift; RGBA in [0, 1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    img = np.empty((H, W, 4))
    for c in range(3):
        ph = rng.uniform(0, 2 * np.pi, 3)
        img[..., c] = (0.5 + 0.2 * np.sin(xx / 7.0 + ph[0]) * np.cos(yy / 11.0 + ph[1])
                       + 0.1 * np.sin((xx + yy) / 3.0 + ph[2]) + rng.normal(0, 0.04, (H, W)))
    img[: H // 3, : W // 3, :3] = 0.85   # flat and bright: the hardest case for FP32 variances
    img[..., 3] = rng.uniform(0, 1, (H, W))
    tgt = img + rng.normal(0, 0.03, img.shape)
    tgt[:, 1:, :3] = 0.7 * tgt[:, 1:, :3] + 0.3 * tgt[:, :-1, :3]
    return np.clip(img, 0, 1).astype(np.float32), np.clip(tgt, 0, 1).astype(np.float32)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("H,W", [(1, 1), (7, 300), (61, 97), (128, 128), (540, 960)])
def test_fine_tune_loss_matches_oracle(H, W):
    img, tgt = _images(H, W, 100 + H + W)
    loss, dL = ms.fine_tune_loss(_dev(img), _dev(tgt))
    torch.cuda.synchronize()
    want, g = OL.fine_tune_loss(img.astype(np.float64), tgt.astype(np.float64))
    got = float(loss.item())
    assert abs(got - want) <= 2e-4 * abs(want) + 1e-7, (got, want)
    d = dL.cpu().numpy().astype(np.float64)
    assert np.all(d[..., 3] == 0.0)
    err = np.abs(d[..., :3] - g)
    scale = np.abs(g).max()
    print({"H": H, "W": W, "loss_rel": abs(got - want) / want, "grad_max_err_over_max": float(err.max() / scale),
           "grad_mean_err_over_max": float(err.mean() / scale)})
    assert err.max() <= 1e-4 * scale, (err.max(), scale)


def test_lambda_one_is_the_l1_kernel_and_calls_repeat():
    img, tgt = _images(200, 333, 7)
    X, T = _dev(img), _dev(tgt)
    ws = torch.empty(_lib.lib().ms_fine_tune_loss_workspace_size(200, 333), dtype=torch.uint8, device="cuda")
    l_a, g_a = ms.fine_tune_loss(X, T, lam=1.0, workspace=ws)
    l_b, g_b = ms.l1_loss(X, T)
    assert abs(l_a.item() - l_b.item()) <= 1e-6 * l_b.item()
    assert torch.allclose(g_a, g_b, rtol=1e-6, atol=0)
    r1 = ms.fine_tune_loss(X, T, workspace=ws)
    r2 = ms.fine_tune_loss(X, T, workspace=ws)
    assert abs(r1[0].item() - r2[0].item()) <= 1e-6 * r1[0].item()   # the loss is overwritten, not accumulated
    assert torch.equal(r1[1], r2[1])


def test_fine_tune_loss_invalid_arguments():
    L = _lib.lib()
    X = torch.zeros(8, 8, 4, device="cuda")
    out = torch.zeros(8, 8, 4, device="cuda")
    loss = torch.zeros(1, device="cuda")
    ws = torch.empty(L.ms_fine_tune_loss_workspace_size(8, 8), dtype=torch.uint8, device="cuda")
    p = lambda t: C.c_void_p(t.data_ptr())
    assert L.ms_fine_tune_loss(p(X), p(X), 8, 8, 1.5, p(out), p(loss), p(ws), ws.numel(), None) == _lib.MS_ERR_INVALID
    assert L.ms_fine_tune_loss(p(X), p(X), 8, 8, 0.6, p(out), p(loss), p(ws), 16, None) == _lib.MS_ERR_INVALID
    assert b"workspace" in L.ms_last_error()
    assert L.ms_fine_tune_loss(p(X), p(X), 8, 8, 0.6, p(out), p(loss), p(ws), ws.numel(), None) == _lib.MS_OK
    torch.cuda.synchronize()
    assert abs(loss.item()) < 1e-6 and torch.count_nonzero(out).item() == 0   # identical (zero) images
