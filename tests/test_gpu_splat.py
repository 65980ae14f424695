"""GPU parity of the source-Gaussian splat render (ms_splat_render) against the oracle."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import synthetic  # noqa: E402
from synthetic import Scene  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_07754_gb300._lib as L
    L.lib()


from gpu_util import dev, err_report  # noqa: E402
import paper_2502_07754_gb300 as ms  # noqa: E402


def _gpu_splat(sc, cams, rgb32):
    sr = ms.SplatRenderer(sc.n, cams)
    flat = sr.render(dev(sc.means), dev(sc.log_scales), dev(sc.quats), dev(sc.opacity), dev(rgb32))
    torch.cuda.synchronize()
    return [t.cpu().numpy().astype(np.float64) for t in sr.images(flat)], sr


def test_splat_fronto_parallel_closed_form():
    sh = np.zeros((1, 1, 3), np.float32)
    sh[0, 0] = [0.4, -0.1, 0.2]
    sc = Scene(np.zeros((1, 3), np.float32), np.log(np.array([[0.2, 0.2, 1e-4]], np.float32)),
               np.array([[1, 0, 0, 0]], np.float32), np.array([0.8], np.float32), sh, 0, False)
    cam = synthetic.make_camera((0.0, 0.0, 4.0), 96, 80)
    rgb = oracle.gaussian_colors(sc).astype(np.float32)
    (img,), _ = _gpu_splat(sc, [cam], rgb)
    ref, _ = oracle.splat_render(sc, cam, rgb=rgb.astype(np.float64))
    rep = err_report(img, ref)
    assert rep["n_over_tol"] == 0 and rep["max_abs"] < 1e-6, rep
    assert img[..., 3].max() > 0.7


def test_splat_views_vs_oracle():
    sc = synthetic.surface_scene(6000, 5501, degree=1, clustered=True)
    dirs = synthetic.fibonacci_dirs(3)
    cams = [synthetic.make_camera(d * r, w, h) for d, r, (w, h) in zip(dirs, [3.0, 3.6, 4.4],
                                                                        [(97, 61), (128, 96), (40, 150)])]
    rgb = oracle.gaussian_colors(sc, cam_center=cams[0].C).astype(np.float32)
    imgs, sr = _gpu_splat(sc, cams, rgb)
    assert sr.last_info.culled_tris == 0
    for v, cam in enumerate(cams):
        ref, nf = oracle.splat_render(sc, cam, rgb=rgb.astype(np.float64))
        rep = err_report(imgs[v], ref)
        assert rep["n_over_tol"] == 0, (v, rep)
        assert nf.max() > 3


def test_splat_eight_view_workload_windows():
    """The eight 1080p cameras of the learned-initializer workload on a 200k-Gaussian
    clustered scene: 24 x 24 windows of every view vs the oracle."""
    w = synthetic.workload(5, n=200_000)
    sc = w.scene
    rgb = oracle.gaussian_colors(sc, cam_center=w.cameras[0].C).astype(np.float32)
    imgs, _ = _gpu_splat(sc, w.cameras, rgb)
    worst = 0.0
    for v, cam in enumerate(w.cameras):
        x0, y0 = 900 + 13 * v, 500 + 7 * v
        ref, _ = oracle.splat_render(sc, cam, rgb=rgb.astype(np.float64), window=(x0, y0, x0 + 24, y0 + 24))
        rep = err_report(imgs[v][y0:y0 + 24, x0:x0 + 24], ref)
        worst = max(worst, rep["max_abs"])
        assert rep["n_over_tol"] == 0, (v, rep)
    print("8-view splat window max abs err", worst)
