"""GPU ray tracing of the triangle soup (ms_bvh_build, ms_raytrace) against the FP64
oracle (oracle/raytrace.py): primary rays alone, and with a point light's shadows, on the
implicit fan layout and on explicit triangles; and the traced primary image against the
rasteriser's."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import synthetic  # noqa: E402
from oracle import raytrace as RT  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_07754_gb300._lib as L
    L.lib()


import paper_2502_07754_gb300 as ms  # noqa: E402
from gpu_util import dev, err_report, oracle_mesh_f32  # noqa: E402


def _soup(n, seed_scene=1):
    w = synthetic.workload(seed_scene, n=n)
    cam = w.cameras[0]
    xyz, rgb, a = oracle_mesh_f32(w.scene, 8, cam.C)
    return w, cam, xyz, rgb, a


@pytest.mark.parametrize("light", [None, (2.5, -1.5, 3.0)])
def test_fan_soup_traced_like_the_oracle(light):
    w, cam, xyz, rgb, a = _soup(300)
    K = 8
    tris = oracle.fan_tris(300, K)
    rt = ms.RayTracer(300 * K, K)
    X, Cc, A = dev(xyz), dev(rgb), dev(a)
    rt.build(X)
    img = rt.trace(X, Cc, A, cam, light=light, ambient=0.3).cpu().numpy().astype(np.float64)
    st, ov = rt.status()
    assert st == 0 and ov == 0
    win = (32, 32, 96, 96)
    ref = RT.render(xyz.astype(np.float64), rgb.astype(np.float64), a.astype(np.float64), tris, cam,
                    light=light, ambient=0.3, window=win)
    rep = err_report(img[win[1]:win[3], win[0]:win[2]], ref)
    print(json.dumps({"case": "fan-soup", "light": light, **rep}))
    assert rep["n_over_tol"] == 0, rep
    if light is not None:
        plain = RT.render(xyz.astype(np.float64), rgb.astype(np.float64), a.astype(np.float64), tris, cam,
                          window=win)
        assert np.abs(plain - ref).max() > 1e-2      # the light does cast shadows here


def test_primary_rays_equal_the_raster():
    """Traced and rasterised images of the same fan soup: the same fragments, barycentrics
    and order (both decide crossings like the FP64 definition)."""
    w, cam, xyz, rgb, a = _soup(1000)
    rt = ms.RayTracer(1000 * 8, 8)
    X, Cc, A = dev(xyz), dev(rgb), dev(a)
    rt.build(X)
    traced = rt.trace(X, Cc, A, cam, T_eps=1e-5).cpu().numpy().astype(np.float64)
    raster = ms.Renderer(1000, 8, cam).forward(X, Cc, A).cpu().numpy().astype(np.float64)
    rep = err_report(traced, raster)
    print(json.dumps({"case": "trace-vs-raster", **rep}))
    assert rep["n_over_tol"] == 0, rep    # a difference would need a centre within rounding of an edge


def _quad(z, half, rgb, a):
    xyz = np.array([[-half, -half, z], [half, -half, z], [half, half, z], [-half, half, z]], np.float32)
    return xyz, np.tile(rgb, (4, 1)).astype(np.float32), np.full(4, a, np.float32), np.array([[0, 1, 2], [0, 2, 3]])


def test_explicit_triangles_with_stacked_shadows():
    """Receiver quad, two partial occluders between it and the light: explicit triangles
    (shared quad corners), shadows multiplying, against the oracle over the whole image."""
    cam = synthetic.make_camera((0.3, -0.2, 3.0), 48, 40, fov_y_deg=45.0)
    parts = [_quad(0.0, 1.5, [0.8, 0.6, 0.4], 1.0), _quad(0.6, 0.5, [0.2, 0.3, 0.9], 0.4),
             _quad(1.1, 0.35, [0.9, 0.1, 0.1], 0.5)]
    xs, cs, as_, ts, off = [], [], [], [], 0
    for x, c, al, t in parts:
        xs.append(x + np.array([0.15 * off, -0.1 * off, 0.0], np.float32))
        cs.append(c); as_.append(al); ts.append(t + off)
        off += 4
    x, c, al, t = np.concatenate(xs), np.concatenate(cs), np.concatenate(as_), np.concatenate(ts).astype(np.int32)
    light = (1.2, 0.8, 4.0)
    rt = ms.RayTracer(t.shape[0])
    X, Cc, A, Tr = dev(x), dev(c), dev(al), dev(t)
    rt.build(X, Tr)
    img = rt.trace(X, Cc, A, cam, tris=Tr, light=light, ambient=0.2).cpu().numpy().astype(np.float64)
    ref = RT.render(x.astype(np.float64), c.astype(np.float64), al.astype(np.float64), t, cam, light=light,
                    ambient=0.2)
    rep = err_report(img, ref)
    print(json.dumps({"case": "stacked-shadows", **rep}))
    assert rep["n_over_tol"] == 0, rep
