"""GPU parity of fan conversion and the forward render against the oracle (C ABI path)."""
import json
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import synthetic  # noqa: E402
from synthetic import Camera, Scene  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-4   # per-channel absolute image tolerance (FP32 kernels vs FP64 oracle)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_07754_gb300._lib as L
    L.lib()


from gpu_util import dev, err_report, fp64_report, gpu_mesh, gpu_render, oracle_mesh_f32, oracle_render  # noqa: E402


def _check_mesh(sc, K, cam_center, axis_rule=1):
    xg, cg, ag = (t.cpu().numpy().astype(np.float64) for t in gpu_mesh(sc, K, cam_center, axis_rule))
    xo, co, ao = oracle.mesh_build(sc, K=K, cam_center=cam_center, axis_rule=axis_rule)
    ex = np.abs(xg - xo).max() / max(1.0, np.abs(xo).max())
    ec = np.abs(cg - co).max()
    ea = np.abs(ag - ao).max()
    assert ex < 1e-6 and ec < 1e-6 and ea < 1e-6, (ex, ec, ea)


def test_mesh_build_workload1():
    w = synthetic.workload(1)
    _check_mesh(w.scene, 8, w.cameras[0].C)
    _check_mesh(w.scene, 8, None)


def test_mesh_build_sh3_f32_and_bf16():
    sc = synthetic.surface_scene(20000, 41, degree=3)
    _check_mesh(sc, 8, np.array([0.5, 1.0, 3.0], np.float32))
    sc16 = synthetic.surface_scene(20000, 42, degree=3, bf16=True)
    _check_mesh(sc16, 6, np.array([0.5, 1.0, 3.0], np.float32))
    _check_mesh(sc16, 12, np.array([0.5, 1.0, 3.0], np.float32), axis_rule=0)


@pytest.mark.parametrize("deg", [1, 2])
def test_mesh_build_low_degrees(deg):
    sc = synthetic.surface_scene(3000, 43 + deg, degree=deg)
    _check_mesh(sc, 8, np.array([0.0, 0.2, 3.0], np.float32))


def test_render_workload1_all_variants_identical():
    w = synthetic.workload(1)
    cam = w.cameras[0]
    xyz, rgb, a = oracle_mesh_f32(w.scene, 8, cam.C)
    orc, nf, culled = oracle_render(xyz, rgb, a, 8, cam)
    assert culled == 0
    base = None
    for tile, kb in [(16, 16), (16, 8), (8, 16), (8, 8), (32, 8), (32, 16)]:
        img, r, _ = gpu_render(xyz, rgb, a, 8, cam, tile=tile, kbuf=kb)
        rep = err_report(img, orc)
        print(json.dumps({"workload": "random-1k", "tile": tile, "kbuf": kb, **rep}))
        assert rep["max_abs"] <= TOL, rep
        if base is None:
            base = img
        else:
            assert np.array_equal(img, base)   # same fragments, same order, same arithmetic


def _check_fp64(rep, n_px):
    # decisions may differ from FP64 on fewer than 0.1% of the pixels, and everywhere else
    # the image is within the tolerance of the FP64 oracle's
    assert rep["decision_mismatch"] < 1e-3 * n_px, rep
    assert rep["max_abs_outside_mismatch"] <= TOL, rep


def test_render_workload2_full_frame():
    w = synthetic.workload(2)
    cam = w.cameras[0]
    xyz, rgb, a = oracle_mesh_f32(w.scene, 8, cam.C)
    img, r, _ = gpu_render(xyz, rgb, a, 8, cam)
    rep, _ = fp64_report(img, xyz, rgb, a, 8, cam)
    print(json.dumps({"workload": w.name, **rep, "pairs": r.last_info.pairs,
                      "extra_passes": r.last_info.extra_passes}))
    _check_fp64(rep, cam.width * cam.height)


def test_render_workload3_windows():
    w = synthetic.workload(3)
    cam = w.cameras[0]
    xyz, rgb, a = oracle_mesh_f32(w.scene, 8, cam.C)
    img, r, _ = gpu_render(xyz, rgb, a, 8, cam)
    # the image centre (sphere, blobs), the torus rim, and one seeded random window
    wins = [(912, 492, 1008, 588), (1500, 560, 1596, 656)]
    rng = np.random.default_rng(7)
    x0, y0 = int(rng.integers(0, 1920 - 96)), int(rng.integers(0, 1080 - 96))
    wins.append((x0, y0, x0 + 96, y0 + 96))
    for win in wins:
        g = img[win[1]:win[3], win[0]:win[2]]
        rep, _ = fp64_report(g, xyz, rgb, a, 8, cam, window=win)
        print(json.dumps({"workload": w.name, "window": win, **rep, "extra_passes": r.last_info.extra_passes}))
        _check_fp64(rep, 96 * 96)


# ---------------------------------------------------------------------------- edge cases

def _one_scene(means, log_s, quats, sigma, rgb=(0.8, 0.3, 0.2)):
    n = len(means)
    sh = np.zeros((n, 1, 3), np.float32)
    C0 = 0.5 / math.sqrt(math.pi)
    sh[:, 0, :] = (np.array(rgb) - 0.5) / C0
    return Scene(np.array(means, np.float32), np.array(log_s, np.float32), np.array(quats, np.float32),
                 np.array(sigma, np.float32), sh, 0)


def test_empty_and_invisible_scenes():
    cam = synthetic.make_camera((0.0, 0.0, 4.0), 64, 48)
    import paper_2502_07754_gb300 as ms
    r = ms.Renderer(0, 8, cam, ms.render_params(bg=(0.1, 0.2, 0.3)))
    e = torch.empty(0, 3, device="cuda")
    out = r.forward(e, e, torch.empty(0, device="cuda")).cpu().numpy()
    assert np.allclose(out[..., :3], [0.1, 0.2, 0.3]) and (out[..., 3] == 0).all()
    # everything behind the camera
    sc = _one_scene([[0, 0, 6.0], [0.2, 0, 7.0]], [[-9, -1, -1]] * 2, [[1, 0, 0, 0]] * 2, [0.9, 0.9])
    xyz, rgb, a = oracle_mesh_f32(sc, 8)
    img, r, _ = gpu_render(xyz, rgb, a, 8, cam)
    assert (img[..., 3] == 0).all()
    assert r.last_info.culled_tris == 16


def test_near_plane_straddling_fan():
    cam = synthetic.make_camera((0.0, 0.0, 1.0), 64, 64)
    # a big fan whose boundary crosses the camera plane: some triangles culled
    # thin axis 2; the fan spans the x axis and a direction tilted towards +z, so its
    # boundary reaches behind the camera plane
    sc = _one_scene([[0, 0, 0.5]], [[math.log(0.6), math.log(0.5), -9]], [[1, 0, 0, 0]], [0.7])
    sc.quats[0] = [math.cos(0.6), math.sin(0.6), 0, 0]
    xyz, rgb, a = oracle_mesh_f32(sc, 8)
    orc, nf, culled = oracle_render(xyz, rgb, a, 8, cam)
    img, r, _ = gpu_render(xyz, rgb, a, 8, cam)
    assert culled > 0 and r.last_info.culled_tris == culled
    assert err_report(img, orc)["max_abs"] <= TOL


def test_deep_stack_forces_buffer_overflow():
    """60 nearly coplanar fans over the same pixels: more pending fragments than the
    buffer holds, so pixels take extra passes -- the order must still be exact."""
    rng = np.random.default_rng(3)
    n = 60
    means = np.c_[rng.normal(0, 0.02, (n, 2)), rng.normal(0, 0.002, n)]
    q = rng.normal(0, 0.05, (n, 4)) + np.array([math.sqrt(0.5), 0, -math.sqrt(0.5), 0])   # thin axis -> z
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    sc = _one_scene(means, [[-9, math.log(0.15), math.log(0.12)]] * n, q, rng.uniform(0.05, 0.3, n))
    sc.sh[:, 0, :] = rng.normal(0, 1, (n, 3))
    cam = synthetic.make_camera((0.3, 0.2, 2.0), 96, 80)
    xyz, rgb, a = oracle_mesh_f32(sc, 8)
    orc, nf, _ = oracle_render(xyz, rgb, a, 8, cam)
    assert nf.max() > 40
    for kb in (8, 16):
        img, r, _ = gpu_render(xyz, rgb, a, 8, cam, kbuf=kb, T_eps=1e-30)
        assert r.last_info.extra_passes > 0
        rep = err_report(img, orc)
        print(json.dumps({"case": "deep-stack", "kbuf": kb, **rep, "extra_passes": r.last_info.extra_passes}))
        assert rep["max_abs"] <= TOL, rep


def test_capacity_overflow_is_reported_and_recovered():
    import paper_2502_07754_gb300 as ms
    from paper_2502_07754_gb300 import _lib
    w = synthetic.workload(1)
    cam = w.cameras[0]
    xyz, rgb, a = oracle_mesh_f32(w.scene, 8, cam.C)
    r = ms.Renderer(1000, 8, cam, ms.render_params(pair_capacity=100))
    X, Cc, A = dev(xyz), dev(rgb), dev(a)
    r.forward(X, Cc, A, check_status=False)
    st, inf = r.info()
    assert st == _lib.MS_ERR_CAPACITY and inf.overflow == 1 and inf.pairs > 100
    out = r.forward(X, Cc, A).cpu().numpy()
    orc, _, _ = oracle_render(xyz, rgb, a, 8, cam)
    assert err_report(out, orc)["max_abs"] <= TOL


def test_invalid_arguments_rejected():
    import ctypes as C
    import paper_2502_07754_gb300 as ms
    from paper_2502_07754_gb300 import _lib
    L = _lib.lib()
    cam = ms.camera_struct(synthetic.make_camera((0.0, 0.0, 4.0), 64, 64))
    p = ms.render_params(tile=12)
    assert L.ms_render(None, None, None, 0, 8, C.byref(cam), C.byref(p), None, None, 0, None) == _lib.MS_ERR_INVALID
    p = ms.render_params()
    assert L.ms_render(None, None, None, 10, 2, C.byref(cam), C.byref(p), None, None, 0, None) == _lib.MS_ERR_INVALID
    assert b"K=2" in L.ms_last_error()
