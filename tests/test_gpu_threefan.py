"""GPU parity of the three-fan conversion of 3D Gaussians (ms_mesh_build_3d) against
oracle/threefan.py, and of the render of the three-fan soup against the oracle's render of
the shared-vertex mesh."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synthetic  # noqa: E402
from oracle import threefan as TF  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_07754_gb300._lib as L
    L.lib()


import oracle  # noqa: E402
import paper_2502_07754_gb300 as ms  # noqa: E402
from gpu_util import dev, err_report, scene_tensors  # noqa: E402


@pytest.mark.parametrize("K", [8, 6, 5])
def test_three_fan_conversion_matches_oracle(K):
    sc = synthetic.random_scene(2000, 70 + K, degree=3)
    cc = np.array([0.3, -0.2, 3.5], np.float32)
    m, s, q, o, sh = scene_tensors(sc)
    x, c, a = ms.mesh_build_3d(m, s, q, o, sh, sc.sh_degree, K=K, cam_center=cc)
    ux, uc, ua, tris, nv = TF.three_fan_build(sc, K=K, cam_center=cc)
    fx, fc, fa, src = TF.as_implicit_fans(ux, uc, ua, K, nv)
    gx, gc, ga = (t.cpu().numpy() for t in (x, c, a))
    assert gx.shape == fx.shape
    assert np.abs(gx - fx).max() < 4e-6
    assert np.abs(gc - fc).max() < 2e-6
    assert np.abs(ga - fa).max() < 2e-7
    # every copy of a shared vertex (centre, axis tips) is the same bits in every fan
    order = np.argsort(src, kind="stable")
    s_sorted = src[order]
    first = np.r_[True, s_sorted[1:] != s_sorted[:-1]]
    head = order[np.maximum.accumulate(np.where(first, np.arange(src.size), 0))]
    for arr in (gx, gc, ga):
        assert np.array_equal(arr[order], arr[head])
    assert np.count_nonzero(~first) == sc.n * (3 * (K + 1) - nv)   # copies beyond the first


def test_three_fan_render_matches_the_shared_mesh():
    w = synthetic.workload(1, n=300)
    cam = w.cameras[0]
    K = 8
    ux, uc, ua, tris, nv = TF.three_fan_build(w.scene, K=K, cam_center=cam.C)
    ux, uc, ua = ux.astype(np.float32), uc.astype(np.float32), ua.astype(np.float32)
    fx, fc, fa, _ = TF.as_implicit_fans(ux, uc, ua, K, nv)
    r = ms.Renderer(3 * w.scene.n, K, cam)
    img = r.forward(dev(fx), dev(fc), dev(fa)).cpu().numpy().astype(np.float64)
    ref, _, _ = oracle.render(ux.astype(np.float64), uc.astype(np.float64), ua.astype(np.float64), tris, cam)
    rep = err_report(img, ref)
    assert rep["n_over_tol"] == 0, rep
    assert img[..., 3].max() > 0.1


def _close(g, o, rel=1e-2, frac=1e-4):
    atol = frac * max(np.abs(o).max(), 1e-30)
    bad = np.abs(g - o) > rel * np.abs(o) + atol
    return int(bad.sum()), float(np.abs(g - o).max() / max(np.abs(o).max(), 1e-30))


def test_summed_copy_gradients_equal_the_shared_mesh_gradients():
    """The adjoint of the copied-vertex fans, with each copy given the sum of its copies'
    gradients, equals the oracle's reverse pass over the shared-vertex mesh at every copy."""
    w = synthetic.workload(1, n=300)
    cam = w.cameras[0]
    K = 8
    sc = w.scene
    sc.opacity[:] = np.minimum(sc.opacity, 0.99)
    ux, uc, ua, tris, nv = TF.three_fan_build(sc, K=K, cam_center=cam.C)
    ux, uc, ua = ux.astype(np.float32), uc.astype(np.float32), ua.astype(np.float32)
    fx, fc, fa, src = TF.as_implicit_fans(ux, uc, ua, K, nv)
    r = ms.Renderer(3 * sc.n, K, cam)
    X, Cc, A = dev(fx), dev(fc), dev(fa)
    out = r.forward(X, Cc, A)
    dL = np.random.default_rng(5).normal(size=(cam.height, cam.width, 4))
    gx, gc, ga = r.backward(X, Cc, A, out, dev(dL.astype(np.float32)))
    ms.three_fan_sum_copies(sc.n, K, grads=(gx, gc, ga))
    ox, oc, oa = oracle.render_backward(ux.astype(np.float64), uc.astype(np.float64), ua.astype(np.float64), tris,
                                        cam, dL)
    for name, g, o in (("xyz", gx, ox), ("rgb", gc, oc), ("alpha", ga, oa)):
        g = g.cpu().numpy().astype(np.float64)
        nbad, rel = _close(g, o[src])
        assert nbad == 0, (name, nbad, rel)


def test_fine_tune_keeps_the_copies_one_vertex():
    """A few fine-tune steps of a three-fan soup with the gradients left in the render
    workspace, summed over copies, then Adam: the copies stay equal bit for bit."""
    w = synthetic.workload(1, n=300)
    cam = w.cameras[0]
    K = 6
    sc = w.scene
    m, s, q, o, sh = scene_tensors(sc)
    x, c, a = ms.mesh_build_3d(m, s, q, o, sh, sc.sh_degree, K=K, cam_center=cam.C)
    r = ms.Renderer(3 * sc.n, K, cam)
    target = torch.rand(cam.height, cam.width, 4, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    opt = ms.FanAdam(x, c, a, lr_color=5e-3)
    for _ in range(5):
        out = r.forward(x, c, a)
        _, dL = ms.l1_loss(out, target)
        r.backward(x, c, a, out, dL, into_workspace=True)
        ms.three_fan_sum_copies(sc.n, K, renderer=r)
        opt.step_ws(x, c, a, r)
    torch.cuda.synchronize()
    first, n_distinct = ms.three_fan_copies(K)
    first = np.asarray(first)
    slots = 3 * (K + 1)
    for arr in (x, c, a):
        v = arr.cpu().numpy().reshape(sc.n, slots, -1)
        assert np.array_equal(v, v[:, first, :])
    # and the fine-tune moved them
    x0, _, _ = ms.mesh_build_3d(m, s, q, o, sh, sc.sh_degree, K=K, cam_center=cam.C)
    assert (x - x0).abs().max().item() > 0
