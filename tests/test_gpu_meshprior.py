"""Explicit triangles and the mesh-prior mode on the GPU: the centroid-fan conversion
against oracle/meshprior.py, the explicit-mesh render and adjoint against the FP64
oracle's render of the triangles themselves, and the mesh-prior builder and weight
adjoint against the oracle's."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import synthetic  # noqa: E402
from oracle import meshprior as MP  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_07754_gb300._lib as L
    L.lib()


import paper_2502_07754_gb300 as ms  # noqa: E402
from gpu_util import dev, err_report  # noqa: E402


def _close(g, o, rel=1e-2, frac=1e-4):
    atol = frac * max(np.abs(o).max(), 1e-30)
    bad = np.abs(g - o) > rel * np.abs(o) + atol
    return int(bad.sum()), float(np.abs(g - o).max() / max(np.abs(o).max(), 1e-30))


def _mesh(seed=0):
    """Two jittered spheres (shared vertices) with random colours and opacities."""
    V1, F1 = synthetic.sphere_mesh(24, 40, 0.8, (0.1, 0.0, 0.0), jitter=2e-3, seed=seed)
    V2, F2 = synthetic.sphere_mesh(16, 24, 0.4, (-0.4, 0.3, 0.6), jitter=2e-3, seed=seed + 1)
    V = np.concatenate([V1, V2])
    F = np.concatenate([F1, F2 + V1.shape[0]]).astype(np.int32)
    rng = np.random.Generator(np.random.PCG64(seed + 2))
    rgb = rng.random((V.shape[0], 3)).astype(np.float32)
    a = rng.uniform(0.2, 0.9, V.shape[0]).astype(np.float32)
    return V, rgb, a, F


def test_centroid_fans_match_the_oracle():
    V, rgb, a, F = _mesh(3)
    fx, fc, fa = (t.cpu().numpy() for t in ms.tris_to_fans(dev(V), dev(rgb), dev(a), dev(F)))
    ox, oc, oa = MP.as_centroid_fans(V[F].astype(np.float64), rgb[F].astype(np.float64), a[F].astype(np.float64))
    for g, o in ((fx, ox), (fc, oc), (fa, oa)):
        o32 = np.asarray(o, np.float32).reshape(g.shape)
        # the centroid is the nearest binary32 value of the exact mean (the oracle rounds its
        # FP64 mean, so the two can differ by one unit in rare double-rounding cases)
        ulp = np.abs(g.view(np.int32).astype(np.int64) - o32.view(np.int32).astype(np.int64))
        assert ulp.max() <= 1 and (ulp > 0).mean() < 1e-3


def test_explicit_mesh_render_and_adjoint_match_the_triangles():
    V, rgb, a, F = _mesh(5)
    cam = synthetic.make_camera((0.4, 0.3, 3.0), 320, 256)
    r = ms.MeshRenderer(F.shape[0], cam)
    X, Cc, A, Tr = dev(V), dev(rgb), dev(a), dev(F)
    out = r.forward(X, Cc, A, Tr)
    img = out.cpu().numpy().astype(np.float64)
    ref, mm, _ = oracle.decision_mismatch(V.astype(np.float64), rgb.astype(np.float64), a.astype(np.float64), F, cam)
    rep = err_report(img, ref)
    d = np.abs(img - ref).max(-1)
    print(json.dumps({"case": "explicit-mesh", **rep}))
    # the triangles drawn as centroid fans: the same pixels and values as the triangles
    # (a difference would need a pixel centre within rounding of an edge)
    assert rep["n_over_tol"] == 0, rep
    dL = np.random.default_rng(6).normal(size=img.shape)
    gx, gc, ga = r.backward(X, Cc, A, Tr, out, dev(dL.astype(np.float32)))
    ox, oc, oa = oracle.render_backward(V.astype(np.float64), rgb.astype(np.float64), a.astype(np.float64), F, cam,
                                        dL)
    for name, g, o in (("xyz", gx, ox), ("rgb", gc, oc), ("alpha", ga, oa)):
        nbad, rel = _close(g.cpu().numpy().astype(np.float64), o)
        assert nbad == 0, (name, nbad, rel)


def _prior(F, S, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    Vm, Fm = synthetic.sphere_mesh(10, 16, 0.9, jitter=1e-3, seed=seed)
    faces = Vm[Fm][:F].astype(np.float32)
    w = (MP.init_weights(faces.shape[0], S) + rng.normal(0, 0.05, (faces.shape[0], S, 3, 3))).astype(np.float32)
    w = np.where(np.abs(w) < 0.05, np.float32(0.05), w).astype(np.float32)
    rgb = rng.random((faces.shape[0], S, 3, 3)).astype(np.float32)
    alpha = rng.uniform(0.2, 0.9, (faces.shape[0], S, 3)).astype(np.float32)
    return faces, w, rgb, alpha


@pytest.mark.parametrize("S", [1, 4])
def test_mesh_prior_build_matches_the_oracle(S):
    faces, w, rgb, alpha = _prior(400, S, 11)
    fx, fc, fa = (t.cpu().numpy().astype(np.float64) for t in ms.mesh_prior_build(dev(faces), dev(w), dev(rgb),
                                                                               dev(alpha)))
    xyz, c, a, _ = MP.triangle_soup(faces.astype(np.float64), w.astype(np.float64), rgb, alpha)
    ox, oc, oa = MP.as_centroid_fans(xyz, c, a)
    assert np.abs(fx - ox).max() < 2e-6 * max(1.0, np.abs(ox).max())
    assert np.abs(fc - oc).max() < 1e-6 and np.abs(fa - oa).max() < 1e-6


def test_mesh_prior_render_and_weight_adjoint_match_the_oracle():
    """Render the secondary triangles (S = 4 per face) as centroid fans and fold the fan
    adjoint to the weights: against the oracle's reverse pass over the same fan soup, its
    fan-to-triangle map and its weight gradient."""
    faces, w, rgb, alpha = _prior(300, 4, 12)
    cam = synthetic.make_camera((0.2, 0.3, 2.8), 256, 256)
    F, S = faces.shape[0], 4
    fx, fc, fa = ms.mesh_prior_build(dev(faces), dev(w), dev(rgb), dev(alpha))
    r = ms.Renderer(F * S, 3, cam)
    out = r.forward(fx, fc, fa)
    img = out.cpu().numpy().astype(np.float64)
    P, Cf, Af = (t.cpu().numpy().astype(np.float64) for t in (fx, fc, fa))
    ftris = oracle.fan_tris(F * S, 3)
    ref, _, _ = oracle.render(P, Cf, Af, ftris, cam)
    rep = err_report(img, ref)
    assert rep["n_over_tol"] == 0, rep
    dL = np.random.default_rng(7).normal(size=img.shape)
    r.backward(fx, fc, fa, out, dev(dL.astype(np.float32)), into_workspace=True)
    dw, dc, da = (t.cpu().numpy().astype(np.float64) for t in ms.mesh_prior_backward(dev(faces), dev(w), renderer=r))
    gx, gc, ga = oracle.render_backward(P, Cf, Af, ftris, cam, dL)
    tx, tc, ta = MP.fan_grads_to_triangles(gx, gc, ga)
    ow = MP.weight_grads(faces.astype(np.float64), w.astype(np.float64), tx.reshape(F, S, 3, 3))
    for name, g, o in (("w", dw, ow), ("rgb", dc.reshape(-1), tc.reshape(-1)), ("alpha", da.reshape(-1), ta)):
        nbad, rel = _close(g.reshape(o.shape), o)
        assert nbad == 0, (name, nbad, rel)
