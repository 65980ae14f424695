"""Storage order of the Gaussians on the GPU (ms_spatial_order, ms_gather_rows): the
permutation against the Morton order computed here from its stated definition, the row
gather against indexing, and the render and its adjoint unchanged by the order (the method
does not depend on the order of its inputs, except exact depth ties)."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synthetic  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_07754_gb300._lib as L
    L.lib()


import paper_2502_07754_gb300 as ms  # noqa: E402
from gpu_util import dev  # noqa: E402


def _dilate3(x):
    x = x.astype(np.uint64) & np.uint64(0x3FF)
    out = np.zeros_like(x)
    for b in range(10):
        out |= ((x >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b)
    return out


def morton_order(means):
    """(code, index) order of the Morton codes as the header defines them, in binary32."""
    m = np.asarray(means, np.float32)
    lo, hi = m.min(axis=0), m.max(axis=0)
    ext = (hi - lo).astype(np.float32)
    ext = np.where(ext > 0, ext, np.float32(1.0)).astype(np.float32)
    q = np.floor(((m - lo).astype(np.float32) / ext).astype(np.float32) * np.float32(1024.0))
    q = np.clip(q, 0, 1023).astype(np.uint64)
    code = (_dilate3(q[:, 0]) << np.uint64(2)) | (_dilate3(q[:, 1]) << np.uint64(1)) | _dilate3(q[:, 2])
    return np.lexsort((np.arange(len(m)), code)), code


@pytest.mark.parametrize("n", [1, 1000, 70001])
def test_permutation_is_the_morton_order(n):
    sc = synthetic.surface_scene(n, 900 + n, degree=0, clustered=True)
    perm = ms.spatial_order(dev(sc.means)).cpu().numpy()
    want, code = morton_order(sc.means)
    assert sorted(perm.tolist()) == list(range(n))          # a permutation
    assert np.array_equal(perm, want)                        # codes ascending, ties by index
    assert (np.diff(code[perm].astype(np.int64)) >= 0).all()


def test_degenerate_boxes():
    # every mean equal (zero extent on all axes), and a flat axis
    m = np.ones((500, 3), np.float32)
    assert np.array_equal(ms.spatial_order(dev(m)).cpu().numpy(), np.arange(500))
    rng = np.random.default_rng(3)
    m2 = rng.normal(size=(2000, 3)).astype(np.float32)
    m2[:, 1] = 0.25
    want, _ = morton_order(m2)
    assert np.array_equal(ms.spatial_order(dev(m2)).cpu().numpy(), want)


def test_gather_rows_equals_indexing():
    rng = np.random.default_rng(4)
    perm = torch.from_numpy(rng.permutation(3001).astype(np.int32)).cuda()
    for shape, dt in (((3001, 3), torch.float32), ((3001,), torch.float32), ((3001, 16, 3), torch.int16),
                      ((3001, 4), torch.float32)):
        t = torch.randint(-1000, 1000, shape, device="cuda").to(dt)
        assert torch.equal(ms.gather_rows(t, perm), t[perm.long()])


def test_render_and_adjoint_do_not_depend_on_the_order():
    w = synthetic.workload(3, n=60000)
    sc, K = w.scene, w.K
    cam = synthetic.make_camera(np.array([0.3, 0.4, 3.2]), 320, 240)
    shv = sc.sh.view(np.int16) if sc.sh_bf16 else sc.sh
    G = [dev(sc.means), dev(sc.log_scales), dev(sc.quats), dev(sc.opacity), dev(shv)]
    perm, *Gp = ms.spatially_ordered(*G)
    outs, grads = [], []
    for gs in (G, Gp):
        xyz, rgb, a = ms.mesh_build(*gs, sc.sh_degree, K=K, cam_center=cam.C)
        r = ms.Renderer(sc.n, K, cam)
        img = r.forward(xyz, rgb, a).clone()
        dL = torch.full_like(img, 1.0 / img.numel())
        dL[..., 3] = 0
        outs.append(img)
        grads.append(r.backward(xyz, rgb, a, img, dL))
    d = (outs[0] - outs[1]).abs()
    rep = {"max_abs": float(d.max()), "pixels_differing": int((d.amax(-1) > 0).sum())}
    print(json.dumps(rep))
    assert rep["max_abs"] <= 1e-4, rep
    # vertex v of reordered fan g is vertex v of fan perm[g]
    p = perm.long()
    vmap = (p[:, None] * (K + 1) + torch.arange(K + 1, device="cuda")[None, :]).reshape(-1)
    for g0, g1 in zip(grads[0], grads[1]):
        ref = g0[vmap]
        scale = ref.abs().max().item()
        assert scale > 0
        assert torch.allclose(g1, ref, rtol=1e-4, atol=1e-5 * scale), (g1 - ref).abs().max().item() / scale
