"""GPU parity of the pruning step (ms_prune_fans) against oracle.prune_fans: the kept
soup and its Adam moments are data movement, so the comparison is bit-exact."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_07754_gb300._lib as L
    L.lib()


import paper_2502_07754_gb300 as ms  # noqa: E402


def _soup(n, K, frac_low, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    V = n * (K + 1)
    xyz = rng.normal(size=(V, 3)).astype(np.float32)
    rgb = rng.random((V, 3)).astype(np.float32)
    a = rng.uniform(0.0, 1.0, (n, K + 1)).astype(np.float32)
    low = rng.random(n) < frac_low
    a[low] *= np.float32(0.018)                                  # every vertex below exp(-4)
    part = (~low) & (rng.random(n) < 0.2)
    a[part, 0] = np.float32(0.001)                               # dim centre, brighter rim: kept
    a[rng.random(n) < 0.01, :] = np.float32(math.exp(-4.0))      # on the threshold: kept
    m = rng.normal(size=7 * V).astype(np.float32)
    v = rng.random(7 * V).astype(np.float32)
    return xyz, rgb, a.reshape(-1), m, v


@pytest.mark.parametrize("n,K,frac", [(10007, 8, 0.3), (3001, 6, 0.5), (777, 8, 0.0), (500, 8, 1.0), (0, 8, 0.5)])
def test_prune_matches_oracle_bit_for_bit(n, K, frac):
    xyz, rgb, a, m, v = _soup(n, K, frac, 40 + n)
    d = lambda t: torch.from_numpy(np.ascontiguousarray(t)).cuda()
    px, pc, pa, pm, pv, k = ms.prune_fans(d(xyz), d(rgb), d(a), K, m=d(m), v=d(v))
    thr = np.float32(math.exp(-4.0))
    ox, oc, oa, (om, ov), fans = oracle.prune_fans(xyz, rgb, a, K, threshold=thr, moments=(m, v))
    assert k == fans.size
    for got, want in ((px, ox), (pc, oc), (pa, oa), (pm, om), (pv, ov)):
        assert np.array_equal(got.cpu().numpy(), np.asarray(want, np.float32).reshape(got.shape))
    if n > 0 and 0 < frac < 1:
        assert 0 < k < n


def test_prune_without_moments_and_render_after():
    """Pruning without optimiser state, then rendering the kept soup: equal to the render
    of the full soup with the pruned fans' faces left out (the oracle's fan list)."""
    import synthetic
    from gpu_util import err_report
    w = synthetic.workload(1, n=600)
    cam = w.cameras[0]
    K = 8
    xyz, rgb, a = oracle.mesh_build(w.scene, K=K, cam_center=cam.C)
    xyz, rgb, a = xyz.astype(np.float32), rgb.astype(np.float32), a.astype(np.float32).copy()
    rng = np.random.Generator(np.random.PCG64(8))
    a.reshape(600, K + 1)[rng.random(600) < 0.4] *= np.float32(0.05)
    d = lambda t: torch.from_numpy(np.ascontiguousarray(t)).cuda()
    px, pc, pa, pm, pv, k = ms.prune_fans(d(xyz), d(rgb), d(a), K)
    assert pm is None and pv is None
    _, _, _, _, fans = oracle.prune_fans(xyz, rgb, a, K, threshold=np.float32(math.exp(-4.0)))
    assert k == fans.size
    img = ms.Renderer(k, K, cam).forward(px, pc, pa).cpu().numpy().astype(np.float64)
    tris = oracle.fan_tris(600, K).reshape(600, K, 3)[fans].reshape(-1, 3)
    ref, _, _ = oracle.render(xyz.astype(np.float64), rgb.astype(np.float64), a.astype(np.float64), tris, cam)
    rep = err_report(img, ref)
    assert rep["n_over_tol"] == 0, rep


def test_prune_on_a_side_stream_while_the_current_stream_is_busy():
    """The binding orders a named stream after the current one: inputs written and
    outputs allocated on the current stream are ready before the kernels read them, and
    the kept count read back is the kernels' result, not the allocation's zero fill."""
    K, n = 8, 20011
    xyz, rgb, a, m, v = _soup(n, K, 0.3, 7)
    d = lambda t: torch.from_numpy(np.ascontiguousarray(t)).cuda()
    X, Cc, m_d, v_d = d(xyz), d(rgb), d(m), d(v)
    A = torch.zeros(a.size, device="cuda")
    big = torch.randn(4096, 4096, device="cuda")
    for _ in range(8):                                   # keep the current stream busy ...
        big = big @ big / 64.0
    A.copy_(d(a))                                        # ... and write an input behind that work
    side = torch.cuda.Stream()
    px, pc, pa, pm, pv, k = ms.prune_fans(X, Cc, A, K, m=m_d, v=v_d, stream=side)
    torch.cuda.synchronize()
    _, _, oa, (om, _), fans = oracle.prune_fans(xyz, rgb, a, K, threshold=np.float32(math.exp(-4.0)),
                                                moments=(m, v))
    assert k == fans.size and 0 < k < n
    assert np.array_equal(pa.cpu().numpy(), np.asarray(oa, np.float32).reshape(-1))
    assert np.array_equal(pm.cpu().numpy(), np.asarray(om, np.float32).reshape(-1))
