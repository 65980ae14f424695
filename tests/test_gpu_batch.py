"""GPU parity of the multi-view batch render (ms_batch_render / ms_batch_render_backward):
every view of a batch equals the single-view render bit for bit and the oracle within
the image tolerance; the batch adjoint is the sum of the per-view adjoints; a CUDA graph
replay of the whole batch step equals the eager calls."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import synthetic  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_07754_gb300._lib as L
    L.lib()


from gpu_util import dev, err_report, oracle_mesh_f32, oracle_render  # noqa: E402
import paper_2502_07754_gb300 as ms  # noqa: E402
from paper_2502_07754_gb300 import _lib  # noqa: E402

K = 6


def _ragged_views():
    """Six cameras on a sphere of radius 3-5 with ragged sizes (odd, thin, one pixel)."""
    dirs = synthetic.fibonacci_dirs(6)
    sizes = [(97, 61), (128, 128), (200, 75), (64, 200), (33, 17), (1, 1)]
    radii = [3.0, 3.5, 4.0, 4.5, 5.0, 3.2]
    return [synthetic.make_camera(d * r, w, h) for d, r, (w, h) in zip(dirs, radii, sizes)]


@pytest.fixture(scope="module")
def soup():
    sc = synthetic.surface_scene(20000, 4401, degree=3, clustered=True)
    return oracle_mesh_f32(sc, K, cam_center=np.array([0.3, 0.2, 4.0], np.float32))


def _single(xyz, rgb, a, cam, prm):
    n = xyz.shape[0] // (K + 1)
    r = ms.Renderer(n, K, cam, prm)
    out = r.forward(xyz, rgb, a)
    return out, r


@pytest.mark.parametrize("tile,kbuf", [(16, 8), (8, 16), (32, 8)])
def test_batch_views_equal_single_renders(soup, tile, kbuf):
    X, Cc, A = (dev(t) for t in soup)
    cams = _ragged_views()
    n = X.shape[0] // (K + 1)
    br = ms.BatchRenderer(n, K, cams, ms.render_params(tile=tile, kbuf=kbuf))
    flat = br.forward(X, Cc, A)
    imgs = br.images(flat)
    for v, cam in enumerate(cams):
        one, _ = _single(X, Cc, A, cam, ms.render_params(tile=tile, kbuf=kbuf))
        assert imgs[v].shape == one.shape
        assert torch.equal(imgs[v], one), (v, (imgs[v] - one).abs().max().item())


def test_batch_vs_oracle(soup):
    X, Cc, A = (dev(t) for t in soup)
    cams = _ragged_views()
    n = X.shape[0] // (K + 1)
    br = ms.BatchRenderer(n, K, cams)
    imgs = [t.cpu().numpy().astype(np.float64) for t in br.images(br.forward(X, Cc, A))]
    for v, cam in enumerate(cams):
        ref, _, _ = oracle_render(*soup, K, cam)
        rep = err_report(imgs[v], ref)
        assert rep["n_over_tol"] == 0, (v, rep)


def test_batch_backward_is_sum_of_views(soup):
    X, Cc, A = (dev(t) for t in soup)
    cams = _ragged_views()
    n = X.shape[0] // (K + 1)
    br = ms.BatchRenderer(n, K, cams)
    flat = br.forward(X, Cc, A)
    g = torch.Generator(device="cuda").manual_seed(7)
    dL = torch.randn(flat.shape, device="cuda", generator=g)
    gb = br.backward(X, Cc, A, flat, dL)
    tot = [torch.zeros_like(X), torch.zeros_like(Cc), torch.zeros_like(A)]
    for v, cam in enumerate(cams):
        out, r = _single(X, Cc, A, cam, ms.render_params())
        dv = br.images(dL)[v].contiguous()
        r.backward(X, Cc, A, out, dv, *tot)
    for a, b in zip(gb, tot):
        scale = b.abs().max().item()
        assert scale > 0
        assert torch.allclose(a, b, rtol=1e-5, atol=1e-6 * scale), (a - b).abs().max().item()


def test_batch_graph_replay_matches_eager(soup):
    X, Cc, A = (dev(t) for t in soup)
    cams = _ragged_views()
    n = X.shape[0] // (K + 1)
    br = ms.BatchRenderer(n, K, cams)
    ref = br.forward(X, Cc, A)            # sizes the capacities
    g = torch.Generator(device="cuda").manual_seed(11)
    dL = torch.randn(ref.shape, device="cuda", generator=g)
    ref_g = br.backward(X, Cc, A, ref, dL)
    flat = br.new_flat()
    grads = [torch.zeros_like(X), torch.zeros_like(Cc), torch.zeros_like(A)]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        br.forward(X, Cc, A, flat, check_status=False)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    launches0 = ms._lib.lib().ms_kernel_launches()
    with torch.cuda.graph(graph):
        for t in grads:
            t.zero_()
        br.forward(X, Cc, A, flat, check_status=False)
        br.backward(X, Cc, A, flat, dL, *grads)
    assert ms._lib.lib().ms_kernel_launches() > launches0
    for _ in range(2):
        flat.fill_(-1.0)
        graph.replay()
        torch.cuda.synchronize()
        st, inf = br.info()
        assert st == _lib.MS_OK and inf.overflow == 0
        assert torch.equal(flat, ref)
        for a, b in zip(grads, ref_g):
            assert torch.allclose(a, b, rtol=1e-5, atol=1e-6 * b.abs().max().item())


def test_batch_invalid_arguments(soup):
    L = _lib.lib()
    cams = (_lib.Camera * 40)(*([ms.camera_struct(_ragged_views()[0])] * 40))
    prm = ms.render_params()
    assert L.ms_batch_workspace_size(100, K, cams, 0, C.byref(prm)) == 0
    assert L.ms_batch_workspace_size(100, K, cams, 33, C.byref(prm)) == 0
    assert L.ms_batch_workspace_size(100, K, cams, 32, C.byref(prm)) > 0
    X, Cc, A = (dev(t) for t in soup)
    n = X.shape[0] // (K + 1)
    ws = torch.empty(L.ms_batch_workspace_size(n, K, cams, 2, C.byref(prm)), dtype=torch.uint8, device="cuda")
    out = torch.empty(61, 97, 4, device="cuda")
    outs = (C.c_void_p * 2)(out.data_ptr(), None)
    s = L.ms_batch_render(C.c_void_p(X.data_ptr()), C.c_void_p(Cc.data_ptr()), C.c_void_p(A.data_ptr()), n, K, cams,
                          2, C.byref(prm), outs, C.c_void_p(ws.data_ptr()), ws.numel(), None)
    assert s == _lib.MS_ERR_INVALID
    s = L.ms_batch_render(C.c_void_p(X.data_ptr()), C.c_void_p(Cc.data_ptr()), C.c_void_p(A.data_ptr()), n, K, cams,
                          33, C.byref(prm), outs, C.c_void_p(ws.data_ptr()), ws.numel(), None)
    assert s == _lib.MS_ERR_INVALID


def test_batch_sixteen_view_workload_windows():
    """The 16-camera, mixed-resolution (512^2 .. 1080p) rig of the batched workload on a
    200k-Gaussian clustered scene: sampled 20 x 20 windows of every view vs the oracle."""
    w = synthetic.workload(4, n=200_000)
    soup = oracle_mesh_f32(w.scene, w.K)
    X, Cc, A = (dev(t) for t in soup)
    n = X.shape[0] // (w.K + 1)
    br = ms.BatchRenderer(n, w.K, w.cameras)
    imgs = br.images(br.forward(X, Cc, A))
    assert br.last_info.culled_tris == 0
    rng = np.random.Generator(np.random.PCG64(404))
    worst = 0.0
    for v, cam in enumerate(w.cameras):
        x0 = int(rng.integers(cam.width // 4, cam.width // 2))
        y0 = int(rng.integers(cam.height // 4, cam.height // 2))
        win = (x0, y0, x0 + 20, y0 + 20)
        ref, _, _ = oracle_render(*soup, w.K, cam, window=win)
        got = imgs[v][y0:y0 + 20, x0:x0 + 20].cpu().numpy().astype(np.float64)
        rep = err_report(got, ref)
        worst = max(worst, rep["max_abs"])
        assert rep["n_over_tol"] == 0, (v, rep)
    print("16-view window max abs err", worst)


def test_batch_autotune_picks_a_candidate_and_renders_identically(soup):
    X, Cc, A = (dev(t) for t in soup)
    cams = _ragged_views()
    n = X.shape[0] // (K + 1)
    br = ms.BatchRenderer(n, K, cams)
    ref = br.forward(X, Cc, A).clone()
    res = br.autotune(X, Cc, A, reps=2, headroom=0.05)
    ms_ = list(res.cand_ms)
    assert all(t > 0 for t in ms_), ms_                 # tile 8, 16, 32 x buffer 8, 16
    assert res.best in range(6) and res.best_ms == min(ms_)
    assert br.params.tile == 8 << (res.best // 2) and br.params.kbuf == 8 << (res.best % 2)
    assert br.params.pair_capacity >= res.pairs and br.params.frag_capacity >= res.frags
    out = br.forward(X, Cc, A)
    assert torch.equal(out, ref)


def test_counted_adam_replays_with_advancing_step():
    """Adam with the step number on the device, captured once in a CUDA graph and replayed
    three times, equals three host-numbered Adam steps."""
    g = torch.Generator(device="cuda").manual_seed(5)
    V = 10007
    p1 = [torch.randn(V, 3, device="cuda", generator=g), torch.rand(V, 3, device="cuda", generator=g),
          torch.rand(V, device="cuda", generator=g)]
    p2 = [t.clone() for t in p1]
    grads = [torch.randn(V, 3, device="cuda", generator=g), torch.randn(V, 3, device="cuda", generator=g),
             torch.randn(V, device="cuda", generator=g)]
    a1 = ms.FanAdam(*p1, lr_color=1e-2)
    a2 = ms.FanAdam(*p2, lr_color=1e-2, device_step=True)
    for _ in range(3):
        a1.step(*p1, *grads)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        a2.step(*p2, *grads)
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    assert int(a2.d_step.item()) == 3
    for x, y in zip(p1, p2):
        assert torch.allclose(x, y, rtol=1e-6, atol=1e-7), (x - y).abs().max().item()
