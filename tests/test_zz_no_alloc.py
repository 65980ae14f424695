"""ms_render_noalloc: the forward render for callers that cannot allocate device memory
(a plugin inside a host application that owns the GPU memory budget, a service that
reserves its device memory at start-up and allocates nothing afterwards).  Its scratch is
a fixed 64 MiB array inside the library.  This file is
collected last on purpose: if it fails, a run that stops at the first failure has already
run every other test."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synthetic  # noqa: E402

pytestmark = pytest.mark.gpu


def test_noalloc_render_matches_workspace_render_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_07754_gb300 as ms
    from paper_2502_07754_gb300 import _lib
    from gpu_util import dev, oracle_mesh_f32
    L = _lib.lib()
    w = synthetic.workload(1)
    cam = w.cameras[0]
    xyz, rgb, a = oracle_mesh_f32(w.scene, 8, cam.C)
    X, Cc, A = dev(xyz), dev(rgb), dev(a)
    ref = ms.Renderer(w.scene.n, 8, cam).forward(X, Cc, A)
    torch.cuda.synchronize()
    cs = ms.camera_struct(cam)
    p = ms.render_params()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        out = torch.full((cam.height, cam.width, 4), float("nan"), device="cuda")
        info = _lib.RenderInfo()
        st = L.ms_render_noalloc(C.c_void_p(X.data_ptr()), C.c_void_p(Cc.data_ptr()), C.c_void_p(A.data_ptr()),
                                 w.scene.n, 8, C.byref(cs), C.byref(p), C.c_void_p(out.data_ptr()), C.byref(info),
                                 stream)
        assert st == _lib.MS_OK, L.ms_last_error()
        assert info.pairs > 0 and info.overflow == 0
        assert torch.isfinite(out).all()
        # the same kernels on the same inputs: the image must be identical, not merely close
        assert torch.equal(out, ref), (out - ref).abs().max().item()


def test_noalloc_render_rejects_scenes_beyond_its_array():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_07754_gb300 as ms
    from paper_2502_07754_gb300 import _lib
    L = _lib.lib()
    cam = ms.camera_struct(synthetic.make_camera((0.0, 0.0, 3.0), 1920, 1080))
    p = ms.render_params()
    x = torch.zeros(9_000_000, 3, device="cuda")
    out = torch.empty(1080, 1920, 4, device="cuda")
    st = L.ms_render_noalloc(C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()), 1_000_000,
                             8, C.byref(cam), C.byref(p), C.c_void_p(out.data_ptr()), None,
                             C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == _lib.MS_ERR_INVALID
    assert b"ms_render_noalloc holds" in L.ms_last_error()
