"""The C-ABI library builds, loads without a GPU and exports every entry point that
include/*.h declares; host-side argument checks run without touching the device."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        names += re.findall(r"MS_API\s+[\w\s\*]+?\b(ms_\w+)\s*\(", txt)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("ms_mesh_build", "ms_render", "ms_render_backward", "ms_render_workspace_size",
                     "ms_render_get_info", "ms_l1_loss", "ms_adam_step"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2502_07754_gb300 import _lib
    L = _lib.lib()
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing
    assert L.ms_version().startswith(b"meshsplats")


def test_python_binding_covers_every_symbol():
    from paper_2502_07754_gb300 import _lib
    assert set(declared_symbols()) <= set(_lib._SIGS)


def test_host_side_validation_without_gpu():
    import paper_2502_07754_gb300 as ms
    from paper_2502_07754_gb300 import _lib
    import synthetic
    L = _lib.lib()
    cam = ms.camera_struct(synthetic.make_camera((0.0, 0.0, 4.0), 64, 64))
    p = ms.render_params()
    assert L.ms_render_workspace_size(100, 8, C.byref(cam), C.byref(p)) > 0
    assert L.ms_render_workspace_size(100, 2, C.byref(cam), C.byref(p)) == 0
    bad = ms.render_params(tile=12)
    assert L.ms_render(None, None, None, 0, 8, C.byref(cam), C.byref(bad), None, None, 0, None) == _lib.MS_ERR_INVALID
    assert b"tile" in L.ms_last_error()
    assert L.ms_render(None, None, None, 5, 8, C.byref(cam), C.byref(p), None, None, 0, None) == _lib.MS_ERR_INVALID
    cam.znear = 0.0
    assert L.ms_render(None, None, None, 0, 8, C.byref(cam), C.byref(p), None, None, 0, None) == _lib.MS_ERR_INVALID
    assert b"znear" in L.ms_last_error()
    fp = _lib.FanParams(2, 2.7, 0.2, 1)
    assert L.ms_mesh_build(None, None, None, None, None, 0, 0, 10, C.byref(fp), None, None, None, None, None,
                           None) == _lib.MS_ERR_INVALID


def test_host_side_validation_of_the_fine_tune_entry_points():
    """Argument checks of the full loss, pruning, the three-fan conversion and the pixel
    index bound return before any device work."""
    import paper_2502_07754_gb300 as ms
    from paper_2502_07754_gb300 import _lib
    import synthetic
    L = _lib.lib()
    assert L.ms_fine_tune_loss_workspace_size(-1, 5) == 0
    assert L.ms_fine_tune_loss_workspace_size(1080, 1920) >= 9 * 4 * 1080 * 1920
    dummy = C.c_void_p(256)   # never dereferenced: every call below fails its checks first
    assert L.ms_fine_tune_loss(dummy, dummy, 8, 8, 1.5, dummy, dummy, dummy, 1 << 20, None) == _lib.MS_ERR_INVALID
    assert b"lambda" in L.ms_last_error()
    assert L.ms_fine_tune_loss(dummy, dummy, -3, 8, 0.6, dummy, dummy, dummy, 1 << 20, None) == _lib.MS_ERR_INVALID
    assert L.ms_fine_tune_loss(dummy, dummy, 8, 8, 0.6, dummy, None, dummy, 1 << 20, None) == _lib.MS_ERR_INVALID
    assert L.ms_fine_tune_loss(dummy, dummy, 8, 8, 0.6, dummy, dummy, dummy, 64, None) == _lib.MS_ERR_INVALID
    assert b"workspace" in L.ms_last_error()

    assert L.ms_prune_workspace_size(-1) == 0 and L.ms_prune_workspace_size(10 ** 6) > 0
    args = [dummy, dummy, dummy, None, None, 10, 2, 0.018, dummy, dummy, dummy, None, None, dummy, dummy, 1 << 20, None]
    assert L.ms_prune_fans(*args) == _lib.MS_ERR_INVALID          # K = 2
    args[6] = 8
    args[3] = dummy                                                # m given without m_out
    assert L.ms_prune_fans(*args) == _lib.MS_ERR_INVALID
    assert b"both" in L.ms_last_error()
    args[3] = None
    args[13] = None                                                # no n_kept
    assert L.ms_prune_fans(*args) == _lib.MS_ERR_INVALID

    fp = _lib.FanParams(2, 2.7, 0.2, 1)
    assert L.ms_mesh_build_3d(dummy, dummy, dummy, dummy, dummy, 0, 0, 10, C.byref(fp), None, dummy, dummy, dummy,
                              None) == _lib.MS_ERR_INVALID
    assert L.ms_mesh_build_3d(dummy, dummy, dummy, dummy, dummy, 0, 0, 10, None, None, dummy, dummy, dummy,
                              None) == _lib.MS_ERR_INVALID

    # 2^32 pixels or more over the views of one call: pixel indices are 32-bit in the records
    big = ms.camera_struct(synthetic.make_camera((0.0, 0.0, 4.0), 32768, 32768))
    cams = (_lib.Camera * 5)(*([big] * 5))
    p = ms.render_params()
    p.frag_capacity = 1000
    outs = (C.c_void_p * 5)(*([dummy] * 5))
    st = L.ms_batch_render(None, None, None, 0, 8, cams, 5, C.byref(p), outs, dummy, 1 << 40, None)
    assert st == _lib.MS_ERR_INVALID
    assert b"pixels" in L.ms_last_error()


def test_spatial_order_argument_checks_without_gpu():
    from paper_2502_07754_gb300 import _lib
    L = _lib.lib()
    assert L.ms_spatial_order_workspace_size(-1) == 0
    assert L.ms_spatial_order_workspace_size(1 << 31) == 0
    assert L.ms_spatial_order_workspace_size(1000) > 8 * 1000 * 2
    assert L.ms_spatial_order(None, 10, None, None, 0, None) == _lib.MS_ERR_INVALID
    assert L.ms_spatial_order(None, 0, None, None, 0, None) == _lib.MS_OK       # nothing to order
    assert L.ms_gather_rows(None, 10, 6, None, None, None) == _lib.MS_ERR_INVALID   # row not whole words
    assert b"row" in L.ms_last_error()
    assert L.ms_gather_rows(None, 10, 8, None, None, None) == _lib.MS_ERR_INVALID
