"""Thin torch front end of the C ABI: tensors supply device pointers and the current
stream; every step of the hot path runs in libmeshsplats.so.  There is no CPU or
eager fallback -- a missing library or a non-CUDA tensor is an error."""
from __future__ import annotations

import ctypes as C
import math

import torch

from . import _lib
from ._lib import check, lib

SCALE_MUL = 2.7
OPAC_MUL = 0.2
LR_XYZ_RATIO = math.exp(-3.0)   # Sec. 3: lr_verts = exp(-3) lr_color


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tensor must live on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return C.c_void_p(t.data_ptr())


def _stream(stream=None, *used):
    """Handle of the stream a call runs on.  When the caller names a stream other than the
    current one, that stream first waits for the current stream (where the inputs, outputs
    and workspaces were written or allocated), and every tensor in `used` is marked as used
    on it so that the caching allocator does not hand its memory out again before the
    call's work there has finished."""
    cur = torch.cuda.current_stream()
    if stream is None or stream == cur:
        return C.c_void_p(cur.cuda_stream)
    stream.wait_stream(cur)
    for t in used:
        if t is not None:
            t.record_stream(stream)
    return C.c_void_p(stream.cuda_stream)


def camera_struct(cam) -> _lib.Camera:
    c = _lib.Camera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    R = [float(x) for x in torch.as_tensor(cam.R_cw, dtype=torch.float32).reshape(9).tolist()]
    for i in range(9):
        c.R_cw[i] = R[i]
    Cc = [float(x) for x in torch.as_tensor(cam.C, dtype=torch.float32).reshape(3).tolist()]
    for i in range(3):
        c.C[i] = Cc[i]
    c.znear = float(cam.znear)
    return c


def render_params(tile=16, kbuf=8, T_eps=1e-5, bg=(0.0, 0.0, 0.0), pair_capacity=0, depth_bits=0, face_mask=None):
    """face_mask: None (every face drawn) or a device int32 tensor, one word per fan (bit j:
    face j drawn); the tensor must stay alive while the parameters are used."""
    p = _lib.RenderParams()
    lib().ms_render_params_default(C.byref(p))
    p.tile, p.kbuf, p.T_eps = int(tile), int(kbuf), float(T_eps)
    for i in range(3):
        p.bg[i] = float(bg[i])
    p.pair_capacity = int(pair_capacity)
    p.depth_bits = int(depth_bits)
    if face_mask is not None:
        if face_mask.dtype != torch.int32 or not face_mask.is_cuda or not face_mask.is_contiguous():
            raise ValueError("face_mask must be a contiguous int32 CUDA tensor")
        p.face_mask = face_mask.data_ptr()
    return p


def mesh_build(means, log_scales, quats, opacity, sh, sh_degree, K=8, scale_mul=SCALE_MUL, opac_mul=OPAC_MUL,
               axis_rule=1, cam_center=None, corr=None, stream=None, out=None, mlp=None):
    """Gaussians -> fan soup (xyz, rgb, alpha) on the device.  sh is float32 or a uint16 /
    int16 / bfloat16 tensor of bfloat16 bits, shape (N, (deg+1)^2, 3).  `out` may give the
    three output tensors (V x 3, V x 3, V) to write into.  corr: corrections from
    FanMLP.forward; or mlp: a FanMLP whose inference runs fused into the conversion
    (ms_mesh_build_mlp: the corrections stay on chip)."""
    if corr is not None and mlp is not None:
        raise ValueError("give corr or mlp, not both")
    N = means.shape[0]
    dev = means.device
    V = N * (K + 1)
    if out is not None:
        xyz, rgb, alpha = out
        if xyz.shape != (V, 3) or rgb.shape != (V, 3) or alpha.shape != (V,):
            raise ValueError("out tensors do not match N (K+1) vertices")
    else:
        xyz = torch.empty(V, 3, device=dev, dtype=torch.float32)
        rgb = torch.empty(V, 3, device=dev, dtype=torch.float32)
        alpha = torch.empty(V, device=dev, dtype=torch.float32)
    fp = _lib.FanParams(int(K), float(scale_mul), float(opac_mul), int(axis_rule))
    sh_dtype = 0 if sh.dtype == torch.float32 else 1
    cc = (C.c_float * 3)(*[float(x) for x in cam_center]) if cam_center is not None else None
    if mlp is not None:
        if mlp.n_out != 2 * (K + 1):
            raise ValueError("the FanMLP predicts %d outputs, K = %d needs %d" % (mlp.n_out, K, 2 * (K + 1)))
        check(lib().ms_mesh_build_mlp(_ptr(means), _ptr(log_scales), _ptr(quats), _ptr(opacity), _ptr(sh), sh_dtype,
                                      int(sh_degree), N, C.byref(fp), cc, _ptr(mlp.packed), _ptr(xyz), _ptr(rgb),
                                      _ptr(alpha), _stream(stream, xyz, rgb, alpha)))
        return xyz, rgb, alpha
    check(lib().ms_mesh_build(_ptr(means), _ptr(log_scales), _ptr(quats), _ptr(opacity), _ptr(sh), sh_dtype,
                              int(sh_degree), N, C.byref(fp), cc, _ptr(corr), _ptr(xyz), _ptr(rgb), _ptr(alpha),
                              _stream(stream, xyz, rgb, alpha)))
    return xyz, rgb, alpha


def mesh_build_3d(means, log_scales, quats, opacity, sh, sh_degree, K=8, scale_mul=SCALE_MUL, opac_mul=OPAC_MUL,
                  cam_center=None, stream=None):
    """3D Gaussians -> three fans per Gaussian (ms_mesh_build_3d): (xyz, rgb, alpha) with
    3 N (K+1) vertices, to be rendered as 3 N fans of K triangles."""
    N = means.shape[0]
    dev = means.device
    V = 3 * N * (K + 1)
    xyz = torch.empty(V, 3, device=dev, dtype=torch.float32)
    rgb = torch.empty(V, 3, device=dev, dtype=torch.float32)
    alpha = torch.empty(V, device=dev, dtype=torch.float32)
    fp = _lib.FanParams(int(K), float(scale_mul), float(opac_mul), 1)
    sh_dtype = 0 if sh.dtype == torch.float32 else 1
    cc = (C.c_float * 3)(*[float(x) for x in cam_center]) if cam_center is not None else None
    check(lib().ms_mesh_build_3d(_ptr(means), _ptr(log_scales), _ptr(quats), _ptr(opacity), _ptr(sh), sh_dtype,
                                 int(sh_degree), N, C.byref(fp), cc, _ptr(xyz), _ptr(rgb), _ptr(alpha),
                                 _stream(stream, xyz, rgb, alpha)))
    return xyz, rgb, alpha


def spatial_order(means, stream=None):
    """Permutation (int32 device tensor of N) that puts the Gaussians in Morton order of
    their means (ms_spatial_order)."""
    N = int(means.shape[0])
    perm = torch.empty(N, dtype=torch.int32, device=means.device)
    ws = torch.empty(max(int(lib().ms_spatial_order_workspace_size(N)), 256), dtype=torch.uint8, device=means.device)
    check(lib().ms_spatial_order(_ptr(means.contiguous()), N, _ptr(perm), _ptr(ws), ws.numel(),
                                 _stream(stream, perm, ws)))
    return perm


def gather_rows(t, perm, stream=None):
    """Rows of t (first dimension) in the order perm (ms_gather_rows): out[i] = t[perm[i]]."""
    t = t.contiguous()
    out = torch.empty_like(t)
    n = int(t.shape[0])
    row = t.element_size() * (t.numel() // max(n, 1))
    check(lib().ms_gather_rows(_ptr(t), n, row, _ptr(perm), _ptr(out), _stream(stream, out)))
    return out


def spatially_ordered(means, *attrs, stream=None):
    """The Gaussians' arrays (means first, then any per-Gaussian arrays) in Morton order of
    the means, and the permutation: (perm, means', *attrs')."""
    perm = spatial_order(means, stream=stream)
    return (perm, gather_rows(means, perm, stream=stream)) + tuple(gather_rows(a, perm, stream=stream) for a in attrs)


def three_fan_copies(K):
    """Copy map of one Gaussian's 3 (K+1) three-fan vertex slots (ms_three_fan_copies):
    (first-copy slot of every slot as a list, number of distinct vertices)."""
    buf = (C.c_int32 * (3 * (K + 1)))()
    n = lib().ms_three_fan_copies(int(K), buf)
    if n < 0:
        raise ValueError(f"K={K} outside 3..16")
    return list(buf), int(n)


def three_fan_sum_copies(N, K, grads=None, renderer=None, stream=None):
    """Gives every copy of a shared three-fan vertex the sum of its copies' gradients
    (ms_three_fan_sum_copies), in place: either grads = (d_xyz, d_rgb, d_alpha) or the
    gradient sums a renderer's backward left in its workspace."""
    if renderer is not None:
        check(lib().ms_three_fan_sum_copies(None, None, None, renderer.grad_ptr(), int(N), int(K),
                                            _stream(stream, renderer.ws)))
        return None
    d_xyz, d_rgb, d_alpha = grads
    check(lib().ms_three_fan_sum_copies(_ptr(d_xyz), _ptr(d_rgb), _ptr(d_alpha), None, int(N), int(K),
                                        _stream(stream, d_xyz, d_rgb, d_alpha)))
    return grads


class Renderer:
    """Owns a render workspace for one (fan count, K, camera, params) and grows its pair
    capacity when a render reports MS_ERR_CAPACITY."""

    def __init__(self, n_fans: int, K: int, cam, params=None, device="cuda"):
        self.n_fans, self.K = int(n_fans), int(K)
        self.cam = cam if isinstance(cam, _lib.Camera) else camera_struct(cam)
        self.params = params if params is not None else render_params()
        self.device = torch.device(device)
        self._alloc()

    def _alloc(self):
        n = lib().ms_render_workspace_size(self.n_fans, self.K, C.byref(self.cam), C.byref(self.params))
        if n == 0:
            raise ValueError("invalid render configuration")
        self.ws = torch.empty(int(n), dtype=torch.uint8, device=self.device)

    @property
    def shape(self):
        return (self.cam.height, self.cam.width)

    def info(self, stream=None):
        inf = _lib.RenderInfo()
        st = lib().ms_render_get_info(_ptr(self.ws), C.byref(inf), _stream(stream))
        return st, inf

    def forward(self, xyz, rgb, alpha, out=None, check_status=True, stream=None):
        if out is None:
            out = torch.empty(self.cam.height, self.cam.width, 4, device=xyz.device, dtype=torch.float32)
        for _ in range(4):
            check(lib().ms_render(_ptr(xyz), _ptr(rgb), _ptr(alpha), self.n_fans, self.K, C.byref(self.cam),
                                  C.byref(self.params), _ptr(out), _ptr(self.ws), self.ws.numel(),
                                  _stream(stream, out, self.ws)))
            if not check_status:
                return out
            st, inf = self.info(stream)
            if st == _lib.MS_ERR_CAPACITY:
                if inf.pairs > inf.pair_capacity:
                    self.params.pair_capacity = int(inf.pairs * 1.25) + 4096
                if inf.frags > inf.frag_capacity:
                    self.params.frag_capacity = int(inf.frags * 1.25) + 65536
                self._alloc()
                continue
            check(st)
            self.last_info = inf
            return out
        raise _lib.MSError(_lib.MS_ERR_CAPACITY, "pair capacity did not converge")

    def backward(self, xyz, rgb, alpha, out_rgba, dL, d_xyz=None, d_rgb=None, d_alpha=None, stream=None,
                 into_workspace=False):
        """Accumulates the adjoint into (d_xyz, d_rgb, d_alpha); with into_workspace the
        gradients stay in the workspace for FanAdam.step_ws and None is returned."""
        if into_workspace:
            check(lib().ms_render_backward(_ptr(xyz), _ptr(rgb), _ptr(alpha), self.n_fans, self.K,
                                           C.byref(self.cam), C.byref(self.params), _ptr(out_rgba),
                                           _ptr(dL.contiguous()), None, None, None, _ptr(self.ws), self.ws.numel(),
                                           _stream(stream, self.ws)))
            return None
        if d_xyz is None:
            d_xyz = torch.zeros_like(xyz)
            d_rgb = torch.zeros_like(rgb)
            d_alpha = torch.zeros_like(alpha)
        check(lib().ms_render_backward(_ptr(xyz), _ptr(rgb), _ptr(alpha), self.n_fans, self.K, C.byref(self.cam),
                                       C.byref(self.params), _ptr(out_rgba), _ptr(dL.contiguous()), _ptr(d_xyz),
                                       _ptr(d_rgb), _ptr(d_alpha), _ptr(self.ws), self.ws.numel(),
                                       _stream(stream, d_xyz, d_rgb, d_alpha, self.ws)))
        return d_xyz, d_rgb, d_alpha

    def grad_ptr(self):
        """Device address of the gradients a backward with into_workspace left behind."""
        off = lib().ms_render_grad_offset(self.n_fans, self.K, C.byref(self.cam), 1, C.byref(self.params))
        return C.c_void_p(self.ws.data_ptr() + int(off))


def tris_to_fans(xyz, rgb, alpha, tris=None, stream=None):
    """Explicit triangles (tris: T x 3 int32 device tensor, or None for a soup of
    consecutive vertex triples) as centroid fans of K = 3 (ms_tris_to_fans): returns the
    fan soup (4T x 3, 4T x 3, 4T)."""
    T = int(tris.shape[0]) if tris is not None else xyz.shape[0] // 3
    fx = torch.empty(4 * T, 3, device=xyz.device)
    fc = torch.empty(4 * T, 3, device=xyz.device)
    fa = torch.empty(4 * T, device=xyz.device)
    check(lib().ms_tris_to_fans(_ptr(xyz), _ptr(rgb), _ptr(alpha), _ptr(tris) if tris is not None else None, T,
                                _ptr(fx), _ptr(fc), _ptr(fa), _stream(stream, fx, fc, fa)))
    return fx, fc, fa


class MeshRenderer:
    """Explicit-topology render (ms_mesh_render / ms_mesh_render_backward): triangles index
    a shared vertex array; owns the workspace and grows its capacities on MS_ERR_CAPACITY."""

    def __init__(self, n_tris: int, cam, params=None, device="cuda"):
        self.T = int(n_tris)
        self.cam = cam if isinstance(cam, _lib.Camera) else camera_struct(cam)
        self.params = params if params is not None else render_params()
        self.device = torch.device(device)
        self._alloc()

    def _alloc(self):
        n = lib().ms_mesh_workspace_size(self.T, C.byref(self.cam), C.byref(self.params))
        if n == 0:
            raise ValueError("invalid render configuration")
        self.ws = None
        self.ws = torch.empty(int(n), dtype=torch.uint8, device=self.device)

    def _render_ws(self):
        soup = (4 * self.T * 28 + 255) // 256 * 256
        return C.c_void_p(self.ws.data_ptr() + soup)

    def forward(self, xyz, rgb, alpha, tris, out=None, stream=None):
        if out is None:
            out = torch.empty(self.cam.height, self.cam.width, 4, device=xyz.device)
        tp = _ptr(tris) if tris is not None else None
        for _ in range(4):
            check(lib().ms_mesh_render(_ptr(xyz), _ptr(rgb), _ptr(alpha), tp, self.T, C.byref(self.cam),
                                       C.byref(self.params), _ptr(out), _ptr(self.ws), self.ws.numel(),
                                       _stream(stream, out, self.ws)))
            inf = _lib.RenderInfo()
            st = lib().ms_render_get_info(self._render_ws(), C.byref(inf), _stream(stream))
            if st == _lib.MS_ERR_CAPACITY:
                if inf.pairs > inf.pair_capacity:
                    self.params.pair_capacity = int(inf.pairs * 1.25) + 4096
                if inf.frags > inf.frag_capacity:
                    self.params.frag_capacity = int(inf.frags * 1.25) + 65536
                self._alloc()
                continue
            check(st)
            self.last_info = inf
            return out
        raise _lib.MSError(_lib.MS_ERR_CAPACITY, "capacity did not converge")

    def backward(self, xyz, rgb, alpha, tris, out_rgba, dL, d_xyz=None, d_rgb=None, d_alpha=None, stream=None):
        if d_xyz is None:
            d_xyz, d_rgb, d_alpha = torch.zeros_like(xyz), torch.zeros_like(rgb), torch.zeros_like(alpha)
        check(lib().ms_mesh_render_backward(_ptr(xyz), _ptr(rgb), _ptr(alpha), _ptr(tris) if tris is not None else None,
                                            self.T, C.byref(self.cam), C.byref(self.params), _ptr(out_rgba),
                                            _ptr(dL.contiguous()), _ptr(d_xyz), _ptr(d_rgb), _ptr(d_alpha),
                                            _ptr(self.ws), self.ws.numel(),
                                            _stream(stream, d_xyz, d_rgb, d_alpha, self.ws)))
        return d_xyz, d_rgb, d_alpha


class RayTracer:
    """Ray tracing of a triangle soup with shadows (ms_bvh_build, ms_raytrace): tris is a
    T x 3 int32 device tensor, or None with K for the implicit fan topology."""

    def __init__(self, n_tris: int, K: int = 0, device="cuda"):
        self.T, self.K = int(n_tris), int(K)
        self.bvh = torch.empty(max(int(lib().ms_bvh_workspace_size(self.T)), 256), dtype=torch.uint8,
                               device=torch.device(device))

    def build(self, xyz, tris=None, stream=None):
        check(lib().ms_bvh_build(_ptr(xyz), _ptr(tris) if tris is not None else None, self.T, self.K,
                                 _ptr(self.bvh), self.bvh.numel(), _stream(stream, self.bvh)))

    def trace(self, xyz, rgb, alpha, cam, tris=None, light=None, ambient=1.0, T_eps=0.0, bg=(0.0, 0.0, 0.0),
              out=None, stream=None):
        cs = cam if isinstance(cam, _lib.Camera) else camera_struct(cam)
        if out is None:
            out = torch.empty(cs.height, cs.width, 4, device=xyz.device)
        lt = (C.c_float * 3)(*[float(x) for x in light]) if light is not None else None
        bgv = (C.c_float * 3)(*[float(x) for x in bg])
        check(lib().ms_raytrace(_ptr(xyz), _ptr(rgb), _ptr(alpha), _ptr(tris) if tris is not None else None, self.T,
                                self.K, _ptr(self.bvh), C.byref(cs), lt, float(ambient), float(T_eps), bgv, _ptr(out),
                                _stream(stream, out)))
        return out

    def status(self, stream=None):
        n = C.c_int32(0)
        st = lib().ms_bvh_status(_ptr(self.bvh), C.byref(n), _stream(stream))
        return st, n.value


def mesh_prior_build(faces, w, rgb, alpha, stream=None):
    """Secondary triangles of the mesh prior (ms_mesh_prior_build) as centroid fans:
    faces F x 3 x 3, w and rgb F x S x 3 x 3, alpha F x S x 3 -> fan soup (4FS x 3, 4FS x 3,
    4FS), to render as F S fans of K = 3."""
    F, S = int(w.shape[0]), int(w.shape[1])
    fx = torch.empty(4 * F * S, 3, device=w.device)
    fc = torch.empty(4 * F * S, 3, device=w.device)
    fa = torch.empty(4 * F * S, device=w.device)
    check(lib().ms_mesh_prior_build(_ptr(faces), _ptr(w), _ptr(rgb), _ptr(alpha), F, S, _ptr(fx), _ptr(fc), _ptr(fa),
                                    _stream(stream, fx, fc, fa)))
    return fx, fc, fa


def mesh_prior_backward(faces, w, fan_grads=None, renderer=None, out=None, stream=None):
    """Gradients of the weights and per-vertex attributes (ms_mesh_prior_backward) from the
    fan soup's gradients: three tensors, or the sums a renderer's backward left in its
    workspace.  Returns (d_w, d_rgb, d_alpha), added to `out` when given."""
    F, S = int(w.shape[0]), int(w.shape[1])
    if out is None:
        out = (torch.zeros_like(w), torch.zeros(F, S, 3, 3, device=w.device), torch.zeros(F, S, 3, device=w.device))
    dw, dc, da = out
    if renderer is not None:
        g = (None, None, None, renderer.grad_ptr())
    else:
        g = (_ptr(fan_grads[0]), _ptr(fan_grads[1]), _ptr(fan_grads[2]), None)
    check(lib().ms_mesh_prior_backward(_ptr(faces), _ptr(w), *g, F, S, _ptr(dw), _ptr(dc), _ptr(da),
                                       _stream(stream, dw, dc, da)))
    return dw, dc, da


class BatchRenderer:
    """Owns a workspace for rendering one fan soup into several views of any sizes with
    one pass of the pipeline (ms_batch_render).  Outputs of all views live in one flat
    device buffer (view v at pixel offset pix_base[v]), so the loss over the batch is
    one launch; `images(flat)` gives per-view H x W x 4 views of it."""

    def __init__(self, n_fans: int, K: int, cams, params=None, device="cuda"):
        cams = list(cams)
        if not 1 <= len(cams) <= _lib.MAX_VIEWS:
            raise ValueError(f"1..{_lib.MAX_VIEWS} views")
        self.n_fans, self.K, self.n_views = int(n_fans), int(K), len(cams)
        self.cams = (_lib.Camera * self.n_views)(
            *[c if isinstance(c, _lib.Camera) else camera_struct(c) for c in cams])
        self.params = params if params is not None else render_params()
        self.device = torch.device(device)
        self.pix_base = []
        n = 0
        for c in self.cams:
            self.pix_base.append(n)
            n += c.width * c.height
        self.n_pixels = n
        self._alloc()

    def _alloc(self):
        n = lib().ms_batch_workspace_size(self.n_fans, self.K, self.cams, self.n_views, C.byref(self.params))
        if n == 0:
            raise ValueError("invalid render configuration")
        self.ws = None
        self.ws = torch.empty(int(n), dtype=torch.uint8, device=self.device)

    def new_flat(self, fill=None):
        t = torch.empty(self.n_pixels, 4, device=self.device, dtype=torch.float32)
        if fill is not None:
            t.fill_(fill)
        return t

    def images(self, flat):
        """Per-view (H, W, 4) views of a flat n_pixels x 4 buffer."""
        return [flat[b:b + c.width * c.height].view(c.height, c.width, 4) for b, c in zip(self.pix_base, self.cams)]

    def _ptrs(self, flat):
        if flat.shape != (self.n_pixels, 4) or not flat.is_contiguous() or not flat.is_cuda:
            raise ValueError("expected a contiguous device buffer of n_pixels x 4 floats")
        base = flat.data_ptr()
        return (C.c_void_p * self.n_views)(*[base + 16 * b for b in self.pix_base])

    def info(self, stream=None):
        inf = _lib.RenderInfo()
        st = lib().ms_render_get_info(_ptr(self.ws), C.byref(inf), _stream(stream))
        return st, inf

    def forward(self, xyz, rgb, alpha, flat=None, check_status=True, stream=None):
        if flat is None:
            flat = self.new_flat()
        outs = self._ptrs(flat)
        for _ in range(4):
            check(lib().ms_batch_render(_ptr(xyz), _ptr(rgb), _ptr(alpha), self.n_fans, self.K, self.cams,
                                        self.n_views, C.byref(self.params), outs, _ptr(self.ws), self.ws.numel(),
                                        _stream(stream, flat, self.ws)))
            if not check_status:
                return flat
            st, inf = self.info(stream)
            if st == _lib.MS_ERR_CAPACITY:
                if inf.pairs > inf.pair_capacity:
                    self.params.pair_capacity = int(inf.pairs * 1.25) + 4096
                if inf.frags > inf.frag_capacity:
                    self.params.frag_capacity = int(inf.frags * 1.25) + 65536
                self._alloc()
                continue
            check(st)
            self.last_info = inf
            return flat
        raise _lib.MSError(_lib.MS_ERR_CAPACITY, "capacity did not converge")

    def autotune(self, xyz, rgb, alpha, reps=3, headroom=0.05, stream=None):
        """Runs ms_batch_autotune (tile, pending buffer, list capacities) on this scene
        and adopts the fastest candidate; returns the ms_tune_result."""
        flat = self.new_flat()
        dL = torch.full_like(flat, 1.0 / flat.numel())
        grads = [torch.empty_like(xyz), torch.empty_like(rgb), torch.empty_like(alpha)]
        sizes = []
        for tile in (8, 16):
            for kbuf in (8, 16):
                p = _lib.RenderParams.from_buffer_copy(self.params)
                p.tile, p.kbuf = tile, kbuf
                sizes.append(lib().ms_batch_workspace_size(self.n_fans, self.K, self.cams, self.n_views, C.byref(p)))
        ws = torch.empty(max(sizes), dtype=torch.uint8, device=self.device)
        res = _lib.TuneResult()
        best = _lib.RenderParams()
        for _ in range(2):
            st = lib().ms_batch_autotune(_ptr(xyz), _ptr(rgb), _ptr(alpha), self.n_fans, self.K, self.cams,
                                         self.n_views, C.byref(self.params), self._ptrs(flat), self._ptrs(dL),
                                         _ptr(grads[0]), _ptr(grads[1]), _ptr(grads[2]), _ptr(ws), ws.numel(),
                                         int(reps), float(headroom), C.byref(best), C.byref(res), _stream(stream))
            if st == _lib.MS_OK and all(res.cand_ms[c] != -2.0 for c in range(_lib.TUNE_CANDIDATES)):
                break
            want = max(res.cand_ws_bytes[c] for c in range(_lib.TUNE_CANDIDATES))
            if want <= ws.numel():
                break
            ws = None
            ws = torch.empty(int(want), dtype=torch.uint8, device=self.device)
        check(st)
        self.params = best
        self._alloc()
        return res

    def grad_ptr(self):
        off = lib().ms_render_grad_offset(self.n_fans, self.K, self.cams, self.n_views, C.byref(self.params))
        return C.c_void_p(self.ws.data_ptr() + int(off))

    def backward(self, xyz, rgb, alpha, flat, dL_flat, d_xyz=None, d_rgb=None, d_alpha=None, stream=None,
                 into_workspace=False):
        if into_workspace:
            check(lib().ms_batch_render_backward(_ptr(xyz), _ptr(rgb), _ptr(alpha), self.n_fans, self.K, self.cams,
                                                 self.n_views, C.byref(self.params), self._ptrs(flat),
                                                 self._ptrs(dL_flat), None, None, None, _ptr(self.ws),
                                                 self.ws.numel(), _stream(stream, self.ws)))
            return None
        if d_xyz is None:
            d_xyz = torch.zeros_like(xyz)
            d_rgb = torch.zeros_like(rgb)
            d_alpha = torch.zeros_like(alpha)
        check(lib().ms_batch_render_backward(_ptr(xyz), _ptr(rgb), _ptr(alpha), self.n_fans, self.K, self.cams,
                                             self.n_views, C.byref(self.params), self._ptrs(flat),
                                             self._ptrs(dL_flat), _ptr(d_xyz), _ptr(d_rgb), _ptr(d_alpha),
                                             _ptr(self.ws), self.ws.numel(),
                                             _stream(stream, d_xyz, d_rgb, d_alpha, self.ws)))
        return d_xyz, d_rgb, d_alpha


class SplatRenderer(BatchRenderer):
    """Renders the source Gaussians themselves (ms_splat_render) into several views:
    the reference image that the fans approximate.  Same flat-buffer layout as
    BatchRenderer."""

    def __init__(self, n_gaussians: int, cams, params=None, device="cuda", axis_rule=1):
        self.axis_rule = int(axis_rule)
        super().__init__(n_gaussians, 8, cams, params, device)

    def _alloc(self):
        n = lib().ms_splat_workspace_size(self.n_fans, self.cams, self.n_views, C.byref(self.params))
        if n == 0:
            raise ValueError("invalid render configuration")
        self.ws = None
        self.ws = torch.empty(int(n), dtype=torch.uint8, device=self.device)

    def render(self, means, log_scales, quats, opacity, rgb, flat=None, stream=None):
        """rgb: N x 3 colour per Gaussian (float32, device)."""
        if flat is None:
            flat = self.new_flat()
        outs = self._ptrs(flat)
        for _ in range(4):
            check(lib().ms_splat_render(_ptr(means), _ptr(log_scales), _ptr(quats), _ptr(opacity), _ptr(rgb),
                                        self.n_fans, self.axis_rule, self.cams, self.n_views, C.byref(self.params),
                                        outs, _ptr(self.ws), self.ws.numel(), _stream(stream, flat, self.ws)))
            st, inf = self.info(stream)
            if st == _lib.MS_ERR_CAPACITY:
                if inf.pairs > inf.pair_capacity:
                    self.params.pair_capacity = int(inf.pairs * 1.25) + 4096
                if inf.frags > inf.frag_capacity:
                    self.params.frag_capacity = int(inf.frags * 1.25) + 65536
                self._alloc()
                continue
            check(st)
            self.last_info = inf
            return flat
        raise _lib.MSError(_lib.MS_ERR_CAPACITY, "capacity did not converge")

    def forward(self, *a, **k):
        raise TypeError("SplatRenderer draws Gaussians: use render()")

    def backward(self, *a, **k):
        raise TypeError("the splat render has no adjoint")


class RenderFn(torch.autograd.Function):
    """Differentiable render of a fan soup; gradients for vertex positions, colours and
    opacities come from ms_render_backward (visibility held fixed)."""

    @staticmethod
    def forward(ctx, xyz, rgb, alpha, renderer: Renderer):
        out = renderer.forward(xyz.detach(), rgb.detach(), alpha.detach())
        ctx.renderer = renderer
        ctx.save_for_backward(xyz, rgb, alpha, out)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        xyz, rgb, alpha, out = ctx.saved_tensors
        d = ctx.renderer.backward(xyz.detach(), rgb.detach(), alpha.detach(), out, grad_out.contiguous())
        return d[0], d[1], d[2], None


def render(xyz, rgb, alpha, renderer: Renderer):
    return RenderFn.apply(xyz, rgb, alpha, renderer)


def l1_loss(img_rgba, target_rgba, stream=None):
    """Returns (loss as a 1-element device tensor, dL/d img_rgba)."""
    dL = torch.empty_like(img_rgba)
    loss = torch.empty(1, device=img_rgba.device, dtype=torch.float32)
    check(lib().ms_l1_loss(_ptr(img_rgba), _ptr(target_rgba), img_rgba.numel() // 4, _ptr(dL), _ptr(loss),
                           _stream(stream, dL, loss)))
    return loss, dL


def fine_tune_loss(img_rgba, target_rgba, lam=0.6, workspace=None, stream=None):
    """Eq. 3 read as lam * L1 + (1 - lam)(1 - SSIM) of H x W x 4 images: returns (loss as a
    1-element device tensor, dL/d img_rgba).  `workspace` (a uint8 device tensor of
    ms_fine_tune_loss_workspace_size bytes) may be passed to avoid an allocation per call."""
    H, W = int(img_rgba.shape[0]), int(img_rgba.shape[1])
    need = lib().ms_fine_tune_loss_workspace_size(H, W)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=img_rgba.device)
    dL = torch.empty_like(img_rgba)
    loss = torch.empty(1, device=img_rgba.device, dtype=torch.float32)
    check(lib().ms_fine_tune_loss(_ptr(img_rgba), _ptr(target_rgba), H, W, float(lam), _ptr(dL), _ptr(loss),
                                  _ptr(workspace), workspace.numel(), _stream(stream, dL, loss, workspace)))
    return loss, dL


def prune_fans(xyz, rgb, alpha, K, threshold=math.exp(-4.0), m=None, v=None, stream=None):
    """Pruning step (ms_prune_fans): removes the fans whose K + 1 vertex opacities are all
    below `threshold` and compacts the rest (and, if given, their Adam moments m, v in the
    FanAdam layout).  Returns (xyz, rgb, alpha, m, v, n_kept) with the kept fans only
    (reads the kept count back, so it synchronises the stream)."""
    n = xyz.shape[0] // (K + 1)
    outs = [torch.empty_like(t) for t in (xyz, rgb, alpha)]
    mo = torch.empty_like(m) if m is not None else None
    vo = torch.empty_like(v) if v is not None else None
    n_kept = torch.zeros(1, dtype=torch.int64, device=xyz.device)
    ws = torch.empty(max(lib().ms_prune_workspace_size(n), 1), dtype=torch.uint8, device=xyz.device)
    check(lib().ms_prune_fans(_ptr(xyz), _ptr(rgb), _ptr(alpha), _ptr(m) if m is not None else None,
                              _ptr(v) if v is not None else None, n, int(K), float(threshold), *[_ptr(t) for t in outs],
                              _ptr(mo) if mo is not None else None, _ptr(vo) if vo is not None else None, _ptr(n_kept),
                              _ptr(ws), ws.numel(), _stream(stream, *outs, mo, vo, n_kept, ws)))
    if stream is not None:
        stream.synchronize()   # the count is read on the host; .item() waits on the current stream only
    k = int(n_kept.item())
    Vk = k * (K + 1)
    # the kernel writes the kept moments in the layout of the kept soup, [xyz 3Vk | rgb 3Vk |
    # alpha Vk], at the front of the output
    cut = lambda t: t[:7 * Vk] if t is not None else None
    return outs[0][:Vk], outs[1][:Vk], outs[2][:Vk], cut(mo), cut(vo), k


def prune_faces(xyz, rgb, alpha, K, face_mask=None, threshold=math.exp(-4.0), m=None, v=None, stream=None):
    """Per-face pruning step (ms_prune_faces): clears the faces whose three vertex
    opacities are all below `threshold` in each fan's face mask (int32 tensor, one word per
    fan; None = all faces), removes fans left without faces and compacts the rest with
    their Adam moments and masks.  Returns (xyz, rgb, alpha, m, v, face_mask, n_kept);
    reads the kept count back, so it synchronises the stream."""
    n = xyz.shape[0] // (K + 1)
    outs = [torch.empty_like(t) for t in (xyz, rgb, alpha)]
    mo = torch.empty_like(m) if m is not None else None
    vo = torch.empty_like(v) if v is not None else None
    mask_o = torch.empty(max(n, 1), dtype=torch.int32, device=xyz.device)
    n_kept = torch.zeros(1, dtype=torch.int64, device=xyz.device)
    ws = torch.empty(max(lib().ms_prune_workspace_size(n), 1), dtype=torch.uint8, device=xyz.device)
    opt = lambda t: _ptr(t) if t is not None else None
    check(lib().ms_prune_faces(_ptr(xyz), _ptr(rgb), _ptr(alpha), opt(m), opt(v), opt(face_mask), n, int(K),
                               float(threshold), *[_ptr(t) for t in outs], opt(mo), opt(vo), _ptr(mask_o),
                               _ptr(n_kept), _ptr(ws), ws.numel(),
                               _stream(stream, *outs, mo, vo, mask_o, n_kept, ws)))
    (stream or torch.cuda.current_stream()).synchronize()
    k = int(n_kept.item())
    Vk = k * (K + 1)
    cut = lambda t: t[:7 * Vk] if t is not None else None
    return outs[0][:Vk], outs[1][:Vk], outs[2][:Vk], cut(mo), cut(vo), mask_o[:k], k


def mse(img_rgba, target_rgba, stream=None):
    """Mean squared RGB error (1-element device tensor)."""
    out = torch.empty(1, device=img_rgba.device, dtype=torch.float32)
    check(lib().ms_mse(_ptr(img_rgba), _ptr(target_rgba), img_rgba.numel() // 4, _ptr(out), _stream(stream, out)))
    return out


def fan_corrections(xyz0, a0, xyz1, a1, K, stream=None):
    """Corrections (N x 2(K+1)) that turn the converted soup into the fine-tuned one."""
    N = xyz0.shape[0] // (K + 1)
    corr = torch.empty(N, 2 * (K + 1), device=xyz0.device, dtype=torch.float32)
    check(lib().ms_fan_corrections(_ptr(xyz0), _ptr(a0), _ptr(xyz1), _ptr(a1), N, int(K), _ptr(corr),
                                   _stream(stream, corr)))
    return corr


class FanAdam:
    """Adam over the fan soup: colours/opacities at lr_color, positions at exp(-3) lr_color.
    With device_step=True the step number lives on the device (ms_adam_step_counted), so
    the update can be captured in a CUDA graph and replayed."""

    def __init__(self, xyz, rgb, alpha, lr_color=5e-3, betas=(0.9, 0.999), eps=1e-15, device_step=False):
        self.V = xyz.shape[0]
        self.lr_color = lr_color
        self.betas, self.eps = betas, eps
        self.m = torch.zeros(7 * self.V, device=xyz.device)
        self.v = torch.zeros(7 * self.V, device=xyz.device)
        self.t = 0
        self.d_step = torch.zeros(1, dtype=torch.int32, device=xyz.device) if device_step else None

    def step_ws(self, xyz, rgb, alpha, renderer, stream=None):
        """One step from the gradients a renderer's backward left in its workspace."""
        if self.d_step is None:
            self.t += 1
        check(lib().ms_adam_step_ws(_ptr(xyz), _ptr(rgb), _ptr(alpha), renderer.grad_ptr(), _ptr(self.m),
                                    _ptr(self.v), self.V, self.t if self.d_step is None else 0,
                                    _ptr(self.d_step) if self.d_step is not None else None,
                                    float(self.lr_color), float(self.lr_color * LR_XYZ_RATIO),
                                    float(self.betas[0]), float(self.betas[1]), float(self.eps), _stream(stream)))

    def step(self, xyz, rgb, alpha, d_xyz, d_rgb, d_alpha, stream=None):
        if self.d_step is not None:
            check(lib().ms_adam_step_counted(_ptr(xyz), _ptr(rgb), _ptr(alpha), _ptr(d_xyz), _ptr(d_rgb),
                                             _ptr(d_alpha), _ptr(self.m), _ptr(self.v), self.V, _ptr(self.d_step),
                                             float(self.lr_color), float(self.lr_color * LR_XYZ_RATIO),
                                             float(self.betas[0]), float(self.betas[1]), float(self.eps),
                                             _stream(stream)))
            return
        self.t += 1
        check(lib().ms_adam_step(_ptr(xyz), _ptr(rgb), _ptr(alpha), _ptr(d_xyz), _ptr(d_rgb), _ptr(d_alpha),
                                 _ptr(self.m), _ptr(self.v), self.V, self.t, float(self.lr_color),
                                 float(self.lr_color * LR_XYZ_RATIO), float(self.betas[0]), float(self.betas[1]),
                                 float(self.eps), _stream(stream)))


class FanMLP:
    """The learned fan initializer (ms_mlp_*): FP32 master weights, their packed bf16
    copy, Adam state, and calls for inputs, inference and training steps."""

    N_IN, HIDDEN = 16, 128

    def __init__(self, K=8, weights=None, seed=0, device="cuda"):
        self.K = int(K)
        self.n_out = 2 * (self.K + 1)
        if self.n_out > 32:
            raise ValueError("K <= 15")
        self.device = torch.device(device)
        if weights is None:
            g = torch.Generator().manual_seed(seed)
            W1 = torch.randn(self.N_IN, self.HIDDEN, generator=g) * math.sqrt(2.0 / self.N_IN)
            W2 = torch.randn(self.HIDDEN, self.HIDDEN, generator=g) * math.sqrt(2.0 / self.HIDDEN)
            W3 = torch.zeros(self.HIDDEN, self.n_out)
            weights = (W1, W2, W3)
        flat = torch.cat([torch.as_tensor(w, dtype=torch.float32).reshape(-1) for w in weights])
        self.W = flat.to(self.device).contiguous()
        n1, n2 = self.N_IN * self.HIDDEN, self.HIDDEN * self.HIDDEN
        self.sizes = (n1, n2, self.HIDDEN * self.n_out)
        self.m = torch.zeros_like(self.W)
        self.v = torch.zeros_like(self.W)
        self.step = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.grads = torch.zeros_like(self.W)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.packed = torch.zeros(int(lib().ms_mlp_packed_bytes()), dtype=torch.uint8, device=self.device)
        self.ws = None
        self.pack()

    def weights(self):
        n1, n2, n3 = self.sizes
        return (self.W[:n1].view(self.N_IN, self.HIDDEN), self.W[n1:n1 + n2].view(self.HIDDEN, self.HIDDEN),
                self.W[n1 + n2:].view(self.HIDDEN, self.n_out))

    def pack(self, stream=None):
        W1, W2, W3 = self.weights()
        check(lib().ms_mlp_pack(_ptr(W1), _ptr(W2), _ptr(W3), self.n_out, _ptr(self.packed), _stream(stream)))

    @staticmethod
    def _gauss(log_scales, quats, opacity, sh, sh_degree):
        sh_dtype = 0 if sh.dtype == torch.float32 else 1
        return _ptr(log_scales), _ptr(quats), _ptr(opacity), _ptr(sh), sh_dtype, int(sh_degree)

    def features(self, log_scales, quats, opacity, sh, sh_degree, stream=None):
        N = log_scales.shape[0]
        X = torch.empty(N, self.N_IN, device=self.device)
        check(lib().ms_mlp_features(*self._gauss(log_scales, quats, opacity, sh, sh_degree), N, _ptr(X),
                                    _stream(stream, X)))
        return X

    def forward(self, log_scales, quats, opacity, sh, sh_degree, out=None, stream=None):
        """Corrections N x 2(K+1) for ms_mesh_build."""
        N = log_scales.shape[0]
        corr = out if out is not None else torch.empty(N, self.n_out, device=self.device)
        check(lib().ms_mlp_forward(*self._gauss(log_scales, quats, opacity, sh, sh_degree), N, _ptr(self.packed),
                                   self.n_out, _ptr(corr), _stream(stream, corr)))
        return corr

    def compute_grads(self, X, T, stream=None):
        """Gradients of the mean squared error (into self.grads) and the loss (device)."""
        n = X.shape[0]
        need = int(lib().ms_mlp_train_workspace_size(n))
        if self.ws is None or self.ws.numel() < need:
            self.ws = torch.empty(max(need, 256), dtype=torch.uint8, device=self.device)
        check(lib().ms_mlp_grads(_ptr(X), _ptr(T), n, self.n_out, _ptr(self.packed), _ptr(self.grads),
                                 _ptr(self.loss), _ptr(self.ws), self.ws.numel(), _stream(stream, self.ws)))
        return self.grads, self.loss

    def adam(self, lr=1e-3, betas=(0.9, 0.999), eps=1e-8, stream=None):
        check(lib().ms_mlp_adam(_ptr(self.W), _ptr(self.grads), _ptr(self.m), _ptr(self.v), self.n_out,
                                _ptr(self.step), float(lr), float(betas[0]), float(betas[1]), float(eps),
                                _ptr(self.packed), _stream(stream)))

    def train_step(self, X, T, lr=1e-3, stream=None):
        self.compute_grads(X, T, stream)
        self.adam(lr, stream=stream)
        return self.loss

    def status(self, stream=None):
        t = C.c_int32(0)
        st = lib().ms_mlp_status(_ptr(self.packed), C.byref(t), _stream(stream))
        return st, t.value
