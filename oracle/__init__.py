"""NumPy front end of the plain CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  It shares no code with the CUDA library; see ms_oracle.c for what
each function computes and which passage of the paper it follows.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

SCALE_MUL = 2.7      # Sec. 3, Eq. 2: scale_mul
NO_TRIAG = 8         # Sec. 3: no_triag = 8 in all experiments
OPAC_MUL = 0.2       # Sec. 3: opac_mul = 0.2 in all experiments

_lib = None


class OrcCamera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32),
                ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("R_cw", C.c_float * 9), ("C", C.c_float * 3), ("znear", C.c_float)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        L.orc_mesh_build.argtypes = [C.c_int64, P, P, P, P, P, C.c_int, C.c_int, C.c_int, C.c_double,
                                     C.c_double, C.c_int, P, P, P, P, P]
        L.orc_render.argtypes = [C.c_int64, P, P, P, C.c_int64, P, P, P, C.c_int, C.c_int, C.c_int,
                                 C.c_int, C.c_int, C.c_int, P, P, P]
        L.orc_render_backward.argtypes = [C.c_int64, P, P, P, C.c_int64, P, P, P, C.c_int, C.c_int,
                                          C.c_int, C.c_int, C.c_int, P, P, P, P]
        L.orc_render_ex.argtypes = [C.c_int64, P, P, P, C.c_int64, P, P, P, C.c_int, C.c_int, C.c_int,
                                    C.c_int, C.c_int, C.c_int, C.c_int, P, P, P, P]
        L.orc_render_backward_ex.argtypes = [C.c_int64, P, P, P, C.c_int64, P, P, P, C.c_int, C.c_int,
                                             C.c_int, C.c_int, C.c_int, C.c_int, P, P, P, P]
        L.orc_sh_basis.argtypes = [C.c_int, P, P]
        L.orc_quat_to_rot.argtypes = [P, P]
        L.orc_fan_tris.argtypes = [C.c_int64, C.c_int32, P]
        L.orc_project.argtypes = [P, P, P, P]
        L.orc_splat_render.argtypes = [C.c_int64, P, P, P, P, P, C.c_int, C.c_double, P, P, C.c_int, C.c_int,
                                       C.c_int, C.c_int, C.c_int, P, P]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def camera_struct(cam) -> OrcCamera:
    c = OrcCamera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    R = np.asarray(cam.R_cw, np.float32).reshape(9)
    for i in range(9):
        c.R_cw[i] = float(R[i])
    Cc = np.asarray(cam.C, np.float32).reshape(3)
    for i in range(3):
        c.C[i] = float(Cc[i])
    c.znear = float(cam.znear)
    return c


def threads_used() -> int:
    return int(lib().orc_last_threads())


def quat_to_rot(q) -> np.ndarray:
    q = _c(q, np.float64)
    R = np.zeros(9)
    lib().orc_quat_to_rot(_p(q), _p(R))
    return R.reshape(3, 3)


def sh_basis(degree: int, d) -> np.ndarray:
    d = _c(d, np.float64)
    Y = np.zeros(16)
    if lib().orc_sh_basis(int(degree), _p(d), _p(Y)) != 0:
        raise ValueError("degree")
    return Y[: (degree + 1) ** 2]


def project(cam, p):
    """Returns (decided float32 (xs, ys, Z, valid), FP64 (xs, ys, Z)) for one world point."""
    cs = camera_struct(cam)
    p = _c(p, np.float64)
    dec = np.zeros(4, np.float32)
    val = np.zeros(3)
    lib().orc_project(C.byref(cs), _p(p), _p(dec), _p(val))
    return dec, val


def fan_tris(n: int, K: int) -> np.ndarray:
    t = np.zeros((n * K, 3), np.int32)
    lib().orc_fan_tris(int(n), int(K), _p(t))
    return t


def mesh_build(scene, K=NO_TRIAG, scale_mul=SCALE_MUL, opac_mul=OPAC_MUL, axis_rule=1,
               cam_center=None, corr=None):
    """Gaussians -> fan soup (xyz, rgb, alpha), FP64."""
    n = scene.n
    V = n * (K + 1)
    xyz, rgb, alpha = np.zeros((V, 3)), np.zeros((V, 3)), np.zeros(V)
    sh = _c(scene.sh, np.uint16 if scene.sh_bf16 else np.float32)
    cc = _c(cam_center, np.float32) if cam_center is not None else None
    cr = _c(corr, np.float64) if corr is not None else None
    rc = lib().orc_mesh_build(n, _p(_c(scene.means, np.float32)), _p(_c(scene.log_scales, np.float32)),
                              _p(_c(scene.quats, np.float32)), _p(_c(scene.opacity, np.float32)), _p(sh),
                              1 if scene.sh_bf16 else 0, int(scene.sh_degree), int(K), float(scale_mul),
                              float(opac_mul), int(axis_rule), _p(cc), _p(cr), _p(xyz), _p(rgb), _p(alpha))
    if rc:
        raise ValueError(f"orc_mesh_build failed ({rc})")
    return xyz, rgb, alpha


def _window(cam, window):
    if window is None:
        return 0, 0, int(cam.width), int(cam.height)
    return tuple(int(v) for v in window)


# Decisions (coverage, order): "fp64" the plain FP64 definition (the default); "fp32" both
# by the binary32 formulas on binary32 projections; "rel32" coverage by the binary32
# formulas on fan-relative rounded FP64 projections and order by the FP64 depth -- the
# decisions the library's kernels take (see ms_oracle.c).
DECIDE = {"fp32": 0, "fp64": 1, "rel32": 2}


def render(xyz, rgb, alpha, tris, cam, bg=(0.0, 0.0, 0.0), window=None, brute=False, nthreads=0, decide="fp64",
           signature=False):
    """Returns (rgba (h, w, 4) float64, fragments per pixel (h, w) int32, culled triangle count),
    plus per-pixel uint64 hashes of the ordered triangle ids when signature=True.  decide:
    "fp32" takes coverage and order by the binary32 formulas, "fp64" by the plain FP64
    definition (see ms_oracle.c)."""
    x0, y0, x1, y1 = _window(cam, window)
    out = np.zeros((max(y1 - y0, 0), max(x1 - x0, 0), 4))
    nfrag = np.zeros(out.shape[:2], np.int32)
    sig = np.zeros(out.shape[:2], np.uint64) if signature else None
    nc = np.zeros(1, np.int64)
    xyz, rgb, alpha = _c(xyz, np.float64), _c(rgb, np.float64), _c(alpha, np.float64)
    tris = _c(tris, np.int32)
    cs = camera_struct(cam)
    bgv = _c(bg, np.float64)
    rc = lib().orc_render_ex(xyz.shape[0], _p(xyz), _p(rgb), _p(alpha), tris.shape[0], _p(tris), C.byref(cs),
                             _p(bgv), x0, y0, x1, y1, int(bool(brute)), int(nthreads), DECIDE[decide], _p(out),
                             _p(nfrag), _p(sig), _p(nc))
    if rc:
        raise RuntimeError(f"orc_render failed ({rc})")
    if signature:
        return out, nfrag, int(nc[0]), sig
    return out, nfrag, int(nc[0])


def decision_mismatch(xyz, rgb, alpha, tris, cam, window=None, nthreads=0, decide="rel32"):
    """Renders the window with the given decisions and with FP64 decisions.  Returns (image
    with FP64 decisions, boolean mask of the pixels whose fragment sets or order differ
    between the two, image with the given decisions)."""
    ia, _, _, sa = render(xyz, rgb, alpha, tris, cam, window=window, nthreads=nthreads, decide=decide,
                          signature=True)
    i64, _, _, s64 = render(xyz, rgb, alpha, tris, cam, window=window, nthreads=nthreads, decide="fp64",
                            signature=True)
    return i64, sa != s64, ia


def render_backward(xyz, rgb, alpha, tris, cam, dL, bg=(0.0, 0.0, 0.0), window=None, nthreads=0, decide="fp64"):
    """Exact reverse pass; returns (d_xyz, d_rgb, d_alpha) in FP64."""
    x0, y0, x1, y1 = _window(cam, window)
    xyz, rgb, alpha = _c(xyz, np.float64), _c(rgb, np.float64), _c(alpha, np.float64)
    tris = _c(tris, np.int32)
    dL = _c(dL, np.float64)
    assert dL.shape == (y1 - y0, x1 - x0, 4)
    V = xyz.shape[0]
    gx, gc, ga = np.zeros((V, 3)), np.zeros((V, 3)), np.zeros(V)
    cs = camera_struct(cam)
    bgv = _c(bg, np.float64)
    rc = lib().orc_render_backward_ex(V, _p(xyz), _p(rgb), _p(alpha), tris.shape[0], _p(tris), C.byref(cs),
                                      _p(bgv), x0, y0, x1, y1, int(nthreads), DECIDE[decide], _p(dL), _p(gx),
                                      _p(gc), _p(ga))
    if rc:
        raise RuntimeError(f"orc_render_backward failed ({rc})")
    return gx, gc, ga


def gaussian_colors(scene, cam_center=None):
    """Colour of every Gaussian (N x 3, FP64): the colour its fan's vertices carry."""
    _, rgb, _ = mesh_build(scene, K=3, cam_center=cam_center)
    return np.ascontiguousarray(rgb.reshape(scene.n, 4, 3)[:, 0, :])


def splat_render(scene, cam, rgb=None, axis_rule=1, trunc=SCALE_MUL, bg=(0.0, 0.0, 0.0), window=None,
                 nthreads=0, cam_center=None):
    """Source-Gaussian render of the window (see ms_oracle_splat.c).  Returns
    (rgba (h, w, 4) float64, fragments per pixel (h, w) int32)."""
    if rgb is None:
        rgb = gaussian_colors(scene, cam_center)
    x0, y0, x1, y1 = _window(cam, window)
    out = np.zeros((max(y1 - y0, 0), max(x1 - x0, 0), 4))
    nfrag = np.zeros(out.shape[:2], np.int32)
    bgv = np.asarray(bg, np.float64)
    camc = camera_struct(cam)
    rc = lib().orc_splat_render(scene.n, _p(_c(scene.means, np.float32)), _p(_c(scene.log_scales, np.float32)),
                                _p(_c(scene.quats, np.float32)), _p(_c(scene.opacity, np.float32)),
                                _p(_c(rgb, np.float64)), int(axis_rule), float(trunc), C.byref(camc), _p(bgv),
                                x0, y0, x1, y1, int(nthreads), _p(out), _p(nfrag))
    if rc != 0:
        raise RuntimeError(f"orc_splat_render failed ({rc})")
    return out, nfrag


def l1_loss_grad(rgb_img, target_rgb):
    """L1 = mean |C - C*| over the RGB channels (Eq. 3 with lambda = 1); returns (loss, dL/dC)."""
    d = rgb_img - target_rgb
    n = d.size
    return float(np.abs(d).sum() / n), np.sign(d) / n


def adam_step(params, grads, m, v, step, lrs, betas=(0.9, 0.999), eps=1e-15):
    """Adam (Sec. 3 'Optimization and Pruning': colours and opacities at lr_color,
    positions at exp(-3) lr_color), FP64, in place on lists of arrays; the opacity
    (last entry) is clamped to [0, 1] after the step."""
    b1, b2 = betas
    for i, (p, g) in enumerate(zip(params, grads)):
        m[i][...] = b1 * m[i] + (1 - b1) * g
        v[i][...] = b2 * v[i] + (1 - b2) * g * g
        mh = m[i] / (1 - b1 ** step)
        vh = v[i] / (1 - b2 ** step)
        p -= lrs[i] * mh / (np.sqrt(vh) + eps)
    np.clip(params[-1], 0.0, 1.0, out=params[-1])


LR_XYZ_RATIO = float(np.exp(-3.0))   # Sec. 3: vertex positions learn at exp(-3) times lr_color


def fan_adam_step(xyz, rgb, alpha, d_xyz, d_rgb, d_alpha, m, v, step, lr_color, betas=(0.9, 0.999), eps=1e-15):
    """One Adam step of the fan soup as Sec. 3 ("Optimization and Pruning") sets it up:
    colours and opacities at lr_color, vertex positions at exp(-3) lr_color, the opacity
    clamped to [0, 1] afterwards.  xyz, rgb (V x 3) and alpha (V) are updated in place;
    m and v are the moments in the layout [xyz 3V | rgb 3V | alpha V] (zero before step 1),
    updated in place; step counts from 1."""
    V = np.asarray(alpha).size
    views = lambda t: [t[:3 * V].reshape(V, 3), t[3 * V:6 * V].reshape(V, 3), t[6 * V:7 * V]]
    adam_step([xyz, rgb, alpha], [d_xyz, d_rgb, d_alpha], views(m), views(v), step,
              [lr_color * LR_XYZ_RATIO, lr_color, lr_color], betas, eps)


PRUNE_THRESHOLD = float(np.exp(-4.0))


def prune_fans(xyz, rgb, alpha, K, threshold=PRUNE_THRESHOLD, moments=()):
    """Pruning step of Sec. 3 ("Optimization and Pruning") at fan granularity: a face goes
    when all three of its vertices have opacity below the threshold (exp(-4)); a fan whose
    faces all go is removed with its K + 1 vertices, the other fans are kept whole and in
    order.  (All of a fan's faces qualify exactly when all of its vertices are below the
    threshold, since every face holds the centre and each boundary vertex is in a face.)
    moments: arrays in the optimiser layout [xyz 3V | rgb 3V | alpha V], compacted alike.
    Returns (xyz, rgb, alpha, [moments...], kept fan indices)."""
    a = np.asarray(alpha).reshape(-1, K + 1)
    keep = ~np.all(a < threshold, axis=1)
    fans = np.nonzero(keep)[0]
    vsel = (fans[:, None] * (K + 1) + np.arange(K + 1)).reshape(-1)
    V = a.size
    out_m = []
    for m in moments:
        m = np.asarray(m)
        out_m.append(np.concatenate([m[:3 * V].reshape(V, 3)[vsel].reshape(-1),
                                     m[3 * V:6 * V].reshape(V, 3)[vsel].reshape(-1), m[6 * V:7 * V][vsel]]))
    return (np.asarray(xyz).reshape(V, 3)[vsel], np.asarray(rgb).reshape(V, 3)[vsel], np.asarray(alpha).reshape(V)[vsel],
            out_m, fans)


def face_masks(alpha, K, threshold=PRUNE_THRESHOLD, face_mask=None):
    """Per-face pruning rule of Sec. 3 ("Optimization and Pruning") as one mask word per
    fan: bit j (face (c, b_j, b_{j+1 mod K})) is set unless all three of the face's vertex
    opacities are below the threshold, and stays clear once an earlier mask cleared it."""
    a = np.asarray(alpha).reshape(-1, K + 1)
    low = a < threshold
    b = low[:, 1:]
    dead = low[:, :1] & b & np.roll(b, -1, axis=1)
    m = ((~dead).astype(np.int64) << np.arange(K)).sum(axis=1)
    if face_mask is not None:
        m &= np.asarray(face_mask, np.int64)
    return m


def prune_faces(xyz, rgb, alpha, K, face_mask=None, threshold=PRUNE_THRESHOLD, moments=()):
    """Pruning step of Sec. 3 per face: the faces of face_masks go; a fan left with no face
    is removed with its K + 1 vertices (its vertices are used by no face), every other fan
    is kept whole and in order (each of its vertices lies in a kept face or is the shared
    centre).  moments: arrays in the optimiser layout [xyz 3V | rgb 3V | alpha V], compacted
    alike.  Returns (xyz, rgb, alpha, [moments...], masks of the kept fans, kept fan
    indices)."""
    masks = face_masks(alpha, K, threshold, face_mask)
    fans = np.nonzero(masks != 0)[0]
    a = np.asarray(alpha).reshape(-1, K + 1)
    vsel = (fans[:, None] * (K + 1) + np.arange(K + 1)).reshape(-1)
    V = a.size
    out_m = []
    for m in moments:
        m = np.asarray(m)
        out_m.append(np.concatenate([m[:3 * V].reshape(V, 3)[vsel].reshape(-1),
                                     m[3 * V:6 * V].reshape(V, 3)[vsel].reshape(-1), m[6 * V:7 * V][vsel]]))
    return (np.asarray(xyz).reshape(V, 3)[vsel], np.asarray(rgb).reshape(V, 3)[vsel],
            np.asarray(alpha).reshape(V)[vsel], out_m, masks[fans], fans)


def masked_fan_tris(n, K, masks=None):
    """Triangles (fan topology) of the faces a mask keeps, in triangle order."""
    t = fan_tris(n, K)
    if masks is None:
        return t
    keep = ((np.asarray(masks, np.int64)[:, None] >> np.arange(K)) & 1).astype(bool).reshape(-1)
    return t[keep]
