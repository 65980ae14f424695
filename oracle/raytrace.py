"""Plain FP64 reference of ray-traced rendering of the fan soup -- TEST INFRASTRUCTURE
ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import this
module; it shares no code with the CUDA library.

The paper's motivation (Sec. 1 and the discussion of ray-tracing renderers) is that a
triangle soup can be ray traced with secondary effects such as shadows; it gives no
shading model.  Readings:

* Primary rays: the pixel-centre ray of the pinhole camera; every triangle it crosses in
  front of the near plane is a fragment with the ray's barycentrics (which equal the
  rasteriser's perspective-correct ones), ordered by view depth, ties by triangle index, and
  composited front to back exactly as in the rasterised render.
* Shadows: a point light L.  A fragment at p gets the light transmittance S, the product
  of (1 - a_g) over every other triangle g that the segment from p to L crosses (a_g the
  triangle's interpolated opacity at the crossing); its colour c becomes c (k + (1 - k) S)
  with an ambient share k.  k = 1 (or a light that nothing occludes) gives the plain render.
* Intersections are decided in FP64 (Moller-Trumbore), edges closed; a crossing at the
  segment's ends (parameter <= 1e-9 or >= 1 - 1e-9) does not count.
"""
from __future__ import annotations

import numpy as np

EPS_T = 1e-9


def _hits(orig, d, P0, P1, P2):
    """Ray orig + t d against all triangles: (t, u, v) arrays and a mask of hits (t > 0)."""
    e1, e2 = P1 - P0, P2 - P0
    pv = np.cross(d, e2)
    det = np.einsum("ij,ij->i", e1, pv)
    ok = np.abs(det) > 1e-300
    inv = np.where(ok, 1.0 / np.where(ok, det, 1.0), 0.0)
    tv = orig - P0
    u = np.einsum("ij,ij->i", tv, pv) * inv
    qv = np.cross(tv, e1)
    v = (qv @ d) * inv
    t = np.einsum("ij,ij->i", e2, qv) * inv
    mask = ok & (u >= 0) & (v >= 0) & (u + v <= 1)
    return t, u, v, mask


def render(xyz, rgb, alpha, tris, cam, light=None, ambient=1.0, bg=(0.0, 0.0, 0.0), window=None):
    """Ray-traced RGBA of the window (x0, y0, x1, y1) (default: the whole image), FP64."""
    xyz = np.asarray(xyz, np.float64)
    rgb = np.asarray(rgb, np.float64)
    alpha = np.asarray(alpha, np.float64)
    tris = np.asarray(tris, np.int64)
    x0, y0, x1, y1 = window if window is not None else (0, 0, cam.width, cam.height)
    R = np.asarray(cam.R_cw, np.float64).reshape(3, 3)     # rows: camera axes in world
    C = np.asarray(cam.C, np.float64)
    P0, P1, P2 = xyz[tris[:, 0]], xyz[tris[:, 1]], xyz[tris[:, 2]]
    bg = np.asarray(bg, np.float64)
    out = np.zeros((y1 - y0, x1 - x0, 4))
    for py in range(y0, y1):
        for px in range(x0, x1):
            dc = np.array([(px + 0.5 - cam.cx) / cam.fx, (py + 0.5 - cam.cy) / cam.fy, 1.0])
            d = R.T @ dc                                      # world direction with unit view depth
            t, u, v, m = _hits(C, d, P0, P1, P2)
            m &= t > cam.znear                                # t is the view depth Z here
            idx = np.nonzero(m)[0]
            order = idx[np.lexsort((idx, t[idx]))]
            T, col = 1.0, np.zeros(3)
            for g in order:
                w = np.array([1.0 - u[g] - v[g], u[g], v[g]])
                a = float(w @ alpha[tris[g]])
                c = w @ rgb[tris[g]]
                if light is not None and ambient < 1.0:
                    c = c * (ambient + (1.0 - ambient) * transmittance(C + t[g] * d, light, g, P0, P1, P2,
                                                                         alpha[tris]))
                col += T * a * c
                T *= 1.0 - a
            out[py - y0, px - x0, :3] = col + T * bg
            out[py - y0, px - x0, 3] = 1.0 - T
    return out


def transmittance(p, light, own, P0, P1, P2, tri_alpha):
    """Product of (1 - a_g) over the triangles g != own crossed by the segment p -> light."""
    d = np.asarray(light, np.float64) - p
    t, u, v, m = _hits(p, d, P0, P1, P2)
    m &= (t > EPS_T) & (t < 1.0 - EPS_T)
    m[own] = False
    S = 1.0
    for g in np.nonzero(m)[0]:
        w = np.array([1.0 - u[g] - v[g], u[g], v[g]])
        S *= 1.0 - float(w @ tri_alpha[g])
    return S
