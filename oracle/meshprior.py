"""Plain FP64 reference of the mesh-prior mode -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import this
module; it shares no code with the CUDA library.

Sec. 3, the mesh-prior paragraphs (the convex-combination equation for the secondary
triangles): on top of a geometry mesh, every face (m_1, m_2, m_3) carries a fixed number
of disjoint secondary triangles whose vertices are convex combinations
v_i = a_i1 m_1 + a_i2 m_2 + a_i3 m_3 (a_i on the simplex) with trainable weights, and
trainable per-vertex colour and opacity.  Readings:

* The simplex constraint is kept by the parameterisation a_ik = w_ik^2 / sum_j w_ij^2 of
  free weights w (non-negative, summing to 1, reaching exact zeros, smooth where any w is
  non-zero); the paper does not say how the constraint is enforced.
* Initialisation "based on the faces": with one triangle per face, the face itself
  (a_i = e_i); with four, its midpoint subdivision (corner triangles, then the middle one).
  The weights start at w = sqrt(a).
* A secondary triangle renders like any triangle of the soup.  Drawn as a fan of K = 3
  around its centroid, whose colour and opacity are the means of the three vertices', it
  covers the same pixels with the same interpolated values, which is how the fan renderer
  takes it.
"""
from __future__ import annotations

import numpy as np

# Barycentric corners of the initial secondary triangles of one face.
INIT = {
    1: np.array([[[1, 0, 0], [0, 1, 0], [0, 0, 1]]], np.float64),
    4: np.array([[[1, 0, 0], [.5, .5, 0], [.5, 0, .5]],
                 [[.5, .5, 0], [0, 1, 0], [0, .5, .5]],
                 [[.5, 0, .5], [0, .5, .5], [0, 0, 1]],
                 [[.5, .5, 0], [0, .5, .5], [.5, 0, .5]]], np.float64),
}


def init_weights(n_faces: int, n_sub: int) -> np.ndarray:
    """w (F, n_sub, 3 vertices, 3 corners) with a = w^2 / sum w^2 the initial layout."""
    return np.broadcast_to(np.sqrt(INIT[n_sub]), (n_faces, n_sub, 3, 3)).copy()


def simplex_weights(w: np.ndarray) -> np.ndarray:
    w = np.asarray(w, np.float64)
    q = w * w
    return q / q.sum(axis=-1, keepdims=True)


def secondary_vertices(faces: np.ndarray, w: np.ndarray) -> np.ndarray:
    """faces (F, 3 corners, 3 coords), w (F, S, 3, 3) -> vertices (F, S, 3, 3 coords)."""
    a = simplex_weights(w)
    return np.einsum("fsik,fkc->fsic", a, np.asarray(faces, np.float64))


def triangle_soup(faces, w, rgb, alpha):
    """Secondary triangles as an explicit soup: (xyz (3T, 3), rgb (3T, 3), alpha (3T),
    tris (T, 3)); rgb (F, S, 3, 3) and alpha (F, S, 3) are the per-vertex attributes."""
    v = secondary_vertices(faces, w).reshape(-1, 3)
    T = v.shape[0] // 3
    return v, np.asarray(rgb, np.float64).reshape(-1, 3), np.asarray(alpha, np.float64).reshape(-1), \
        np.arange(3 * T, dtype=np.int32).reshape(T, 3)


def as_centroid_fans(xyz, rgb, alpha):
    """Triangle soup -> fan soup of K = 3 (centroid, v1, v2, v3 per triangle), the
    centroid carrying the means of the three vertices' colour and opacity."""
    x = np.asarray(xyz, np.float64).reshape(-1, 3, 3)
    c = np.asarray(rgb, np.float64).reshape(-1, 3, 3)
    a = np.asarray(alpha, np.float64).reshape(-1, 3)
    fx = np.concatenate([x.mean(axis=1, keepdims=True), x], axis=1).reshape(-1, 3)
    fc = np.concatenate([c.mean(axis=1, keepdims=True), c], axis=1).reshape(-1, 3)
    fa = np.concatenate([a.mean(axis=1, keepdims=True), a], axis=1).reshape(-1)
    return fx, fc, fa


def fan_grads_to_triangles(g_xyz, g_rgb, g_alpha):
    """Adjoint of as_centroid_fans: the centroid's gradients go a third to each vertex."""
    gx = np.asarray(g_xyz, np.float64).reshape(-1, 4, 3)
    gc = np.asarray(g_rgb, np.float64).reshape(-1, 4, 3)
    ga = np.asarray(g_alpha, np.float64).reshape(-1, 4)
    return ((gx[:, 1:] + gx[:, :1] / 3.0).reshape(-1, 3), (gc[:, 1:] + gc[:, :1] / 3.0).reshape(-1, 3),
            (ga[:, 1:] + ga[:, :1] / 3.0).reshape(-1))


def weight_grads(faces, w, g_vertices):
    """dL/dw from dL/dv (F, S, 3, 3 coords): dL/da_ik = dL/dv_i . m_k, then through
    a_ik = w_ik^2 / Q_i (Q_i = sum_j w_ij^2): dL/dw_ij = (2 w_ij / Q_i)(dL/da_ij - sum_k a_ik dL/da_ik)."""
    w = np.asarray(w, np.float64)
    a = simplex_weights(w)
    Q = (w * w).sum(axis=-1, keepdims=True)
    ga = np.einsum("fsic,fkc->fsik", np.asarray(g_vertices, np.float64), np.asarray(faces, np.float64))
    return 2.0 * w / Q * (ga - (a * ga).sum(axis=-1, keepdims=True))
