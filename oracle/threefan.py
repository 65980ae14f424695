"""Plain FP64 reference of the three-fan conversion of 3D Gaussians -- TEST
INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import this
module; it shares no code with the CUDA library.

Sec. 3 "Transformation for 3D Gaussians" (the equation of the three scaled rotation
vectors and the vertex equation that follows it): all three axes are kept,
sr_k = scale_mul exp(s_k) r_k (r_k the columns of the rotation of the normalised
quaternion); one fan per pair of axes (1, 2), (1, 3), (2, 3), each with K boundary vertices
v_i = m + cos(t_i) sr_a + sin(t_i) sr_b at the angles t_i = -pi + 2 pi i / K (the reading
of the flat case), and K triangles (m, v_i, v_{i+1 mod K}); 3K triangles per Gaussian.
Colour and opacity as in the flat case: every vertex carries the Gaussian's colour, the
centre its opacity sigma and the boundary vertices opac_mul sigma.  Readings:

* "Shared points at surface intersections": the fans meet where a boundary vertex is an
  axis tip m +- sr_k, which two fans reach when both contain the angle giving that tip;
  such a vertex is stored once.  Angles that are multiples of pi/2 take the exact cosine
  and sine (0, +-1), so a tip is exactly m +- sr_k in every fan that reaches it.
* Vertex order: the centre, then the boundary vertices of fan (1, 2), (1, 3), (2, 3) in
  angle order, each tip at its first appearance.
"""
from __future__ import annotations

import math

import numpy as np

from . import SCALE_MUL, OPAC_MUL, gaussian_colors, quat_to_rot

PLANES = ((0, 1), (0, 2), (1, 2))


def angle_cos_sin(i: int, K: int):
    """cos and sin of t_i = -pi + 2 pi i / K, exact where t_i is a multiple of pi/2."""
    if (4 * i) % K == 0:
        q = (4 * i) // K                      # t_i = (q - 2) pi / 2
        return ((-1.0, 0.0), (0.0, -1.0), (1.0, 0.0), (0.0, 1.0))[q % 4]
    t = -math.pi + 2.0 * math.pi * i / K
    return math.cos(t), math.sin(t)


def _tip(i: int, K: int, a: int, b: int):
    """(axis, sign) of the tip the angle i reaches in the fan spanned by axes a, b, or None."""
    c, s = angle_cos_sin(i, K)
    if c in (1.0, -1.0):
        return (a, int(c))
    if s in (1.0, -1.0):
        return (b, int(s))
    return None


def fan_layout(K: int):
    """Unique-vertex layout of one Gaussian: (number of vertices, for each fan the vertex
    index of each of its K boundary vertices).  Index 0 is the centre."""
    seen = {}
    idx = []
    n = 1
    for a, b in PLANES:
        row = []
        for i in range(K):
            key = _tip(i, K, a, b)
            if key is not None and key in seen:
                row.append(seen[key])
                continue
            row.append(n)
            if key is not None:
                seen[key] = n
            n += 1
        idx.append(row)
    return n, idx


def three_fan_build(scene, K: int = 8, scale_mul: float = SCALE_MUL, opac_mul: float = OPAC_MUL, cam_center=None):
    """Gaussians -> unique-vertex mesh.  Returns (xyz V x 3, rgb V x 3, alpha V,
    tris T x 3 int32, vertices per Gaussian); V = N nv, T = N 3K, FP64."""
    nv, idx = fan_layout(K)
    N = scene.n
    cols = gaussian_colors(scene, cam_center=cam_center)
    xyz = np.zeros((N, nv, 3))
    rgb = np.repeat(cols[:, None, :], nv, axis=1)
    alpha = np.empty((N, nv))
    tris = np.empty((N, 3 * K, 3), np.int32)
    cs = [angle_cos_sin(i, K) for i in range(K)]
    for g in range(N):
        R = quat_to_rot(scene.quats[g].astype(np.float64))
        m = scene.means[g].astype(np.float64)
        sr = [scale_mul * math.exp(float(scene.log_scales[g, k])) * R[:, k] for k in range(3)]
        xyz[g, 0] = m
        for p, (a, b) in enumerate(PLANES):
            for i in range(K):
                c, s = cs[i]
                xyz[g, idx[p][i]] = m + c * sr[a] + s * sr[b]
                tris[g, p * K + i] = (g * nv, g * nv + idx[p][i], g * nv + idx[p][(i + 1) % K])
        sigma = float(scene.opacity[g])
        alpha[g, 0] = sigma
        alpha[g, 1:] = opac_mul * sigma
    return xyz.reshape(-1, 3), rgb.reshape(-1, 3), alpha.reshape(-1), tris.reshape(-1, 3), nv


def as_implicit_fans(xyz, rgb, alpha, K: int, nv: int):
    """The same mesh as 3 implicit fans per Gaussian (centre + K boundary vertices each,
    shared vertices copied into every fan that uses them), and for every fan vertex the
    index of the unique vertex it copies (to sum the copies' gradients)."""
    _, idx = fan_layout(K)
    N = xyz.shape[0] // nv
    src = np.empty((N, 3, K + 1), np.int64)
    for g in range(N):
        for p in range(3):
            src[g, p, 0] = g * nv
            src[g, p, 1:] = g * nv + np.asarray(idx[p])
    src = src.reshape(-1)
    return xyz[src], rgb[src], alpha[src], src
