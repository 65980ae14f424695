"""Seeded synthetic inputs for the MeshSplats hot path.

This module draws Gaussian scenes and pinhole cameras and nothing else: it holds
none of the method's arithmetic (no fan construction, no SH evaluation, no
projection, no rasterisation).  Both the FP64 oracle and the CUDA path consume
the arrays it returns, so they see identical bytes.

Gaussian record (Sec. 3, Eq. 1 "GS" and the GaMeS flat parameterisation):
  means      (N, 3)  float32   position m
  log_scales (N, 3)  float32   s, with exp(s) the per-axis scale
  quats      (N, 4)  float32   rotation quaternion (w, x, y, z), unit length
  opacity    (N,)    float32   activated opacity sigma in [0, 1]
  sh         (N, (d+1)^2, 3)   float32, or uint16 holding bfloat16 bits
Camera (Sec. 3 "Rendering MeshSplats in Nvdiffrast", the MVP transform):
  OpenCV axes (x right, y down, z forward), X_cam = R_cw (p - C),
  pixel = (fx X/Z + cx, fy Y/Z + cy), row 0 at the top.

Workloads (seed = 1000 + workload number):
  1  1,000 random Gaussians, SH degree 0, K=8, 128x128, camera at distance 4
  2  200,000 flat Gaussians on a unit sphere plus a torus, SH degree 3, 800x800
  3  1,000,000 clustered flat Gaussians, SH degree 3 in bfloat16, 1920x1080
  4  3,000,000 clustered flat Gaussians, K=6, 16 cameras of mixed resolution
  5  3,000,000 clustered flat Gaussians, K=8, 8 cameras at 1920x1080
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SPHERE_R = 1.0
TORUS_R = 1.6
TORUS_r = 0.3
SPHERE_AREA = 4.0 * math.pi * SPHERE_R ** 2
TORUS_AREA = 4.0 * math.pi ** 2 * TORUS_R * TORUS_r


@dataclasses.dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    R_cw: np.ndarray          # (3, 3) float32, rows = camera x, y, z axes in world
    C: np.ndarray             # (3,) float32 camera centre in world
    znear: float = 0.01

    def as_tuple(self):
        return (self.width, self.height, self.fx, self.fy, self.cx, self.cy,
                self.R_cw.astype(np.float32).reshape(9), self.C.astype(np.float32), self.znear)


@dataclasses.dataclass
class Scene:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity: np.ndarray
    sh: np.ndarray
    sh_degree: int
    sh_bf16: bool = False

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def sh_f32(self) -> np.ndarray:
        """SH coefficients as float32 (exact widening of bfloat16 bits)."""
        if not self.sh_bf16:
            return self.sh
        return (self.sh.astype(np.uint32) << 16).view(np.float32)


@dataclasses.dataclass
class Workload:
    name: str
    scene: Scene
    K: int
    cameras: list
    target_scene: Scene | None = None


def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float32 to bfloat16 (round to nearest even); returns uint16 bits."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    return ((u + rounding) >> 16).astype(np.uint16)


def look_at(C, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0)) -> np.ndarray:
    """World-to-camera rotation with rows (right, down, forward)."""
    C = np.asarray(C, np.float64)
    z = np.asarray(target, np.float64) - C
    z /= np.linalg.norm(z)
    up = np.asarray(up, np.float64)
    if abs(np.dot(z, up / np.linalg.norm(up))) > 0.99:
        up = np.array([0.0, 0.0, 1.0])
    x = np.cross(z, up)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    return np.stack([x, y, z]).astype(np.float32)


def make_camera(C, width, height, fov_y_deg=60.0, target=(0.0, 0.0, 0.0), znear=0.01) -> Camera:
    f = (height / 2.0) / math.tan(math.radians(fov_y_deg) / 2.0)
    return Camera(width, height, float(np.float32(f)), float(np.float32(f)),
                  width / 2.0, height / 2.0, look_at(C, target),
                  np.asarray(C, np.float32), znear)


def rotmat_to_quat(R: np.ndarray) -> np.ndarray:
    """(N,3,3) proper rotations -> (N,4) unit quaternions (w,x,y,z) (input construction only)."""
    m = R.astype(np.float64)
    tr = m[:, 0, 0] + m[:, 1, 1] + m[:, 2, 2]
    q = np.empty((m.shape[0], 4))
    # Shepperd's method, branch on the largest diagonal term.
    cands = np.stack([tr, m[:, 0, 0], m[:, 1, 1], m[:, 2, 2]], 1)
    k = np.argmax(cands, 1)
    for case in range(4):
        i = np.nonzero(k == case)[0]
        if i.size == 0:
            continue
        a = m[i]
        if case == 0:
            s = np.sqrt(1.0 + tr[i]) * 2
            q[i] = np.stack([0.25 * s, (a[:, 2, 1] - a[:, 1, 2]) / s,
                             (a[:, 0, 2] - a[:, 2, 0]) / s, (a[:, 1, 0] - a[:, 0, 1]) / s], 1)
        elif case == 1:
            s = np.sqrt(1.0 + a[:, 0, 0] - a[:, 1, 1] - a[:, 2, 2]) * 2
            q[i] = np.stack([(a[:, 2, 1] - a[:, 1, 2]) / s, 0.25 * s,
                             (a[:, 0, 1] + a[:, 1, 0]) / s, (a[:, 0, 2] + a[:, 2, 0]) / s], 1)
        elif case == 2:
            s = np.sqrt(1.0 + a[:, 1, 1] - a[:, 0, 0] - a[:, 2, 2]) * 2
            q[i] = np.stack([(a[:, 0, 2] - a[:, 2, 0]) / s, (a[:, 0, 1] + a[:, 1, 0]) / s,
                             0.25 * s, (a[:, 1, 2] + a[:, 2, 1]) / s], 1)
        else:
            s = np.sqrt(1.0 + a[:, 2, 2] - a[:, 0, 0] - a[:, 1, 1]) * 2
            q[i] = np.stack([(a[:, 1, 0] - a[:, 0, 1]) / s, (a[:, 0, 2] + a[:, 2, 0]) / s,
                             (a[:, 1, 2] + a[:, 2, 1]) / s, 0.25 * s], 1)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _sh_coeffs(rng, n, degree, sigma0=0.5, sigma_hi=0.2):
    nb = (degree + 1) ** 2
    sh = rng.normal(0.0, sigma_hi, size=(n, nb, 3))
    sh[:, 0, :] = rng.normal(0.0, sigma0, size=(n, 3))
    return sh.astype(np.float32)


def random_scene(n: int, seed: int, degree: int = 0) -> Scene:
    """Workload 1 recipe: means U[-1,1]^3, log-scales U[-4,-2]^3, quats normalize(N(0,I4)),
    opacity sigmoid(N(0,1)), SH degree-0 coefficients N(0, 0.5)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    means = rng.uniform(-1.0, 1.0, (n, 3)).astype(np.float32)
    log_scales = rng.uniform(-4.0, -2.0, (n, 3)).astype(np.float32)
    q = rng.normal(0.0, 1.0, (n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opacity = _sigmoid(rng.normal(0.0, 1.0, n)).astype(np.float32)
    sh = _sh_coeffs(rng, n, degree)
    return Scene(means, log_scales, q.astype(np.float32), opacity, sh, degree)


def _sample_sphere(rng, n):
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v * SPHERE_R, v.copy()


def _torus_point(u, v):
    cu, su, cv, sv = np.cos(u), np.sin(u), np.cos(v), np.sin(v)
    p = np.stack([(TORUS_R + TORUS_r * cv) * cu, (TORUS_R + TORUS_r * cv) * su, TORUS_r * sv], 1)
    nrm = np.stack([cv * cu, cv * su, sv], 1)
    return p, nrm


def _sample_torus(rng, n):
    out_u, out_v = [np.zeros(0)], [np.zeros(0)]
    need = n
    while need > 0:
        u = rng.uniform(0, 2 * np.pi, 2 * need + 16)
        v = rng.uniform(0, 2 * np.pi, 2 * need + 16)
        keep = rng.uniform(0, 1, u.size) < (TORUS_R + TORUS_r * np.cos(v)) / (TORUS_R + TORUS_r)
        out_u.append(u[keep][:need])
        out_v.append(v[keep][:need])
        need -= out_u[-1].size
    return _torus_point(np.concatenate(out_u), np.concatenate(out_v)) + (
        np.concatenate(out_u), np.concatenate(out_v))


def _surface_points(rng, n, clustered: bool, n_blobs=256, blob_std=0.05):
    """Points and unit normals on the sphere + torus, split by area.  With clustered,
    half of them fall in Gaussian blobs (std blob_std, measured along the surface)."""
    n_uniform = n // 2 if clustered else n
    frac_sphere = SPHERE_AREA / (SPHERE_AREA + TORUS_AREA)
    ns = int(round(n_uniform * frac_sphere))
    ps, ns_ = _sample_sphere(rng, ns)
    pt, nt, _, _ = _sample_torus(rng, n_uniform - ns)
    P, Nrm = [ps, pt], [ns_, nt]
    if clustered:
        n_bl = n - n_uniform
        nb_s = int(round(n_blobs * frac_sphere))
        cs, _ = _sample_sphere(rng, nb_s)
        _, _, cu, cv = _sample_torus(rng, n_blobs - nb_s)
        which = rng.integers(0, n_blobs, n_bl)
        off = rng.normal(0.0, blob_std, (n_bl, 2))
        on_s = which < nb_s
        i_s = np.nonzero(on_s)[0]
        if i_s.size:
            c = cs[which[i_s]]
            t1 = np.cross(c, np.array([0.0, 0.0, 1.0]))
            bad = np.linalg.norm(t1, axis=1) < 1e-6
            t1[bad] = np.array([1.0, 0.0, 0.0])
            t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
            t2 = np.cross(c, t1)
            p = c + off[i_s, :1] * t1 + off[i_s, 1:] * t2
            p /= np.linalg.norm(p, axis=1, keepdims=True)
            P.append(p * SPHERE_R)
            Nrm.append(p.copy())
        i_t = np.nonzero(~on_s)[0]
        if i_t.size:
            k = which[i_t] - nb_s
            u = cu[k] + off[i_t, 0] / (TORUS_R + TORUS_r * np.cos(cv[k]))
            v = cv[k] + off[i_t, 1] / TORUS_r
            p, nrm = _torus_point(u, v)
            P.append(p)
            Nrm.append(nrm)
    P = np.concatenate(P)
    Nrm = np.concatenate(Nrm)
    perm = rng.permutation(P.shape[0])
    return P[perm], Nrm[perm]


def surface_scene(n: int, seed: int, degree: int = 3, clustered: bool = False,
                  bf16: bool = False, thin_ratio: float = 1e-3) -> Scene:
    """Flat Gaussians on the sphere + torus.  Axis 0 of each Gaussian is the surface
    normal and is thin: s0 = s1 + log(thin_ratio); s1, s2 = log(0.5 sqrt(A/N)) + N(0, 0.25)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    P, Nrm = _surface_points(rng, n, clustered)
    helper = np.where(np.abs(Nrm[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    t1 = np.cross(Nrm, helper)
    t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
    t2 = np.cross(Nrm, t1)
    phi = rng.uniform(0, 2 * np.pi, n)[:, None]
    r2 = np.cos(phi) * t1 + np.sin(phi) * t2
    r3 = np.cross(Nrm, r2)
    R = np.stack([Nrm, r2, r3], axis=2)          # columns r1 (normal), r2, r3
    quats = rotmat_to_quat(R).astype(np.float32)
    base = math.log(0.5 * math.sqrt((SPHERE_AREA + TORUS_AREA) / n))
    s12 = base + rng.normal(0.0, 0.25, (n, 2))
    s0 = s12[:, :1] + math.log(thin_ratio)
    log_scales = np.concatenate([s0, s12], 1).astype(np.float32)
    opacity = _sigmoid(rng.normal(0.0, 1.0, n)).astype(np.float32)
    sh = _sh_coeffs(rng, n, degree)
    if bf16:
        sh = to_bf16_bits(sh)
    return Scene(P.astype(np.float32), log_scales, quats, opacity, sh, degree, bf16)


def jittered(scene: Scene, std: float, seed: int) -> Scene:
    rng = np.random.Generator(np.random.PCG64(seed))
    m = (scene.means + rng.normal(0.0, std, scene.means.shape)).astype(np.float32)
    return dataclasses.replace(scene, means=m)


def fibonacci_dirs(n: int) -> np.ndarray:
    i = np.arange(n) + 0.5
    z = 1.0 - 2.0 * i / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = np.pi * (3.0 - math.sqrt(5.0)) * i
    return np.stack([r * np.cos(phi), z, r * np.sin(phi)], 1)


def orbit_camera(radius, elev_deg, width, height, azim_deg=0.0):
    e, a = math.radians(elev_deg), math.radians(azim_deg)
    C = radius * np.array([math.cos(e) * math.sin(a), math.sin(e), math.cos(e) * math.cos(a)])
    return make_camera(C, width, height)


def workload(idx: int, n: int | None = None) -> Workload:
    """The five workloads; n overrides the Gaussian count (for small parity cases)."""
    seed = 1000 + idx
    if idx == 1:
        sc = random_scene(n or 1000, seed, degree=0)
        cam = make_camera((0.0, 0.0, 4.0), 128, 128)
        return Workload("random-1k-K8-128px", sc, 8, [cam])
    if idx == 2:
        sc = surface_scene(n or 200_000, seed, degree=3)
        return Workload("surfaces-200k-K8-800px", sc, 8, [orbit_camera(4.0, 20.0, 800, 800)])
    if idx == 3:
        sc = surface_scene(n or 1_000_000, seed, degree=3, clustered=True, bf16=True)
        tgt = jittered(sc, 1e-3, seed + 100)
        return Workload("clustered-1M-K8-1080p", sc, 8, [orbit_camera(3.0, 20.0, 1920, 1080)], tgt)
    if idx == 4:
        sc = surface_scene(n or 3_000_000, seed, degree=3, clustered=True, bf16=True)
        rng = np.random.Generator(np.random.PCG64(seed + 200))
        res = [(512, 512), (800, 800), (1280, 720), (1920, 1080)]
        cams = []
        for d in fibonacci_dirs(16):
            w, h = res[int(rng.integers(0, 4))]
            cams.append(make_camera(d * rng.uniform(3.0, 5.0), w, h))
        tgt = jittered(sc, 1e-3, seed + 100)
        return Workload("clustered-3M-K6-16views", sc, 6, cams, tgt)
    if idx == 5:
        sc = surface_scene(n or 3_000_000, seed, degree=3, clustered=True, bf16=True)
        cams = [make_camera(d * 3.5, 1920, 1080) for d in fibonacci_dirs(8)]
        return Workload("clustered-3M-K8-8views-1080p", sc, 8, cams)
    raise ValueError(idx)


def sphere_mesh(n_lat: int, n_lon: int, radius: float = 1.0, centre=(0.0, 0.0, 0.0), jitter: float = 0.0,
                seed: int = 0):
    """A UV-tessellated sphere with shared vertices: (vertices V x 3 float32, faces T x 3
    int32, outward winding).  `jitter` moves every vertex by N(0, jitter) so no two
    triangles are exactly coplanar or meet a pixel centre exactly."""
    rng = np.random.Generator(np.random.PCG64(seed))
    verts = [(0.0, 0.0, radius)]
    for i in range(1, n_lat):
        th = np.pi * i / n_lat
        for j in range(n_lon):
            ph = 2 * np.pi * j / n_lon
            verts.append((radius * np.sin(th) * np.cos(ph), radius * np.sin(th) * np.sin(ph), radius * np.cos(th)))
    verts.append((0.0, 0.0, -radius))
    V = np.asarray(verts) + np.asarray(centre)
    if jitter:
        V = V + rng.normal(0.0, jitter, V.shape)
    ring = lambda i, j: 1 + (i - 1) * n_lon + (j % n_lon)
    faces = []
    for j in range(n_lon):
        faces.append((0, ring(1, j), ring(1, j + 1)))
    for i in range(1, n_lat - 1):
        for j in range(n_lon):
            a, b, c, d = ring(i, j), ring(i, j + 1), ring(i + 1, j), ring(i + 1, j + 1)
            faces.append((a, c, b))
            faces.append((b, c, d))
    south = len(verts) - 1
    for j in range(n_lon):
        faces.append((south, ring(n_lat - 1, j + 1), ring(n_lat - 1, j)))
    return V.astype(np.float32), np.asarray(faces, np.int32)


def mesh_prior_weights(n_faces: int, n_sub: int, jitter: float = 0.0, seed: int = 0) -> np.ndarray:
    """Weights w (F, n_sub, 3 vertices, 3 corners) of secondary triangles laid out on each
    face: one triangle per face covering it (n_sub = 1), or its midpoint subdivision (four:
    the three corner triangles, then the middle one).  Each entry is the square root of the
    layout's barycentric coordinate, plus N(0, jitter) noise when jitter > 0."""
    h = 0.5 ** 0.5
    layouts = {1: [[[1, 0, 0], [0, 1, 0], [0, 0, 1]]],
               4: [[[1, 0, 0], [h, h, 0], [h, 0, h]], [[h, h, 0], [0, 1, 0], [0, h, h]],
                   [[h, 0, h], [0, h, h], [0, 0, 1]], [[h, h, 0], [0, h, h], [h, 0, h]]]}
    w = np.broadcast_to(np.asarray(layouts[n_sub], np.float64), (n_faces, n_sub, 3, 3)).copy()
    if jitter > 0:
        w += np.random.Generator(np.random.PCG64(seed)).normal(0.0, jitter, w.shape)
    return w
