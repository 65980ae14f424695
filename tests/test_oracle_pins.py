"""Pins of the CPU oracle against closed forms, invariants, library routines and
brute force -- nothing here compares the oracle with itself.  CPU only."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synthetic
from synthetic import Camera, Scene

HERE = os.path.dirname(os.path.abspath(__file__))


def flat_camera(w=16, h=16):
    """Identity pose, unit focal length, principal point at 0: a point (x, y, 1) lands
    exactly on screen position (x, y) in binary32 as well as in FP64."""
    return Camera(w, h, 1.0, 1.0, 0.0, 0.0, np.eye(3, dtype=np.float32), np.zeros(3, np.float32), 0.01)


# --------------------------------------------------------------------------------------
# Paper constants (values printed in the paper, tests/golden/paper_constants.json)
# --------------------------------------------------------------------------------------

def test_paper_constants():
    g = json.load(open(os.path.join(HERE, "golden", "paper_constants.json")))
    assert oracle.SCALE_MUL == g["scale_mul"]["value"]
    assert oracle.NO_TRIAG == g["no_triag"]["value"]
    assert oracle.OPAC_MUL == g["opac_mul"]["value"]
    assert math.isclose(g["lr_verts_over_lr_color"]["value"], math.exp(-3), rel_tol=1e-15)
    assert math.isclose(g["prune_opacity_threshold"]["value"], math.exp(-4), rel_tol=1e-15)


# --------------------------------------------------------------------------------------
# Rotation (Sec. 3: Sigma = R S S^T R^T, R = [r1 r2 r3])
# --------------------------------------------------------------------------------------

def test_rotation_closed_forms():
    assert np.allclose(oracle.quat_to_rot([1, 0, 0, 0]), np.eye(3), atol=0)
    # 90 degrees about +z: x -> y, y -> -x
    c = math.cos(math.pi / 4)
    R = oracle.quat_to_rot([c, 0, 0, c])
    assert np.allclose(R, [[0, -1, 0], [1, 0, 0], [0, 0, 1]], atol=1e-15)
    # 180 degrees about +x
    assert np.allclose(oracle.quat_to_rot([0, 1, 0, 0]), np.diag([1, -1, -1]), atol=1e-15)
    rng = np.random.default_rng(0)
    for _ in range(100):
        q = rng.normal(size=4) * rng.uniform(0.1, 10)
        R = oracle.quat_to_rot(q)
        assert np.abs(R.T @ R - np.eye(3)).max() < 1e-14
        assert abs(np.linalg.det(R) - 1) < 1e-14
        assert np.abs(oracle.quat_to_rot(-q) - R).max() < 1e-15
        # rotation about the axis of the quaternion leaves the axis fixed
        ax = q[1:] / np.linalg.norm(q[1:])
        assert np.abs(R @ ax - ax).max() < 1e-13


# --------------------------------------------------------------------------------------
# Spherical harmonics (colour, Sec. 3 Eq. 1 "c often expressed in SH")
# --------------------------------------------------------------------------------------

def test_sh_matches_scipy_real_harmonics():
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(1)
    for _ in range(50):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        theta, phi = math.acos(d[2]), math.atan2(d[1], d[0])
        Y = oracle.sh_basis(3, d)
        for l in range(4):
            for m in range(-l, l + 1):
                yc = complex(sp.sph_harm_y(l, abs(m), theta, phi))
                if m < 0:
                    ref = math.sqrt(2) * yc.imag
                elif m == 0:
                    ref = yc.real
                else:
                    ref = math.sqrt(2) * yc.real
                assert abs(Y[l * l + m + l] - ref) < 1e-12, (l, m)


def test_sh_orthonormal_by_quadrature():
    # Gauss-Legendre in cos(theta) x uniform phi integrates the products exactly.
    z, wz = np.polynomial.legendre.leggauss(8)
    nphi = 16
    G = np.zeros((16, 16))
    for zi, wi in zip(z, wz):
        s = math.sqrt(1 - zi * zi)
        for k in range(nphi):
            ph = 2 * math.pi * k / nphi
            Y = oracle.sh_basis(3, [s * math.cos(ph), s * math.sin(ph), zi])
            G += wi * (2 * math.pi / nphi) * np.outer(Y, Y)
    assert np.abs(G - np.eye(16)).max() < 1e-13


def test_sh_degree0_colour_closed_form():
    sc = synthetic.random_scene(64, 7, degree=0)
    xyz, rgb, a = oracle.mesh_build(sc, K=8, cam_center=[0, 0, 4])
    C0 = 1.0 / (2.0 * math.sqrt(math.pi))
    want = np.maximum(0.0, 0.5 + C0 * sc.sh[:, 0, :].astype(np.float64))
    assert np.abs(rgb.reshape(64, 9, 3) - want[:, None, :]).max() < 1e-15


def test_sh_clamps_negative_colour():
    sc = synthetic.random_scene(4, 3, degree=0)
    sc.sh[:] = -10.0
    _, rgb, _ = oracle.mesh_build(sc, K=8)
    assert (rgb == 0).all()


# --------------------------------------------------------------------------------------
# Fan conversion (Sec. 3, Eq. 2 and the vertex equation)
# --------------------------------------------------------------------------------------

def one_gaussian(m, log_s, q, sigma=0.5):
    return Scene(np.array([m], np.float32), np.array([log_s], np.float32), np.array([q], np.float32),
                 np.array([sigma], np.float32), np.zeros((1, 1, 3), np.float32), 0)


def test_fan_hand_computed():
    # identity rotation, s = (ln eps, ln 1, ln 2): a = 2.7 (0,1,0), b = 5.4 (0,0,1)
    sc = one_gaussian([1, 2, 3], [math.log(1e-3), 0.0, math.log(2.0)], [1, 0, 0, 0], sigma=0.5)
    xyz, rgb, alpha = oracle.mesh_build(sc, K=4, axis_rule=0)
    want = np.array([[1, 2, 3],            # centre
                     [1, 2 - 2.7, 3],      # theta = -pi
                     [1, 2, 3 - 5.4],      # theta = -pi/2
                     [1, 2 + 2.7, 3],      # theta = 0
                     [1, 2, 3 + 5.4]])     # theta = pi/2
    assert np.abs(xyz - want).max() < 1e-6   # inputs are binary32
    assert np.allclose(alpha, [0.5, 0.1, 0.1, 0.1, 0.1], atol=1e-7, rtol=0)
    assert np.allclose(rgb, 0.5)


@pytest.mark.parametrize("K", [3, 6, 8, 12])
def test_fan_geometry_invariants(K):
    sc = synthetic.random_scene(200, 11, degree=0)
    xyz, rgb, alpha = oracle.mesh_build(sc, K=K, axis_rule=1)
    xyz = xyz.reshape(-1, K + 1, 3)
    alpha = alpha.reshape(-1, K + 1)
    for g in range(sc.n):
        R = oracle.quat_to_rot(sc.quats[g].astype(np.float64))
        s = sc.log_scales[g].astype(np.float64)
        keep = sorted(np.argsort(s, kind="stable")[1:])
        a = 2.7 * math.exp(s[keep[0]]) * R[:, keep[0]]
        b = 2.7 * math.exp(s[keep[1]]) * R[:, keep[1]]
        m = sc.means[g].astype(np.float64)
        assert np.abs(xyz[g, 0] - m).max() < 1e-15
        d = xyz[g, 1:] - m
        # on the ellipse: ((v-m).a/|a|^2)^2 + ((v-m).b/|b|^2)^2 = 1
        e = (d @ a / (a @ a)) ** 2 + (d @ b / (b @ b)) ** 2
        assert np.abs(e - 1).max() < 1e-12
        # vertex 0 at theta = -pi is m - a
        assert np.abs(xyz[g, 1] - (m - a)).max() < 1e-14
        # polygon area (K/2) r1 r2 sin(2 pi / K)
        area = 0.5 * np.linalg.norm(np.cross(d, np.roll(d, -1, axis=0)), axis=1).sum()
        r1, r2 = np.linalg.norm(a), np.linalg.norm(b)
        assert abs(area - 0.5 * K * r1 * r2 * math.sin(2 * math.pi / K)) < 1e-12 * max(1.0, area)
        assert abs(alpha[g, 0] / alpha[g, 1] - 5.0) < 1e-12


def test_axis_rules_agree_on_flat_gaussians():
    sc = synthetic.surface_scene(500, 5, degree=0)
    a0 = oracle.mesh_build(sc, K=8, axis_rule=0)
    a1 = oracle.mesh_build(sc, K=8, axis_rule=1)
    for u, v in zip(a0, a1):
        assert np.array_equal(u, v)


def test_corrections_zero_is_plain_conversion():
    sc = synthetic.random_scene(50, 9, degree=0)
    plain = oracle.mesh_build(sc, K=8)
    zero = oracle.mesh_build(sc, K=8, corr=np.zeros((50, 18)))
    for u, v in zip(plain, zero):
        assert np.array_equal(u, v)
    corr = np.zeros((50, 18))
    corr[:, 1:9] = 0.5            # boundary radius x 1.5
    corr[:, 9] = math.log(2.0)    # centre opacity x 2 (clamped at 1)
    xyz, _, alpha = oracle.mesh_build(sc, K=8, corr=corr)
    m = xyz.reshape(50, 9, 3)[:, :1]
    d_plain = plain[0].reshape(50, 9, 3)[:, 1:] - m
    assert np.abs(xyz.reshape(50, 9, 3)[:, 1:] - m - 1.5 * d_plain).max() < 1e-14
    assert np.allclose(alpha.reshape(50, 9)[:, 0], np.minimum(1.0, 2 * sc.opacity.astype(np.float64)))


# --------------------------------------------------------------------------------------
# Camera (Sec. 3: MVP transform to screen)
# --------------------------------------------------------------------------------------

def test_camera_principal_point_and_fov_edge():
    cam = synthetic.make_camera((0.0, 0.0, 4.0), 128, 96, fov_y_deg=60.0)
    dec, val = oracle.project(cam, [0.0, 0.0, 0.0])
    assert abs(val[0] - 64) < 1e-12 and abs(val[1] - 48) < 1e-12 and abs(val[2] - 4) < 1e-12
    assert dec[3] == 1.0
    # a point on the upper edge of the vertical field of view maps to row 0 (y down)
    y = 4.0 * math.tan(math.radians(30.0))
    _, val = oracle.project(cam, [0.0, y, 0.0])
    assert abs(val[1]) < 1e-4 and abs(val[0] - 64) < 1e-9
    # +x world is to the right on screen for this camera
    _, val = oracle.project(cam, [0.5, 0.0, 0.0])
    assert val[0] > 64


# --------------------------------------------------------------------------------------
# Coverage: top-left rule, watertightness, brute force (Sec. 3 rasterisation)
# --------------------------------------------------------------------------------------

DECISIONS = ("fp64", "rel32", "fp32")   # every decision mode of the oracle obeys the coverage pins


def _render_2d(verts2d, tris, w=16, h=16, rgb=None, alpha=None, z=None, decide="fp64"):
    V = len(verts2d)
    zz = np.ones(V) if z is None else np.asarray(z, np.float64)
    xyz = np.array([[x * zz[i], y * zz[i], zz[i]] for i, (x, y) in enumerate(verts2d)])
    rgb = np.ones((V, 3)) if rgb is None else rgb
    alpha = np.full(V, 0.5) if alpha is None else alpha
    return oracle.render(xyz, rgb, alpha, np.asarray(tris, np.int32), flat_camera(w, h), brute=True, decide=decide)


@pytest.mark.parametrize("decide", DECISIONS)
def test_top_left_rule_square(decide):
    # square [2.5, 10.5]^2 from two triangles: the top and left edges own their pixel centres
    v = [(2.5, 2.5), (10.5, 2.5), (10.5, 10.5), (2.5, 10.5)]
    for tris in ([[0, 1, 2], [0, 2, 3]], [[1, 2, 3], [1, 3, 0]], [[0, 2, 1], [3, 2, 0]]):
        _, nf, _ = _render_2d(v, tris, decide=decide)
        want = np.zeros((16, 16), np.int32)
        want[2:10, 2:10] = 1
        assert np.array_equal(nf, want)


def _fraction_side(a, b, p):
    return (b[0] - a[0]) * (p[1] - a[1]) - (b[1] - a[1]) * (p[0] - a[0])


@pytest.mark.parametrize("decide", DECISIONS)
def test_fan_watertight_exact_ties(decide):
    """A fan whose spokes and rims pass exactly through pixel centres: every centre
    inside is covered once, including the shared centre vertex."""
    c = (8.5, 8.5)
    ring = [(14.5, 8.5), (12.5, 12.5), (8.5, 14.5), (4.5, 12.5), (2.5, 8.5), (4.5, 4.5), (8.5, 2.5), (12.5, 4.5)]
    K = len(ring)
    verts = [c] + ring
    tris = [[0, 1 + j, 1 + (j + 1) % K] for j in range(K)]
    for order in (tris, [[t[0], t[2], t[1]] for t in tris]):
        _, nf, _ = _render_2d(verts, order, decide=decide)
        F = [(Fraction(x), Fraction(y)) for x, y in ring]
        # orientation: interior where the edge function is positive
        sgn = 1 if _fraction_side(F[0], F[1], (Fraction(c[0]), Fraction(c[1]))) > 0 else -1
        for py in range(16):
            for px in range(16):
                p = (Fraction(2 * px + 1, 2), Fraction(2 * py + 1, 2))
                sides = [sgn * _fraction_side(F[j], F[(j + 1) % K], p) for j in range(K)]
                if p in F:
                    assert nf[py, px] <= 1
                    continue
                if min(sides) > 0:
                    want = 1
                elif min(sides) < 0:
                    want = 0
                else:
                    j = sides.index(0)
                    a, b = F[j], F[(j + 1) % K]
                    ex, ey = (b[0] - a[0]) * sgn, (b[1] - a[1]) * sgn
                    want = int(ey < 0 or (ey == 0 and ex > 0))
                assert nf[py, px] == want, (px, py)


@pytest.mark.parametrize("decide", DECISIONS)
def test_brute_force_equals_bbox_mode(decide):
    w = synthetic.workload(1, n=300)
    xyz, rgb, a = oracle.mesh_build(w.scene, K=8, cam_center=w.cameras[0].C)
    tris = oracle.fan_tris(w.scene.n, 8)
    xyz = xyz.astype(np.float32)
    r1, n1, _ = oracle.render(xyz, rgb, a, tris, w.cameras[0], brute=True, decide=decide)
    r2, n2, _ = oracle.render(xyz, rgb, a, tris, w.cameras[0], brute=False, nthreads=3, decide=decide)
    assert np.array_equal(n1, n2)
    assert np.array_equal(r1, r2)


@pytest.mark.parametrize("decide", DECISIONS)
def test_fronto_parallel_fan_pixel_count_matches_area(decide):
    K = 8
    sc = one_gaussian([0, 0, 0], [math.log(0.4), math.log(0.3), -8.0], [1, 0, 0, 0], sigma=0.5)
    cam = synthetic.make_camera((0.0, 0.0, 4.0), 256, 256)
    xyz, rgb, a = oracle.mesh_build(sc, K=K, axis_rule=1)
    _, nf, _ = oracle.render(xyz.astype(np.float32), rgb, a, oracle.fan_tris(1, K), cam, decide=decide)
    s = cam.fy / 4.0
    r1, r2 = 2.7 * 0.4 * s, 2.7 * 0.3 * s
    area = 0.5 * K * r1 * r2 * math.sin(2 * math.pi / K)
    perim = K * 2 * max(r1, r2) * math.sin(math.pi / K)
    assert nf.max() == 1
    assert abs(nf.sum() - area) < perim


# --------------------------------------------------------------------------------------
# Interpolation (Sec. 3: vertex colours interpolated, linear opacity across the mesh)
# --------------------------------------------------------------------------------------

def _ray_hits(cam, px, py, P0, n):
    R = np.asarray(cam.R_cw, np.float64)   # binary32 rows: invert exactly, not by transpose
    d = np.linalg.solve(R, np.array([(px + 0.5 - cam.cx) / cam.fx, (py + 0.5 - cam.cy) / cam.fy, 1.0]))
    C = np.asarray(cam.C, np.float64)
    t = (n @ (P0 - C)) / (n @ d)
    return C + t * d


def test_perspective_correct_interpolation_of_world_linear_attributes():
    rng = np.random.default_rng(3)
    cam = synthetic.make_camera((0.3, 0.2, 3.0), 64, 64)
    P = np.array([[-0.8, -0.6, 0.3], [0.9, -0.4, -0.5], [0.1, 0.8, 0.4]], np.float32).astype(np.float64)
    A = rng.normal(size=(4, 3))   # three colour channels and alpha, linear in world space
    b = rng.uniform(0.3, 0.6, 4)
    vals = P @ A.T + b
    rgb = vals[:, :3]
    alpha = np.full(3, 1.0)
    img, nf, _ = oracle.render(P, rgb, alpha, np.array([[0, 1, 2]], np.int32), cam)
    n = np.cross(P[1] - P[0], P[2] - P[0])
    ys, xs = np.nonzero(nf == 1)
    assert xs.size > 200
    for px, py in zip(xs, ys):
        X = _ray_hits(cam, px, py, P[0], n)
        assert np.abs(img[py, px, :3] - (A[:3] @ X + b[:3])).max() < 1e-9
    # opacity interpolates the same way: single fragment, colour 1 => output alpha = alpha(X)
    alpha = vals[:, 3] * 0 + np.array([0.2, 0.9, 0.5])
    img, nf, _ = oracle.render(P, np.ones((3, 3)), alpha, np.array([[0, 1, 2]], np.int32), cam)
    Aa, *_ = np.linalg.lstsq(np.c_[P, np.ones(3)], alpha, rcond=None)
    for px, py in list(zip(xs, ys))[::7]:
        X = _ray_hits(cam, px, py, P[0], n)
        want = Aa[:3] @ X + Aa[3]
        assert abs(img[py, px, 3] - want) < 1e-9
        assert abs(img[py, px, 0] - want) < 1e-9


def test_fronto_parallel_interpolation_is_affine_in_screen():
    # flat camera, all vertices at the same depth: mu = screen barycentrics
    v = [(1.2, 1.7), (14.1, 3.3), (5.6, 13.9)]
    rgb = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]])
    img, nf, _ = _render_2d(v, [[0, 1, 2]], rgb=rgb, alpha=np.ones(3), z=[2.0, 2.0, 2.0])
    V = np.array(v)
    for py, px in zip(*np.nonzero(nf)):
        lam = np.linalg.solve(np.c_[V, np.ones(3)].T, [px + 0.5, py + 0.5, 1.0])
        assert np.abs(img[py, px, :3] - lam).max() < 1e-12


# --------------------------------------------------------------------------------------
# Compositing (Sec. 3: layers blended front to back through alpha)
# --------------------------------------------------------------------------------------

def test_two_layer_closed_form_and_depth_order():
    big = [(-40.0, -40.0), (80.0, -40.0), (-40.0, 80.0)]
    c1, a1, c2, a2 = np.array([0.9, 0.2, 0.1]), 0.35, np.array([0.1, 0.7, 0.4]), 0.6
    # the far triangle comes first in index order; depth must decide
    verts = big + big
    rgb = np.vstack([np.tile(c2, (3, 1)), np.tile(c1, (3, 1))])
    alpha = np.array([a2] * 3 + [a1] * 3)
    img, nf, _ = _render_2d(verts, [[0, 1, 2], [3, 4, 5]], rgb=rgb, alpha=alpha, z=[3.0] * 3 + [2.0] * 3)
    assert (nf == 2).all()
    want = a1 * c1 + (1 - a1) * a2 * c2
    assert np.abs(img[..., :3] - want).max() < 1e-14
    assert np.abs(img[..., 3] - (1 - (1 - a1) * (1 - a2))).max() < 1e-14


def test_equal_depth_ties_go_to_lower_triangle_index():
    big = [(-40.0, -40.0), (80.0, -40.0), (-40.0, 80.0)]
    c0, c1 = np.array([1.0, 0, 0]), np.array([0, 0, 1.0])
    rgb = np.vstack([np.tile(c0, (3, 1)), np.tile(c1, (3, 1))])
    img, _, _ = _render_2d(big + big, [[0, 1, 2], [3, 4, 5]], rgb=rgb, alpha=np.full(6, 0.5), z=[2.0] * 6)
    assert np.abs(img[..., :3] - (0.5 * c0 + 0.25 * c1)).max() < 1e-15


def test_zero_alpha_gives_background():
    w = synthetic.workload(1, n=200)
    xyz, rgb, a = oracle.mesh_build(w.scene, K=8)
    bg = (0.2, 0.3, 0.4)
    img, nf, _ = oracle.render(xyz.astype(np.float32), rgb, np.zeros_like(a), oracle.fan_tris(200, 8),
                               w.cameras[0], bg=bg)
    assert nf.sum() > 0
    assert np.abs(img[..., :3] - np.array(bg)).max() == 0 and np.abs(img[..., 3]).max() == 0


def test_opaque_fans_reproduce_zbuffer():
    """sigma = 1 and opac_mul = 1: the image is the colour of the nearest surface,
    found here by FP64 ray-triangle intersection (no screen-space rasterisation)."""
    w = synthetic.workload(1, n=150)
    sc = w.scene
    sc.opacity[:] = 1.0
    cam = w.cameras[0]
    K = 8
    xyz, rgb, a = oracle.mesh_build(sc, K=K, opac_mul=1.0, cam_center=cam.C)
    xyz = xyz.astype(np.float32).astype(np.float64)
    tris = oracle.fan_tris(sc.n, K)
    img, nf, _ = oracle.render(xyz, rgb, a, tris, cam)
    R = np.asarray(cam.R_cw, np.float64)
    C = np.asarray(cam.C, np.float64)
    H, W = cam.height, cam.width
    px, py = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    D = np.stack([(px - cam.cx) / cam.fx, (py - cam.cy) / cam.fy, np.ones_like(px)], -1) @ np.linalg.inv(R).T
    best_t = np.full((H, W), np.inf)
    best_c = np.zeros((H, W, 3))
    margin = np.full((H, W), np.inf)
    for t in range(tris.shape[0]):
        P0, P1, P2 = xyz[tris[t]]
        e1, e2 = P1 - P0, P2 - P0
        h = np.cross(D, e2)
        det = h @ e1
        ok = np.abs(det) > 1e-300
        s = C - P0
        u = (h @ s) / np.where(ok, det, 1)
        q = np.cross(s, e1)
        v = (D @ q) / np.where(ok, det, 1)
        tt = (e2 @ q) / np.where(ok, det, 1)
        mn = np.minimum(np.minimum(u, v), 1 - u - v)
        hit = ok & (mn > 0) & (tt > 0)
        near_edge = ok & (np.abs(mn) < 1e-3)
        margin[near_edge] = 0
        upd = hit & (tt < best_t)
        # depth near-ties between surfaces are excluded as well
        close = hit & (np.abs(tt - best_t) < 1e-6 * best_t)
        margin[close] = 0
        best_t[upd] = tt[upd]
        best_c[upd] = rgb[tris[t][0]]
    good = margin > 0
    assert good.mean() > 0.9
    covered = np.isfinite(best_t) & good
    assert np.abs(img[..., :3][covered] - best_c[covered]).max() < 1e-12
    assert np.abs(img[..., 3][covered] - 1.0).max() < 1e-12
    assert (nf[~np.isfinite(best_t) & good] == 0).all()


def test_permutation_invariance():
    w = synthetic.workload(1, n=400)
    sc = w.scene
    cam = w.cameras[0]
    K = 8
    xyz, rgb, a = oracle.mesh_build(sc, K=K, cam_center=cam.C)
    img, _, _ = oracle.render(xyz.astype(np.float32), rgb, a, oracle.fan_tris(sc.n, K), cam)
    perm = np.random.default_rng(5).permutation(sc.n)
    vperm = (perm[:, None] * (K + 1) + np.arange(K + 1)).reshape(-1)
    img2, _, _ = oracle.render(xyz[vperm].astype(np.float32), rgb[vperm], a[vperm],
                               oracle.fan_tris(sc.n, K), cam)
    assert np.abs(img - img2).max() < 1e-13


def test_near_plane_culls_triangles():
    cam = synthetic.make_camera((0.0, 0.0, 2.0), 32, 32)
    xyz = np.array([[0, 0, 0], [0.5, 0, 0], [0, 0.5, 0], [0, 0, 0], [0.5, 0, 0], [0, 0, 3.0]])
    img, nf, culled = oracle.render(xyz, np.ones((6, 3)), np.ones(6), np.array([[0, 1, 2], [3, 4, 5]], np.int32), cam)
    assert culled == 1
    assert nf.max() == 1


# --------------------------------------------------------------------------------------
# Reverse pass vs central finite differences of the forward
# --------------------------------------------------------------------------------------

def _fd_scene():
    w = synthetic.workload(1, n=40)
    cam = synthetic.make_camera((0.0, 0.0, 2.5), 64, 64)
    sc = w.scene
    sc.opacity[:] = np.clip(sc.opacity, 0.05, 0.9)
    xyz, rgb, a = oracle.mesh_build(sc, K=8, cam_center=cam.C)
    xyz = xyz.astype(np.float32).astype(np.float64)
    return xyz, rgb, a, oracle.fan_tris(sc.n, 8), cam


def test_reverse_pass_matches_finite_differences():
    """Loss = sum of random weights times the output over a window around one fan; the
    analytic reverse pass must match central differences of the forward.  Position
    steps stay below a quarter ulp of the binary32 coordinate, so coverage and order
    (decided in binary32) are identical at +h and -h: visibility is held fixed."""
    xyz, rgb, a, tris, cam = _fd_scene()
    rng = np.random.default_rng(8)
    img, nf, _ = oracle.render(xyz, rgb, a, tris, cam)
    gx_all, _, _ = oracle.render_backward(xyz, rgb, a, tris, cam, np.ones_like(img))
    active = np.nonzero(np.abs(gx_all).sum(1) > 1e-6)[0]
    assert active.size > 30
    checks = 0
    for v in rng.choice(active, 10, replace=False):
        g = v // 9
        pts = np.array([oracle.project(cam, xyz[9 * g + k])[1][:2] for k in range(9)])
        x0, y0 = np.maximum(np.floor(pts.min(0)).astype(int) - 2, 0)
        x1, y1 = np.minimum(np.ceil(pts.max(0)).astype(int) + 3, [cam.width, cam.height])
        Wt = np.zeros_like(img)
        Wt[y0:y1, x0:x1] = rng.normal(size=(y1 - y0, x1 - x0, 4))
        gx, gc, ga = oracle.render_backward(xyz, rgb, a, tris, cam, Wt)
        win = (x0, y0, x1, y1)
        Wl = Wt[y0:y1, x0:x1]

        def loss(x, c, al):
            return float((oracle.render(x, c, al, tris, cam, window=win, nthreads=1)[0] * Wl).sum())

        for r in range(3):
            h = float(np.spacing(np.float32(xyz[v, r]))) / 8
            xp, xm = xyz.copy(), xyz.copy()
            xp[v, r] += h
            xm[v, r] -= h
            fd = (loss(xp, rgb, a) - loss(xm, rgb, a)) / (2 * h)
            assert abs(fd - gx[v, r]) <= 1e-6 * abs(gx[v, r]) + 1e-6, (v, r, fd, gx[v, r])
            checks += 1
        h = 1e-6
        cp, cm = rgb.copy(), rgb.copy()
        cp[v, 1] += h
        cm[v, 1] -= h
        fd = (loss(xyz, cp, a) - loss(xyz, cm, a)) / (2 * h)
        assert abs(fd - gc[v, 1]) <= 1e-7 * abs(gc[v, 1]) + 1e-9
        ap, am = a.copy(), a.copy()
        ap[v] += h
        am[v] -= h
        fd = (loss(xyz, rgb, ap) - loss(xyz, rgb, am)) / (2 * h)
        assert abs(fd - ga[v]) <= 1e-6 * abs(ga[v]) + 1e-9
        checks += 2
    assert checks == 50
