"""Pins of the ray-tracing oracle (oracle/raytrace.py): primary rays reproduce the
rasterised composite; shadow rays scale a fragment's colour by k + (1 - k) S with S the
product of (1 - a) over the triangles between it and a point light."""
import numpy as np

import oracle
import synthetic
from oracle import raytrace as RT


def _quad(z, half, rgb, a):
    """Two triangles spanning [-half, half]^2 in the plane z, uniform colour and opacity."""
    xyz = np.array([[-half, -half, z], [half, -half, z], [half, half, z], [-half, half, z]], np.float64)
    tris = np.array([[0, 1, 2], [0, 2, 3]])
    return xyz, np.tile(rgb, (4, 1)).astype(np.float64), np.full(4, a, np.float64), tris


def _merge(*parts):
    xs, cs, as_, ts, off = [], [], [], [], 0
    for x, c, a, t in parts:
        xs.append(x); cs.append(c); as_.append(a); ts.append(t + off)
        off += x.shape[0]
    return np.concatenate(xs), np.concatenate(cs), np.concatenate(as_), np.concatenate(ts)


def test_primary_rays_reproduce_the_raster():
    w = synthetic.workload(1, n=80)
    cam = w.cameras[0]
    K = 8
    xyz, rgb, a = oracle.mesh_build(w.scene, K=K, cam_center=cam.C)
    tris = oracle.fan_tris(80, K)
    win = (44, 44, 84, 84)
    ras, nf, _ = oracle.render(xyz, rgb, a, tris, cam, window=win)
    ray = RT.render(xyz, rgb, a, tris, cam, window=win)
    assert nf.max() >= 2
    d = np.abs(ras - ray).max(axis=2)
    # only pixel centres within rounding of a triangle edge may be decided differently
    assert np.count_nonzero(d > 1e-9) <= 0.005 * d.size, np.count_nonzero(d > 1e-9)


def test_full_ambient_ignores_the_light():
    cam = synthetic.make_camera((0.0, 0.0, 3.0), 32, 32)
    recv = _quad(0.0, 1.0, [0.8, 0.4, 0.2], 0.9)
    occ = _quad(0.5, 0.3, [0.1, 0.1, 0.1], 0.5)
    x, c, a, t = _merge(recv, occ)
    plain = RT.render(x, c, a, t, cam)
    lit = RT.render(x, c, a, t, cam, light=(0.0, 0.0, 10.0), ambient=1.0)
    assert np.array_equal(plain, lit)


def test_shadow_of_a_uniform_occluder():
    """Receiver plane z = 0 (opacity 1), a square occluder of opacity 0.6 at z = 0.5 off to
    the side of the view, light at (2, 0, 2): a receiver point p is shadowed where the
    segment to the light meets z = 0.5 (at p + (L - p)/4) inside the square; shadowed
    points get k + (1 - k)(1 - 0.6), the rest 1."""
    cam = synthetic.make_camera((0.0, 0.0, 3.0), 40, 40, fov_y_deg=40.0)
    col = np.array([0.8, 0.6, 0.4])
    recv = _quad(0.0, 2.0, col, 1.0)
    xo = np.array([[0.6, -0.2, 0.5], [1.0, -0.2, 0.5], [1.0, 0.2, 0.5], [0.6, 0.2, 0.5]])   # not under the view axis
    occ = (xo, np.tile([0.0, 0.0, 0.0], (4, 1)).astype(np.float64), np.full(4, 0.6), np.array([[0, 1, 2], [0, 2, 3]]))
    x, c, a, t = _merge(recv, occ)
    k = 0.25
    L = np.array([2.0, 0.0, 2.0])
    img = RT.render(x, c, a, t, cam, light=L, ambient=k)
    plain = RT.render(x, c, a, t, cam)
    checked = shadowed = 0
    R = np.asarray(cam.R_cw, np.float64).reshape(3, 3)
    for py in range(40):
        for px in range(40):
            d = R.T @ np.array([(px + 0.5 - cam.cx) / cam.fx, (py + 0.5 - cam.cy) / cam.fy, 1.0])
            # first hit: the occluder if the ray meets it, else the receiver
            p_occ = cam.C + d * ((0.5 - cam.C[2]) / d[2])
            if 0.6 - 1e-6 <= p_occ[0] <= 1.0 + 1e-6 and -0.2 - 1e-6 <= p_occ[1] <= 0.2 + 1e-6:
                continue                                    # the occluder is in front here: skip
            p = cam.C + d * ((0.0 - cam.C[2]) / d[2])      # receiver point
            q = (p + 0.25 * (L - p))[:2]                     # where the segment to the light meets z = 0.5
            inside = 0.6 < q[0] < 1.0 and -0.2 < q[1] < 0.2
            margin = min(abs(q[0] - 0.6), abs(q[0] - 1.0), abs(q[1] + 0.2), abs(q[1] - 0.2))
            if margin < 1e-6:
                continue
            S = 0.4 if inside else 1.0
            assert np.allclose(img[py, px, :3], plain[py, px, :3] * (k + (1 - k) * S), rtol=1e-12, atol=1e-14)
            checked += 1
            shadowed += inside
    assert checked > 1000 and shadowed > 20


def test_stacked_occluders_multiply():
    p = np.array([0.0, 0.0, 0.0])
    light = (0.0, 0.0, 3.0)
    o1 = _quad(1.0, 0.5, [0, 0, 0], 0.3)
    o2 = _quad(2.0, 0.5, [0, 0, 0], 0.5)
    x, c, a, t = _merge(_quad(0.0, 0.5, [1, 1, 1], 1.0), o1, o2)
    P0, P1, P2 = x[t[:, 0]], x[t[:, 1]], x[t[:, 2]]
    S = RT.transmittance(p + np.array([0.1, 0.05, 0.0]), light, 0, P0, P1, P2, a[t])
    assert abs(S - 0.7 * 0.5) < 1e-15


def test_no_self_shadow_from_the_own_triangle():
    x, c, a, t = _quad(0.0, 1.0, [1, 1, 1], 0.9)
    P0, P1, P2 = x[t[:, 0]], x[t[:, 1]], x[t[:, 2]]
    # a point of triangle 0, light behind the plane: the segment leaves from triangle 0
    # itself (excluded) and crosses nothing else
    S = RT.transmittance(np.array([0.5, -0.5, 0.0]), (0.2, -0.3, -2.0), 0, P0, P1, P2, a[t])
    assert S == 1.0
