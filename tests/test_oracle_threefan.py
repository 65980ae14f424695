"""Pins of the three-fan conversion oracle (oracle/threefan.py): Sec. 3 "Transformation
for 3D Gaussians" -- three orthogonal fans per Gaussian, shared tips, 3K triangles."""
import math

import numpy as np
import pytest

import oracle
import synthetic
from oracle import threefan as TF


def _scene(n, seed, degree=0):
    return synthetic.random_scene(n, seed, degree=degree)


@pytest.mark.parametrize("K,nv", [(8, 19), (12, 31), (6, 17), (5, 15), (4, 7)])
def test_vertex_counts(K, nv):
    """1 + 3K boundary slots minus the tips reached by two fans: with 4 | K all six tips
    are shared (1 + 3K - 6); with K even but not 4 | K only +-sr_1 (fans (1,2) and (1,3)
    both contain t = -pi and 0); with K odd only -sr_1 (t = -pi)."""
    assert TF.fan_layout(K)[0] == nv


def test_angles_at_quarter_turns_are_exact():
    K = 8
    assert TF.angle_cos_sin(0, K) == (-1.0, 0.0)
    assert TF.angle_cos_sin(2, K) == (0.0, -1.0)
    assert TF.angle_cos_sin(4, K) == (1.0, 0.0)
    assert TF.angle_cos_sin(6, K) == (0.0, 1.0)
    c, s = TF.angle_cos_sin(1, K)
    assert abs(c - math.cos(-3 * math.pi / 4)) < 1e-16 and abs(s - math.sin(-3 * math.pi / 4)) < 1e-16


def test_vertices_on_the_ellipsoid_and_in_their_planes():
    sc = _scene(50, 11)
    K = 8
    xyz, rgb, a, tris, nv = TF.three_fan_build(sc, K=K)
    _, idx = TF.fan_layout(K)
    for g in range(sc.n):
        R = oracle.quat_to_rot(sc.quats[g].astype(np.float64))
        # columns sr_k = (scale_mul exp(s_k)) r_k, the scalar formed first as the equation reads
        A = (TF.SCALE_MUL * np.exp(sc.log_scales[g].astype(np.float64)))[None, :] * R
        m = sc.means[g].astype(np.float64)
        v = xyz[g * nv:(g + 1) * nv]
        assert np.array_equal(v[0], m)
        u = np.linalg.solve(A, (v[1:] - m).T).T          # coordinates along sr_1, sr_2, sr_3
        assert np.abs(np.linalg.norm(u, axis=1) - 1.0).max() < 1e-12
        for p, (i, j) in enumerate(TF.PLANES):
            k = 3 - i - j                                  # the axis normal to fan p
            rows = np.asarray(idx[p]) - 1
            assert np.abs(u[rows, k]).max() < 1e-12
        # each tip m +- sr_k is one vertex, and no two vertices nearly coincide (a tip
        # reached by two fans is stored once)
        for k in range(3):
            for sgn in (1.0, -1.0):
                d = np.linalg.norm(v - (m + sgn * A[:, k]), axis=1)
                assert np.count_nonzero(d < 1e-12 * np.linalg.norm(A[:, k])) == 1
        gaps = np.linalg.norm(v[:, None] - v[None, :], axis=2) + np.eye(nv)
        assert gaps.min() > 1e-6 * np.linalg.norm(A, axis=0).min()


def test_fan_areas_and_triangle_count():
    sc = _scene(20, 12)
    K = 8
    xyz, rgb, a, tris, nv = TF.three_fan_build(sc, K=K)
    assert tris.shape == (sc.n * 3 * K, 3)
    for g in range(sc.n):
        s = TF.SCALE_MUL * np.exp(sc.log_scales[g].astype(np.float64))
        for p, (i, j) in enumerate(TF.PLANES):
            t = tris[(g * 3 + p) * K:(g * 3 + p + 1) * K]
            P = xyz[t]
            area = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1).sum()
            want = 0.5 * K * s[i] * s[j] * math.sin(2 * math.pi / K)
            assert abs(area - want) < 1e-12 * want


def test_colour_and_opacity_follow_the_flat_rule():
    sc = _scene(30, 13, degree=1)
    cc = np.array([0.2, -0.1, 3.0], np.float32)
    xyz, rgb, a, tris, nv = TF.three_fan_build(sc, K=8, cam_center=cc)
    cols = oracle.gaussian_colors(sc, cam_center=cc)
    a = a.reshape(sc.n, nv)
    assert np.array_equal(rgb.reshape(sc.n, nv, 3), np.repeat(cols[:, None], nv, axis=1))
    assert np.array_equal(a[:, 0], sc.opacity.astype(np.float64))
    assert np.allclose(a[:, 1:], 0.2 * sc.opacity.astype(np.float64)[:, None], rtol=0, atol=1e-17)


def test_flat_fan_matches_the_flat_conversion():
    """Fan (2, 3) of a Gaussian whose smallest scale is on axis 1 is the flat conversion's
    fan (which drops the smallest axis and keeps the other two in order)."""
    sc = _scene(40, 14)
    sc.log_scales[:, 0] = sc.log_scales[:, 1:].min(axis=1) - 1.0
    K = 8
    xyz, rgb, a, tris, nv = TF.three_fan_build(sc, K=K)
    fx, fc, fa = oracle.mesh_build(sc, K=K, axis_rule=1)
    _, idx = TF.fan_layout(K)
    for g in range(sc.n):
        ours = xyz[g * nv + np.asarray(idx[2])]
        flat = fx.reshape(sc.n, K + 1, 3)[g, 1:]
        scale = np.abs(flat - fx.reshape(sc.n, K + 1, 3)[g, 0]).max()
        assert np.abs(ours - flat).max() <= 1e-12 * max(scale, 1.0)
        assert np.array_equal(fa.reshape(sc.n, K + 1)[g], a.reshape(sc.n, nv)[g, [0] + list(idx[2])])


def test_implicit_fan_copies_render_like_the_shared_mesh():
    w = synthetic.workload(1, n=60)
    cam = w.cameras[0]
    K = 8
    xyz, rgb, a, tris, nv = TF.three_fan_build(w.scene, K=K, cam_center=cam.C)
    fx, fc, fa, src = TF.as_implicit_fans(xyz, rgb, a, K, nv)
    assert fx.shape[0] == w.scene.n * 3 * (K + 1)
    assert np.array_equal(fx, xyz[src])
    shared, _, _ = oracle.render(xyz, rgb, a, tris, cam)
    fans, _, _ = oracle.render(fx, fc, fa, oracle.fan_tris(w.scene.n * 3, K), cam)
    assert np.array_equal(shared, fans)
    assert shared[..., 3].max() > 0.1


@pytest.mark.parametrize("K", list(range(3, 17)))
def test_library_copy_map_matches_the_oracle(K):
    """ms_three_fan_copies (host code of the library, no device work) against the copy map
    of the oracle's implicit-fan layout: two slots are copies exactly when they copy the
    same unique vertex, and each slot maps to the first of them."""
    import paper_2502_07754_gb300 as ms
    first, n = ms.three_fan_copies(K)
    nv, _ = TF.fan_layout(K)
    assert n == nv
    src = TF.as_implicit_fans(np.zeros((nv, 3)), np.zeros((nv, 3)), np.zeros(nv), K, nv)[3]
    want = [int(np.nonzero(src == src[s])[0].min()) for s in range(src.size)]
    assert first == want
