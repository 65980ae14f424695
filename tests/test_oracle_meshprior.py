"""Pins of the mesh-prior oracle (oracle/meshprior.py): secondary triangles as convex
combinations of the geometry faces (Sec. 3, the mesh-prior paragraphs)."""
import numpy as np

import oracle
import synthetic
from oracle import meshprior as MP


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _faces(F, seed):
    rng = _rng(seed)
    c = rng.normal(0, 0.5, (F, 1, 3))
    return c + rng.normal(0, 0.2, (F, 3, 3))


def test_one_triangle_per_face_starts_as_the_face():
    faces = _faces(30, 1)
    v = MP.secondary_vertices(faces, MP.init_weights(30, 1))
    assert np.array_equal(v[:, 0], faces)


def test_midpoint_subdivision_tiles_the_face():
    faces = _faces(25, 2)
    v = MP.secondary_vertices(faces, MP.init_weights(25, 4))
    area = lambda t: 0.5 * np.linalg.norm(np.cross(t[..., 1, :] - t[..., 0, :], t[..., 2, :] - t[..., 0, :]), axis=-1)
    assert np.allclose(area(v).sum(axis=1), area(faces), rtol=1e-13, atol=0)
    mid = 0.5 * (faces[:, 0] + faces[:, 1])
    assert np.allclose(v[:, 0, 1], mid, rtol=0, atol=1e-15) and np.array_equal(v[:, 0, 0], faces[:, 0])


def test_weights_stay_on_the_simplex_and_vertices_in_the_face():
    rng = _rng(3)
    faces = _faces(40, 4)
    w = rng.normal(size=(40, 2, 3, 3))
    a = MP.simplex_weights(w)
    assert np.all(a >= 0) and np.allclose(a.sum(-1), 1.0, rtol=0, atol=1e-15)
    v = MP.secondary_vertices(faces, w)
    # barycentric coordinates of each vertex w.r.t. its face, recovered by least squares
    for f in range(40):
        M = np.stack([faces[f, 1] - faces[f, 0], faces[f, 2] - faces[f, 0]], axis=1)
        for s in range(2):
            for i in range(3):
                uv, res, _, _ = np.linalg.lstsq(M, v[f, s, i] - faces[f, 0], rcond=None)
                assert np.linalg.norm(M @ uv - (v[f, s, i] - faces[f, 0])) < 1e-13   # in the face's plane
                assert uv.min() >= -1e-13 and uv.sum() <= 1 + 1e-13                 # inside the face


def test_weight_gradient_matches_finite_differences():
    rng = _rng(5)
    faces = _faces(6, 6)
    w = rng.normal(size=(6, 4, 3, 3))
    C = rng.normal(size=(6, 4, 3, 3))
    L = lambda ww: float((MP.secondary_vertices(faces, ww) ** 2 * C).sum())
    g_v = 2.0 * MP.secondary_vertices(faces, w) * C
    g = MP.weight_grads(faces, w, g_v)
    h = 1e-6
    for idx in [(0, 0, 0, 0), (2, 3, 1, 2), (5, 1, 2, 1), (3, 2, 0, 1)]:
        wp, wm = w.copy(), w.copy()
        wp[idx] += h
        wm[idx] -= h
        fd = (L(wp) - L(wm)) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-7 * max(1.0, abs(fd)), (idx, fd, g[idx])


def test_centroid_fans_render_like_the_triangles():
    """Four secondary triangles per face (the midpoint subdivision, which tiles the face)
    over a small synthetic mesh: the triangle soup and its K = 3 centroid fans give the
    same image (FP64 oracle, both ways).  (Secondary triangles of one face that overlap lie
    in one plane, so their order at a pixel is a depth tie decided by rounding; splitting a
    triangle into a fan can change that rounding, so overlapping layouts are not compared.)"""
    w = synthetic.workload(1, n=10)
    cam = w.cameras[0]
    faces = _faces(40, 7) * 0.8
    rng = _rng(8)
    S = 4
    wts = MP.init_weights(40, S)
    rgb = rng.random((40, S, 3, 3))
    alpha = rng.uniform(0.2, 0.9, (40, S, 3))
    x, c, a, tris = MP.triangle_soup(faces, wts, rgb, alpha)
    fx, fc, fa = MP.as_centroid_fans(x, c, a)
    tri_img, nf, _ = oracle.render(x, c, a, tris, cam)
    fan_img, _, _ = oracle.render(fx, fc, fa, oracle.fan_tris(tris.shape[0], 3), cam)
    assert nf.max() > 2 and tri_img[..., 3].max() > 0.3
    assert np.abs(tri_img - fan_img).max() < 1e-12


def test_centroid_fan_adjoint():
    rng = _rng(9)
    T = 7
    x = rng.normal(size=(3 * T, 3))
    gx = rng.normal(size=(4 * T, 3))
    gc = rng.normal(size=(4 * T, 3))
    ga = rng.normal(size=4 * T)
    tx, tc, ta = MP.fan_grads_to_triangles(gx, gc, ga)
    # <J v, g> = <v, J^T g> for the linear map triangle -> fan
    fx, _, _ = MP.as_centroid_fans(x, x, x[:, 0])
    assert abs((fx * gx).sum() - (x * tx).sum()) < 1e-12
