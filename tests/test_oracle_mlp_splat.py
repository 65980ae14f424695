"""CPU pins of the learned-initializer reference (oracle/mlp.py) and of the
source-Gaussian render (oracle/ms_oracle_splat.c): closed forms, finite differences,
round trips and brute-force re-derivations that a slip in either would break."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp
import synthetic
from synthetic import Scene


# ------------------------------------------------------------------------ bfloat16

def test_bf16_rounding_ties_to_even_and_exact_values():
    u = 2.0 ** -8
    cases = {1.0: 1.0, 1.0 + u: 1.0, 1.0 + 3 * u: 1.0 + 4 * u, 1.0 + u + 2.0 ** -20: 1.0 + 2 * u,
             -1.0 - u: -1.0, 3.0: 3.0, 0.0: 0.0, 2.0 ** -130: 2.0 ** -130}
    for x, want in cases.items():
        assert mlp.bf16_round(np.array([x]))[0] == want, x
    r = mlp.bf16_round(np.random.default_rng(0).normal(size=1000))
    bits = r.astype(np.float32).view(np.uint32)
    assert np.all(bits & 0xFFFF == 0)


# ------------------------------------------------------------------------ GELU

def test_gelu_closed_forms():
    x = np.linspace(-6, 6, 121)
    g = mlp.gelu(x)
    assert np.allclose(g - mlp.gelu(-x), x, atol=1e-15)          # erf odd
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert abs(mlp.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15   # Phi(1)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(x), fd, atol=1e-9)
    assert abs(mlp.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15


# ------------------------------------------------------------------------ network

def _net(seed=1, n=37, n_out=18):
    rng = np.random.Generator(np.random.PCG64(seed))
    X = rng.normal(size=(n, 16))
    X[:, 15] = 1.0
    W1 = rng.normal(0, 0.3, (16, 128))
    W2 = rng.normal(0, 0.1, (128, 128))
    W3 = rng.normal(0, 0.1, (128, n_out))
    T = rng.normal(size=(n, n_out))
    return X, W1, W2, W3, T


def test_zero_output_layer_gives_zero_corrections():
    X, W1, W2, _, _ = _net()
    y, _ = mlp.forward(X, W1, W2, np.zeros((128, 18)))
    assert np.all(y == 0.0)


def test_fp64_network_gradients_match_central_differences():
    X, W1, W2, W3, T = _net()
    y, cache = mlp.forward(X, W1, W2, W3, round_bf16=False)
    _, dy = mlp.mse_grad(y, T)
    g = mlp.backward(cache, dy)
    Ws = [W1, W2, W3]
    rng = np.random.default_rng(3)
    for li in range(3):
        for _ in range(6):
            i, j = (int(rng.integers(0, s)) for s in Ws[li].shape)
            h = 1e-6
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[li][i, j] += h
            Wm[li][i, j] -= h
            lp, _ = mlp.mse_grad(mlp.forward(X, *Wp, round_bf16=False)[0], T)
            lm, _ = mlp.mse_grad(mlp.forward(X, *Wm, round_bf16=False)[0], T)
            fd = (lp - lm) / (2 * h)
            assert abs(g[li][i, j] - fd) <= 1e-7 * max(1.0, abs(fd)), (li, i, j, g[li][i, j], fd)


def test_bf16_network_stays_within_rounding_of_fp64():
    X, W1, W2, W3, _ = _net()
    y64, _ = mlp.forward(X, W1, W2, W3, round_bf16=False)
    y16, _ = mlp.forward(X, W1, W2, W3, round_bf16=True)
    scale = np.abs(y64).max()
    assert np.abs(y16 - y64).max() < 0.05 * scale     # 8-bit significands, two layers
    assert np.abs(y16 - y64).max() > 0.0             # the rounding points are active


def test_adam_first_step_closed_form():
    p = [np.array([1.0, -2.0, 0.5])]
    g = [np.array([0.3, -4.0, 2.0])]
    m = [np.zeros(3)]
    v = [np.zeros(3)]
    mlp.adam(p, g, m, v, 1, 0.01, eps=0.0)
    # first step: m_hat = g, v_hat = g^2, so the update is lr * sign(g)
    assert np.allclose(p[0], [0.99, -1.99, 0.49], atol=1e-15, rtol=0)


# ------------------------------------------------------------------------ features

def test_features_of_a_constructed_gaussian():
    X = mlp.features(np.zeros((1, 3)), np.log([[0.1, 0.2, 0.001]]), [[2.0, 0.0, 0.0, 0.0]], [0.7],
                     [[0.1, -0.2, 0.3]])
    want = [math.log(0.1), math.log(0.2), math.log(0.001), 1, 0, 0, 0, 0.7, 0.1, -0.2, 0.3, 1.0, 0.5, 0.005,
            math.log(0.01), 1.0]
    assert np.allclose(X[0], want, atol=1e-12)


def test_corrections_round_trip_through_the_conversion():
    """Targets extracted from a 'fine-tune' that scaled boundary offsets by (1 + dr) and
    opacities by exp(do) are dr, do; converting with them reproduces the moved fans."""
    sc = synthetic.surface_scene(50, 7, degree=0)
    K = 8
    xyz0, _, a0 = oracle.mesh_build(sc, K=K)
    rng = np.random.Generator(np.random.PCG64(9))
    corr = np.zeros((sc.n, 2 * (K + 1)))
    corr[:, 1:K + 1] = rng.uniform(-0.3, 0.3, (sc.n, K))
    corr[:, K + 1:] = rng.uniform(-0.5, 0.0, (sc.n, K + 1))
    xyz1, _, a1 = oracle.mesh_build(sc, K=K, corr=corr)
    got = mlp.corrections_from_finetune(xyz0, a0, xyz1, a1, K)
    assert np.allclose(got[:, 1:], corr[:, 1:], atol=1e-9)
    assert np.all(got[:, 0] == 0.0)


# ------------------------------------------------------------------------ source-Gaussian render

def _one_scene(means, log_scales, quats, opac, dc):
    n = len(means)
    sh = np.zeros((n, 1, 3), np.float32)
    sh[:, 0, :] = np.asarray(dc, np.float32)
    return Scene(np.asarray(means, np.float32), np.asarray(log_scales, np.float32), np.asarray(quats, np.float32),
                 np.asarray(opac, np.float32), sh, 0, False)


def _world_rays(cam, px, py):
    R = np.asarray(cam.R_cw, np.float32).astype(np.float64).reshape(3, 3)
    f32 = lambda v: float(np.float32(v))          # the camera travels as binary32
    dc = np.stack([(px - f32(cam.cx)) / f32(cam.fx), (py - f32(cam.cy)) / f32(cam.fy), np.ones_like(px)], -1)
    return dc @ R          # rows: R^T dc


def test_splat_fronto_parallel_isotropic_closed_form():
    sc = _one_scene([[0, 0, 0]], [[math.log(0.2), math.log(0.2), math.log(1e-4)]], [[1, 0, 0, 0]], [0.8],
                    [[0.4, -0.1, 0.2]])
    s = math.exp(float(sc.log_scales[0, 0]))       # the binary32 inputs, widened
    sig = float(sc.opacity[0])
    cam = synthetic.make_camera((0.0, 0.0, 4.0), 96, 80)
    img, nf = oracle.splat_render(sc, cam)
    py, px = np.mgrid[0:80, 0:96].astype(np.float64) + 0.5
    d = _world_rays(cam, px, py)
    C = np.asarray(cam.C, np.float32).astype(np.float64)
    t = -C[2] / d[..., 2]
    P = C + t[..., None] * d
    r2 = P[..., 0] ** 2 + P[..., 1] ** 2
    col = 0.5 + 0.5 * math.sqrt(1.0 / math.pi) * np.array([0.4, -0.1, 0.2], np.float32).astype(np.float64)
    a = np.where(r2 <= (2.7 * s) ** 2, sig * np.exp(-r2 / (2 * s * s)), 0.0)
    assert np.abs(img[..., 3] - a).max() < 1e-9
    assert np.abs(img[..., :3] - a[..., None] * col).max() < 1e-9
    assert nf.sum() == np.count_nonzero(a) and nf.sum() > 100


def test_splat_two_layers_and_permutation():
    sc = _one_scene([[0, 0, 0.3], [0, 0, 0]], [[-1.5, -1.5, -9], [-1.2, -1.2, -9]], [[1, 0, 0, 0]] * 2,
                    [0.6, 0.9], [[0.5, 0.0, 0.0], [0.0, 0.5, 0.0]])
    cam = synthetic.make_camera((0.0, 0.0, 4.0), 33, 33)
    img, _ = oracle.splat_render(sc, cam)
    col = oracle.gaussian_colors(sc)
    c = img[16, 16]
    # the pixel centre (16.5, 16.5) is the principal point: both splats hit at u = v = 0
    a1, a2 = float(sc.opacity[0]), float(sc.opacity[1])
    want = a1 * col[0] + (1 - a1) * a2 * col[1]
    assert np.allclose(c[:3], want, atol=1e-12)
    assert abs(c[3] - (1 - (1 - a1) * (1 - a2))) < 1e-12
    perm = np.array([1, 0])
    sc2 = _one_scene(sc.means[perm], sc.log_scales[perm], sc.quats[perm], sc.opacity[perm],
                     sc.sh[perm, 0, :])
    img2, _ = oracle.splat_render(sc2, cam)
    assert np.array_equal(img, img2)


@pytest.mark.parametrize("eye,tol", [((0.0, 0.0, 3.5), 1e-9), ((0.5, 0.8, 3.5), 1e-6)])
def test_splat_tilted_matches_a_linear_solve(eye, tol):
    """A tilted splat against a world-space linear solve of m + u u_a + v u_b = C + t d.
    On the axis-aligned camera R_cw is exact; on the oblique one its binary32 entries are
    orthonormal to ~1e-7 only, so the camera-space and world-space geometry agree to that
    level (the tolerance)."""
    rng = np.random.Generator(np.random.PCG64(21))
    q = rng.normal(size=(1, 4))
    sc = _one_scene([[0.1, -0.05, 0.2]], [[-1.3, -9.0, -1.6]], q, [0.7], [[0.2, 0.1, -0.3]])
    cam = synthetic.make_camera(eye, 64, 48)
    img, _ = oracle.splat_render(sc, cam)
    R = oracle.quat_to_rot(sc.quats[0].astype(np.float64))
    ua, ub = R[:, 0], R[:, 2]                 # axis 1 has the smallest scale
    sa, sb = math.exp(float(sc.log_scales[0, 0])), math.exp(float(sc.log_scales[0, 2]))
    m = sc.means[0].astype(np.float64)
    C = np.asarray(cam.C, np.float32).astype(np.float64)
    col = oracle.gaussian_colors(sc)[0]
    n_in = 0
    for py in range(48):
        for px in range(64):
            d = _world_rays(cam, np.array(px + 0.5), np.array(py + 0.5))
            u, v, t = np.linalg.solve(np.stack([ua, ub, -d], 1), C - m)
            inside = (u / (2.7 * sa)) ** 2 + (v / (2.7 * sb)) ** 2 <= 1 and t > 0
            a = float(sc.opacity[0]) * math.exp(-0.5 * (u * u / sa ** 2 + v * v / sb ** 2)) if inside else 0.0
            n_in += inside
            assert abs(img[py, px, 3] - a) < tol, (px, py)
            assert np.allclose(img[py, px, :3], a * col, atol=tol)
    assert n_in > 50
