"""GPU parity of the learned fan initializer (tensor-core MLP) against oracle/mlp.py:
inputs, inference, the gradients of a training step, and corrections consumed by the
fan conversion.

Tolerance of the network outputs: both sides round the same operands to bfloat16, but
a pre-activation accumulated in FP32 (GPU) or FP64 (oracle) can round to neighbouring
bfloat16 values, one unit (2^-8 relative) in some hidden activations; an output then
moves by at most 2^-8 sum_k |h2_k W3_kj| from the last layer plus what the first hidden
layer passes on, so the test allows 2^-6 sum_k |h2_k W3_kj| + 1e-5.  The weight
gradients are compared entry by entry against a bound propagated the same way through
the forward and backward passes (_grad_bounds)."""
import json
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import mlp  # noqa: E402
import synthetic  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_07754_gb300._lib as L
    L.lib()


from gpu_util import dev, scene_tensors  # noqa: E402
import paper_2502_07754_gb300 as ms  # noqa: E402

K = 8
NOUT = 2 * (K + 1)


def _weights(seed, zero_out=False):
    rng = np.random.Generator(np.random.PCG64(seed))
    W1 = rng.normal(0, 0.35, (16, 128))
    W2 = rng.normal(0, 0.12, (128, 128))
    W3 = np.zeros((128, NOUT)) if zero_out else rng.normal(0, 0.1, (128, NOUT))
    return [w.astype(np.float32) for w in (W1, W2, W3)]


def _gpu_features(sc):
    _, s, q, o, sh = scene_tensors(sc)
    net = ms.FanMLP(K=K)
    return net.features(s, q, o, sh, sc.sh_degree).cpu().numpy().astype(np.float64)


def test_features_match_oracle():
    for bf in (False, True):
        sc = synthetic.surface_scene(5000, 61, degree=3, clustered=True, bf16=bf)
        got = _gpu_features(sc)
        want = mlp.scene_features(sc)
        err = np.abs(got - want) / np.maximum(1.0, np.abs(want))
        assert err.max() < 2e-6, (bf, err.max(), np.unravel_index(err.argmax(), err.shape))


@pytest.mark.parametrize("n", [1, 127, 128, 1000, 20011])
def test_inference_matches_oracle(n):
    sc = synthetic.surface_scene(n, 62 + n, degree=3, clustered=True, bf16=True)
    W = _weights(5)
    net = ms.FanMLP(K=K, weights=W)
    _, s, q, o, sh = scene_tensors(sc)
    got = net.forward(s, q, o, sh, sc.sh_degree).cpu().numpy().astype(np.float64)
    X = net.features(s, q, o, sh, sc.sh_degree).cpu().numpy().astype(np.float64)
    y, cache = mlp.forward(X, *[w.astype(np.float64) for w in W])
    cond = np.abs(cache["h2"]) @ np.abs(cache["w3"])
    tol = 2.0 ** -6 * cond + 1e-5
    d = np.abs(got - y)
    assert np.all(d <= tol), (d.max(), (d / tol).max())
    assert np.median(d) < 1e-2 * np.median(np.abs(y)) + 1e-6
    st, t = net.status()
    assert st == 0 and t == 0


def test_zero_output_layer_gives_zero_corrections_on_gpu():
    sc = synthetic.surface_scene(3000, 63, degree=0)
    net = ms.FanMLP(K=K, weights=_weights(6, zero_out=True))
    _, s, q, o, sh = scene_tensors(sc)
    corr = net.forward(s, q, o, sh, sc.sh_degree)
    assert torch.count_nonzero(corr).item() == 0


def _gelu2(z):
    # second derivative of the exact GELU: phi(z) (2 - z^2)
    return np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi) * (2.0 - z * z)


def _grad_bounds(cache, dy, T):
    """Per-entry bounds on |GPU - oracle| for dW1, dW2, dW3, propagated through the network
    from the two ways the sides may differ: a value rounded to bfloat16 (h1, h2, dy, dz2,
    dz1) may land on the neighbouring bfloat16 value (one bfloat16 unit, at most 2^-7 of
    the value) because the GPU's FP32 value before rounding differs from the oracle's FP64
    value, and the tensor cores accumulate k products in FP32 (k 2^-24 sum |a b|).  Inputs
    and weights are the same bfloat16 values on both sides."""
    a = np.abs
    u8, u24 = 2.0 ** -7, 2.0 ** -24
    acc = lambda A, B: A.shape[1] * u24 * (a(A) @ a(B))
    x, w1, w2, w3 = cache["x"], cache["w1"], cache["w2"], cache["w3"]
    z1, h1, z2, h2 = cache["z1"], cache["h1"], cache["z2"], cache["h2"]
    gp1, gp2 = a(mlp.gelu_grad(z1)), a(mlp.gelu_grad(z2))
    e_z1 = acc(x, w1)
    e_h1 = u8 * a(h1) + gp1 * e_z1
    e_z2 = e_h1 @ a(w2) + acc(h1, w2)
    e_h2 = u8 * a(h2) + gp2 * e_z2
    y = h2 @ w3
    e_y = e_h2 @ a(w3) + acc(h2, w3)
    dyr = mlp.bf16_round(dy)
    # dy = 2 (y - T) / size in FP32 (its rounding and y's error), then rounded to bfloat16
    e_dy = 2.0 * (e_y + 4 * u24 * (a(y) + a(T))) / dy.size + u8 * a(dyr)
    e_w3 = e_h2.T @ a(dyr) + a(h2).T @ e_dy + acc(h2.T, dyr)
    g2 = dyr @ w3.T
    e_g2 = e_dy @ a(w3.T) + acc(dyr, w3.T)
    dz2 = mlp.bf16_round(g2 * mlp.gelu_grad(z2))
    e_dz2 = e_g2 * gp2 + a(g2) * a(_gelu2(z2)) * e_z2 + u8 * a(dz2)
    e_w2 = e_h1.T @ a(dz2) + a(h1).T @ e_dz2 + acc(h1.T, dz2)
    g1 = dz2 @ w2.T
    e_g1 = e_dz2 @ a(w2.T) + acc(dz2, w2.T)
    dz1 = mlp.bf16_round(g1 * mlp.gelu_grad(z1))
    e_dz1 = e_g1 * gp1 + a(g1) * a(_gelu2(z1)) * e_z1 + u8 * a(dz1)
    e_w1 = a(x).T @ e_dz1 + acc(x.T, dz1)
    return e_w1, e_w2, e_w3


@pytest.mark.parametrize("n", [200, 4096, 30001])
def test_gradients_match_oracle(n):
    sc = synthetic.surface_scene(n, 64 + n, degree=3, clustered=True)
    W = _weights(7)
    net = ms.FanMLP(K=K, weights=W)
    _, s, q, o, sh = scene_tensors(sc)
    X = net.features(s, q, o, sh, sc.sh_degree)
    rng = np.random.Generator(np.random.PCG64(8))
    T = rng.normal(0, 0.2, (n, NOUT)).astype(np.float32)
    grads, loss = net.compute_grads(X, dev(T))
    g = grads.cpu().numpy().astype(np.float64)
    Xo = X.cpu().numpy().astype(np.float64)
    y, cache = mlp.forward(Xo, *[w.astype(np.float64) for w in W])
    lo, dy = mlp.mse_grad(y, T.astype(np.float64))
    want = mlp.backward(cache, dy)
    bounds = _grad_bounds(cache, dy, T.astype(np.float64))
    off = 0
    for name, wv, eb in zip(("dW1", "dW2", "dW3"), want, bounds):
        gv = g[off:off + wv.size].reshape(wv.shape)
        off += wv.size
        err = np.abs(gv - wv)
        # an absolute floor 2^-20 below the matrix's largest entry: the tensor cores align
        # the products of an accumulation group to its largest one, so entries made of
        # vanishing products (dead GELU units, ~1e-25) carry errors relative to that scale
        eb = eb + 2.0 ** -20 * np.abs(wv).max()
        ratio = err / (eb + 1e-30)
        worst = np.unravel_index(int(np.argmax(ratio)), ratio.shape)
        print(json.dumps({"n": n, "grad": name, "max_err_over_bound": float(ratio.max()), "at": [int(i) for i in worst],
                          "gpu": float(gv[worst]), "oracle": float(wv[worst]), "bound": float(eb[worst])}))
        # element by element within the derived bound (twice it, for the bound's own
        # first-order terms), and the typical entry far inside it
        assert (err <= 2.0 * eb + 1e-30).all(), (name, float(ratio.max()))
        # the bound is a worst case (every rounding on the other side); a misplaced or
        # sign-flipped entry in a sum that cancels can hide under it, so the typical
        # entry must also sit far inside it (an FP32 simulation gives ratios ~1e-6)
        assert np.median(err / (eb + 1e-30)) < 1e-2, name
        rel = np.linalg.norm(gv - wv) / np.linalg.norm(wv)
        print(json.dumps({"n": n, "grad": name, "max_err_over_bound": float((err / (eb + 1e-30)).max()),
                          "median_err_over_bound": float(np.median(err / (eb + 1e-30))), "frobenius_rel": rel}))
        assert rel < 2e-2, (name, rel)
    assert abs(loss.item() - lo) <= 1e-3 * lo
    st, t = net.status()
    assert st == 0 and t == 0


def test_training_steps_reduce_the_loss():
    sc = synthetic.surface_scene(8192, 65, degree=3, clustered=True)
    net = ms.FanMLP(K=K, seed=3)
    _, s, q, o, sh = scene_tensors(sc)
    X = net.features(s, q, o, sh, sc.sh_degree)
    # a smooth target of the inputs: the network can fit it
    Xn = X.cpu().numpy()
    T = np.tanh(Xn[:, :NOUT % 16 + 2].sum(1, keepdims=True)) * np.linspace(-0.2, 0.2, NOUT)[None, :]
    Tt = dev(T.astype(np.float32))
    first = None
    for i in range(60):
        l = net.train_step(X, Tt, lr=3e-3).item()
        first = l if first is None else first
    assert l < 0.3 * first, (first, l)
    assert int(net.step.item()) == 60


def test_corrections_drive_the_conversion_like_the_oracle():
    sc = synthetic.surface_scene(4000, 66, degree=3, clustered=True, bf16=True)
    net = ms.FanMLP(K=K, weights=_weights(9))
    m, s, q, o, sh = scene_tensors(sc)
    corr = net.forward(s, q, o, sh, sc.sh_degree) * 0.05
    cc = np.array([0.3, 0.2, 3.0], np.float32)
    xyz, rgb, a = ms.mesh_build(m, s, q, o, sh, sc.sh_degree, K=K, cam_center=cc, corr=corr.contiguous())
    xo, co, ao = oracle.mesh_build(sc, K=K, cam_center=cc, corr=corr.cpu().numpy().astype(np.float64))
    assert np.abs(xyz.cpu().numpy() - xo).max() < 2e-6
    assert np.abs(a.cpu().numpy() - ao).max() < 2e-6
    assert np.abs(rgb.cpu().numpy() - co).max() < 2e-6


def _scaled_weights(seed, k, scale):
    rng = np.random.Generator(np.random.PCG64(seed))
    n_out = 2 * (k + 1)
    W1 = rng.normal(0, 0.35, (16, 128))
    W2 = rng.normal(0, 0.12, (128, 128))
    W3 = rng.normal(0, 0.1 * scale, (128, n_out))
    return [w.astype(np.float32) for w in (W1, W2, W3)]


@pytest.mark.parametrize("k,n,deg,bf", [(8, 4000, 3, True), (8, 130, 3, False), (15, 1000, 2, True),
                                        (3, 777, 1, False), (6, 300, 0, True)])
def test_fused_inference_conversion_equals_the_two_launches(k, n, deg, bf):
    """ms_mesh_build_mlp (inference fused into the conversion, corrections kept on chip)
    gives the fan soup of ms_mlp_forward then ms_mesh_build bit for bit: ragged tiles,
    K = 15 (staged in two chunks of Gaussians per tile), every SH degree; and the soup
    matches the oracle's conversion with the same corrections."""
    sc = synthetic.surface_scene(n, 70 + k, degree=deg, clustered=True, bf16=bf)
    net = ms.FanMLP(K=k, weights=_scaled_weights(11 + k, k, 0.5))
    m, s, q, o, sh = scene_tensors(sc)
    cc = np.array([0.3, 0.2, 3.0], np.float32)
    corr = net.forward(s, q, o, sh, sc.sh_degree)
    want = ms.mesh_build(m, s, q, o, sh, sc.sh_degree, K=k, cam_center=cc, corr=corr)
    got = ms.mesh_build(m, s, q, o, sh, sc.sh_degree, K=k, cam_center=cc, mlp=net)
    for a, b in zip(got, want):
        assert torch.equal(a, b)
    assert net.status() == (0, 0)   # no tensor-core wait expired
    xo, co, ao = oracle.mesh_build(sc, K=k, cam_center=cc, corr=corr.cpu().numpy().astype(np.float64))
    assert np.abs(got[0].cpu().numpy() - xo).max() < 2e-6 * max(1.0, np.abs(xo).max())
    assert np.abs(got[1].cpu().numpy() - co).max() < 2e-6
    assert np.abs(got[2].cpu().numpy() - ao).max() < 2e-6


def test_fused_conversion_rejects_bad_arguments():
    sc = synthetic.surface_scene(50, 3, degree=0)
    m, s, q, o, sh = scene_tensors(sc)
    net = ms.FanMLP(K=8)
    with pytest.raises(ValueError):
        ms.mesh_build(m, s, q, o, sh, 0, K=6, mlp=net)          # packed for K = 8
    with pytest.raises(ValueError):
        ms.mesh_build(m, s, q, o, sh, 0, K=8, mlp=net, corr=torch.zeros(50, 18, device="cuda"))
