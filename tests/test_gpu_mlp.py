"""GPU parity of the learned fan initializer (tensor-core MLP) against oracle/mlp.py:
inputs, inference, the gradients of a training step, and corrections consumed by the
fan conversion.

Tolerance of the network outputs: both sides round the same operands to bfloat16, but
a pre-activation accumulated in FP32 (GPU) or FP64 (oracle) can round to neighbouring
bfloat16 values, one unit (2^-8 relative) in some hidden activations; an output then
moves by at most 2^-8 sum_k |h2_k W3_kj| from the last layer plus what the first hidden
layer passes on, so the test allows 2^-6 sum_k |h2_k W3_kj| + 1e-5."""
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
    off = 0
    for name, wv in zip(("dW1", "dW2", "dW3"), want):
        gv = g[off:off + wv.size].reshape(wv.shape)
        off += wv.size
        rel = np.linalg.norm(gv - wv) / np.linalg.norm(wv)
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
