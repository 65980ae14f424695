"""What the learned initializer gains over the plain conversion: fans converted with
the MLP's corrections start closer to the source-Gaussian render and reach the plain
conversion's fine-tuned PSNR in fewer fine-tune steps (the network is trained on pairs
from fine-tunes of other scenes; everything runs on the GPU)."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synthetic  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_07754_gb300._lib as L
    L.lib()


import paper_2502_07754_gb300 as ms  # noqa: E402
from paper_2502_07754_gb300 import initializer as I  # noqa: E402


def test_trained_initializer_beats_plain_conversion():
    K, n, steps = 8, 20000, 80
    cams = [synthetic.make_camera(d * 3.5, 256, 192) for d in synthetic.fibonacci_dirs(6)]
    cc = cams[0].C
    sets = [I.make_pairs(I.Gaussians.from_scene(synthetic.surface_scene(n, s, degree=3, clustered=True, bf16=True)),
                         cams, K, steps, cc, lr_color=2e-3) for s in (21, 22)]
    for p in sets:   # the fine-tune itself improves the plain conversion
        assert p.curves[0][-1][1] > p.curves[0][0][1] + 3.0
    pairs = I.PairSet(torch.cat([p.X for p in sets]).contiguous(), torch.cat([p.T for p in sets]).contiguous())
    net = ms.FanMLP(K=K, seed=1)
    l0, l1 = I.train(net, pairs, 200, lr=2e-3)
    assert l1 < 0.9 * l0
    held_out = I.Gaussians.from_scene(synthetic.surface_scene(n, 29, degree=3, clustered=True, bf16=True))
    out = I.compare(held_out, cams, K, net, steps, cc, eval_every=10, lr_color=2e-3)
    print(json.dumps(out))
    plain, mlp = out["plain"], out["mlp"]
    assert mlp[0][1] > plain[0][1] + 2.0                     # better start
    assert out["steps_to_plain_final"] is not None and out["steps_to_plain_final"] < steps
    assert mlp[-1][1] >= plain[-1][1] - 0.1                  # and no worse at the end
    st, t = net.status()
    assert st == 0 and t == 0
