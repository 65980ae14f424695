"""The fine-tuning of Sec. 3 on the GPU: per-face pruning (ms_prune_faces) bit for bit
against the oracle, the masked render against the oracle's render of the kept faces, and
the whole loop (Eq. 3 loss over two views, adjoint, two-learning-rate Adam, pruning every
few epochs) against the same loop run by the FP64 oracle."""
import json
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import synthetic  # noqa: E402
from oracle import loss as oloss  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_07754_gb300._lib as L
    L.lib()


import paper_2502_07754_gb300 as ms  # noqa: E402
from paper_2502_07754_gb300.finetune import FanFineTune  # noqa: E402
from gpu_util import dev, err_report, oracle_mesh_f32  # noqa: E402

THR = float(np.float32(math.exp(-4.0)))


def _designed_alpha(a, n, K, seed):
    """Opacities far from the threshold except by design: a third of the fans all dim
    (removed), a third with a dim centre and boundary vertices 0, 1, 4, 5 dim (faces 0 and
    4 removed), the rest at least 0.05."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a = np.maximum(a.reshape(n, K + 1), np.float32(0.05))
    kind = rng.integers(0, 3, n)
    a[kind == 0] = np.float32(0.005)
    part = kind == 1
    a[part, 0] = np.float32(0.005)
    a[np.ix_(part, 1 + np.array([0, 1, 4, 5]))] = np.float32(0.005)
    return a.reshape(-1).astype(np.float32)


@pytest.mark.parametrize("n,K,with_mask", [(3001, 8, False), (2500, 6, True), (0, 8, False)])
def test_prune_faces_matches_oracle_bit_for_bit(n, K, with_mask):
    rng = np.random.Generator(np.random.PCG64(30 + n))
    V = n * (K + 1)
    xyz = rng.normal(size=(V, 3)).astype(np.float32)
    rgb = rng.random((V, 3)).astype(np.float32)
    a = _designed_alpha(rng.random(V).astype(np.float32), n, K, 31) if n else np.zeros(0, np.float32)
    m = rng.normal(size=7 * V).astype(np.float32)
    v = rng.random(7 * V).astype(np.float32)
    early = rng.integers(0, 1 << K, max(n, 1)).astype(np.int32)[:n] if with_mask else None
    px, pc, pa, pm, pv, mask, k = ms.prune_faces(dev(xyz), dev(rgb), dev(a), K,
                                                 face_mask=dev(early) if early is not None else None,
                                                 threshold=THR, m=dev(m), v=dev(v))
    ox, oc, oa, (om, ov), omask, fans = oracle.prune_faces(xyz, rgb, a, K, face_mask=early, threshold=THR,
                                                          moments=(m, v))
    assert k == fans.size
    for got, want in ((px, ox), (pc, oc), (pa, oa), (pm, om), (pv, ov)):
        assert np.array_equal(got.cpu().numpy(), np.asarray(want, np.float32).reshape(got.shape))
    assert np.array_equal(mask.cpu().numpy().astype(np.int64), omask)


def test_masked_render_matches_the_kept_faces():
    w = synthetic.workload(1, n=400)
    cam = w.cameras[0]
    K = 8
    xyz, rgb, a = oracle_mesh_f32(w.scene, K, cam.C)
    a = _designed_alpha(a, 400, K, 5)
    px, pc, pa, _, _, mask, k = ms.prune_faces(dev(xyz), dev(rgb), dev(a), K, threshold=THR)
    r = ms.Renderer(k, K, cam, ms.render_params(face_mask=mask))
    img = r.forward(px, pc, pa).cpu().numpy().astype(np.float64)
    ox, oc, oa, _, omask, fans = oracle.prune_faces(xyz, rgb, a, K, threshold=THR)
    ref, _, _ = oracle.render(ox.astype(np.float64), oc.astype(np.float64), oa.astype(np.float64),
                              oracle.masked_fan_tris(fans.size, K, omask), cam)
    rep = err_report(img, ref)
    assert rep["n_over_tol"] == 0, rep
    assert 0 < k < 400 and (omask != (1 << K) - 1).any()


def test_fine_tune_loop_matches_the_oracle_loop():
    """Twelve epochs of the full loop on 400 Gaussians and two 128 x 128 views (pruning
    every 4 epochs, lr_color 1e-3 so that no opacity crosses the threshold by drift): the
    per-epoch losses agree to 1e-4 relative, the same faces are pruned, and the final
    renders agree to 2e-3 (Adam normalises every gradient, so vertices with near-zero
    gradients -- sign decided by rounding -- move by up to lr per step on either side
    without changing the image much)."""
    w = synthetic.workload(1, n=400)
    K = 8
    cams = [w.cameras[0], synthetic.make_camera((1.5, 0.5, 3.6), 128, 128)]
    xyz, rgb, a = oracle_mesh_f32(w.scene, K, cams[0].C)
    a = _designed_alpha(a, 400, K, 6)
    tgt_scene = synthetic.jittered(w.scene, 2e-2, 77)
    txyz, trgb, ta = oracle_mesh_f32(tgt_scene, K, cams[0].C)
    br = ms.BatchRenderer(400, K, cams)
    targets = br.forward(dev(txyz), dev(trgb), dev(ta)).clone()
    tgt_np = [t.cpu().numpy().astype(np.float64) for t in br.images(targets)]
    lr, epochs, every = 1e-3, 12, 4
    ft = FanFineTune(dev(xyz), dev(rgb), dev(a), K, cams, targets, lr_color=lr, prune_every=every, threshold=THR)
    gpu_losses = ft.run(epochs)
    # the oracle loop
    X, Cc, A = xyz.astype(np.float64), rgb.astype(np.float64), a.astype(np.float64)
    m, v = np.zeros(7 * X.shape[0]), np.zeros(7 * X.shape[0])
    mask = None
    orc_losses = []
    for ep in range(1, epochs + 1):
        n = X.shape[0] // (K + 1)
        tris = oracle.masked_fan_tris(n, K, mask)
        gx, gc, ga = np.zeros_like(X), np.zeros_like(Cc), np.zeros_like(A)
        total = 0.0
        for cam, tgt in zip(cams, tgt_np):
            img, _, _ = oracle.render(X, Cc, A, tris, cam)
            l, g = oloss.fine_tune_loss(img, tgt, 0.6)
            total += l / len(cams)
            dL = np.zeros_like(img)
            dL[..., :3] = g / len(cams)
            x_, c_, a_ = oracle.render_backward(X, Cc, A, tris, cam, dL)
            gx += x_
            gc += c_
            ga += a_
        orc_losses.append(total)
        oracle.fan_adam_step(X, Cc, A, gx, gc, ga, m, v, ep, lr)
        if ep % every == 0:
            X, Cc, A, (m, v), mask, _ = oracle.prune_faces(X, Cc, A, K, face_mask=mask, threshold=THR,
                                                           moments=(m, v))
    rel = np.abs(np.array(gpu_losses) - np.array(orc_losses)) / np.array(orc_losses)
    assert ft.n_fans == X.shape[0] // (K + 1)
    assert np.array_equal(ft.face_mask.cpu().numpy().astype(np.int64), mask)
    flat = ft.br.new_flat()
    ft.br.forward(ft.xyz, ft.rgb, ft.alpha, flat)
    worst = 0.0
    tris = oracle.masked_fan_tris(X.shape[0] // (K + 1), K, mask)
    for cam, img in zip(cams, ft.br.images(flat)):
        ref, _, _ = oracle.render(X, Cc, A, tris, cam)
        worst = max(worst, float(np.abs(img.cpu().numpy() - ref).max()))
    print(json.dumps({"loss_rel_err_max": float(rel.max()), "final_image_max_abs": worst,
                      "prunes": ft.history, "loss_first": orc_losses[0], "loss_last": orc_losses[-1]}))
    assert rel.max() < 1e-4, rel
    assert worst < 2e-3, worst
    assert orc_losses[-1] < orc_losses[0]
    assert ft.history and ft.history[0][2] < ft.history[0][1]
