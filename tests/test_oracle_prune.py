"""Pins of the pruning oracle (oracle.prune_fans): Sec. 3 "Optimization and Pruning",
faces with all three vertex opacities below exp(-4) go, and with them every fan left
with no face."""
import math

import numpy as np

import oracle
import synthetic


def test_threshold_is_exp_minus_four():
    assert oracle.PRUNE_THRESHOLD == math.exp(-4.0)
    assert abs(oracle.PRUNE_THRESHOLD - 0.018315638888734179) < 1e-17


def test_hand_example():
    K = 3
    t = oracle.PRUNE_THRESHOLD
    alpha = np.array([0.001, 0.002, 0.0, 0.003,        # fan 0: all below -> removed
                      0.01, 0.5, 0.001, 0.001,         # fan 1: centre below, one boundary above -> kept
                      t, 0.0, 0.0, 0.0,                # fan 2: the centre sits exactly on the threshold -> kept
                      0.9, 0.18, 0.18, 0.18])          # fan 3: kept
    V = alpha.size
    xyz = np.arange(3 * V, dtype=np.float64).reshape(V, 3)
    rgb = -xyz
    m = np.arange(7 * V, dtype=np.float64)
    v = m * 10
    px, pc, pa, (pm, pv), fans = oracle.prune_fans(xyz, rgb, alpha, K, moments=(m, v))
    assert list(fans) == [1, 2, 3]
    assert np.array_equal(px, xyz[4:])
    assert np.array_equal(pc, rgb[4:])
    assert np.array_equal(pa, alpha[4:])
    Vk = 12
    assert np.array_equal(pm[:3 * Vk], m[12:3 * V])                  # xyz segment, vertices 4..15
    assert np.array_equal(pm[3 * Vk:6 * Vk], m[3 * V + 12:6 * V])    # rgb segment
    assert np.array_equal(pm[6 * Vk:], m[6 * V + 4:7 * V])           # alpha segment
    assert np.array_equal(pv, np.concatenate([v[12:3 * V], v[3 * V + 12:6 * V], v[6 * V + 4:7 * V]]))


def test_pruning_twice_is_pruning_once():
    rng = np.random.Generator(np.random.PCG64(3))
    K, n = 8, 500
    alpha = rng.uniform(0, 0.03, n * (K + 1))
    xyz = rng.normal(size=(n * (K + 1), 3))
    a1 = oracle.prune_fans(xyz, xyz, alpha, K)
    a2 = oracle.prune_fans(a1[0], a1[1], a1[2], K)
    assert 0 < len(a1[4]) < n
    assert np.array_equal(a2[4], np.arange(len(a1[4])))


def test_render_equals_render_without_the_pruned_faces():
    """The pruned soup renders exactly like the full soup with the pruned fans' faces
    left out of the triangle list; and every face left out has all vertices below the
    threshold."""
    w = synthetic.workload(1, n=400)
    cam = w.cameras[0]
    K = 8
    xyz, rgb, a = oracle.mesh_build(w.scene, K=K, cam_center=cam.C)
    rng = np.random.Generator(np.random.PCG64(5))
    a = a.copy()
    low = rng.random(400) < 0.4
    a.reshape(400, K + 1)[low] *= 0.05     # 40% of the fans drop below the threshold everywhere
    px, pc, pa, _, fans = oracle.prune_fans(xyz, rgb, a, K)
    assert 0 < fans.size < 400
    tris = oracle.fan_tris(400, K).reshape(400, K, 3)[fans].reshape(-1, 3)
    full, _, _ = oracle.render(xyz, rgb, a, tris, cam)
    pruned, _, _ = oracle.render(px, pc, pa, oracle.fan_tris(fans.size, K), cam)
    assert np.array_equal(full, pruned)
    gone = np.setdiff1d(np.arange(400), fans)
    assert np.all(a.reshape(400, K + 1)[gone] < oracle.PRUNE_THRESHOLD)


# ------------------------------------------------------------------ per-face pruning

def test_face_masks_hand_example():
    """K = 4 fans (faces (c,b0,b1), (c,b1,b2), (c,b2,b3), (c,b3,b0)), threshold t:
    a dim centre with one bright boundary vertex b2 keeps exactly the two faces holding b2;
    a bright centre keeps every face; an all-dim fan keeps none; a face whose three
    opacities sit exactly on the threshold stays (below means strictly below)."""
    t = float(np.float32(math.exp(-4.0)))
    lo, hi = 0.001, 0.5
    alpha = np.array([
        [lo, lo, lo, hi, lo],    # b2 bright: faces 1 and 2
        [hi, lo, lo, lo, lo],    # centre bright: all faces
        [lo, lo, lo, lo, lo],    # all dim: none
        [t, t, t, t, t],         # on the threshold: all kept
    ])
    m = oracle.face_masks(alpha.reshape(-1), 4, threshold=t)
    assert list(m) == [0b0110, 0b1111, 0b0000, 0b1111]


def test_prune_faces_removes_faceless_fans_and_keeps_earlier_removals():
    rng = np.random.Generator(np.random.PCG64(4))
    K, n = 8, 500
    xyz = rng.normal(size=(n * (K + 1), 3))
    rgb = rng.random((n * (K + 1), 3))
    a = rng.uniform(0.0, 1.0, (n, K + 1))
    a[rng.random(n) < 0.3] *= 0.01
    a[:, 0][rng.random(n) < 0.5] = 0.001
    a = a.reshape(-1)
    px, pc, pa, _, masks, fans = oracle.prune_faces(xyz, rgb, a, K)
    # without an earlier mask the removed fans are exactly those of the fan rule
    _, _, _, _, fans_f = oracle.prune_fans(xyz, rgb, a, K)
    assert np.array_equal(fans, fans_f)
    assert (masks != 0).all() and masks.max() < (1 << K)
    # an earlier mask stays applied, and pruning again with the result changes nothing
    early = rng.integers(0, 1 << K, n)
    _, _, pa2, _, m2, f2 = oracle.prune_faces(xyz, rgb, a, K, face_mask=early)
    full = oracle.face_masks(a, K)
    assert np.array_equal(m2, (full & early)[f2])
    _, _, _, _, m3, f3 = oracle.prune_faces(px, pc, pa, K, face_mask=masks)
    assert np.array_equal(f3, np.arange(fans.size)) and np.array_equal(m3, masks)


def test_masked_render_equals_render_of_the_kept_triangles():
    """Drawing a pruned soup through its face masks is drawing the kept faces' triangles:
    the explicit triangle list of masked_fan_tris is the reference."""
    w = synthetic.workload(1, n=200)
    cam = w.cameras[0]
    K = 8
    xyz, rgb, a = oracle.mesh_build(w.scene, K=K, cam_center=cam.C)
    rng = np.random.Generator(np.random.PCG64(9))
    a = a.copy().reshape(-1, K + 1)
    a[rng.random(200) < 0.5, 0] = 0.001          # dim centres: rim faces may go
    a[:, 1:][rng.random((200, K)) < 0.5] = 0.001
    a = a.reshape(-1)
    px, pc, pa, _, masks, fans = oracle.prune_faces(xyz, rgb, a, K)
    kept = oracle.masked_fan_tris(fans.size, K, masks)
    full_tris = oracle.fan_tris(200, K).reshape(200, K, 3)
    bits = ((oracle.face_masks(a, K)[:, None] >> np.arange(K)) & 1).astype(bool)
    ref, _, _ = oracle.render(xyz, rgb, a, full_tris[bits], cam)
    img, _, _ = oracle.render(px, pc, pa, kept, cam)
    assert np.allclose(img, ref, atol=0, rtol=0) or np.abs(img - ref).max() < 1e-12
    assert int(bits.sum()) < 200 * K      # some faces did go
