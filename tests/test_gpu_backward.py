"""GPU adjoint (ms_render_backward) against the oracle's exact reverse pass and FP64
central finite differences; L1 loss and Adam against the oracle."""
import json
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import synthetic  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


from gpu_util import dev, gpu_render, oracle_mesh_f32  # noqa: E402


def _gpu_grads(r, X, Cc, A, out, dL):
    dLt = dev(dL.astype(np.float32))
    gx, gc, ga = r.backward(X, Cc, A, torch.from_numpy(out.astype(np.float32)).cuda(), dLt)
    torch.cuda.synchronize()
    return gx.cpu().numpy().astype(np.float64), gc.cpu().numpy().astype(np.float64), ga.cpu().numpy().astype(np.float64)


def _close(g, o, rel=1e-2, frac=1e-4):
    atol = frac * max(np.abs(o).max(), 1e-30)
    bad = np.abs(g - o) > rel * np.abs(o) + atol
    return int(bad.sum()), float(np.abs(g - o).max() / max(np.abs(o).max(), 1e-30))


def test_backward_matches_oracle_reverse_pass():
    w = synthetic.workload(1)
    cam = w.cameras[0]
    sc = w.scene
    sc.opacity[:] = np.minimum(sc.opacity, 0.99)
    xyz, rgb, a = oracle_mesh_f32(sc, 8, cam.C)
    img, r, (X, Cc, A) = gpu_render(xyz, rgb, a, 8, cam)
    dL = np.random.default_rng(0).normal(size=img.shape)
    gx, gc, ga = _gpu_grads(r, X, Cc, A, img, dL)
    ox, oc, oa = oracle.render_backward(xyz.astype(np.float64), rgb, a, oracle.fan_tris(sc.n, 8), cam, dL)
    for name, g, o in (("xyz", gx, ox), ("rgb", gc, oc), ("alpha", ga, oa)):
        nbad, rel = _close(g, o)
        print(json.dumps({"grad": name, "n_bad": nbad, "max_rel_to_max": rel}))
        assert nbad == 0, (name, nbad, rel)


def test_backward_deep_stack_matches_oracle_reverse_pass():
    """The adjoint where the forward needed extra passes: 60 nearly coplanar fans over the
    same pixels (more pending fragments than the buffer holds), compositing without early
    termination, against the oracle's exact reverse pass entry by entry."""
    rng = np.random.default_rng(3)
    n = 60
    means = np.c_[rng.normal(0, 0.02, (n, 2)), rng.normal(0, 0.002, n)].astype(np.float32)
    q = rng.normal(0, 0.05, (n, 4)) + np.array([math.sqrt(0.5), 0, -math.sqrt(0.5), 0])
    q = (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(np.float32)
    sh = np.zeros((n, 1, 3), np.float32)
    sh[:, 0, :] = rng.normal(0, 1, (n, 3))
    sc = synthetic.Scene(means, np.array([[-9, math.log(0.15), math.log(0.12)]] * n, np.float32), q,
                         rng.uniform(0.05, 0.3, n).astype(np.float32), sh, 0)
    cam = synthetic.make_camera((0.3, 0.2, 2.0), 96, 80)
    xyz, rgb, a = oracle_mesh_f32(sc, 8)
    for kb in (8, 16):
        img, r, (X, Cc, A) = gpu_render(xyz, rgb, a, 8, cam, kbuf=kb, T_eps=1e-30)
        assert r.last_info.extra_passes > 0
        dL = np.random.default_rng(1).normal(size=img.shape)
        gx, gc, ga = _gpu_grads(r, X, Cc, A, img, dL)
        ox, oc, oa = oracle.render_backward(xyz.astype(np.float64), rgb, a, oracle.fan_tris(n, 8), cam, dL)
        for name, g, o in (("xyz", gx, ox), ("rgb", gc, oc), ("alpha", ga, oa)):
            nbad, rel = _close(g, o)
            print(json.dumps({"case": "deep-stack", "kbuf": kb, "grad": name, "n_bad": nbad, "max_rel_to_max": rel}))
            assert nbad == 0, (name, nbad, rel)


def test_backward_clustered_1m_window_matches_oracle_reverse_pass():
    """The adjoint of the 1M-Gaussian 1080p render with the loss gradient confined to a
    96 x 96 window over the blobs (deep, nearly coplanar stacks): every vertex gradient
    against the oracle's reverse pass over that window."""
    w = synthetic.workload(3)
    cam = w.cameras[0]
    sc = w.scene
    xyz, rgb, a = oracle_mesh_f32(sc, 8, cam.C)
    img, r, (X, Cc, A) = gpu_render(xyz, rgb, a, 8, cam, T_eps=1e-30)
    x0, y0, x1, y1 = win = (912, 492, 1008, 588)
    dLw = np.random.default_rng(2).normal(size=(y1 - y0, x1 - x0, 4))
    dL = np.zeros(img.shape)
    dL[y0:y1, x0:x1] = dLw
    gx, gc, ga = _gpu_grads(r, X, Cc, A, img, dL)
    ox, oc, oa = oracle.render_backward(xyz.astype(np.float64), rgb, a, oracle.fan_tris(sc.n, 8), cam, dLw,
                                        window=win)
    touched = (np.abs(ox).sum(1) + np.abs(oc).sum(1) + np.abs(oa)) > 0
    assert touched.sum() > 1000
    for name, g, o in (("xyz", gx, ox), ("rgb", gc, oc), ("alpha", ga, oa)):
        nbad, rel = _close(g, o)
        print(json.dumps({"case": "clustered-1M-window", "grad": name, "n_bad": nbad, "max_rel_to_max": rel,
                          "vertices": int(touched.sum())}))
        assert nbad == 0, (name, nbad, rel)


def test_autograd_function_matches_direct_backward():
    import paper_2502_07754_gb300 as ms
    w = synthetic.workload(1, n=300)
    cam = w.cameras[0]
    xyz, rgb, a = oracle_mesh_f32(w.scene, 8, cam.C)
    r = ms.Renderer(300, 8, cam)
    X = dev(xyz).requires_grad_()
    Cc = dev(rgb).requires_grad_()
    A = dev(a).requires_grad_()
    out = ms.render(X, Cc, A, r)
    wts = torch.randn_like(out)
    (out * wts).sum().backward()
    gx, gc, ga = r.backward(X.detach(), Cc.detach(), A.detach(), out.detach(), wts)
    # float atomics accumulate in a run-dependent order: equal up to rounding
    for u, v in ((X.grad, gx), (Cc.grad, gc), (A.grad, ga)):
        assert torch.allclose(u, v, rtol=1e-4, atol=1e-5 * v.abs().max().item())


def _project_np(cam, P):
    R = np.asarray(cam.R_cw, np.float64)
    Xc = (P - np.asarray(cam.C, np.float64)) @ R.T
    return cam.fx * Xc[:, 0] / Xc[:, 2] + cam.cx, cam.fy * Xc[:, 1] / Xc[:, 2] + cam.cy, Xc[:, 2]


def test_finetune_gradients_vs_fp64_finite_differences():
    """Workload 3 (1M clustered Gaussians, 1080p, L1 against the jittered scene): GPU
    gradients of 64 fans checked against central differences of the FP64 oracle."""
    w = synthetic.workload(3)
    cam = w.cameras[0]
    K = 8
    xyz, rgb, a = oracle_mesh_f32(w.scene, K, cam.C)
    txyz, trgb, ta = oracle_mesh_f32(w.target_scene, K, cam.C)
    img, r, (X, Cc, A) = gpu_render(xyz, rgb, a, K, cam)
    H, W = cam.height, cam.width
    n = w.scene.n
    xs, ys, zs = _project_np(cam, xyz.astype(np.float64))
    xs, ys = xs.reshape(n, K + 1), ys.reshape(n, K + 1)
    bx0, bx1 = np.floor(xs.min(1)).astype(int) - 2, np.ceil(xs.max(1)).astype(int) + 3
    by0, by1 = np.floor(ys.min(1)).astype(int) - 2, np.ceil(ys.max(1)).astype(int) + 3
    area = (np.clip(bx1, 0, W) - np.clip(bx0, 0, W)) * (np.clip(by1, 0, H) - np.clip(by0, 0, H))
    rng = np.random.default_rng(11)
    cand = rng.permutation(np.nonzero((area >= 80) & (bx0 > 0) & (by0 > 0) & (bx1 < W) & (by1 < H))[0])
    tgtP = txyz.astype(np.float64)
    dL = np.zeros((H, W, 4))
    picked = []
    for g in cand:
        if len(picked) == 64:
            break
        win = (bx0[g], by0[g], bx1[g], by1[g])
        # fans that can touch the window (3 px margin around their FP64 projections)
        sel = np.nonzero((bx1 + 3 >= win[0]) & (bx0 - 3 <= win[2]) & (by1 + 3 >= win[1]) & (by0 - 3 <= win[3]))[0]
        if g not in sel:
            continue
        vsel = (sel[:, None] * (K + 1) + np.arange(K + 1)).reshape(-1)
        tris = oracle.fan_tris(sel.size, K)
        P = xyz[vsel].astype(np.float64)
        own = np.nonzero(sel == g)[0][0]
        # covered pixels of this fan alone
        _, nf1, _ = oracle.render(P[own * 9:own * 9 + 9], rgb[vsel][own * 9:own * 9 + 9].astype(np.float64),
                                  a[vsel][own * 9:own * 9 + 9].astype(np.float64), oracle.fan_tris(1, K), cam,
                                  window=win)
        if nf1.sum() < 50:
            continue
        # the jittered target moves fans by ~0.3 px: the same selection covers the window
        tgt, _, _ = oracle.render(tgtP[vsel], trgb[vsel].astype(np.float64), ta[vsel].astype(np.float64),
                                  tris, cam, window=win)
        picked.append((g, win, sel, vsel, tris, own, tgt))
    assert len(picked) == 64
    # dL of the full-image L1 loss, from the oracle's images, inside every picked window
    scale = 1.0 / (3 * H * W)
    for g, win, sel, vsel, tris, own, tgt in picked:
        C_o, _, _ = oracle.render(xyz[vsel].astype(np.float64), rgb[vsel].astype(np.float64),
                                  a[vsel].astype(np.float64), tris, cam, window=win)
        dL[win[1]:win[3], win[0]:win[2], :3] = np.sign(C_o[..., :3] - tgt[..., :3]) * scale
    gx, gc, ga = _gpu_grads(r, X, Cc, A, img, dL)
    worst = 0.0
    skipped = 0
    for g, win, sel, vsel, tris, own, tgt in picked:
        P0 = xyz[vsel].astype(np.float64)
        C0 = rgb[vsel].astype(np.float64)
        A0 = a[vsel].astype(np.float64)
        # other picked fans' windows may overlap this one; the loss is restricted to this window
        dLw = dL[win[1]:win[3], win[0]:win[2]]

        def loss(P, Cv, Av):
            o, _, _, sig = oracle.render(P, Cv, Av, tris, cam, window=win, nthreads=1, signature=True)
            return float((np.abs(o[..., :3] - tgt[..., :3]) * (dLw[..., :3] != 0)).sum() * scale), sig

        _, sig0 = loss(P0, C0, A0)

        def fd_position(li, c):
            # central difference with visibility held fixed, as the adjoint defines it: a
            # step that changes any pixel's fragments or their order (FP64 decisions flip
            # on sub-ulp moves between nearly coplanar surfels) is redrawn 16x smaller; a
            # component that still flips sits on a visibility boundary and is left out
            h = float(np.spacing(np.float32(P0[li, c]))) / 8
            for _ in range(4):
                Pp, Pm = P0.copy(), P0.copy()
                Pp[li, c] += h
                Pm[li, c] -= h
                (lp, sp), (lm, sm) = loss(Pp, C0, A0), loss(Pm, C0, A0)
                if np.array_equal(sp, sig0) and np.array_equal(sm, sig0):
                    return (lp - lm) / (2 * h)
                h /= 16
            return None

        fd, gg = [], []
        for k in range(K + 1):
            li, vi = own * (K + 1) + k, g * (K + 1) + k
            for c in range(3):
                d = fd_position(li, c)
                if d is None:
                    skipped += 1
                    continue
                fd.append(d)
                gg.append(gx[vi, c])
            for c in range(3):
                h = 1e-6
                Cp, Cm = C0.copy(), C0.copy()
                Cp[li, c] += h
                Cm[li, c] -= h
                fd.append((loss(P0, Cp, A0)[0] - loss(P0, Cm, A0)[0]) / (2 * h))
                gg.append(gc[vi, c])
            h = 1e-6
            Ap, Am = A0.copy(), A0.copy()
            Ap[li] += h
            Am[li] -= h
            fd.append((loss(P0, C0, Ap)[0] - loss(P0, C0, Am)[0]) / (2 * h))
            gg.append(ga[vi])
        fd, gg = np.array(fd), np.array(gg)
        rel = np.linalg.norm(gg - fd) / max(np.linalg.norm(fd), 1e-30)
        worst = max(worst, rel)
        assert rel <= 1e-2, (g, rel)
    print(json.dumps({"fd_fans": 64, "worst_rel_err": worst, "position_components_on_a_visibility_boundary": skipped}))
    assert skipped <= 64 * 27 // 20, skipped   # nearly all components are differentiable


def test_l1_loss_and_adam_match_oracle():
    import paper_2502_07754_gb300 as ms
    rng = np.random.default_rng(2)
    a_img = rng.uniform(0, 1, (37, 53, 4)).astype(np.float32)
    b_img = rng.uniform(0, 1, (37, 53, 4)).astype(np.float32)
    loss, dL = ms.l1_loss(dev(a_img), dev(b_img))
    lo, go = oracle.l1_loss_grad(a_img[..., :3].astype(np.float64), b_img[..., :3].astype(np.float64))
    assert abs(loss.item() - lo) < 1e-6
    assert np.abs(dL.cpu().numpy()[..., :3] - go).max() < 1e-9 and (dL.cpu().numpy()[..., 3] == 0).all()
    V = 1000
    P = [rng.normal(size=(V, 3)), rng.uniform(0, 1, (V, 3)), rng.uniform(0, 1, V)]
    Pg = [dev(p.astype(np.float32)) for p in P]
    P = [p.astype(np.float32).astype(np.float64) for p in P]
    opt = ms.FanAdam(*Pg, lr_color=5e-3)
    mo, vo = np.zeros(7 * V), np.zeros(7 * V)
    for step in range(1, 4):
        G = [rng.normal(size=p.shape) * 1e-2 for p in P]
        Gg = [dev(gr.astype(np.float32)) for gr in G]
        opt.step(*Pg, *Gg)
        oracle.fan_adam_step(*P, *[gr.astype(np.float32).astype(np.float64) for gr in G], mo, vo, step, 5e-3)
    assert np.abs(opt.m.cpu().numpy() - mo).max() < 1e-6
    for pg, po in zip(Pg, P):
        assert np.abs(pg.cpu().numpy() - po).max() < 1e-5


def test_gradients_left_in_workspace_drive_adam_like_explicit_arrays():
    """ms_render_backward with NULL gradient arrays leaves the same gradients in the
    workspace as in explicit arrays (up to the summation order of the float atomics), and
    ms_adam_step_ws on them equals ms_adam_step on the same gradients as arrays.  (Adam's
    first step moves a parameter by lr * sign(g), so the two paths are compared on
    identical gradients: a sum that cancels to ~0 may take either sign in another run.)"""
    import paper_2502_07754_gb300 as ms
    w = synthetic.workload(3, n=30000)
    sc = w.scene
    cam = synthetic.make_camera(np.array([0.3, 0.4, 3.2]), 320, 240)
    xyz0, rgb0, a0 = (dev(t) for t in oracle_mesh_f32(sc, w.K, cam_center=cam.C))
    r = ms.Renderer(sc.n, w.K, cam)
    out = r.forward(xyz0, rgb0, a0)
    g = torch.Generator(device="cuda").manual_seed(3)
    target = torch.rand(out.shape, device="cuda", generator=g)
    _, dL = ms.l1_loss(out, target)
    V = xyz0.shape[0]
    grads = r.backward(xyz0, rgb0, a0, out, dL)
    assert r.backward(xyz0, rgb0, a0, out, dL, into_workspace=True) is None
    torch.cuda.synchronize()
    off = r.grad_ptr().value - r.ws.data_ptr()
    ws_g = r.ws[off:off + 32 * V].view(torch.float32).view(V, 8).clone()
    as_arrays = (ws_g[:, 0:3].contiguous(), ws_g[:, 4:7].contiguous(), ws_g[:, 3].contiguous())
    for a, b in zip(grads, as_arrays):
        scale = a.abs().max().item()
        assert scale > 0
        assert torch.allclose(a, b, rtol=1e-4, atol=1e-5 * scale), (a - b).abs().max().item() / scale
    params = []
    for fused in (False, True):
        x, c, al = xyz0.clone(), rgb0.clone(), a0.clone()
        opt = ms.FanAdam(x, c, al, lr_color=1e-3)
        if fused:
            opt.step_ws(x, c, al, r)
        else:
            opt.step(x, c, al, *as_arrays)
        torch.cuda.synchronize()
        params.append((x, c, al))
    for p_ref, p_ws in zip(*params):
        assert torch.allclose(p_ref, p_ws, rtol=3e-7, atol=1e-9), (p_ref - p_ws).abs().max().item()   # <= 2 ulp
    moved = (params[1][0] != xyz0).float().mean().item()
    assert moved > 0.01   # the step did something


def test_backward_after_fragment_overflow_stays_in_bounds():
    """A forward whose fragment buffer is too small reports MS_ERR_CAPACITY; the backward
    on that workspace (whose record ranges beyond the capacity and adjoint slots hold
    whatever the memory held before) must still finish without a CUDA error."""
    import ctypes as C
    import paper_2502_07754_gb300 as ms
    from paper_2502_07754_gb300 import _lib
    L = _lib.lib()
    w = synthetic.workload(1)
    cam = w.cameras[0]
    xyz, rgb, a = oracle_mesh_f32(w.scene, 8, cam.C)
    X, Cc, A = dev(xyz), dev(rgb), dev(a)
    full = ms.Renderer(w.scene.n, 8, cam)
    full.forward(X, Cc, A)
    frags = full.last_info.frags
    cs = ms.camera_struct(cam)
    p = ms.render_params()
    p.frag_capacity = max(1, frags // 2)
    nbytes = L.ms_render_workspace_size(w.scene.n, 8, C.byref(cs), C.byref(p))
    g = torch.Generator(device="cuda").manual_seed(9)
    ws = torch.randint(0, 256, (nbytes + 256,), dtype=torch.uint8, device="cuda", generator=g)
    base = (256 - ws.data_ptr() % 256) % 256
    wsp = C.c_void_p(ws.data_ptr() + base)
    out = torch.zeros(cam.height, cam.width, 4, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda t: C.c_void_p(t.data_ptr())
    assert L.ms_render(ptr(X), ptr(Cc), ptr(A), w.scene.n, 8, C.byref(cs), C.byref(p), ptr(out), wsp, nbytes,
                       stream) == _lib.MS_OK
    info = _lib.RenderInfo()
    assert L.ms_render_get_info(wsp, C.byref(info), stream) == _lib.MS_ERR_CAPACITY
    assert info.overflow == 1 and info.frags > info.frag_capacity
    dL = torch.randn(out.shape, device="cuda", generator=g)
    grads = [torch.zeros_like(X), torch.zeros_like(Cc), torch.zeros_like(A)]
    assert L.ms_render_backward(ptr(X), ptr(Cc), ptr(A), w.scene.n, 8, C.byref(cs), C.byref(p), ptr(out), ptr(dL),
                                *[ptr(t) for t in grads], wsp, nbytes, stream) == _lib.MS_OK
    torch.cuda.synchronize()   # raises if a kernel faulted
    # the renderer's own workspace still renders and differentiates normally afterwards
    gx, gc, ga = full.backward(X, Cc, A, full.forward(X, Cc, A), dL)
    torch.cuda.synchronize()
    assert torch.isfinite(gx).all() and torch.isfinite(gc).all() and torch.isfinite(ga).all()
