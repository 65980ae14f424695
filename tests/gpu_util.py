"""Helpers shared by the GPU parity tests: move seeded synthetic inputs to the device,
run the CUDA path through the C ABI, and run the oracle on the same bytes."""
import numpy as np
import torch

import oracle
import synthetic
import paper_2502_07754_gb300 as ms


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def scene_tensors(sc):
    sh = dev(sc.sh.view(np.int16)) if sc.sh_bf16 else dev(sc.sh)
    return dev(sc.means), dev(sc.log_scales), dev(sc.quats), dev(sc.opacity), sh


def gpu_mesh(sc, K, cam_center=None, axis_rule=1, corr=None):
    m, s, q, o, sh = scene_tensors(sc)
    return ms.mesh_build(m, s, q, o, sh, sc.sh_degree, K=K, axis_rule=axis_rule, cam_center=cam_center, corr=corr)


def oracle_mesh_f32(sc, K, cam_center=None, axis_rule=1):
    """Fan soup from the oracle, rounded to float32: the common input of both renderers."""
    xyz, rgb, a = oracle.mesh_build(sc, K=K, cam_center=cam_center, axis_rule=axis_rule)
    return xyz.astype(np.float32), rgb.astype(np.float32), a.astype(np.float32)


def gpu_render(xyz, rgb, a, K, cam, **kw):
    n_fans = xyz.shape[0] // (K + 1)
    r = ms.Renderer(n_fans, K, cam, ms.render_params(**kw))
    X, Cc, A = dev(xyz), dev(rgb), dev(a)
    out = r.forward(X, Cc, A)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64), r, (X, Cc, A)


def oracle_render(xyz, rgb, a, K, cam, window=None, bg=(0.0, 0.0, 0.0), decide="fp64"):
    n_fans = xyz.shape[0] // (K + 1)
    return oracle.render(xyz.astype(np.float64), rgb.astype(np.float64), a.astype(np.float64),
                         oracle.fan_tris(n_fans, K), cam, bg=bg, window=window, decide=decide)


def fp64_report(img, xyz, rgb, a, K, cam, window=None, tol=1e-4):
    """GPU image (of the window) against the oracle with FP64 decisions.  The kernels decide
    coverage in binary32 on fan-relative positions; the pixels where those decisions differ
    from FP64 ones are found on the oracle (its "rel32" mode) and reported.  Returns the
    error report over all pixels plus the mismatch count and the largest error outside the
    mismatched pixels."""
    n_fans = xyz.shape[0] // (K + 1)
    ref, mm, _ = oracle.decision_mismatch(xyz.astype(np.float64), rgb.astype(np.float64), a.astype(np.float64),
                                          oracle.fan_tris(n_fans, K), cam, window=window)
    rep = err_report(img, ref, tol)
    d = np.abs(img - ref).max(axis=-1)
    rep["decision_mismatch"] = int(mm.sum())
    rep["max_abs_outside_mismatch"] = float(d[~mm].max()) if (~mm).any() else 0.0
    return rep, ref


def err_report(gpu, orc, tol=1e-4):
    d = np.abs(gpu - orc)
    return {"max_abs": float(d.max()) if d.size else 0.0, "mean_abs": float(d.mean()) if d.size else 0.0,
            "n_over_tol": int((d > tol).sum()), "n": int(d.size)}
