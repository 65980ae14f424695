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


def oracle_render(xyz, rgb, a, K, cam, window=None, bg=(0.0, 0.0, 0.0)):
    n_fans = xyz.shape[0] // (K + 1)
    return oracle.render(xyz.astype(np.float64), rgb.astype(np.float64), a.astype(np.float64),
                         oracle.fan_tris(n_fans, K), cam, bg=bg, window=window)


def err_report(gpu, orc, tol=1e-4):
    d = np.abs(gpu - orc)
    return {"max_abs": float(d.max()) if d.size else 0.0, "mean_abs": float(d.mean()) if d.size else 0.0,
            "n_over_tol": int((d > tol).sum()), "n": int(d.size)}
