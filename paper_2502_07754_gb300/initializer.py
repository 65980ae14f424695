"""The learned fan initializer end to end: source-Gaussian targets, fine-tuning of the
converted fans (Sec. 3 "Fine-tuning"), training pairs from the fine-tunes, training of
the tensor-core MLP, and the comparison of MLP-initialized and plain conversions under
the same fine-tune.  Every step runs in libmeshsplats.so; this module only sequences the
calls and holds the buffers."""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch

from . import api
from .api import BatchRenderer, FanAdam, FanMLP, SplatRenderer


@dataclass
class Gaussians:
    """Device tensors of a scene (means, log_scales, quats, opacity, sh)."""
    means: torch.Tensor
    log_scales: torch.Tensor
    quats: torch.Tensor
    opacity: torch.Tensor
    sh: torch.Tensor
    sh_degree: int

    @property
    def n(self):
        return self.means.shape[0]

    @classmethod
    def from_scene(cls, sc, device="cuda"):
        import numpy as np
        d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        sh = d(sc.sh.view(np.int16)) if sc.sh_bf16 else d(sc.sh)
        return cls(d(sc.means), d(sc.log_scales), d(sc.quats), d(sc.opacity), sh, sc.sh_degree)


def psnr(m: float) -> float:
    return -10.0 * math.log10(max(m, 1e-20))


def convert(G: Gaussians, K: int, cam_center, corr=None, mlp=None):
    """The conversion, with corrections given, or predicted by `mlp` inside the same kernel."""
    return api.mesh_build(G.means, G.log_scales, G.quats, G.opacity, G.sh, G.sh_degree, K=K, cam_center=cam_center,
                          corr=corr, mlp=mlp)


def gaussian_colors(G: Gaussians, cam_center):
    """Colour of every Gaussian (what its fan's vertices carry), N x 3."""
    _, rgb, _ = convert(G, 3, cam_center)
    return rgb.view(G.n, 4, 3)[:, 0, :].contiguous()


def source_targets(G: Gaussians, cams, cam_center, params=None):
    """The source Gaussians rendered into every view (flat buffer, BatchRenderer layout)."""
    sr = SplatRenderer(G.n, cams, params)
    return sr.render(G.means, G.log_scales, G.quats, G.opacity, gaussian_colors(G, cam_center))


class FineTuner:
    """L1 fine-tune of a fan soup against target images of several views: batch render,
    L1, batch adjoint, two-learning-rate Adam (Sec. 3 "Optimization and Pruning")."""

    def __init__(self, n_fans, K, cams, lr_color=5e-4, params=None, headroom=1.5):
        self.br = BatchRenderer(n_fans, K, cams, params)
        self.lr_color = lr_color
        self.headroom = headroom

    def run(self, xyz, rgb, a, targets, steps, eval_every=0):
        """Optimises (xyz, rgb, a) in place; returns [(step, PSNR)] at step 0, every
        eval_every steps and after the last step."""
        br = self.br
        flat = br.new_flat()
        br.forward(xyz, rgb, a, flat)
        inf = br.last_info   # leave room for the soup to move during the fine-tune
        br.params.pair_capacity = int(inf.pairs * self.headroom) + 4096
        br.params.frag_capacity = int(inf.frags * self.headroom) + 65536
        br._alloc()
        grads = [torch.zeros_like(xyz), torch.zeros_like(rgb), torch.zeros_like(a)]
        adam = FanAdam(xyz, rgb, a, lr_color=self.lr_color)
        curve = []
        for s in range(steps + 1):
            check = s % 16 == 0 or s == steps
            br.forward(xyz, rgb, a, flat, check_status=check)
            if s == 0 or s == steps or (eval_every and s % eval_every == 0):
                curve.append((s, psnr(api.mse(flat, targets).item())))
            if s == steps:
                break
            _, dL = api.l1_loss(flat, targets)
            for t in grads:
                t.zero_()
            br.backward(xyz, rgb, a, flat, dL, *grads)
            adam.step(xyz, rgb, a, *grads)
        return curve


@dataclass
class PairSet:
    X: torch.Tensor          # N x 16 inputs
    T: torch.Tensor          # N x 2(K+1) corrections
    curves: list = field(default_factory=list)


def make_pairs(G: Gaussians, cams, K, steps, cam_center, lr_color=5e-4, keep_every=1):
    """Training pairs from one fine-tune of the plain conversion against the source
    Gaussians: (inputs of every keep_every-th Gaussian, corrections its fan received)."""
    targets = source_targets(G, cams, cam_center)
    xyz0, rgb0, a0 = convert(G, K, cam_center)
    xyz, rgb, a = xyz0.clone(), rgb0.clone(), a0.clone()
    curve = FineTuner(G.n, K, cams, lr_color).run(xyz, rgb, a, targets, steps)
    T = api.fan_corrections(xyz0, a0, xyz, a, K)
    net = FanMLP(K=K)
    X = net.features(G.log_scales, G.quats, G.opacity, G.sh, G.sh_degree)
    if keep_every > 1:
        X, T = X[::keep_every].contiguous(), T[::keep_every].contiguous()
    return PairSet(X, T, [curve])


def train(net: FanMLP, pairs: PairSet, steps, lr=2e-3):
    """Full-batch Adam on the mean squared error of the corrections; returns the loss
    before the first and after the last step."""
    first = net.train_step(pairs.X, pairs.T, lr=lr).item()
    for _ in range(steps - 1):
        net.train_step(pairs.X, pairs.T, lr=lr)
    net.compute_grads(pairs.X, pairs.T)
    return first, net.loss.item()


def compare(G: Gaussians, cams, K, net: FanMLP, steps, cam_center, eval_every=10, lr_color=5e-4):
    """Plain conversion + fine-tune vs MLP-initialized conversion + the same fine-tune,
    both judged by PSNR against the source-Gaussian render of the same views."""
    targets = source_targets(G, cams, cam_center)
    out = {}
    for name in ("plain", "mlp"):
        xyz, rgb, a = convert(G, K, cam_center, mlp=net if name == "mlp" else None)
        out[name] = FineTuner(G.n, K, cams, lr_color).run(xyz, rgb, a, targets, steps, eval_every)
    final_plain = out["plain"][-1][1]
    reach = next((s for s, p in out["mlp"] if p >= final_plain), None)
    out["steps_to_plain_final"] = reach
    out["steps"] = steps
    return out
