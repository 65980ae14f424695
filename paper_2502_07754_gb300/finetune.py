"""The fine-tuning of Sec. 3 ("Fine-tuning", "Loss Function", "Optimization and Pruning")
as a loop over the library's entry points: every step renders all views in one batch,
takes the loss of Eq. 3 (lam L1 + (1 - lam)(1 - SSIM), ms_fine_tune_loss) per view, runs
the adjoint into the render workspace and the two-learning-rate Adam step; every
`prune_every` epochs (an epoch is one step over all views) the faces whose three vertex
opacities are all below exp(-4) are removed (ms_prune_faces) and fans left without faces
are dropped with their Adam moments.  With `three_fan` (a soup of ms_mesh_build_3d), the
gradients of the copies of each shared vertex are summed before the update, so the copies
stay one vertex (no pruning then: removing single fans would split a Gaussian's copies).
Every step is a library kernel; Python only sequences the calls."""
from __future__ import annotations

import math

import torch

from . import api
from .api import BatchRenderer, FanAdam

PRUNE_THRESHOLD = math.exp(-4.0)


class FanFineTune:
    def __init__(self, xyz, rgb, alpha, K, cams, targets, lr_color=5e-3, lam=0.6, prune_every=10,
                 threshold=PRUNE_THRESHOLD, params=None, three_fan=False, n_gaussians=None):
        """xyz, rgb, alpha: the fan soup (optimised in place until a pruning step replaces
        the tensors; read them back from the attributes).  targets: the views' target
        images as one flat (pixels of all views) x 4 tensor in BatchRenderer order."""
        self.K = int(K)
        self.cams = list(cams)
        self.xyz, self.rgb, self.alpha = xyz, rgb, alpha
        self.targets = targets
        self.lam = float(lam)
        self.prune_every = 0 if three_fan else int(prune_every)
        self.threshold = float(threshold)
        self.three_fan = bool(three_fan)
        self.n_gaussians = n_gaussians
        self.params = params if params is not None else api.render_params()
        self.face_mask = None
        self.adam = FanAdam(xyz, rgb, alpha, lr_color=lr_color)
        self.epoch = 0
        self.history = []
        self._build_renderer()

    @property
    def n_fans(self):
        return self.xyz.shape[0] // (self.K + 1)

    def _build_renderer(self):
        if self.face_mask is not None:
            self.params.face_mask = self.face_mask.data_ptr()
        self.br = BatchRenderer(self.n_fans, self.K, self.cams, self.params)
        self.flat = self.br.new_flat()
        self.dL = torch.zeros_like(self.flat)
        need = max(api.lib().ms_fine_tune_loss_workspace_size(c.height, c.width) for c in self.br.cams)
        self.loss_ws = torch.empty(max(need, 1), dtype=torch.uint8, device=self.flat.device)

    def loss(self):
        """Renders all views; returns the mean of the views' losses (device tensor) and
        leaves dL/d(image) of that mean in self.dL."""
        br = self.br
        br.forward(self.xyz, self.rgb, self.alpha, self.flat)
        total = torch.zeros(1, device=self.flat.device)
        nv = len(self.cams)
        for img, tgt, g in zip(br.images(self.flat), br.images(self.targets), br.images(self.dL)):
            l, d = api.fine_tune_loss(img, tgt, lam=self.lam, workspace=self.loss_ws)
            g.copy_(d / nv)
            total += l / nv
        return total

    def step(self):
        """One epoch: loss of all views, adjoint, Adam; pruning when the epoch count reaches a
        multiple of prune_every.  Returns the loss before the update (device tensor)."""
        total = self.loss()
        self.br.backward(self.xyz, self.rgb, self.alpha, self.flat, self.dL, into_workspace=True)
        if self.three_fan:
            api.three_fan_sum_copies(self.n_gaussians, self.K, renderer=self.br)
        self.adam.step_ws(self.xyz, self.rgb, self.alpha, self.br)
        self.epoch += 1
        if self.prune_every and self.epoch % self.prune_every == 0:
            self.prune()
        return total

    def prune(self):
        a = self.adam
        x, c, al, m, v, mask, k = api.prune_faces(self.xyz, self.rgb, self.alpha, self.K, face_mask=self.face_mask,
                                                  threshold=self.threshold, m=a.m, v=a.v)
        self.history.append((self.epoch, self.n_fans, k))
        self.xyz, self.rgb, self.alpha = x.clone(), c.clone(), al.clone()
        a.m, a.v, a.V = m.clone(), v.clone(), self.xyz.shape[0]
        self.face_mask = mask.clone()
        self._build_renderer()

    def run(self, epochs):
        return [float(self.step().item()) for _ in range(epochs)]
