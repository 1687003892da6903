"""Training-side consumers of the rasterizer's backward, on the GPU:

    image_loss -> ls_image_loss  (L = 0.6 L1 + 0.2 L2 + 0.2 (1 - SSIM), the
                                  appendix "Loss Functions", and dL/dimage)
    Adam       -> ls_adam        (per-tensor moments; scales in log space,
                                  opacities in logit space)

Argument marshalling only; the arithmetic runs in libls.so.
"""
from __future__ import annotations

import ctypes

import torch

from . import _native as N
from .raster import Splats, _p, _stream

WEIGHTS = (0.6, 0.2, 0.2)


class ImageLoss:
    """Reusable workspace for one image size."""

    def __init__(self, height, width, weights=WEIGHTS, device="cuda"):
        self.H, self.W = int(height), int(width)
        self.weights = tuple(float(w) for w in weights)
        self.device = torch.device(device)
        self.ws_bytes = N.lib().ls_image_loss_workspace(self.H, self.W)
        if self.ws_bytes == 0:
            raise ValueError("image size out of range")
        self._ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
        self.out = torch.zeros(4, dtype=torch.float32, device=self.device)  # total, L1, L2, SSIM

    def __call__(self, pred, target, grad=None):
        """Enqueues the loss (self.out) and, when `grad` is given
        ([H, W, 3] float32), writes dL/dpred into it."""
        for t in (pred, target) + ((grad,) if grad is not None else ()):
            if not (t.is_cuda and t.is_contiguous() and t.dtype == torch.float32 and tuple(t.shape) == (self.H, self.W, 3)):
                raise ValueError("expected contiguous float32 CUDA tensors of shape [H, W, 3]")
        ws = ctypes.c_void_p((self._ws.data_ptr() + 255) // 256 * 256)
        w1, w2, w3 = self.weights
        N.check(N.lib().ls_image_loss(self.H, self.W, _p(pred), _p(target), w1, w2, w3, _p(self.out), _p(grad), ws,
                                      self.ws_bytes, _stream()), "ls_image_loss")
        return self.out


def adam_(param, grad, m1, m2, step, lr, beta1=0.9, beta2=0.999, eps=1e-15, mode=0):
    """One Adam step of `param` in place (ls_adam); mode 0 identity, 1 log, 2 logit."""
    N.check(N.lib().ls_adam(param.numel(), _p(param), _p(grad), _p(m1), _p(m2), int(step), float(lr), float(beta1),
                            float(beta2), float(eps), int(mode), _stream()), "ls_adam")


class Adam:
    """Adam over the five parameter tensors of a Splats, each with its own
    rate and space: means and quaternions as they are, scales in log space,
    opacities in logit space, SH coefficients as they are."""

    MODES = dict(means=0, scales=1, quats=0, opac=2, sh=0)

    def __init__(self, splats: Splats, lrs, betas=(0.9, 0.999), eps=1e-15):
        self.sp = splats
        self.lrs = dict(lrs)
        self.betas = betas
        self.eps = eps
        self.step_count = 0
        self.m1 = {k: torch.zeros_like(getattr(splats, k)) for k in self.MODES}
        self.m2 = {k: torch.zeros_like(getattr(splats, k)) for k in self.MODES}

    def step(self, grads):
        self.step_count += 1
        for k, mode in self.MODES.items():
            lr = self.lrs.get(k, 0.0)
            if lr == 0.0:
                continue
            adam_(getattr(self.sp, k), grads[k], self.m1[k], self.m2[k], self.step_count, lr, self.betas[0],
                  self.betas[1], self.eps, mode)


# The densification thresholds of the appendix table (3DLS row) and the 3DGS
# row beside it.
DENSIFY_3DLS = dict(grad2d=0.0002, grow_scale2d=0.05, grow_scale3d=0.006, prune_scale2d=0.15, prune_scale3d=0.4,
                    prune_opacity=0.025)
DENSIFY_3DGS = dict(grad2d=0.0002, grow_scale2d=0.05, grow_scale3d=0.01, prune_scale2d=0.15, prune_scale3d=0.1,
                    prune_opacity=0.005)


class DensifyStats:
    """Per-primitive densification statistics (ls_densify_accumulate) and
    the refinement decision (ls_densify_decide): flags bit 0 duplicate,
    bit 1 split, bit 2 prune."""

    def __init__(self, n, device="cuda"):
        self.n = int(n)
        self.device = torch.device(device)
        self.grad_accum = torch.zeros(self.n, dtype=torch.float32, device=self.device)
        self.count = torch.zeros(self.n, dtype=torch.int32, device=self.device)
        self.max_radius = torch.zeros(self.n, dtype=torch.float32, device=self.device)
        self.flags = torch.zeros(self.n, dtype=torch.uint8, device=self.device)
        self.counts = torch.zeros(3, dtype=torch.int64, device=self.device)

    def reset(self):
        self.grad_accum.zero_()
        self.count.zero_()
        self.max_radius.zero_()

    def accumulate(self, g2d, proj, cam, n_cams=1):
        from .raster import cam_struct
        N.check(N.lib().ls_densify_accumulate(self.n, _p(g2d), _p(proj), ctypes.byref(cam_struct(cam)), int(n_cams),
                                              _p(self.grad_accum), _p(self.count), _p(self.max_radius), _stream()),
                "ls_densify_accumulate")

    def decide(self, splats: Splats, extent, thresholds=DENSIFY_3DLS, use_scale2d=False, use_prune_scale3d=False):
        p = N.LsDensifyParams()
        for k, v in thresholds.items():
            setattr(p, k, float(v))
        p.use_scale2d = int(use_scale2d)
        p.use_prune_scale3d = int(use_prune_scale3d)
        N.check(N.lib().ls_densify_decide(self.n, _p(self.grad_accum), _p(self.count), _p(self.max_radius),
                                          _p(splats.scales), _p(splats.opac), float(extent), ctypes.byref(p),
                                          _p(self.flags), _p(self.counts), _stream()), "ls_densify_decide")
        return self.flags, self.counts
