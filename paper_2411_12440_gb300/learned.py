"""Learned per-tile termination (a8): the MLP that proposes, per tile, the
camera depth beyond which no pixel of the tile is still compositing, and the
truncated render that uses the proposal and falls back exactly when it is
refuted.

Every computation runs in libls.so: the tensor-core MLP forward/backward and
Adam (ls_mlp_*), the tile features and labels, and the truncated render.
This module holds parameters and drives training.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import _native as N
from .raster import _p, _stream

NPARAM = 7361
IN, HID, FEATURES = 48, 64, 35
OFF_W1, OFF_B1 = 0, HID * IN
OFF_W2, OFF_B2 = OFF_B1 + HID, OFF_B1 + HID + HID * HID
OFF_W3, OFF_B3 = OFF_B2 + HID, OFF_B2 + 2 * HID


def init_params(seed):
    """He initialisation of the packed parameters (w1t | b1 | w2t | b2 | w3 | b3)."""
    rng = np.random.default_rng(seed)
    p = np.zeros(NPARAM)
    p[OFF_W1:OFF_B1] = rng.normal(0, math.sqrt(2.0 / FEATURES), HID * IN)
    p[OFF_W2:OFF_B2] = rng.normal(0, math.sqrt(2.0 / HID), HID * HID)
    p[OFF_W3:OFF_B3] = rng.normal(0, math.sqrt(1.0 / HID), HID)
    return p


class TerminationMLP:
    """Packed FP32 master parameters plus the FP16 weights the kernels read."""

    def __init__(self, params=None, device="cuda", seed=0):
        self.device = torch.device(device)
        p = init_params(seed) if params is None else np.asarray(params, np.float64)
        self.master = torch.tensor(p, dtype=torch.float32, device=self.device)
        self.w1t = torch.empty(HID * IN, dtype=torch.float16, device=self.device)
        self.w2t = torch.empty(HID * HID, dtype=torch.float16, device=self.device)
        self.w3 = torch.empty(HID, dtype=torch.float16, device=self.device)
        self.b1 = torch.empty(HID, dtype=torch.float32, device=self.device)
        self.b2 = torch.empty(HID, dtype=torch.float32, device=self.device)
        self.b3 = torch.empty(1, dtype=torch.float32, device=self.device)
        self.m1 = torch.zeros(NPARAM, dtype=torch.float32, device=self.device)
        self.m2 = torch.zeros(NPARAM, dtype=torch.float32, device=self.device)
        self.grad = torch.zeros(NPARAM, dtype=torch.float32, device=self.device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.step_count = 0
        self.sync_weights()

    def sync_weights(self):
        """FP16/FP32 working copies from the master parameters."""
        m = self.master
        self.w1t.copy_(m[OFF_W1:OFF_B1])
        self.b1.copy_(m[OFF_B1:OFF_W2])
        self.w2t.copy_(m[OFF_W2:OFF_B2])
        self.b2.copy_(m[OFF_B2:OFF_W3])
        self.w3.copy_(m[OFF_W3:OFF_B3])
        self.b3.copy_(m[OFF_B3:])

    def c(self):
        s = N.LsMlp()
        s.w1t, s.b1, s.w2t, s.b2, s.w3, s.b3 = (t.data_ptr() for t in
                                                (self.w1t, self.b1, self.w2t, self.b2, self.w3, self.b3))
        return s

    def forward(self, x16, out=None):
        m = int(x16.shape[0])
        y = out if out is not None else torch.empty(m, dtype=torch.float32, device=self.device)
        N.check(N.lib().ls_mlp_forward(m, _p(x16), ctypes.byref(self.c()), _p(y), _stream()), "ls_mlp_forward")
        return y

    def grad_of(self, x16, target, under_weight=4.0):
        """Accumulated gradient and loss of the asymmetric squared error."""
        self.grad.zero_()
        self.loss.zero_()
        N.check(N.lib().ls_mlp_backward(int(x16.shape[0]), _p(x16), ctypes.byref(self.c()), _p(target),
                                        float(under_weight), _p(self.grad), _p(self.loss), _stream()),
                "ls_mlp_backward")
        return self.grad, self.loss

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step_count += 1
        N.check(N.lib().ls_mlp_adam(self.step_count, lr, beta1, beta2, eps, _p(self.master), _p(self.grad),
                                    _p(self.m1), _p(self.m2), ctypes.byref(self.c()), _stream()), "ls_mlp_adam")

    def train_step(self, x16, target, lr=1e-3, under_weight=4.0):
        self.grad_of(x16, target, under_weight)
        self.adam(lr)
        return self.loss

    def params(self):
        return self.master.detach().cpu().numpy().astype(np.float64)

    def save(self, path, **meta):
        np.savez(path, params=self.params(), **meta)

    @staticmethod
    def load(path, device="cuda"):
        d = np.load(path)
        mlp = TerminationMLP(d["params"], device=device)
        mlp.meta = {k: d[k] for k in d.files if k != "params"}
        return mlp
