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
from .raster import Rasterizer, RenderParams, Splats, _p, _stream, cam_struct, tiles_of

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


# ---------------------------------------------------------------------------
# truncated render
# ---------------------------------------------------------------------------
LOG_KEEP_ALL = math.log(64.0)  # target of tiles in which some pixel never stops


class LearnedRenderer:
    """Forward render of one camera with learned (or given) per-tile
    termination depths; exact fallback for refuted tiles."""

    def __init__(self, splats: Splats, cam, params: RenderParams | None = None, device="cuda", margin_keys=1.25):
        self.splats = splats
        self.cam = cam
        self.params = params or RenderParams()
        self.params.sh_degree = splats.sh_degree
        self.device = torch.device(device)
        self.status = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.stats = torch.zeros(4, dtype=torch.int64, device=self.device)
        H, W = cam["height"], cam["width"]
        self.image = torch.empty((H, W, 3), dtype=torch.float32, device=self.device)
        self.T = torch.empty((H, W), dtype=torch.float32, device=self.device)
        self.n_last = torch.empty((H, W), dtype=torch.int32, device=self.device)
        self.tiles = tiles_of(cam, self.params)
        self.dstar = torch.empty(self.tiles, dtype=torch.float32, device=self.device)
        self._c = cam_struct(cam)
        self._pc = self.params.c()
        rz = Rasterizer(self.params, device=self.device)
        _, tc = rz.project(splats, [cam], counts=True)
        self.capacity = int(tc.sum(dtype=torch.int64).item() * margin_keys) + 1024
        wsb = N.lib().ls_render_learned_workspace(splats.n, ctypes.byref(self._c), ctypes.byref(self._pc),
                                                  self.capacity)
        self._ws = torch.empty(wsb + 256, dtype=torch.uint8, device=self.device)
        self._ws_ptr = (self._ws.data_ptr() + 255) // 256 * 256
        self._ws_bytes = wsb

    def render(self, mlp: TerminationMLP | None = None, margin=0.0, dstar_in=None, t_thr=None, stats=True):
        """mlp, or per-tile depths dstar_in [tiles]; t_thr None = exact;
        stats=False leaves counters() as they were (and skips counting the
        keys before truncation)."""
        sp = self.splats
        thr = self.params.t_min if t_thr is None else t_thr
        net = ctypes.byref(mlp.c()) if mlp is not None else None
        if mlp is None and dstar_in is None:
            raise ValueError("an MLP or per-tile depths")
        N.check(N.lib().ls_render_learned(sp.n, _p(sp.means), _p(sp.scales), _p(sp.quats), _p(sp.opac), _p(sp.sh),
                                          ctypes.byref(self._c), ctypes.byref(self._pc), net, float(margin),
                                          _p(dstar_in), float(thr), self.capacity, _p(self.image), _p(self.T),
                                          _p(self.n_last), _p(self.dstar), _p(self.stats if stats else None),
                                          ctypes.c_void_p(self._ws_ptr), self._ws_bytes, _p(self.status), _stream()),
                "ls_render_learned")
        return self.image, self.T

    def counters(self):
        """(keys before truncation, kept, held-out sorted, refuted tiles)."""
        return tuple(int(v) for v in self.stats.cpu().tolist())

    def check(self):
        s = int(self.status.item())
        if s != 0:
            raise N.LsError(s, "ls_render_learned")


# ---------------------------------------------------------------------------
# training data and training
# ---------------------------------------------------------------------------
def tile_examples(rz: Rasterizer, splats: Splats, cam):
    """(features [m, 48] fp16, targets [m] fp32) of the non-empty tiles of one
    plain render: the target is the log of the depth at which the tile's last
    pixel stopped, LOG_KEEP_ALL when some pixel never stops.  A rasterizer
    whose t_min is a threshold t_thr gives the targets of the truncated render
    at t_thr: a pixel stops at the first entry that would take T below it."""
    image, T, state = rz.forward(splats, cam)
    nt = tiles_of(cam, rz.params)
    labels = torch.empty(nt, dtype=torch.float32, device=rz.device)
    rz.render_stats(state["proj"], splats.n, cam, state["ranges"], state["vals"], labels=labels)
    x, total = rz.tile_features(state["proj"], splats.n, cam)
    keep = total > 0
    y = torch.where(torch.isinf(labels), torch.full_like(labels, LOG_KEEP_ALL),
                    torch.log(torch.clamp(labels, min=1e-3)))
    return x[keep], y[keep]


def train(mlp: TerminationMLP, x, y, steps=2000, batch=65536, lr=1e-3, under_weight=4.0, seed=0, log_every=0):
    """Adam on shuffled minibatches of (x, y), all on the GPU."""
    g = torch.Generator(device=x.device)
    g.manual_seed(seed)
    m = x.shape[0]
    losses = []
    for s in range(steps):
        idx = torch.randint(0, m, (min(batch, m),), device=x.device, generator=g)
        loss = mlp.train_step(x[idx].contiguous(), y[idx].contiguous(), lr=lr, under_weight=under_weight)
        if log_every and (s % log_every == 0 or s == steps - 1):
            losses.append((s, float(loss.item())))
    return losses
