"""Kernel fits of procedural patterns (Sec. 5.1, "Exploring Kernel
Distributions", Fig. 5): stripes, checkerboards and concentric circles at
several frequencies, fitted by primitives rendered with each kernel of the
family (Appendix B, Eq. 21-25, with the alignment factors of its last
paragraph), on the same primitive count and step budget.

Every step runs on the GPU through libls.so: projection, duplicate/sort and
forward blend (ls_project, ls_duplicate_sort, ls_render_fwd), the 6:2:2
training loss and its gradient (ls_image_loss), the backward
(ls_render_bwd) and Adam (ls_adam).  This module only sets up the scene and
loops.

The pattern recipe (the paper shows the patterns but prints no parameters):
a square image of side S, grey levels 0.1 and 0.9; stripes are vertical
bands of `freq` periods across the image; a checkerboard has square cells
with `freq` periods across; circles are rings of `freq` periods from the
centre to the nearest edge.  Primitives start on a jittered n x n grid in
the plane z = 4 in front of an identity camera (60 degree field of view),
isotropic with a standard deviation of half the grid spacing, opacity 0.5,
grey 0.5 (SH degree 0).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import raster, scenes, training

PATTERNS = ("stripes", "checkerboard", "circles")
# Appendix B: the kernel family and its distribution-alignment factors
KERNELS = {"linear": (0, 2.5), "gaussian": (1, 1.0), "laplacian": (2, 1.0), "cosine": (3, 2.5),
           "quadratic": (4, 6.0)}
LO, HI = 0.1, 0.9
Z0 = 4.0


def pattern(kind, freq, size):
    """[size, size, 3] float32 target of the given kind and frequency."""
    c = np.arange(size, dtype=np.float64) + 0.5
    y, x = np.meshgrid(c, c, indexing="ij")
    if kind == "stripes":
        on = np.floor(x * freq / size * 2.0) % 2 == 0
    elif kind == "checkerboard":
        on = (np.floor(x * freq / size * 2.0) + np.floor(y * freq / size * 2.0)) % 2 == 0
    elif kind == "circles":
        r = np.hypot(x - size / 2.0, y - size / 2.0)
        on = np.floor(r * freq / (size / 2.0) * 2.0) % 2 == 0
    else:
        raise ValueError(kind)
    v = np.where(on, HI, LO).astype(np.float32)
    return np.repeat(v[..., None], 3, axis=2)


def init_scene(n_side, size, seed=0):
    """Primitives on a jittered n_side x n_side grid covering the image."""
    cam = scenes.identity_camera(size, size)
    rng = np.random.default_rng(seed)
    sp = size / n_side  # grid spacing in pixels
    g = (np.arange(n_side) + 0.5) * sp
    py, px = np.meshgrid(g, g, indexing="ij")
    px = px.reshape(-1) + rng.uniform(-0.25, 0.25, n_side * n_side) * sp
    py = py.reshape(-1) + rng.uniform(-0.25, 0.25, n_side * n_side) * sp
    n = n_side * n_side
    f = cam["fx"]
    means = np.stack([(px - cam["cx"]) * Z0 / f, (py - cam["cy"]) * Z0 / f, np.full(n, Z0)], 1)
    s = 0.5 * sp * Z0 / f
    scales = np.full((n, 3), s)
    quats = np.zeros((n, 4))
    quats[:, 0] = 1.0
    quats += rng.normal(0, 0.05, (n, 4))
    opac = np.full(n, 0.5)
    sh = np.zeros((n, 1, 3))
    sh[:, 0] = scenes.dc_for_colour(np.full(3, 0.5))
    return scenes.Scene(means.astype(np.float32), scales.astype(np.float32), quats.astype(np.float32),
                        opac.astype(np.float32), sh.astype(np.float32), 0), cam


DEFAULT_LRS = dict(means=2e-3, scales=1e-2, quats=2e-3, opac=5e-2, sh=2e-2)


def fit(kind, freq, kernel="linear", size=256, n_side=48, steps=300, seed=0, lrs=None, device="cuda",
        record_every=25):
    """Fit one pattern with one kernel; returns the loss curve and the final
    PSNR / L1 against the target."""
    kid, lam = KERNELS[kernel]
    scene, cam = init_scene(n_side, size, seed)
    sp = raster.Splats.from_scene(scene, device=device)
    rz = raster.Rasterizer(raster.RenderParams(kernel=kid, lam=lam, sh_degree=0), device=device)
    target = torch.from_numpy(pattern(kind, freq, size)).to(device)
    loss = training.ImageLoss(size, size, device=device)
    opt = training.Adam(sp, lrs or DEFAULT_LRS)
    gimg = torch.empty((size, size, 3), dtype=torch.float32, device=device)
    gout = dict(means=torch.empty_like(sp.means), scales=torch.empty_like(sp.scales),
                quats=torch.empty_like(sp.quats), opac=torch.empty_like(sp.opac), sh=torch.empty_like(sp.sh))
    curve = []
    for step in range(steps):
        image, T, state = rz.forward(sp, cam, sync_capacity=True)
        out = loss(image, target, gimg)
        if step % record_every == 0 or step == steps - 1:
            curve.append((step, float(out[0].item())))
        rz.render_bwd(sp, cam, state, gimg, None, out=gout)
        opt.step(gout)
    image, _, _ = rz.forward(sp, cam, sync_capacity=True)
    out = loss(image, target)
    torch.cuda.synchronize(device)
    rz.check_status("pattern fit")
    l2 = float(out[2].item())
    return {"pattern": kind, "freq": freq, "kernel": kernel, "lambda": lam, "prims": sp.n, "steps": steps,
            "loss_curve": curve, "loss": float(out[0].item()), "l1": float(out[1].item()), "mse": l2,
            "psnr_db": math.inf if l2 == 0 else -10.0 * math.log10(l2), "ssim": float(out[3].item())}


def sweep(patterns=PATTERNS, freqs=(4, 16), kernels=tuple(KERNELS), **kw):
    """Every (pattern, frequency, kernel) on the same budget: {pattern/freq: {kernel: psnr}}."""
    table = {}
    for kind in patterns:
        for fq in freqs:
            row = {}
            for k in kernels:
                row[k] = fit(kind, fq, k, **kw)
            table["%s/%d" % (kind, fq)] = row
    return table
