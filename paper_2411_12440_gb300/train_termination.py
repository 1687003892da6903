"""Trains the per-tile termination MLP on plain renders and calibrates its
margin; writes an .npz (packed parameters, margin, threshold, record).

    python -m paper_2411_12440_gb300.train_termination --renders 20000 \
        --out paper_2411_12440_gb300/data/termination_mlp.npz

Targets come from plain renders at T_min = t_thr (the depth at which each
tile's last pixel would take T below t_thr); scenes are the 3M-primitive
cluster recipe with seeds 100..107, cameras of uneven size on the ring.
Rendering, features, the network's forward/backward and Adam all run in
libls.so on the GPU.

Calibration, on held-out views of the training scenes, picks the margin
added to the network's log depth and, for comparison, the one global depth
(the same for every tile and view) that sorts the fewest keys: the method
without the network.  `--from` recalibrates stored weights without training.
"""
from __future__ import annotations

import argparse
import math
import time

import numpy as np
import torch

from . import raster, scenes
from .learned import LearnedRenderer, TerminationMLP, tile_examples, train


MARGINS = (0.0, 0.1, 0.2, 0.3, 0.4, 0.6)
# global depths tried for the no-network baseline: geometric from 1 to 32
CONSTANTS = tuple(float(v) for v in np.geomspace(1.0, 32.0, 31))


def sorted_keys(views, t_thr, **kw):
    """Keys sorted (kept + held out) over the views, with an MLP or depths."""
    P = raster.RenderParams(sh_degree=3)
    tot = 0
    for spx, cam in views:
        lr = LearnedRenderer(spx, cam, P)
        if "const" in kw:
            lr.render(dstar_in=torch.full((lr.tiles,), kw["const"], device=lr.device), t_thr=t_thr)
        else:
            lr.render(kw["mlp"], margin=kw["margin"], t_thr=t_thr)
        torch.cuda.synchronize()
        lr.check()
        _, kept, held, _ = lr.counters()
        tot += kept + held
    return tot


def calibrate(net, views, t_thr):
    """(margin, margin table, constant depth, constant table)."""
    mt = {m: sorted_keys(views, t_thr, mlp=net, margin=m) for m in MARGINS}
    ct = {c: sorted_keys(views, t_thr, const=c) for c in CONSTANTS}
    return min(mt, key=mt.get), mt, min(ct, key=ct.get), ct


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--renders", type=int, default=20000)
    ap.add_argument("--prims", type=int, default=3_000_000)
    ap.add_argument("--scenes", type=int, default=8)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--t-thr", type=float, default=1e-3)
    ap.add_argument("--calib-views", type=int, default=16)
    ap.add_argument("--from", dest="src", default=None, help="recalibrate the weights of this .npz, no training")
    ap.add_argument("--out", required=True)
    args = ap.parse_args()
    torch.manual_seed(0)
    t0 = time.time()
    sc = [raster.Splats.from_scene(scenes.cluster_scene(args.prims, 100 + k, 3)) for k in range(args.scenes)]
    if args.src:
        net = TerminationMLP.load(args.src)
        meta = {k: v for k, v in net.meta.items()
                if k in ("t_thr", "renders", "steps", "examples", "final_loss", "seconds")}
        t_thr = float(meta["t_thr"])
        first_loss = None
    else:
        t_thr = args.t_thr
        rz_lab = raster.Rasterizer(raster.RenderParams(sh_degree=3, t_min=t_thr))
        xs, ys = [], []
        for i in range(args.renders):
            cam = scenes.ring_cameras(1, 10_000 + i)[0]
            x, y = tile_examples(rz_lab, sc[i % args.scenes], cam)
            xs.append(x)
            ys.append(y)
        x, y = torch.cat(xs), torch.cat(ys)
        del xs, ys
        t_data = time.time() - t0
        net = TerminationMLP(seed=0)
        losses = []
        # cosine-decayed learning rate in 10 legs
        legs = 10
        for k in range(legs):
            lr = args.lr * 0.5 * (1 + math.cos(math.pi * k / legs))
            losses += train(net, x, y, steps=args.steps // legs, batch=args.batch, lr=lr, under_weight=1.0, seed=k,
                            log_every=args.steps // legs)
        t_train = time.time() - t0 - t_data
        first_loss = losses[0][1]
        meta = dict(t_thr=t_thr, renders=args.renders, steps=args.steps, examples=int(x.shape[0]),
                    final_loss=losses[-1][1], seconds=np.array([t_data, t_train]))
    # margin and global constant: fewest sorted keys over held-out views of the training scenes
    views = [(sc[k % args.scenes], scenes.ring_cameras(1, 900_000 + k)[0]) for k in range(args.calib_views)]
    margin, mt, const, ct = calibrate(net, views, t_thr)
    net.save(args.out, margin=margin, margin_table=np.array(list(mt.items())), const_dstar=const,
             const_table=np.array(list(ct.items())), calib_views=args.calib_views, **meta)
    print("examples %d, loss %s -> %.4f, margin %.2f (%d keys), constant %.3f (%d keys), keep-all %d keys" %
          (int(meta["examples"]), "%.4f" % first_loss if first_loss is not None else "-", float(meta["final_loss"]),
           margin, mt[margin], const, ct[const], sorted_keys(views, t_thr, const=math.inf)))


if __name__ == "__main__":
    main()
