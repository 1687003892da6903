"""Trains the per-tile termination MLP on plain renders and calibrates its
margin; writes an .npz (packed parameters, margin, threshold, record).

    python -m paper_2411_12440_gb300.train_termination --renders 20000 \
        --out paper_2411_12440_gb300/data/termination_mlp.npz

Targets come from plain renders at T_min = t_thr (the depth at which each
tile's last pixel would take T below t_thr); scenes are the 3M-primitive
cluster recipe with seeds 100..107, cameras of uneven size on the ring.
Rendering, features, the network's forward/backward and Adam all run in
libls.so on the GPU.
"""
from __future__ import annotations

import argparse
import math
import time

import numpy as np
import torch

from . import raster, scenes
from .learned import LearnedRenderer, TerminationMLP, tile_examples, train


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
    ap.add_argument("--out", required=True)
    args = ap.parse_args()
    torch.manual_seed(0)
    t0 = time.time()
    sc = [raster.Splats.from_scene(scenes.cluster_scene(args.prims, 100 + k, 3)) for k in range(args.scenes)]
    rz_lab = raster.Rasterizer(raster.RenderParams(sh_degree=3, t_min=args.t_thr))
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
    # margin: fewest sorted keys over held-out views of the training scenes
    P = raster.RenderParams(sh_degree=3)
    views = [(sc[k % args.scenes], scenes.ring_cameras(1, 900_000 + k)[0]) for k in range(args.calib_views)]
    best = None
    table = {}
    for m in (0.0, 0.1, 0.2, 0.3, 0.4, 0.6):
        tot = 0
        for spx, cam in views:
            lr = LearnedRenderer(spx, cam, P)
            lr.render(net, margin=m, t_thr=args.t_thr)
            torch.cuda.synchronize()
            lr.check()
            _, kept, held, _ = lr.counters()
            tot += kept + held
        table[m] = tot
        if best is None or tot < table[best]:
            best = m
    net.save(args.out, margin=best, t_thr=args.t_thr, renders=args.renders, steps=args.steps,
             examples=int(x.shape[0]), final_loss=losses[-1][1], margin_table=np.array(list(table.items())),
             seconds=np.array([t_data, t_train]))
    print("examples %d, data %.1fs, train %.1fs, loss %.4f -> %.4f, margin %.2f" %
          (x.shape[0], t_data, t_train, losses[0][1], losses[-1][1], best))


if __name__ == "__main__":
    main()
