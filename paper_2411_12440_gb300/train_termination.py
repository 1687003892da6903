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
(the same for every tile and view: the method without the network), each
the one that renders those views fastest; the tables keep time, keys sorted
and tiles refuted per candidate.  `--from` recalibrates stored weights
without training; several `--under-weight` values train one network each on
the same examples.
"""
from __future__ import annotations

import argparse
import math
import time

import numpy as np
import torch

from . import raster, scenes
from .learned import LearnedRenderer, TerminationMLP, tile_examples, train


MARGINS = (0.0, 0.1, 0.2, 0.3, 0.4, 0.6, 0.8)
# global depths tried for the no-network baseline: geometric from 1 to 32
CONSTANTS = tuple(float(v) for v in np.geomspace(1.0, 32.0, 31))


def render_cost(views, t_thr, reps=3, **kw):
    """(milliseconds, keys sorted, tiles refuted) summed over the views, with
    an MLP (mlp, margin) or one global depth (const); the time of a view is
    the median of `reps` renders."""
    P = raster.RenderParams(sh_degree=3)
    ms = keys = refuted = 0
    for spx, cam in views:
        lr = LearnedRenderer(spx, cam, P)
        if "const" in kw:
            args = dict(dstar_in=torch.full((lr.tiles,), kw["const"], device=lr.device), t_thr=t_thr)
        else:
            args = dict(mlp=kw["mlp"], margin=kw["margin"], t_thr=t_thr)
        lr.render(**args)
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            lr.render(**args)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        lr.check()
        _, kept, held, nref = lr.counters()
        ms += sorted(times)[reps // 2]
        keys += kept + held
        refuted += nref
    return ms, keys, refuted


def calibrate(net, views, t_thr):
    """Margin of the network and the no-network global depth, each the one
    that renders the views fastest: (margin, table, depth, table), tables of
    (value, ms, keys sorted, tiles refuted)."""
    mt = {m: render_cost(views, t_thr, mlp=net, margin=m) for m in MARGINS}
    ct = {c: render_cost(views, t_thr, const=c) for c in CONSTANTS}
    return (min(mt, key=lambda m: mt[m][0]), [(m,) + v for m, v in mt.items()],
            min(ct, key=lambda c: ct[c][0]), [(c,) + v for c, v in ct.items()])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--renders", type=int, default=20000)
    ap.add_argument("--prims", type=int, default=3_000_000)
    ap.add_argument("--scenes", type=int, default=8)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--t-thr", type=float, default=1e-3)
    ap.add_argument("--under-weight", type=float, nargs="+", default=[1.0],
                    help="weights of the squared error when the prediction is below the target; one network each")
    ap.add_argument("--calib-views", type=int, default=16)
    ap.add_argument("--from", dest="src", default=None, help="recalibrate the weights of this .npz, no training")
    ap.add_argument("--out", required=True, help="output .npz (with several under-weights: a prefix)")
    args = ap.parse_args()
    torch.manual_seed(0)
    t0 = time.time()
    sc = [raster.Splats.from_scene(scenes.cluster_scene(args.prims, 100 + k, 3)) for k in range(args.scenes)]
    views = [(sc[k % args.scenes], scenes.ring_cameras(1, 900_000 + k)[0]) for k in range(args.calib_views)]
    nets = []
    if args.src:
        net = TerminationMLP.load(args.src)
        meta = {k: v for k, v in net.meta.items()
                if k in ("t_thr", "renders", "steps", "examples", "final_loss", "seconds", "under_weight")}
        nets.append((args.out, net, meta, None))
        t_thr = float(meta["t_thr"])
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
        for uw in args.under_weight:
            t1 = time.time()
            net = TerminationMLP(seed=0)
            losses = []
            # cosine-decayed learning rate in 10 legs
            legs = 10
            for k in range(legs):
                lr = args.lr * 0.5 * (1 + math.cos(math.pi * k / legs))
                losses += train(net, x, y, steps=args.steps // legs, batch=args.batch, lr=lr, under_weight=uw,
                                seed=k, log_every=args.steps // legs)
            meta = dict(t_thr=t_thr, renders=args.renders, steps=args.steps, examples=int(x.shape[0]),
                        final_loss=losses[-1][1], under_weight=uw, seconds=np.array([t_data, time.time() - t1]))
            out = args.out if len(args.under_weight) == 1 else "%s_uw%g.npz" % (args.out.replace(".npz", ""), uw)
            nets.append((out, net, meta, losses[0][1]))
    for out, net, meta, first in nets:
        margin, mt, const, ct = calibrate(net, views, t_thr)
        net.save(out, margin=margin, margin_table=np.array(mt), const_dstar=const, const_table=np.array(ct),
                 calib_views=args.calib_views, **meta)
        best = [r for r in mt if r[0] == margin][0]
        cbest = [r for r in ct if r[0] == const][0]
        print("%s: loss %s -> %.4f, margin %.2f (%.2f ms, %d keys, %d refuted), constant %.3f (%.2f ms, %d keys)" %
              (out, "%.4f" % first if first is not None else "-", float(meta["final_loss"]), margin, best[1], best[2],
               best[3], const, cbest[1], cbest[2]), flush=True)


if __name__ == "__main__":
    main()
