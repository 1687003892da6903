#!/usr/bin/env python
"""Benchmark of the linear-splatting rasterizer hot path on GB300.

One step = the whole differentiable frame: projection (a1), duplication and
radix sort (a2, a3), forward blending (a4), blending adjoint (a5) and
projection adjoint (a6) of a 3M-primitive SH-degree-3 scene at 1920x1080,
inputs resident in HBM.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank renders its own replica of the frame (replicas:
the frame has no exchange step), timing is the max over ranks and `value`
is the total frames/s of all ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "diff_3m_1080p"
METRIC = "1080p fwd+bwd iters/s at 3M prims (fwd frames/s alongside)"
SM_MAX_MHZ = 2070.0
LANES_PER_SM = 128

# DRAM traffic per launch of the dominant kernel from one ncu capture of the
# bench workload (dram__bytes_read.sum + dram__bytes_write.sum), valid only
# while the kernel source is the one measured (sha1 prefix of the file).
NCU_TRAFFIC = {"blend_bwd": {"bytes": 71568128 + 1768704, "src": "d8f0e74f6ecb"}}


def _src_hash(name):
    p = os.path.join(ROOT, "paper_2411_12440_gb300", "csrc", name)
    return hashlib.sha1(open(p, "rb").read()).hexdigest()[:12]


def measure_fp32_issue(dev, iters=200_000):
    """Dependent-free FP32 FMA lane instructions per second (T), from the
    library's probe timed with CUDA events after one warm-up launch."""
    import ctypes
    import torch
    from paper_2411_12440_gb300 import _native as N
    out = torch.zeros(1, dtype=torch.float32, device=dev)
    ops = ctypes.c_int64(0)
    st = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    L = N.lib()
    N.check(L.ls_fp32_issue_probe(iters // 10, 8, ctypes.c_void_p(out.data_ptr()), ctypes.byref(ops), st), "probe")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    N.check(L.ls_fp32_issue_probe(iters, 8, ctypes.c_void_p(out.data_ptr()), ctypes.byref(ops), st), "probe")
    e1.record()
    torch.cuda.synchronize(dev)
    return ops.value / (e0.elapsed_time(e1) * 1e-3) / 1e12


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region:
    one nvidia-smi process streaming a row every 50 ms, started (and its
    first row awaited) before the region and ended after it."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, period_ms=50):
        self.index = index
        self.period_ms = period_ms
        self.rows = []
        self._p = None
        self._t = None
        self._first = threading.Event()

    def _read(self):
        for line in self._p.stdout:
            row = [x.strip() for x in line.split(",")]
            if len(row) >= 9:
                self.rows.append(row)
                self._first.set()

    def __enter__(self):
        try:
            self._p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                        "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                                       stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self._p = None
            return self
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()
        self._first.wait(timeout=5.0)  # the first row: the clocks as the region starts
        return self

    def __exit__(self, *a):
        if self._p is None:
            return
        self._p.terminate()  # our own child, by its handle
        try:
            self._p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self._p.kill()
            self._p.wait(timeout=5)
        self._t.join(timeout=5)

    def summary(self):
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) >= 9:
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def frame_config(prims, cam, tile, ws, prims_override):
    """The `config` of the measured frame, the same for both arms."""
    wl = WORKLOAD if prims_override is None else "%s (prims=%d)" % (WORKLOAD, prims)
    return {"workload": wl, "prims": prims, "width": cam["width"], "height": cam["height"], "sh_degree": 3,
            "tile": "%dx%d" % (tile, tile), "l2": "inputs larger than L2 (708 MB of parameters)",
            "parallelism": "replicas" if ws > 1 else "single"}


class Peaks:
    """Roofline denominators: the measured HBM copy rate (MEASURED_PEAKS.json)
    and the FP32 lane rate SMs x 128 lanes x the maximum SM clock, the SM
    count read from the device; the library's dependent-free FMA probe
    measures the latter beside it."""

    def __init__(self, dev):
        import torch
        self.hbm, self.hbm_src = _peaks()
        self.sms = torch.cuda.get_device_properties(dev).multi_processor_count
        self.alu = self.sms * LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12  # Tops/s, FP32 lane instructions
        self.alu_src = "%d SMs x %d FP32 lanes x %.0f MHz" % (self.sms, LANES_PER_SM, SM_MAX_MHZ)
        self.fma_probe = measure_fp32_issue(dev)

    def entry(self, bound, amount, ms):
        """Roofline object of `amount` bytes (hbm) or FP32 lane operations
        (alu) done in `ms` milliseconds."""
        sec = ms * 1e-3
        if bound == "hbm":
            a = amount / sec / 1e9
            return {"bound": "hbm", "achieved": a, "peak": self.hbm, "unit": "GB/s", "frac": a / self.hbm,
                    "peak_source": self.hbm_src}
        a = amount / sec / 1e12
        return {"bound": "alu", "achieved": a, "peak": self.alu, "unit": "Tops/s", "frac": a / self.alu,
                "peak_source": self.alu_src}

    def lower_bound_ms(self, units):
        """Time of a set of stages if each ran at its roofline."""
        return sum(amount / (self.hbm * 1e9 if b == "hbm" else self.alu * 1e12) * 1e3 for b, amount in units)


def frame_units(R, n_vis, K, n_eval, n_contrib, tiles, kp, sh_bytes=192, pixels=0):
    """Algorithmic work of each kernel of one frame: bytes for the
    HBM-bound stages, FP32 lane operations for the blends.  R records, n_vis
    visible, K tile keys, n_eval evaluated and n_contrib composited pairs."""
    par = 32 + sh_bytes  # scales, quaternion, opacity + SH of a visible primitive
    return {
        # mu for every record, parameters + SH of the visible ones, the 68 B record written (Sec. 3.1 Eq. 1-4)
        "project": ("hbm", 12 * R + (par + 68) * n_vis),
        # depth sort (histogram + 4 passes of 16 B), box per record (order, depth key, footprint, box), key
        # count with stash (box, order, record geometry, 8 B per key written), copy to offsets (8 B read and
        # written per key), tile sort (kp passes of 16 B per key), ranges
        "duplicate_sort": ("hbm", 4 * R + 4 * 16 * R + (16 * R + 16 * n_vis) + (12 * R + 32 * n_vis + 8 * K)
                           + 16 * K + kp * 16 * K + 8 * tiles),
        # FP32 lane operations: 7 per evaluated pair, 11 more per composited pair
        "blend_fwd": ("alu", 7 * n_eval + 11 * n_contrib),
        # recompute 7 per evaluated pair + 40 per contributing pair
        "blend_bwd": ("alu", 7 * n_eval + 40 * n_contrib),
        # parameters + SH and g2d read, gradients of the same size written
        "project_bwd": ("hbm", (2 * (12 + par) + 48 + 4) * R),
        # 48 B per record cleared
        "g2d_clear": ("hbm", 48 * R),
        # n_last read per pixel; a tile's bucket written and read, its order entry written
        "tile_order": ("hbm", 4 * pixels + 12 * tiles),
    }


def dist_setup(args, backend="nccl"):
    """Rank layout from the torchrun environment; one process group over all
    ranks when there is more than one (nccl on the GPUs; gloo in CPU tests)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws, device="cuda"):
    """The largest of every rank's x (the job's time is its slowest rank's)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(ws, ms_per_step):
    """Whole-job steps per second: every rank runs its own replica of the
    frame (weak scaling), so N ranks finish N frames per slowest step."""
    return ws * 1e3 / ms_per_step


# --------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline leg and the reference arm)
# --------------------------------------------------------------------------
def oracle_frame_estimate(scene, cam, P, ncores, frac=0.1, seed=0):
    """Seconds the FP64 oracle needs for one fwd+bwd frame, from a bounded
    sample: the full projection and the full tile lists, then the blend
    forward and backward on a seeded random `frac` of the tiles and the
    projection adjoint on the same fraction of the visible primitives, each
    scaled to the whole frame.  Returns (estimate, what was sampled, seconds
    actually spent)."""
    import numpy as np
    import oracle
    oracle.set_threads(ncores)
    W, H = cam["width"], cam["height"]
    tw, th = P.get("tile_w", 16), P.get("tile_h", 16)
    tiles = ((W + tw - 1) // tw) * ((H + th - 1) // th)
    rng = np.random.default_rng(seed)
    mask = np.zeros(tiles, np.uint8)
    mask[rng.choice(tiles, size=max(1, int(round(frac * tiles))), replace=False)] = 1
    f_tiles = mask.sum() / tiles
    t0 = time.perf_counter()
    proj, vis = oracle.project(scene, cam, P)
    t_proj = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.render(proj, vis, W, H, P, tile_mask=np.zeros(tiles, np.uint8))  # the tile lists alone
    t_lists = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.render(proj, vis, W, H, P, tile_mask=mask)
    t_fwd = time.perf_counter() - t0
    gC = rng.standard_normal((H, W, 3))
    gT = rng.standard_normal((H, W))
    t0 = time.perf_counter()
    oracle.render_bwd(proj, vis, W, H, gC, gT, P, tile_mask=mask)
    t_bwd = time.perf_counter() - t0
    vis_idx = np.nonzero(vis)[0]
    pick = np.sort(rng.choice(vis_idx, size=max(1, int(round(frac * len(vis_idx)))), replace=False))
    sub = scene.subset(pick)
    g2s = rng.standard_normal((len(pick), 9))
    t0 = time.perf_counter()
    oracle.project_bwd(sub, cam, g2s, P)
    t_pbwd = time.perf_counter() - t0
    f_prims = len(pick) / len(vis_idx)
    est = (t_proj + t_lists + max(t_fwd - t_lists, 0.0) / f_tiles + t_lists + max(t_bwd - t_lists, 0.0) / f_tiles
           + t_pbwd / f_prims)
    sample = ("full projection and tile lists; blending fwd+bwd on a seeded random %.3f of the tiles (%d of %d) and "
              "the projection adjoint on %d of %d visible primitives, each scaled to the frame" %
              (f_tiles, int(mask.sum()), tiles, len(pick), len(vis_idx)))
    spent = t_proj + 2 * t_lists + t_fwd + t_bwd + t_pbwd
    return est, sample, spent


def run_reference(args):
    """Reference arm: the FP64 oracle as it stands on the host cores.  Each
    step is one bounded sample of the frame (oracle_frame_estimate); the line
    reports the seconds a step really took as ms_per_step and the frame rate
    the sample extrapolates to as value."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_2411_12440_gb300 import scenes
    oracle.build()
    ncores = os.cpu_count() or 1
    scene, cams, extra = scenes.make_workload(WORKLOAD)
    P = dict(sh_degree=3, antialias=int(extra["antialias"]))
    # each step is one bounded sample (~9 s of host work on 16 cores); the
    # steps and warm-up steps asked for are run as given unless that would
    # take more than ~6 minutes
    steps, warmup = max(1, args.steps), max(0, args.warmup)
    if steps + warmup > 40:
        warmup = min(warmup, 2)
        steps = max(1, min(steps, 40 - warmup))
    ests, spent = [], []
    sample = ""
    for i in range(warmup + steps):
        t0 = time.perf_counter()
        est, sample, _ = oracle_frame_estimate(scene, cams[0], P, ncores)
        if i >= warmup:
            ests.append(est)
            spent.append(time.perf_counter() - t0)
    sec = statistics.median(ests)
    value = 1.0 / sec
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": ws,
            "steps": steps, "warmup": warmup, "ms_per_step": 1e3 * statistics.mean(spent),
            "frame_seconds_estimate": sec, "frame_seconds_estimates": [round(e, 3) for e in ests],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": frame_config(scene.n, cams[0], 16, ws, None),
            "cpu_baseline": {"value": value, "unit": "iters/s", "cores": ncores, "kind": "oracle",
                             "sample": sample, "estimate": "value extrapolates the sample to the whole frame; "
                                                           "ms_per_step is the time one sample took"},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# batched form: 64 cameras of uneven resolution, one graph-captured launch
# --------------------------------------------------------------------------
def bench_batched(dev, reps=10):
    import dataclasses
    import torch
    from paper_2411_12440_gb300 import raster, scenes
    from paper_2411_12440_gb300.batch import Autotuner, BatchRenderer
    scene, cams, extra = scenes.make_workload("batch_3m_64cams")
    sp = raster.Splats.from_scene(scene, device=dev)
    P = raster.RenderParams(sh_degree=3)
    tune = Autotuner(reps=2).tune(sp, cams, P, device=dev)
    Pt = dataclasses.replace(P, tile_w=tune.tile[0], tile_h=tune.tile[1])
    br = BatchRenderer(sp, cams, Pt, blend_batch=tune.blend_batch, device=dev)
    br.plan()
    br.capture()
    for _ in range(2):
        br.render()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        br.render()
    e1.record()
    torch.cuda.synchronize(dev)
    br.check()
    ms_batch = e0.elapsed_time(e1) / reps
    K = int(br.n_keys.item())
    # the blending stage alone, on what the last call left in the workspace
    imgs = br.images.clone()
    br.blend_only()
    torch.cuda.synchronize(dev)
    br.check()
    assert torch.equal(br.images, imgs), "blend-only images differ"
    e0.record()
    for _ in range(reps):
        br.blend_only()
    e1.record()
    torch.cuda.synchronize(dev)
    ms_blend = e0.elapsed_time(e1) / reps
    del br, imgs
    torch.cuda.empty_cache()
    # Roofline of the batched call: its projection and duplicate/sort stages
    # timed through ls_project / ls_duplicate_sort on the same 64 cameras and
    # tile shape; the persistent blend (with its job queue) timed alone
    # through ls_render_batch_blend.  Blend work from the per-camera counting
    # forward (the batched blend walks the same lists with the same per-tile
    # code).
    rzb = raster.Rasterizer(Pt, device=dev)
    proj, tc = rzb.project(sp, cams, counts=True)
    rzb.ensure_capacity(tc)
    R = sp.n * len(cams)
    n_vis = int((proj.view(torch.uint8)[64 * R:68 * R].view(torch.int32) != -1).sum().item())
    del proj, tc
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    t_proj, t_sort = [], []
    for i in range(4):
        ev[0].record()
        proj, _ = rzb.project(sp, cams, counts=False)
        ev[1].record()
        rzb.duplicate_sort(proj, R, cams)
        ev[2].record()
        torch.cuda.synchronize(dev)
        if i:
            t_proj.append(ev[0].elapsed_time(ev[1]))
            t_sort.append(ev[1].elapsed_time(ev[2]))
        del proj
    rzb.check_status("batched stages")
    del rzb
    torch.cuda.empty_cache()
    n_eval = n_contrib = tiles = 0
    rzc = raster.Rasterizer(Pt, device=dev)
    for cam in cams:
        _, _, st = rzc.forward(sp, cam)
        _, _, _, ne, nc = rzc.render_stats(st["proj"], sp.n, cam, st["ranges"], st["vals"])
        n_eval += ne
        n_contrib += nc
        tiles += raster.tiles_of(cam, Pt)
        del st
    rzc.check_status("batched counts")
    del rzc
    torch.cuda.empty_cache()
    kp = (max(1, (tiles - 1).bit_length()) + 7) // 8
    u = frame_units(R, n_vis, K, n_eval, n_contrib, tiles, kp, sh_bytes=192)
    ms_p, ms_s = statistics.median(t_proj), statistics.median(t_sort)
    peaks = Peaks(dev)
    lb = peaks.lower_bound_ms([u["project"], u["duplicate_sort"], u["blend_fwd"]])
    roof = {"project": peaks.entry(*u["project"], ms_p), "duplicate_sort": peaks.entry(*u["duplicate_sort"], ms_s),
            "blend": dict(peaks.entry(*u["blend_fwd"], ms_blend),
                          timing="ls_render_batch_blend (job queue and persistent blend) after the call"),
            "frame": {"lower_bound_ms": lb, "frac": lb / ms_batch,
                      "meaning": "time of the call's stages at their rooflines over its measured time"}}
    roof = {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv) for kk, vv in r.items()} for k, r in roof.items()}
    units_b = {"records": R, "visible": n_vis, "pairs_evaluated": n_eval, "pairs_composited": n_contrib,
               "tiles": tiles}
    # the plain path, one camera at a time, at the faster of the tuned tile
    # shape and its default 16x16
    plain_ms = {}
    for tile in dict.fromkeys([tuple(tune.tile), (16, 16)]):
        rz = raster.Rasterizer(dataclasses.replace(P, tile_w=tile[0], tile_h=tile[1]), device=dev)
        for cam in cams:
            rz.forward(sp, cam, sync_capacity=True)
        torch.cuda.synchronize(dev)
        e0.record()
        for cam in cams:
            rz.forward(sp, cam, sync_capacity=False)
        e1.record()
        torch.cuda.synchronize(dev)
        rz.check_status("plain cameras")
        plain_ms["%dx%d" % tile] = e0.elapsed_time(e1)
        del rz
        torch.cuda.empty_cache()
    plain_tile = min(plain_ms, key=plain_ms.get)
    ms_plain = plain_ms[plain_tile]
    pixels = sum(c["width"] * c["height"] for c in cams)
    return {"workload": "batch_3m_64cams", "cams": len(cams), "prims": scene.n, "pixels": pixels, "tile_keys": K,
            "tile": "%dx%d" % tune.tile, "blend_batch": tune.blend_batch, "graph": True,
            "ms_per_batch": ms_batch, "frames_per_s": len(cams) * 1e3 / ms_batch,
            "plain_ms_per_batch": ms_plain, "plain_frames_per_s": len(cams) * 1e3 / ms_plain,
            "plain_tile": plain_tile, "plain_ms_by_tile": {k: round(v, 3) for k, v in plain_ms.items()},
            "speedup_vs_plain": ms_plain / ms_batch, "roofline": roof, "units": units_b,
            "autotune_ms": {"%dx%d/b%d" % k: round(v, 3) for k, v in tune.table.items()}}


# --------------------------------------------------------------------------
# kernel family: the same frame with the Gaussian kernel as the speed control
# --------------------------------------------------------------------------
def time_frame(sp, cam, P, dev, steps=20, warmup=3):
    """Median forward (project + duplicate/sort + blend) and backward (blend
    adjoint + projection adjoint) ms of one camera, and the frame's units."""
    import torch
    from paper_2411_12440_gb300 import raster, scenes
    rz = raster.Rasterizer(P, device=dev)
    R = sp.n
    H, W = cam["height"], cam["width"]
    w, v = scenes.loss_weights(H, W, seed=7)
    gimg, gT = torch.from_numpy(w).to(dev), torch.from_numpy(v).to(dev)
    gout = dict(means=torch.empty_like(sp.means), scales=torch.empty_like(sp.scales),
                quats=torch.empty_like(sp.quats), opac=torch.empty_like(sp.opac), sh=torch.empty_like(sp.sh))
    proj, tc = rz.project(sp, [cam], counts=True)
    rz.ensure_capacity(tc)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    for i in range(warmup + steps):
        e = evs[i - warmup] if i >= warmup else None
        if e:
            e[0].record()
        proj, _ = rz.project(sp, [cam], counts=False)
        keys, vals, n_keys, ranges = rz.duplicate_sort(proj, R, [cam])
        image, T, n_last = rz.render_fwd(proj, R, cam, ranges, vals)
        if e:
            e[1].record()
        rz.render_bwd(sp, cam, dict(proj=proj, ranges=ranges, vals=vals, T=T, n_last=n_last), gimg, gT, out=gout)
        if e:
            e[2].record()
    torch.cuda.synchronize(dev)
    rz.check_status("kernel family")
    fwd = statistics.median(e[0].elapsed_time(e[1]) for e in evs)
    bwd = statistics.median(e[1].elapsed_time(e[2]) for e in evs)
    _, _, _, n_eval, n_contrib = rz.render_stats(proj, R, cam, ranges, vals)
    return {"fwd_ms": fwd, "bwd_ms": bwd, "tile_keys": int(n_keys.item()), "pairs_evaluated": n_eval,
            "pairs_composited": n_contrib}


def bench_kernel_family(sp, cam, antialias, dev):
    """Linear kernel (lambda 2.5) against the Gaussian (lambda 1, support at
    3 sigma or alpha_min) on the same primitives: the paper's speed claim."""
    import dataclasses
    from paper_2411_12440_gb300 import raster
    base = raster.RenderParams(sh_degree=3, antialias=antialias)
    out = {"linear": time_frame(sp, cam, dataclasses.replace(base, kernel=0, lam=2.5), dev),
           "gaussian": time_frame(sp, cam, dataclasses.replace(base, kernel=1, lam=1.0), dev)}
    out["gaussian_over_linear_fwd"] = out["gaussian"]["fwd_ms"] / out["linear"]["fwd_ms"]
    out["gaussian_over_linear_bwd"] = out["gaussian"]["bwd_ms"] / out["linear"]["bwd_ms"]
    return out


# --------------------------------------------------------------------------
# learned termination: 5M primitives, one 1920x1080 view on the ring
# --------------------------------------------------------------------------
def bench_learned(dev, reps=20):
    """Plain forward frame against the learned-termination frame (trained
    network plus calibrated margin, lossy threshold t_thr) and the same
    truncated pipeline without the network: every key kept, and one global
    depth tuned on the training views.  PSNR against the plain frame."""
    import math
    import torch
    from paper_2411_12440_gb300 import raster, scenes
    from paper_2411_12440_gb300.learned import LearnedRenderer, TerminationMLP
    net = TerminationMLP.load(os.path.join(ROOT, "paper_2411_12440_gb300", "data", "termination_mlp.npz"),
                              device=dev)
    margin, t_thr = float(net.meta["margin"]), float(net.meta["t_thr"])
    const = float(net.meta["const_dstar"]) if "const_dstar" in net.meta else None
    scene, cams, _ = scenes.make_workload("learned_5m_1080p")
    cam = cams[0]
    sp = raster.Splats.from_scene(scene, device=dev)
    del scene
    P = raster.RenderParams(sh_degree=3)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    def psnr(img, ref):
        mse = float(((img - ref) ** 2).mean().item())
        return math.inf if mse == 0.0 else -10.0 * math.log10(mse)

    out = {"workload": "learned_5m_1080p", "prims": sp.n, "width": cam["width"], "height": cam["height"],
           "t_thr": t_thr, "margin": margin, "const_dstar": const}
    rz = raster.Rasterizer(P, device=dev)
    img0, _, st0 = rz.forward(sp, cam)
    img0 = img0.clone()
    out["plain"] = {"ms": timed(lambda: rz.forward(sp, cam, sync_capacity=False)),
                    "keys_sorted": int(st0["n_keys"].item())}
    rz.check_status("plain")
    rzt = raster.Rasterizer(raster.RenderParams(sh_degree=3, t_min=t_thr), device=dev)
    rzt.forward(sp, cam)
    out["plain_t_thr"] = {"ms": timed(lambda: rzt.forward(sp, cam, sync_capacity=False))}
    out["plain_t_thr"]["psnr_db"] = psnr(rzt.forward(sp, cam)[0], img0)
    rzt.check_status("plain at t_thr")
    del rz, rzt
    torch.cuda.empty_cache()
    lr = LearnedRenderer(sp, cam, P, device=dev)
    modes = {"mlp": dict(mlp=net, margin=margin),
             "keep_all": dict(dstar_in=torch.full((lr.tiles,), math.inf, device=dev))}
    if const is not None:
        modes["const"] = dict(dstar_in=torch.full((lr.tiles,), const, device=dev))
    for name, kw in modes.items():
        ms = timed(lambda: lr.render(t_thr=t_thr, stats=False, **kw))
        lr.check()
        lr.render(t_thr=t_thr, **kw)  # once more with the counters
        lr.check()
        total, kept, held, refuted = lr.counters()
        out[name] = {"ms": ms, "keys_sorted": kept + held, "keys_kept": kept, "keys_held_sorted": held,
                     "tiles_refuted": refuted, "psnr_db": psnr(lr.image, img0),
                     "max_abs_err": float((lr.image - img0).abs().max().item())}
    out["tiles"] = lr.tiles
    del lr
    torch.cuda.empty_cache()
    # Frame-level roofline of the learned frame: its projection, its sort
    # stages over the keys it actually sorted (kept + held out) and a blend
    # of the work a plain render stopping at t_thr counts, each at its
    # roofline, over the measured frame time.
    rzs = raster.Rasterizer(raster.RenderParams(sh_degree=3, t_min=t_thr), device=dev)
    _, _, st = rzs.forward(sp, cam)
    _, _, _, ne, nc = rzs.render_stats(st["proj"], sp.n, cam, st["ranges"], st["vals"])
    R = sp.n
    n_vis = int((st["proj"].view(torch.uint8)[64 * R:68 * R].view(torch.int32) != -1).sum().item())
    rzs.check_status("learned counts")
    del rzs, st
    torch.cuda.empty_cache()
    u = frame_units(R, n_vis, out["mlp"]["keys_sorted"], ne, nc, out["tiles"], 2, sh_bytes=192)
    peaks = Peaks(dev)
    lb = peaks.lower_bound_ms([u["project"], u["duplicate_sort"], u["blend_fwd"]])
    out["roofline"] = {"frame": {"lower_bound_ms": round(lb, 4), "frac": round(lb / out["mlp"]["ms"], 4),
                                 "meaning": "time of projection, the sort of the keys sorted and the blend at their "
                                            "rooflines over the measured learned frame"},
                       "units": {"visible": n_vis, "keys_sorted": out["mlp"]["keys_sorted"],
                                 "pairs_evaluated_at_t_thr": ne, "pairs_composited_at_t_thr": nc}}
    out["speedup_vs_plain"] = out["plain"]["ms"] / out["mlp"]["ms"]
    out["speedup_vs_keep_all"] = out["keep_all"]["ms"] / out["mlp"]["ms"]
    if const is not None:
        out["speedup_vs_const"] = out["const"]["ms"] / out["mlp"]["ms"]
    return out


def bench_kernel_fit(dev):
    """Pattern fits of Sec. 5.1 (Fig. 5): stripes, checkerboard and circles at
    4 and 16 periods, 256 x 256, 2304 primitives, 300 steps of the library's
    own forward, 6:2:2 loss, backward and Adam, for every kernel of the
    family; PSNR against the target per (pattern, kernel)."""
    from paper_2411_12440_gb300 import fitting
    t0 = time.perf_counter()
    t = fitting.sweep(freqs=(4, 16), size=256, n_side=48, steps=300, device=dev)
    psnr = {k: {kk: round(vv["psnr_db"], 2) for kk, vv in v.items()} for k, v in t.items()}
    best = {k: max(v, key=v.get) for k, v in psnr.items()}
    return {"workload": "patterns_256", "prims": 48 * 48, "steps": 300, "psnr_db": psnr, "best_kernel": best,
            "linear_over_gaussian_db": {k: round(v["linear"] - v["gaussian"], 2) for k, v in psnr.items()},
            "seconds": round(time.perf_counter() - t0, 2)}


def learned_probe():
    """One plain forward frame, then one learned frame (trained network,
    calibrated margin, no counters) of the 5M 1080p workload, after one
    untimed frame of each: the launch list of a profiler run shows both."""
    import torch
    from paper_2411_12440_gb300 import raster, scenes
    from paper_2411_12440_gb300.learned import LearnedRenderer, TerminationMLP
    dev = torch.device("cuda", 0)
    net = TerminationMLP.load(os.path.join(ROOT, "paper_2411_12440_gb300", "data", "termination_mlp.npz"),
                              device=dev)
    margin, t_thr = float(net.meta["margin"]), float(net.meta["t_thr"])
    scene, cams, _ = scenes.make_workload("learned_5m_1080p")
    cam = cams[0]
    sp = raster.Splats.from_scene(scene, device=dev)
    del scene
    P = raster.RenderParams(sh_degree=3)
    rz = raster.Rasterizer(P, device=dev)
    lr = LearnedRenderer(sp, cam, P, device=dev)
    rz.forward(sp, cam)  # capacity from an exact count
    for _ in range(2):
        rz.forward(sp, cam, sync_capacity=False)
        lr.render(mlp=net, margin=margin, t_thr=t_thr, stats=False)
    torch.cuda.synchronize(dev)
    rz.check_status("plain")
    lr.check()
    print(json.dumps({"learned_probe": "learned_5m_1080p", "frames": ["plain", "mlp", "plain", "mlp"]}))


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--prims", type=int, default=None,
                    help="override the primitive count (same recipe; for small profiling cases)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-camera batched measurement")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-termination measurement")
    ap.add_argument("--no-family", action="store_true", help="skip the linear-vs-Gaussian measurement")
    ap.add_argument("--no-fit", action="store_true", help="skip the pattern fits of the kernel family")
    ap.add_argument("--learned-probe", action="store_true",
                    help="one plain and one learned forward frame of the 5M 1080p workload (for a launch list)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.learned_probe:
        return learned_probe()
    args.warmup = max(args.warmup, 3)

    import numpy as np
    import torch
    from paper_2411_12440_gb300 import raster, scenes

    ws, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    scene, cams, extra = scenes.make_workload(WORKLOAD, n=args.prims)
    cam = cams[0]
    P = raster.RenderParams(sh_degree=3, antialias=int(extra["antialias"]))
    rz = raster.Rasterizer(P, device=dev)
    sp = raster.Splats.from_scene(scene, device=dev)
    R = sp.n
    H, W = cam["height"], cam["width"]
    w, v = scenes.loss_weights(H, W, seed=7)
    gimg = torch.from_numpy(w).to(dev)
    gT = torch.from_numpy(v).to(dev)
    g2d = torch.empty((R, 12), dtype=torch.float32, device=dev)
    gout = dict(means=torch.empty_like(sp.means), scales=torch.empty_like(sp.scales),
                quats=torch.empty_like(sp.quats), opac=torch.empty_like(sp.opac), sh=torch.empty_like(sp.sh))

    # One step is the boundary calls of the frame: ls_project,
    # ls_duplicate_sort, ls_render_fwd and ls_render_bwd (which clears its
    # 2D-gradient buffer itself and runs the blend and projection adjoints).
    stage_names = ["project", "duplicate_sort", "render_fwd", "render_bwd"]

    def step(evs=None, bwd=True, splats=None, grad_image=None, grad_t=None, outg=None):
        spx = splats or sp
        rec = (lambda i: evs[i].record()) if evs is not None else (lambda i: None)
        rec(0)
        proj, _ = rz.project(spx, [cam], counts=False)
        rec(1)
        keys, vals, n_keys, ranges = rz.duplicate_sort(proj, R, [cam])
        rec(2)
        image, T, n_last = rz.render_fwd(proj, R, cam, ranges, vals)
        rec(3)
        if not bwd:
            return image, T, None
        state = dict(proj=proj, ranges=ranges, vals=vals, T=T, n_last=n_last)
        g = rz.render_bwd(spx, cam, state, grad_image if grad_image is not None else gimg,
                          grad_t if grad_t is not None else gT, out=outg or gout)
        rec(4)
        return image, T, g

    # The same frame kernel by kernel, for the per-kernel durations of the
    # rooflines: the adjoint as ls_tile_order and ls_blend_bwd_ordered (the
    # longest-first tile order ls_render_bwd uses) into a cleared 2D-gradient
    # buffer (cleared by a device copy through ls_copy), then ls_project_bwd.
    kernel_names = ["project", "duplicate_sort", "blend_fwd", "g2d_clear", "tile_order", "blend_bwd", "project_bwd"]
    g2d_zero = torch.zeros((R, 12), dtype=torch.float32, device=dev)

    def kernel_step(evs):
        evs[0].record()
        proj, _ = rz.project(sp, [cam], counts=False)
        evs[1].record()
        keys, vals, n_keys, ranges = rz.duplicate_sort(proj, R, [cam])
        evs[2].record()
        image, T, n_last = rz.render_fwd(proj, R, cam, ranges, vals)
        evs[3].record()
        raster.copy_(g2d, g2d_zero)
        evs[4].record()
        order = rz.tile_order(cam, n_last)
        evs[5].record()
        rz.blend_bwd_ordered(proj, R, cam, ranges, order, vals, T, n_last, gimg, gT, g2d)
        evs[6].record()
        rz.project_bwd(sp, [cam], proj, g2d, out=gout)
        evs[7].record()

    # capacity from an exact count, then no host syncs inside steps
    proj, tc = rz.project(sp, [cam], counts=True)
    K = rz.ensure_capacity(tc)
    dk = proj.view(torch.uint8)[64 * R:68 * R].view(torch.int32)
    n_vis = int((dk != -1).sum().item())
    keys, vals, n_keys, ranges = rz.duplicate_sort(proj, R, [cam])
    _, _, _, n_eval, n_contrib = rz.render_stats(proj, R, cam, ranges, vals)
    K_box = K
    K = int(n_keys.item())
    del proj, tc
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    rz.check_status("warmup")

    # ---------------------------------------------------------------- timed fwd+bwd
    # The headline: the frame's boundary calls recorded once in a CUDA graph
    # (raster.FrameGraph) and replayed, as a training loop runs them; each
    # replay redoes the whole frame on the resident parameters.
    fg = raster.FrameGraph(rz, sp, cam, gimg, gT)
    for _ in range(args.warmup):
        fg.replay()
    torch.cuda.synchronize()
    rz.check_status("graph warmup")
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        t_start.record()
        for i in range(args.steps):
            fg.replay()
        t_end.record()
        torch.cuda.synchronize()
    barrier(ws)
    total_ms = max_over_ranks(t_start.elapsed_time(t_end), ws)
    rz.check_status("timed steps")

    # The same steps launched call by call from the host, with events between
    # the boundary calls for the per-stage times.
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(stage_names) + 1)] for _ in range(args.steps)]
    barrier(ws)
    torch.cuda.synchronize()
    t_e0 = torch.cuda.Event(enable_timing=True)
    t_e1 = torch.cuda.Event(enable_timing=True)
    t_e0.record()
    for i in range(args.steps):
        step(evs[i])
    t_e1.record()
    torch.cuda.synchronize()
    barrier(ws)
    eager_ms = max_over_ranks(t_e0.elapsed_time(t_e1), ws) / args.steps
    rz.check_status("call-by-call steps")
    stage_ms = {nm: statistics.mean(e[j].elapsed_time(e[j + 1]) for e in evs) for j, nm in enumerate(stage_names)}

    # ---------------------------------------------------------------- kernel by kernel
    kevs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(kernel_names) + 1)] for _ in range(args.steps)]
    for _ in range(2):
        kernel_step(kevs[0])
    torch.cuda.synchronize()
    with ClockSampler(local) as kclocks:
        for i in range(args.steps):
            kernel_step(kevs[i])
        torch.cuda.synchronize()
    rz.check_status("kernel by kernel")
    kernel_ms = {nm: statistics.mean(e[j].elapsed_time(e[j + 1]) for e in kevs)
                 for j, nm in enumerate(kernel_names)}

    # ---------------------------------------------------------------- timed fwd only
    fgf = raster.FrameGraph(rz, sp, cam)
    for _ in range(args.warmup):
        fgf.replay()
    barrier(ws)
    torch.cuda.synchronize()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record()
    for i in range(args.steps):
        fgf.replay()
    f1.record()
    torch.cuda.synchronize()
    barrier(ws)
    fwd_ms = max_over_ranks(f0.elapsed_time(f1), ws) / args.steps
    rz.check_status("timed forward")
    del fgf

    # ---------------------------------------------------------------- e2e through host buffers
    # Every step copies its inputs (all primitive parameters and the loss
    # weights) from pinned host memory and reads the image and all parameter
    # gradients back.  Copies run on streams of their own, double-buffered,
    # so step i+1's upload and step i-1's read-back overlap step i's compute.
    e2e = None
    if not args.no_e2e:
        host_in = [t.cpu().pin_memory() for t in sp.tensors()] + [gimg.cpu().pin_memory(), gT.cpu().pin_memory()]
        names = ("means", "scales", "quats", "opac", "sh")
        slots = []
        for _ in range(2):
            dev_in = [torch.empty_like(t, device=dev) for t in host_in]
            slots.append(dict(
                dev_in=dev_in, splats=raster.Splats(*dev_in[:5], sp.sh_degree),
                host_out=[torch.empty((H, W, 3), dtype=torch.float32).pin_memory()] +
                         [torch.empty(getattr(sp, k).shape, dtype=torch.float32).pin_memory() for k in names]))
        for sl in slots:  # each slot's frame recorded once, on its own input buffers
            for d_, h_ in zip(sl["dev_in"], host_in):
                d_.copy_(h_)
            sl["fg"] = raster.FrameGraph(rz, sl["splats"], cam, sl["dev_in"][5], sl["dev_in"][6])
            sl["grads"], sl["image"] = sl["fg"].grads, sl["fg"].image
        h2d = sum(t.numel() * t.element_size() for t in host_in)
        d2h = sum(t.numel() * t.element_size() for t in slots[0]["host_out"])
        NS = 1  # copy streams per direction (more did not raise the host-link rate)
        s_ups = [torch.cuda.Stream(dev) for _ in range(NS)]
        s_downs = [torch.cuda.Stream(dev) for _ in range(NS)]
        s_comp = torch.cuda.Stream(dev)
        s_up, s_down = s_ups[0], s_downs[0]
        comp_done = [None, None]
        down_done = [None, None]

        def chunked_copy(dsts, srcs, streams, wait):
            """Copy each src into its dst in len(streams) chunks, one per stream,
            after `wait`; returns the events that mark the end of each stream."""
            evs = []
            for j, st_ in enumerate(streams):
                with torch.cuda.stream(st_):
                    if wait is not None:
                        st_.wait_event(wait)
                    for d, h in zip(dsts, srcs):
                        df, hf = d.view(-1), h.view(-1)
                        n = df.numel()
                        lo, hi = n * j // len(streams), n * (j + 1) // len(streams)
                        if hi > lo:  # through the library's host-link copy (ls_copy)
                            raster.copy_(df[lo:hi], hf[lo:hi], st_)
                    ev = torch.cuda.Event()
                    ev.record(st_)
                    evs.append(ev)
            return evs

        def e2e_step(i):
            sl = slots[i % 2]
            # step i-2 has finished reading this slot's inputs
            ups = chunked_copy(sl["dev_in"], host_in, s_ups, comp_done[i % 2])
            with torch.cuda.stream(s_comp):
                for ev in ups:
                    s_comp.wait_event(ev)
                if down_done[i % 2] is not None:
                    for ev in down_done[i % 2]:  # step i-2's results are on the host
                        s_comp.wait_event(ev)
                sl["fg"].replay()  # writes sl["image"] and sl["grads"]
                cd = torch.cuda.Event()
                cd.record(s_comp)
                comp_done[i % 2] = cd
            down_done[i % 2] = chunked_copy(sl["host_out"], [sl["image"]] + [sl["grads"][k] for k in names], s_downs,
                                            cd)

        for i in range(4):
            e2e_step(i)
        torch.cuda.synchronize()
        barrier(ws)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        n_e2e = max(3, args.steps // 2)
        e0.record(s_up)
        for st_ in s_ups[1:] + [s_comp] + s_downs:
            st_.wait_event(e0)
        for i in range(n_e2e):
            e2e_step(i)
        for st_ in s_ups + [s_comp] + s_downs[1:]:
            s_down.wait_stream(st_)
        e1.record(s_down)
        torch.cuda.synchronize()
        barrier(ws)
        e2e_ms = max_over_ranks(e0.elapsed_time(e1), ws) / n_e2e
        rz.check_status("e2e")
        e2e = {"value": job_rate(ws, e2e_ms), "unit": "iters/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "overlap": "uploads, compute (one frame graph per buffer) and read-backs on three streams, "
                          "double-buffered",
               "moves": "every primitive parameter in, the image and every parameter gradient out"}

        # The same steps with the primitives resident on the device, as in a
        # training loop: per step only the step's data (the upstream
        # gradients of the image and of T) comes from pinned host memory and
        # the rendered image goes back; the parameter gradients stay on the
        # device for the optimiser.
        r_in = [gimg.cpu().pin_memory(), gT.cpu().pin_memory()]
        r_slots = [dict(dev_in=[torch.empty_like(t, device=dev) for t in r_in],
                        host_out=[torch.empty((H, W, 3), dtype=torch.float32).pin_memory()]) for _ in range(2)]
        for sl in r_slots:
            for d_, h_ in zip(sl["dev_in"], r_in):
                d_.copy_(h_)
            sl["fg"] = raster.FrameGraph(rz, sp, cam, sl["dev_in"][0], sl["dev_in"][1])
            sl["grads"], sl["image"] = sl["fg"].grads, sl["fg"].image
        r_h2d = sum(t.numel() * t.element_size() for t in r_in)
        r_d2h = sum(t.numel() * t.element_size() for t in r_slots[0]["host_out"])
        comp_done = [None, None]
        down_done = [None, None]

        def r_step(i):
            sl = r_slots[i % 2]
            ups = chunked_copy(sl["dev_in"], r_in, s_ups, comp_done[i % 2])
            with torch.cuda.stream(s_comp):
                for ev in ups:
                    s_comp.wait_event(ev)
                if down_done[i % 2] is not None:
                    for ev in down_done[i % 2]:
                        s_comp.wait_event(ev)
                sl["fg"].replay()
                cd = torch.cuda.Event()
                cd.record(s_comp)
                comp_done[i % 2] = cd
            down_done[i % 2] = chunked_copy(sl["host_out"], [sl["image"]], s_downs, cd)

        for i in range(4):
            r_step(i)
        torch.cuda.synchronize()
        barrier(ws)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s_up)
        for st_ in s_ups[1:] + [s_comp] + s_downs:
            st_.wait_event(e0)
        for i in range(n_e2e):
            r_step(i)
        for st_ in s_ups + [s_comp] + s_downs[1:]:
            s_down.wait_stream(st_)
        e1.record(s_down)
        torch.cuda.synchronize()
        barrier(ws)
        r_ms = max_over_ranks(e0.elapsed_time(e1), ws) / n_e2e
        rz.check_status("e2e resident")
        e2e["resident_parameters"] = {
            "value": job_rate(ws, r_ms), "unit": "iters/s", "h2d_bytes_per_step": r_h2d, "d2h_bytes_per_step": r_d2h,
            "moves": "the upstream image and T gradients in, the image out; parameters and gradients stay resident"}

    ms = total_ms / args.steps
    value = job_rate(ws, ms)

    # ---------------------------------------------------------------- roofline of the dominant kernel
    peaks = Peaks(dev)
    kp = 2
    nt = raster.tiles_of(cam, P)
    units = frame_units(R, n_vis, K, n_eval, n_contrib, nt, kp, sh_bytes=192, pixels=H * W)
    stage_roofs = {k: peaks.entry(*units[k], kernel_ms[k]) for k in kernel_names}
    # the dominant kernel: the longest of the stages that are one launch
    # each (duplicate_sort is a chain of a dozen launches, none of them
    # longer than the blends; the clear and the tile order are small helpers)
    dom = max(("project", "blend_fwd", "blend_bwd", "project_bwd"), key=lambda k: kernel_ms[k])
    roof = dict(stage_roofs[dom])
    if roof["bound"] == "alu":
        roof["peak_check"] = {"measured_fma_tops": round(peaks.fma_probe, 3),
                              "of_peak": round(peaks.fma_probe / peaks.alu, 4)}
    tr = NCU_TRAFFIC.get(dom)
    src = {"blend_fwd": "blend.cu", "blend_bwd": "blend.cu", "project": "project.cu", "project_bwd": "project.cu",
           "duplicate_sort": "sort.cu"}[dom]
    roof["kernel"] = dom
    roof["duration_ms"] = kernel_ms[dom]
    roof["timing"] = ("CUDA events around the kernel's launch on its stream, mean over %d kernel-by-kernel steps of "
                      "the same frame" % args.steps)
    roof["traffic"] = tr["bytes"] if tr and tr.get("src") == _src_hash(src) else None
    stage_roofs = {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv) for kk, vv in r.items()
                       if kk in ("bound", "achieved", "unit", "frac")} for k, r in stage_roofs.items()}
    # the duplicate/sort stage also against the plan's per-unit figures for
    # the classic method (12 B per key + 8 B per record for the duplication,
    # six 8-bit passes over 12-byte (tile | depth, id) keys at 24 B per key
    # per pass plus an 8 B histogram read): what that method would move for
    # the same K, over the time this design takes
    classic_bytes = 12 * K + 8 * R + (24 * 6 + 8) * K
    stage_roofs["duplicate_sort"]["frac_classic_method_bytes"] = round(
        classic_bytes / (kernel_ms["duplicate_sort"] * 1e-3) / 1e9 / peaks.hbm, 4)

    line = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": frame_config(R, cam, P.tile_w, ws, args.prims),
            "launch": "the frame's boundary calls recorded once in a CUDA graph (raster.FrameGraph) and replayed",
            "call_by_call": {"value": job_rate(ws, eager_ms), "ms_per_step": eager_ms,
                             "launch": "the same boundary calls launched one by one from the host"},
            "fwd_fps": job_rate(ws, fwd_ms), "fwd_ms": fwd_ms,
            "stages_ms": {k: round(v, 4) for k, v in stage_ms.items()},
            "kernels_ms": {k: round(v, 4) for k, v in kernel_ms.items()},
            "stage_rooflines": stage_roofs,
            "units": {"tile_keys": K, "box_tile_keys": K_box, "visible": n_vis, "pairs_evaluated": n_eval,
                      "pairs_composited": n_contrib},
            "roofline": roof, "clocks": clocks.summary(), "clocks_kernel_by_kernel": kclocks.summary(), "e2e": e2e,
            # per step: ls_project 1; ls_duplicate_sort 13 + kp (depth histogram, scan, 4 depth passes, boxes,
            # key count, 2-launch warp-count scan, key copy, digit scan, kp tile passes, ranges); ls_render_fwd
            # 1; ls_render_bwd 4 (tile work, tile order, blend adjoint, projection adjoint; its clear is a
            # memset)
            "gpu_launches": args.steps * (1 + (13 + kp) + 1 + 4)}

    if not args.no_batch and args.prims is None:
        line["batched"] = bench_batched(dev)
    if not args.no_family and args.prims is None:
        line["kernel_family"] = bench_kernel_family(sp, cam, int(extra["antialias"]), dev)
    if not args.no_learned and args.prims is None:
        line["learned"] = bench_learned(dev)
    if not args.no_fit and args.prims is None:
        line["kernel_fit"] = bench_kernel_fit(dev)
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        # the median of two samples after one untimed one, as the reference
        # arm takes its steps
        ncores = os.cpu_count() or 1
        Pc = dict(sh_degree=3, antialias=int(extra["antialias"]))
        runs = [oracle_frame_estimate(scene, cam, Pc, ncores) for _ in range(3)][1:]
        est = statistics.median(r[0] for r in runs)
        line["cpu_baseline"] = {"value": 1.0 / est, "unit": "iters/s", "cores": ncores, "kind": "oracle",
                                "sample": runs[0][1] + "; median of 2 samples after 1 untimed",
                                "seconds_spent": round(sum(r[2] for r in runs), 1)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
