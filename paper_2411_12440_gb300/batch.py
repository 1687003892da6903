"""Batched multi-camera rendering: one ls_render_batch call renders every
camera of a set (sizes may differ) over one shared sort and one persistent
blending launch; the call is captured once in a CUDA graph and replayed.

An autotuner picks the tile shape (8x8, 16x16, 32x16) and the number of
records staged per shared-memory batch by timing the real call.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math

import torch

from . import _native as N
from .raster import RenderParams, Splats, _p, _stream, cam_array, cam_struct, tiles_of

TILE_SHAPES = ((8, 8), (16, 16), (32, 16))
BLEND_BATCHES = (32, 64, 128, 256)


class BatchRenderer:
    """Renders `cams` (list of camera dicts, at most 64) of one scene."""

    def __init__(self, splats: Splats, cams, params: RenderParams | None = None, blend_batch=0, device="cuda",
                 margin=1.1):
        if not 1 <= len(cams) <= N.LS_MAX_CAMS:
            raise ValueError("1..%d cameras per batch" % N.LS_MAX_CAMS)
        self.splats = splats
        self.cams = list(cams)
        self.params = dataclasses.replace(params or RenderParams(), sh_degree=splats.sh_degree)
        self.blend_batch = int(blend_batch)
        self.device = torch.device(device)
        self.margin = margin
        self.status = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.n_keys = torch.zeros(1, dtype=torch.int64, device=self.device)
        self.pix = [c["width"] * c["height"] for c in self.cams]
        self.images = torch.empty((sum(self.pix), 3), dtype=torch.float32, device=self.device)
        self._cams_c = cam_array(self.cams)
        self._params_c = self.params.c()
        self.capacity = 0
        self.graph = None
        self._ws = None

    # ---------------------------------------------------------------- planning
    def count_keys(self):
        """Upper bound on the tile keys of the current scene: the support-box
        tiles of every record (one host read); the keys actually made are the
        box tiles the support ellipses reach."""
        from .raster import Rasterizer
        rz = Rasterizer(self.params, device=self.device)
        _, tc = rz.project(self.splats, self.cams, counts=True)
        return int(tc.sum(dtype=torch.int64).item())

    def plan(self, capacity=None):
        K = self.count_keys() if capacity is None else int(capacity)
        self.capacity = int(math.ceil(K * self.margin)) + 1024 if capacity is None else K
        wsb = N.lib().ls_render_batch_workspace(self.splats.n, self._cams_c, len(self.cams),
                                                ctypes.byref(self._params_c), self.capacity)
        if wsb == 0:
            raise ValueError("invalid batch configuration")
        self._ws = torch.empty(wsb + 256, dtype=torch.uint8, device=self.device)
        self._ws_ptr = (self._ws.data_ptr() + 255) // 256 * 256
        self._ws_bytes = wsb
        self.graph = None
        return self.capacity

    # ---------------------------------------------------------------- render
    def render_eager(self):
        if self._ws is None:
            self.plan()
        sp = self.splats
        N.check(N.lib().ls_render_batch(sp.n, _p(sp.means), _p(sp.scales), _p(sp.quats), _p(sp.opac), _p(sp.sh),
                                        self._cams_c, len(self.cams), ctypes.byref(self._params_c),
                                        self.blend_batch, self.capacity, _p(self.images), ctypes.c_void_p(0),
                                        _p(self.n_keys), ctypes.c_void_p(self._ws_ptr), self._ws_bytes,
                                        _p(self.status), _stream()), "ls_render_batch")

    def blend_only(self):
        """The blending stage alone on what the last render left in the
        workspace (ls_render_batch_blend): the same images; for timing."""
        N.check(N.lib().ls_render_batch_blend(self.splats.n, self._cams_c, len(self.cams), ctypes.byref(self._params_c),
                                              self.blend_batch, self.capacity, _p(self.images), ctypes.c_void_p(0),
                                              ctypes.c_void_p(self._ws_ptr), self._ws_bytes, _p(self.status),
                                              _stream()), "ls_render_batch_blend")

    def capture(self):
        """Record the whole batched render in a CUDA graph (after one eager
        call, which also sets the kernels' shared-memory attributes)."""
        self.render_eager()
        torch.cuda.synchronize(self.device)
        self.check()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.render_eager()
        torch.cuda.current_stream(self.device).wait_stream(s)
        self.graph = g
        return g

    def render(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self.render_eager()
        return self.images

    def check(self):
        s = int(self.status.item())
        if s != 0:
            raise N.LsError(s, "ls_render_batch")

    def image(self, c):
        """View of camera c's image [H, W, 3] in the packed output."""
        off = sum(self.pix[:c])
        cam = self.cams[c]
        return self.images[off:off + self.pix[c]].view(cam["height"], cam["width"], 3)


@dataclasses.dataclass
class TuneResult:
    tile: tuple
    blend_batch: int
    ms: float
    table: dict


class Autotuner:
    """Times ls_render_batch for every tile shape and blend batch size and
    keeps the fastest (median of `reps` timed calls after one warm-up)."""

    def __init__(self, tiles=TILE_SHAPES, batches=BLEND_BATCHES, reps=3):
        self.tiles = tiles
        self.batches = batches
        self.reps = reps

    def tune(self, splats: Splats, cams, params: RenderParams | None = None, device="cuda"):
        base = params or RenderParams()
        table = {}
        best = None
        for tw, th in self.tiles:
            P = dataclasses.replace(base, tile_w=tw, tile_h=th)
            br = BatchRenderer(splats, cams, P, device=device)
            br.plan()
            for b in self.batches:
                br.blend_batch = b
                br.render_eager()
                torch.cuda.synchronize(device)
                br.check()
                ts = []
                for _ in range(self.reps):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    br.render_eager()
                    e1.record()
                    torch.cuda.synchronize(device)
                    ts.append(e0.elapsed_time(e1))
                ms = sorted(ts)[len(ts) // 2]
                table[(tw, th, b)] = ms
                if best is None or ms < best[2]:
                    best = ((tw, th), b, ms)
            del br
            torch.cuda.empty_cache()
        return TuneResult(best[0], best[1], best[2], table)
