"""PyTorch-facing API of the linear-splatting rasterizer.

Torch supplies device memory, the current stream and autograd; every stage
of the rasterizer is a call into libls.so (include/ls.h):

    project        -> ls_project         (a1, Sec. 3.1 Eq. 1-4, Eq. 12 support)
    duplicate_sort -> ls_duplicate_sort  (a2 + a3, order of Eq. 6)
    render_fwd     -> ls_render_fwd      (a4, Eq. 6 with the kernel of Eq. 12)
    render_bwd     -> ls_render_bwd      (a5 + a6, adjoint; AGS of Eq. 13-14)

Parameter layout on the device (Splats): means/scales [N, 3], quats [N, 4]
(w, x, y, z), opacities [N] (activated values), SH coefficient-major
[(deg+1)^2 * 3, N].
"""
from __future__ import annotations

import ctypes
import dataclasses
import math

import numpy as np
import torch

from . import _native as N


@dataclasses.dataclass
class RenderParams:
    lam: float = 2.5
    kernel: int = 0
    ags: int = 0
    antialias: int = 0
    eps2d: float = 0.3
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.999
    t_min: float = 1e-4
    tile_w: int = 16
    tile_h: int = 16
    bg: tuple = (0.0, 0.0, 0.0)
    near: float = 0.2
    far: float = 1e4
    sh_degree: int = 0

    @staticmethod
    def from_dict(d=None, **kw):
        p = RenderParams()
        for k, v in dict(d or {}, **kw).items():
            setattr(p, k, v)
        return p

    def c(self):
        s = N.LsParams()
        s.lam = self.lam
        s.kernel = int(self.kernel)
        s.ags = int(self.ags)
        s.antialias = int(self.antialias)
        s.eps2d = self.eps2d
        s.alpha_min = self.alpha_min
        s.alpha_max = self.alpha_max
        s.t_min = self.t_min
        s.tile_w = int(self.tile_w)
        s.tile_h = int(self.tile_h)
        for i in range(3):
            s.bg[i] = float(self.bg[i])
        s.near_plane = self.near
        s.far_plane = self.far
        s.sh_degree = int(self.sh_degree)
        return s


def cam_struct(cam):
    c = N.LsCamera()
    vm = np.asarray(cam["viewmat"], dtype=np.float32).reshape(16)
    for i in range(16):
        c.viewmat[i] = float(vm[i])
    c.fx, c.fy, c.cx, c.cy = cam["fx"], cam["fy"], cam["cx"], cam["cy"]
    c.width, c.height = int(cam["width"]), int(cam["height"])
    return c


def cam_array(cams):
    arr = (N.LsCamera * len(cams))()
    for i, cam in enumerate(cams):
        arr[i] = cam_struct(cam)
    return arr


def tiles_of(cam, params):
    return ((cam["width"] + params.tile_w - 1) // params.tile_w) * ((cam["height"] + params.tile_h - 1) // params.tile_h)


class Splats:
    """Primitive parameters in the library's device layout."""

    def __init__(self, means, scales, quats, opac, sh, sh_degree):
        self.means, self.scales, self.quats, self.opac, self.sh = means, scales, quats, opac, sh
        self.sh_degree = int(sh_degree)

    @property
    def n(self):
        return int(self.means.shape[0])

    @staticmethod
    def sh_to_device_layout(sh):
        """[N, K, 3] -> coefficient-major [K*3, N]."""
        n = sh.shape[0]
        return sh.reshape(n, -1).t().contiguous()

    @staticmethod
    def sh_from_device_layout(sh, n):
        return sh.t().reshape(n, -1, 3)

    @staticmethod
    def from_scene(scene, device="cuda"):
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(device)
        return Splats(t(scene.means), t(scene.scales), t(scene.quats), t(scene.opac),
                      Splats.sh_to_device_layout(t(scene.sh)), scene.sh_degree)

    def tensors(self):
        return self.means, self.scales, self.quats, self.opac, self.sh


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def copy_(dst, src, stream=None):
    """dst <- src (same size, contiguous) between device memory and pinned
    host memory, either way, enqueued on `stream` (default: the current one)."""
    if not (dst.is_contiguous() and src.is_contiguous()):
        raise ValueError("contiguous tensors")
    n = dst.numel() * dst.element_size()
    if n != src.numel() * src.element_size():
        raise ValueError("sizes differ")
    st = ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    N.check(N.lib().ls_copy(_p(dst), _p(src), n, st), "ls_copy")
    return dst


def _dev_check(t, name):
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)


class Rasterizer:
    """Owns the status word and the reusable scratch of one render stream.

    `key_capacity` bounds the number of tile keys; `grow_margin` is the slack
    added when the capacity is (re)sized from an exact count.
    """

    def __init__(self, params: RenderParams | None = None, device="cuda", grow_margin=1.15):
        self.params = params or RenderParams()
        self.device = torch.device(device)
        self.status = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.grow_margin = grow_margin
        self.capacity = 0
        self._bufs = {}
        # ls_render_bwd blends the tiles longest first (ordered workspace)
        self.bwd_tile_order = True

    # ---------------------------------------------------------------- buffers
    def _buf(self, name, nbytes, dtype=torch.uint8):
        """Reusable device buffer of at least nbytes (256-byte aligned)."""
        b = self._bufs.get(name)
        if b is None or b.numel() * b.element_size() < nbytes:
            b = torch.empty(max(nbytes, 256) // torch.tensor([], dtype=dtype).element_size() + 64, dtype=dtype,
                            device=self.device)
            self._bufs[name] = b
        return b

    def reset_status(self):
        self.status.zero_()

    def check_status(self, where="libls"):
        s = int(self.status.item())
        if s != 0:
            raise N.LsError(s, where)

    # ---------------------------------------------------------------- stages
    def project(self, splats: Splats, cams, counts=True):
        P = self.params
        P.sh_degree = splats.sh_degree
        R = len(cams) * splats.n
        for t, nm in zip(splats.tensors(), ("means", "scales", "quats", "opac", "sh")):
            _dev_check(t, nm)
        proj = torch.empty(N.lib().ls_proj_bytes(R) // 4 or 1, dtype=torch.float32, device=self.device)
        tc = torch.empty(max(R, 1), dtype=torch.int32, device=self.device) if counts else None
        ca = cam_array(cams)
        N.check(N.lib().ls_project(splats.n, _p(splats.means), _p(splats.scales), _p(splats.quats), _p(splats.opac),
                                   _p(splats.sh), ca, len(cams), ctypes.byref(P.c()), _p(proj), _p(tc),
                                   _p(self.status), _stream()), "ls_project")
        return proj, tc

    def ensure_capacity(self, tile_counts):
        """Size the key buffers from the support-box tile count, an upper bound
        on the keys (one device->host read)."""
        K = int(tile_counts.sum(dtype=torch.int64).item())
        if K > self.capacity:
            self.capacity = int(math.ceil(K * self.grow_margin)) + 1024
        return K

    def duplicate_sort(self, proj, R, cams, capacity=None):
        P = self.params
        cap = int(capacity if capacity is not None else self.capacity)
        total_tiles = sum(tiles_of(c, P) for c in cams)
        keys = self._buf("keys", 4 * max(cap, 1), torch.int32)
        vals = self._buf("vals", 4 * max(cap, 1), torch.int32)
        n_keys = torch.empty(1, dtype=torch.int64, device=self.device)  # written by the call
        ranges = torch.empty(2 * total_tiles, dtype=torch.int32, device=self.device)
        wsb = N.lib().ls_duplicate_sort_workspace(R, cap, total_tiles)
        ws = self._buf("dup_ws", wsb + 256)
        ws_ptr = (ws.data_ptr() + 255) // 256 * 256
        ca = cam_array(cams)
        N.check(N.lib().ls_duplicate_sort(R, _p(proj), ca, len(cams), ctypes.byref(P.c()), cap, _p(keys), _p(vals),
                                          _p(n_keys), _p(ranges), ctypes.c_void_p(ws_ptr), wsb, _p(self.status),
                                          _stream()), "ls_duplicate_sort")
        return keys, vals, n_keys, ranges

    def render_fwd(self, proj, R, cam, ranges, vals):
        P = self.params
        H, W = cam["height"], cam["width"]
        image = torch.empty((H, W, 3), dtype=torch.float32, device=self.device)
        T = torch.empty((H, W), dtype=torch.float32, device=self.device)
        n_last = torch.empty((H, W), dtype=torch.int32, device=self.device)
        N.check(N.lib().ls_render_fwd(_p(proj), R, ctypes.byref(cam_struct(cam)), ctypes.byref(P.c()), _p(ranges),
                                      _p(vals), _p(image), _p(T), _p(n_last), _p(self.status), _stream()),
                "ls_render_fwd")
        return image, T, n_last

    def render_stats(self, proj, R, cam, ranges, vals, labels=None):
        """Forward blend that also returns (evaluated pairs, composited pairs);
        with `labels` (float [tiles]) also each tile's termination depth."""
        P = self.params
        H, W = cam["height"], cam["width"]
        image = torch.empty((H, W, 3), dtype=torch.float32, device=self.device)
        T = torch.empty((H, W), dtype=torch.float32, device=self.device)
        n_last = torch.empty((H, W), dtype=torch.int32, device=self.device)
        stats = torch.zeros(2, dtype=torch.int64, device=self.device)
        N.check(N.lib().ls_render_stats(_p(proj), R, ctypes.byref(cam_struct(cam)), ctypes.byref(P.c()), _p(ranges),
                                        _p(vals), _p(image), _p(T), _p(n_last), _p(stats), _p(labels),
                                        _p(self.status), _stream()), "ls_render_stats")
        s = stats.cpu().tolist()
        return image, T, n_last, int(s[0]), int(s[1])

    def tile_features(self, proj, R, cam):
        """MLP inputs [tiles, 48] (fp16) and keys per tile [tiles] (int32)."""
        P = self.params
        nt = tiles_of(cam, P)
        x = torch.empty((nt, 48), dtype=torch.float16, device=self.device)
        total = torch.empty(nt, dtype=torch.int32, device=self.device)
        c, pc = cam_struct(cam), P.c()
        wsb = N.lib().ls_tile_features_workspace(ctypes.byref(c), ctypes.byref(pc))
        ws = self._buf("feat_ws", wsb + 256)
        ws_ptr = (ws.data_ptr() + 255) // 256 * 256
        N.check(N.lib().ls_tile_features(_p(proj), R, ctypes.byref(c), ctypes.byref(pc), _p(x), _p(total),
                                         ctypes.c_void_p(ws_ptr), wsb, _stream()), "ls_tile_features")
        return x, total

    def blend_bwd(self, proj, R, cam, ranges, vals, T, n_last, grad_image, grad_T, g2d):
        """a5 alone: accumulates into g2d [R, 12] (zero it first)."""
        N.check(N.lib().ls_blend_bwd(_p(proj), R, ctypes.byref(cam_struct(cam)), ctypes.byref(self.params.c()),
                                     _p(ranges), _p(vals), _p(T), _p(n_last), _p(grad_image), _p(grad_T), _p(g2d),
                                     _p(self.status), _stream()), "ls_blend_bwd")

    def tile_order(self, cam, n_last):
        """Longest-first order of the camera's tiles for the backward blend
        (ls_tile_order): uint32 [tiles]."""
        c, pc = cam_struct(cam), self.params.c()
        order = torch.empty(tiles_of(cam, self.params), dtype=torch.int32, device=self.device)
        wsb = N.lib().ls_tile_order_workspace(ctypes.byref(c), ctypes.byref(pc))
        ws = self._buf("order_ws", wsb + 256)
        ws_ptr = (ws.data_ptr() + 255) // 256 * 256
        N.check(N.lib().ls_tile_order(_p(n_last), ctypes.byref(c), ctypes.byref(pc), _p(order), ctypes.c_void_p(ws_ptr),
                                      wsb, _stream()), "ls_tile_order")
        return order

    def blend_bwd_ordered(self, proj, R, cam, ranges, order, vals, T, n_last, grad_image, grad_T, g2d):
        """a5 alone with tile b of the launch = order[b] (ls_blend_bwd_ordered)."""
        N.check(N.lib().ls_blend_bwd_ordered(_p(proj), R, ctypes.byref(cam_struct(cam)), ctypes.byref(self.params.c()),
                                             _p(ranges), _p(order), _p(vals), _p(T), _p(n_last), _p(grad_image),
                                             _p(grad_T), _p(g2d), _p(self.status), _stream()), "ls_blend_bwd_ordered")

    def project_bwd(self, splats: Splats, cams, proj, g2d, out=None):
        """a6 alone: 3D gradients from g2d (overwritten into `out` when given)."""
        g = out or dict(means=torch.empty_like(splats.means), scales=torch.empty_like(splats.scales),
                        quats=torch.empty_like(splats.quats), opac=torch.empty_like(splats.opac),
                        sh=torch.empty_like(splats.sh))
        N.check(N.lib().ls_project_bwd(splats.n, _p(splats.means), _p(splats.scales), _p(splats.quats),
                                       _p(splats.opac), _p(splats.sh), cam_array(cams), len(cams),
                                       ctypes.byref(self.params.c()), _p(proj), _p(g2d), _p(g["means"]),
                                       _p(g["scales"]), _p(g["quats"]), _p(g["opac"]), _p(g["sh"]), _p(self.status),
                                       _stream()), "ls_project_bwd")
        return g

    def render_bwd(self, splats: Splats, cam, state, grad_image, grad_T=None, want_g2d=False, out=None):
        """a5 + a6 in one ls_render_bwd call (the 2D gradient buffer is
        cleared inside the library); 3D gradients into `out` when given."""
        P = self.params
        n = splats.n
        grad_image = grad_image.contiguous()
        if grad_T is not None:
            grad_T = grad_T.contiguous()
        g = out or dict(means=torch.empty_like(splats.means), scales=torch.empty_like(splats.scales),
                        quats=torch.empty_like(splats.quats), opac=torch.empty_like(splats.opac),
                        sh=torch.empty_like(splats.sh))
        g2d = torch.empty((n, 12), dtype=torch.float32, device=self.device) if want_g2d else None
        c, pc = cam_struct(cam), P.c()
        wsb = 0
        if self.bwd_tile_order:  # room for the longest-first tile order of the backward blend
            wsb = N.lib().ls_render_bwd_workspace_ordered(n, ctypes.byref(c), ctypes.byref(pc))
        wsb = wsb or N.lib().ls_render_bwd_workspace(n)
        ws = self._buf("bwd_ws", wsb + 256)
        ws_ptr = (ws.data_ptr() + 255) // 256 * 256
        N.check(N.lib().ls_render_bwd(n, _p(splats.means), _p(splats.scales), _p(splats.quats), _p(splats.opac),
                                      _p(splats.sh), ctypes.byref(c), ctypes.byref(pc),
                                      _p(state["proj"]), _p(state["ranges"]), _p(state["vals"]), _p(state["T"]),
                                      _p(state["n_last"]), _p(grad_image), _p(grad_T), _p(g["means"]),
                                      _p(g["scales"]), _p(g["quats"]), _p(g["opac"]), _p(g["sh"]), _p(g2d),
                                      ctypes.c_void_p(ws_ptr), wsb, _p(self.status), _stream()), "ls_render_bwd")
        if want_g2d:
            g["g2d"] = g2d
        return g

    # ---------------------------------------------------------------- frames
    def forward(self, splats: Splats, cam, sync_capacity=True):
        """One camera, one frame: returns image [H, W, 3], T [H, W] and the
        state the backward pass needs."""
        proj, tc = self.project(splats, [cam], counts=True)
        R = splats.n
        if sync_capacity or self.capacity == 0:
            self.ensure_capacity(tc)
        keys, vals, n_keys, ranges = self.duplicate_sort(proj, R, [cam])
        image, T, n_last = self.render_fwd(proj, R, cam, ranges, vals)
        state = dict(proj=proj, tile_counts=tc, keys=keys, vals=vals, n_keys=n_keys, ranges=ranges, T=T,
                     n_last=n_last)
        return image, T, state



class FrameGraph:
    """One camera's frame recorded once in a CUDA graph and replayed.

    The recorded calls are the boundary calls of a frame: ls_project,
    ls_duplicate_sort, ls_render_fwd and, with `grad_image`, ls_render_bwd.
    None of them reads a value back to the host (the key count stays on the
    device), so a replay redoes the whole frame on whatever the parameter
    tensors hold at that moment: update them in place between replays (as
    Adam does) and never rebind them.  The outputs live in the graph's own
    memory and are overwritten by every replay (they hold nothing before the
    first): `image`, `T`, `n_keys` and, with a backward, the 3D gradients in
    `grads`.  The key capacity is the
    rasterizer's at capture time; a frame that needs more keys sets
    LS_ERR_CAPACITY in the status word (check it, grow the capacity and
    capture again).  Replaying saves the host launch work and the gaps
    between the frame's ~20 kernels.
    """

    def __init__(self, rasterizer: Rasterizer, splats: Splats, cam, grad_image=None, grad_T=None):
        if rasterizer.device.type != "cuda":
            raise RuntimeError("FrameGraph needs a CUDA device")
        self.rz, self.splats, self.cam = rasterizer, splats, cam
        self.grad_image, self.grad_T = grad_image, grad_T
        self.grads = None
        if grad_image is not None:
            self.grads = dict(means=torch.empty_like(splats.means), scales=torch.empty_like(splats.scales),
                              quats=torch.empty_like(splats.quats), opac=torch.empty_like(splats.opac),
                              sh=torch.empty_like(splats.sh))
        if rasterizer.capacity == 0:
            _, tc = rasterizer.project(splats, [cam], counts=True)
            rasterizer.ensure_capacity(tc)
        dev = rasterizer.device
        self._frame()  # eager once: sets the kernels' shared-memory limits and sizes the scratch
        torch.cuda.synchronize(dev)
        rasterizer.check_status("FrameGraph eager frame")
        self.graph = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(device=dev)
        s.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(s):
            with torch.cuda.graph(self.graph, stream=s):
                self.image, self.T, self.n_keys = self._frame()
        torch.cuda.current_stream(dev).wait_stream(s)

    def _frame(self):
        rz, sp, cam = self.rz, self.splats, self.cam
        proj, _ = rz.project(sp, [cam], counts=False)
        keys, vals, n_keys, ranges = rz.duplicate_sort(proj, sp.n, [cam])
        image, T, n_last = rz.render_fwd(proj, sp.n, cam, ranges, vals)
        if self.grads is not None:
            state = dict(proj=proj, ranges=ranges, vals=vals, T=T, n_last=n_last)
            rz.render_bwd(sp, cam, state, self.grad_image, self.grad_T, out=self.grads)
        return image, T, n_keys

    def replay(self):
        """Launch the recorded frame on the current stream."""
        self.graph.replay()
        return self.image, self.T


class LinearSplatFn(torch.autograd.Function):
    """Differentiable render of one camera: (means, scales, quats, opacities,
    sh[K*3, N]) -> (image [H, W, 3], T [H, W]).  The backward recomputes
    transmittance from the forward's checkpoint (T_final, n_last)."""

    @staticmethod
    def forward(ctx, means, scales, quats, opac, sh, cam, rasterizer, sh_degree):
        sp = Splats(means.contiguous(), scales.contiguous(), quats.contiguous(), opac.contiguous(), sh.contiguous(),
                    sh_degree)
        image, T, state = rasterizer.forward(sp, cam)
        ctx.rasterizer = rasterizer
        ctx.cam = cam
        ctx.sh_degree = sh_degree
        ctx.state = state
        ctx.save_for_backward(sp.means, sp.scales, sp.quats, sp.opac, sp.sh)
        return image, T

    @staticmethod
    def backward(ctx, g_image, g_T):
        means, scales, quats, opac, sh = ctx.saved_tensors
        sp = Splats(means, scales, quats, opac, sh, ctx.sh_degree)
        if g_image is None:
            g_image = torch.zeros((ctx.cam["height"], ctx.cam["width"], 3), device=means.device)
        g = ctx.rasterizer.render_bwd(sp, ctx.cam, ctx.state, g_image, g_T)
        return g["means"], g["scales"], g["quats"], g["opac"], g["sh"], None, None, None


def render(splats: Splats, cam, rasterizer: Rasterizer):
    """Differentiable render through LinearSplatFn."""
    return LinearSplatFn.apply(splats.means, splats.scales, splats.quats, splats.opac, splats.sh, cam, rasterizer,
                               splats.sh_degree)
