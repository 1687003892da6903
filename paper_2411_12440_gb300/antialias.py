"""The anti-aliased variant's 3D smoothing filter (Sec. 4.1, "3DLS+AA", with
the anti-aliasing of Mip-Splatting): per-primitive filter variances from the
training cameras (ls_filter3d_variance), filtered scales and opacities fed to
the rasterizer (ls_filter3d_apply) and the chain rule back
(ls_filter3d_apply_bwd).  The 2D filter is RenderParams.antialias.
Argument marshalling only."""
from __future__ import annotations

import ctypes

import torch

from . import _native as N
from .raster import Splats, _p, _stream, cam_array

FILTER3D_S2 = 0.2


class Filter3D:
    """Filter variances of a set of primitives for a set of cameras."""

    def __init__(self, splats: Splats, cams, near=0.2, s2=FILTER3D_S2):
        self.n = splats.n
        dev = splats.means.device
        self.var = torch.empty(self.n, dtype=torch.float32, device=dev)
        ws = torch.empty(N.lib().ls_filter3d_workspace() + 256, dtype=torch.uint8, device=dev)
        self._ws = ws
        wp = ctypes.c_void_p((ws.data_ptr() + 255) // 256 * 256)
        N.check(N.lib().ls_filter3d_variance(self.n, _p(splats.means), cam_array(cams), len(cams), float(near),
                                             float(s2), _p(self.var), wp, N.lib().ls_filter3d_workspace(), _stream()),
                "ls_filter3d_variance")

    def apply(self, splats: Splats) -> Splats:
        """The primitives as the rasterizer sees them (new scale and opacity
        tensors; means, rotations and SH shared)."""
        s = torch.empty_like(splats.scales)
        o = torch.empty_like(splats.opac)
        N.check(N.lib().ls_filter3d_apply(self.n, _p(splats.scales), _p(splats.opac), _p(self.var), _p(s), _p(o),
                                          _stream()), "ls_filter3d_apply")
        return Splats(splats.means, s, splats.quats, o, splats.sh, splats.sh_degree)

    def backward(self, splats: Splats, g_scales_f, g_opac_f):
        """Gradients of the unfiltered scales and opacities."""
        gs = torch.empty_like(splats.scales)
        go = torch.empty_like(splats.opac)
        N.check(N.lib().ls_filter3d_apply_bwd(self.n, _p(splats.scales), _p(splats.opac), _p(self.var),
                                              _p(g_scales_f), _p(g_opac_f), _p(gs), _p(go), _stream()),
                "ls_filter3d_apply_bwd")
        return gs, go
