"""ls_duplicate_sort_noalloc: the duplication + sort stage for callers that
cannot allocate device memory (a plugin inside a host application that owns
every device allocation, a real-time loop that must not allocate, a small C
program that links only libls.so).  It keeps its scratch in one static device
array instead of a caller-supplied workspace.

Called through the C ABI and checked against ls_duplicate_sort, which takes a
workspace: integer results, so bit-exact, on two calls in a row (the static
scratch keeps the previous call's contents, which must not leak into the
next).  This file is collected last so a run that stops at the first failure
has already run every other test; it also passes on its own.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2411_12440_gb300 import _native as N
from paper_2411_12440_gb300 import raster, scenes
from tests.gpu_helpers import pack_records

pytestmark = pytest.mark.gpu

MAX_RECORDS = 65536
MAX_KEYS = 524288


def _noalloc(proj, R, cams, params, cap):
    keys = torch.zeros(max(cap, 1), dtype=torch.int32, device="cuda")
    vals = torch.zeros(max(cap, 1), dtype=torch.int32, device="cuda")
    n_keys = torch.zeros(1, dtype=torch.int64, device="cuda")
    total = sum(raster.tiles_of(c, params) for c in cams)
    ranges = torch.zeros(2 * total, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    code = N.lib().ls_duplicate_sort_noalloc(R, raster._p(proj), raster.cam_array(cams), len(cams),
                                             ctypes.byref(params.c()), cap, raster._p(keys), raster._p(vals),
                                             raster._p(n_keys), raster._p(ranges), raster._p(status),
                                             raster._stream())
    torch.cuda.synchronize()
    return code, keys, vals, n_keys, ranges, status


def _with_workspace(proj, R, cams, params, cap):
    rz = raster.Rasterizer(params)
    keys, vals, n_keys, ranges = rz.duplicate_sort(proj, R, cams, capacity=cap)
    torch.cuda.synchronize()
    rz.check_status()
    return keys, vals, n_keys, ranges


@pytest.mark.parametrize("tile", [(16, 16), (8, 8)])
def test_noalloc_matches_workspace_entry_point_twice(tile):
    params = raster.RenderParams(tile_w=tile[0], tile_h=tile[1])
    W, H = 640, 400
    cam = scenes.identity_camera(W, H)
    # two different inputs in a row: the second must not see the first's scratch
    for seed, R in ((31, 20_000), (32, 7_001)):
        rec = scenes.random_records(R, W, H, seed=seed, max_ext=30)
        proj, _ = pack_records(rec)
        k_ref, v_ref, n_ref, r_ref = _with_workspace(proj, R, [cam], params, MAX_KEYS)
        K = int(n_ref.item())
        assert 0 < K <= MAX_KEYS
        code, keys, vals, n_keys, ranges, status = _noalloc(proj, R, [cam], params, MAX_KEYS)
        assert code == 0
        assert int(status.item()) == 0
        assert int(n_keys.item()) == K
        assert torch.equal(keys[:K], k_ref[:K])
        assert torch.equal(vals[:K], v_ref[:K])
        assert torch.equal(ranges, r_ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    params = raster.RenderParams()
    cam = scenes.identity_camera(64, 64)
    fake = ctypes.c_void_p(256)
    L = N.lib()
    too_many_records = L.ls_duplicate_sort_noalloc(MAX_RECORDS + 1, fake, raster.cam_array([cam]), 1,
                                                   ctypes.byref(params.c()), 1000, fake, fake, fake, fake, None,
                                                   raster._stream())
    too_many_keys = L.ls_duplicate_sort_noalloc(1000, fake, raster.cam_array([cam]), 1, ctypes.byref(params.c()),
                                                MAX_KEYS + 1, fake, fake, fake, fake, None, raster._stream())
    assert too_many_records == 5 and too_many_keys == 5  # LS_ERR_UNSUPPORTED, nothing enqueued
