"""GPU tests of ls_copy, the host-link copy of end-to-end steps: pinned host
to device and back is exact at odd sizes, and pageable host memory is
refused before anything is enqueued."""
import ctypes

import pytest
import torch

from paper_2411_12440_gb300 import _native as N
from paper_2411_12440_gb300 import raster

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 7, 4096 + 3, 3_000_001])
def test_pinned_round_trip_is_exact(n):
    g = torch.Generator().manual_seed(n)
    h = torch.randint(0, 256, (n,), dtype=torch.uint8, generator=g).pin_memory()
    d = torch.empty(n, dtype=torch.uint8, device="cuda")
    back = torch.empty(n, dtype=torch.uint8).pin_memory()
    raster.copy_(d, h)
    raster.copy_(back, d)
    torch.cuda.synchronize()
    assert torch.equal(back, h)
    assert torch.equal(d.cpu(), h)


def test_pageable_host_memory_is_refused():
    h = torch.zeros(1024, dtype=torch.float32)  # not pinned
    d = torch.ones(1024, dtype=torch.float32, device="cuda")
    code = N.lib().ls_copy(ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(h.data_ptr()), 4096, None)
    torch.cuda.synchronize()
    assert code == 1  # LS_ERR_INVALID_ARG
    assert bool((d == 1).all())
