"""Host-side checks that need no GPU: libls.so builds for sm_103a, loads, and
exports every entry point include/ls.h declares; host argument checks reject
bad calls before anything is launched; struct layouts match the header."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2411_12440_gb300 import build, _native
    build.build()
    return _native.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "ls.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(ls_[a-z_0-9]+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), n


def test_prototypes_cover_header():
    from paper_2411_12440_gb300 import _native
    assert set(_declared()) <= set(_native.PROTOTYPES)


def test_struct_layouts_match_header(L, tmp_path):
    """ctypes mirrors have the size and field offsets gcc gives the C structs."""
    import subprocess
    from paper_2411_12440_gb300 import _native as N
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "ls.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\\n", sizeof(ls_params), offsetof(ls_params, bg), offsetof(ls_params, sh_degree),
         sizeof(ls_camera), offsetof(ls_camera, width));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert got == [ctypes.sizeof(N.LsParams), N.LsParams.bg.offset, N.LsParams.sh_degree.offset,
                   ctypes.sizeof(N.LsCamera), N.LsCamera.width.offset]


def test_version_and_status_strings(L):
    assert L.ls_version() == 1
    assert L.ls_status_string(3) == b"tile-key capacity exceeded"
    assert L.ls_status_string(99) == b"unknown status"
    assert L.ls_proj_bytes(10) == 680


def test_workspace_queries(L):
    a = L.ls_duplicate_sort_workspace(1000, 10000, 256)
    b = L.ls_duplicate_sort_workspace(1000, 20000, 256)
    assert 0 < a < b
    assert L.ls_duplicate_sort_workspace(-1, 10, 10) == 0
    assert L.ls_render_bwd_workspace(1000) >= 48000


def test_host_argument_checks_reject_before_launch(L):
    """Invalid parameters return LS_ERR_INVALID_ARG without touching the GPU
    (the pointers below are never dereferenced)."""
    from paper_2411_12440_gb300 import raster
    from paper_2411_12440_gb300 import scenes
    cam = raster.cam_struct(scenes.identity_camera(64, 64))
    bad = [raster.RenderParams(lam=0.0), raster.RenderParams(tile_w=12), raster.RenderParams(sh_degree=4),
           raster.RenderParams(alpha_max=1.0), raster.RenderParams(kernel=7), raster.RenderParams(near=2, far=1)]
    fake = ctypes.c_void_p(16)
    for p in bad:
        r = L.ls_project(10, fake, fake, fake, fake, fake, ctypes.byref(cam), 1, ctypes.byref(p.c()), fake, None,
                         None, None)
        assert r == 1, p
    good = raster.RenderParams()
    # no cameras / too many cameras
    assert L.ls_project(10, fake, fake, fake, fake, fake, ctypes.byref(cam), 0, ctypes.byref(good.c()), fake, None,
                        None, None) == 1
    assert L.ls_project(10, fake, fake, fake, fake, fake, ctypes.byref(cam), 65, ctypes.byref(good.c()), fake, None,
                        None, None) == 1
    # misaligned quaternion pointer
    assert L.ls_project(10, fake, fake, ctypes.c_void_p(20), fake, fake, ctypes.byref(cam), 1,
                        ctypes.byref(good.c()), fake, None, None, None) == 1
    # zero-size camera
    c2 = raster.cam_struct(dict(scenes.identity_camera(64, 64), width=0))
    assert L.ls_render_fwd(fake, 10, ctypes.byref(c2), ctypes.byref(good.c()), fake, fake, fake, fake, fake, None,
                           None) == 1
    # workspace too small
    assert L.ls_duplicate_sort(100, fake, ctypes.byref(cam), 1, ctypes.byref(good.c()), 1000, fake, fake, fake, fake,
                               ctypes.c_void_p(256), 10, None, None) == 1
    # records not a multiple of the camera count
    cams2 = raster.cam_array([scenes.identity_camera(64, 64)] * 2)
    assert L.ls_duplicate_sort(101, fake, cams2, 2, ctypes.byref(good.c()), 1000, fake, fake, fake, fake,
                               ctypes.c_void_p(256), 1 << 30, None, None) == 1
    # empty problem is valid and launches nothing
    assert L.ls_project(0, None, None, None, None, None, ctypes.byref(cam), 1, ctypes.byref(good.c()), None, None,
                        None, None) == 0


def test_noalloc_rejects_bad_cameras_and_tiles_before_any_arithmetic(L):
    """ls_duplicate_sort_noalloc applies ls_duplicate_sort's own camera and
    parameter rules before it counts tiles: a width near INT_MAX or a tile
    shape outside {8x8, 16x16, 32x16} is an invalid argument, not an
    overflow."""
    from paper_2411_12440_gb300 import raster, scenes
    fake = ctypes.c_void_p(16)
    good = raster.RenderParams()
    huge = raster.cam_array([dict(scenes.identity_camera(64, 64), width=2 ** 31 - 1)])
    assert L.ls_duplicate_sort_noalloc(10, fake, huge, 1, ctypes.byref(good.c()), 100, fake, fake, fake, fake, None,
                                       None) == 1
    cam = raster.cam_array([scenes.identity_camera(64, 64)])
    odd = raster.RenderParams(tile_w=12, tile_h=12)
    assert L.ls_duplicate_sort_noalloc(10, fake, cam, 1, ctypes.byref(odd.c()), 100, fake, fake, fake, fake, None,
                                       None) == 1
    # beyond the static scratch: unsupported, still before any launch
    assert L.ls_duplicate_sort_noalloc(70_000, fake, cam, 1, ctypes.byref(good.c()), 100, fake, fake, fake, fake,
                                       None, None) == 5


def test_debug_sort_wait_setter_checks_arguments(L):
    assert L.ls_debug_set_sort_wait(-1, -1) == 1
    assert L.ls_debug_set_sort_wait(0, -2) == 1
    assert L.ls_debug_set_sort_wait(1000, 0) == 0
    assert L.ls_debug_set_sort_wait(0, -1) == 0  # defaults again


def test_ordered_backward_workspace_size(L):
    from paper_2411_12440_gb300 import raster, scenes
    cam = raster.cam_struct(scenes.identity_camera(100, 60))
    good, odd = raster.RenderParams(), raster.RenderParams(tile_w=12, tile_h=12)
    plain = L.ls_render_bwd_workspace(1000)
    ordered = L.ls_render_bwd_workspace_ordered(1000, ctypes.byref(cam), ctypes.byref(good.c()))
    tiles = 7 * 4  # 100 x 60 pixels in 16 x 16 tiles
    assert ordered == plain + 768 + 2 * 256 and tiles * 4 <= 256
    assert L.ls_render_bwd_workspace_ordered(1000, ctypes.byref(cam), ctypes.byref(odd.c())) == 0
    assert L.ls_render_bwd_workspace_ordered(-1, ctypes.byref(cam), ctypes.byref(good.c())) == 0


def test_dependent_launch_switch_checks_arguments(L):
    assert L.ls_set_dependent_launch(2) == 1 and L.ls_set_dependent_launch(-1) == 1
    assert L.ls_set_dependent_launch(0) == 0
    assert L.ls_set_dependent_launch(1) == 0  # the default again


def test_training_entry_points_reject_bad_arguments_before_launch(L):
    """The loss, Adam, densification and 3D-filter entry points check their
    arguments on the host (no pointer is dereferenced here)."""
    from paper_2411_12440_gb300 import _native as N
    from paper_2411_12440_gb300 import raster, scenes
    fake = ctypes.c_void_p(256)
    assert L.ls_image_loss_workspace(0, 10) == 0 and L.ls_image_loss_workspace(10, 20000) == 0
    assert L.ls_image_loss_workspace(10, 20) > 0
    ws = L.ls_image_loss_workspace(10, 20)
    assert L.ls_image_loss(0, 20, fake, fake, 0.6, 0.2, 0.2, fake, fake, fake, ws, None) == 1
    assert L.ls_image_loss(10, 20, None, fake, 0.6, 0.2, 0.2, fake, fake, fake, ws, None) == 1
    assert L.ls_image_loss(10, 20, fake, fake, float("nan"), 0.2, 0.2, fake, fake, fake, ws, None) == 1
    assert L.ls_image_loss(10, 20, fake, fake, 0.6, 0.2, 0.2, fake, fake, fake, ws - 1, None) == 1
    assert L.ls_image_loss(10, 20, fake, fake, 0.6, 0.2, 0.2, fake, fake, ctypes.c_void_p(300), ws, None) == 1
    assert L.ls_adam(10, fake, fake, fake, fake, 0, 1e-3, 0.9, 0.999, 1e-15, 0, None) == 1  # step 0
    assert L.ls_adam(10, fake, fake, fake, fake, 1, 1e-3, 0.9, 0.999, 1e-15, 3, None) == 1  # mode 3
    assert L.ls_adam(10, fake, fake, fake, fake, 1, 1e-3, 1.0, 0.999, 1e-15, 0, None) == 1  # beta1 1
    assert L.ls_adam(0, None, None, None, None, 1, 1e-3, 0.9, 0.999, 1e-15, 0, None) == 0  # nothing to do
    cam = raster.cam_struct(scenes.identity_camera(64, 64))
    assert L.ls_densify_accumulate(10, fake, fake, ctypes.byref(cam), 0, fake, fake, fake, None) == 1
    assert L.ls_densify_accumulate(10, fake, ctypes.c_void_p(260), ctypes.byref(cam), 1, fake, fake, fake,
                                   None) == 1  # misaligned records
    p = N.LsDensifyParams()
    assert L.ls_densify_decide(10, fake, fake, fake, fake, fake, 0.0, ctypes.byref(p), fake, None, None) == 1
    assert L.ls_densify_decide(10, fake, fake, fake, fake, fake, 1.0, None, fake, None, None) == 1
    cams = raster.cam_array([scenes.identity_camera(64, 64)])
    wsf = L.ls_filter3d_workspace()
    assert L.ls_filter3d_variance(10, fake, cams, 1, 0.0, 0.2, fake, fake, wsf, None) == 1  # near 0
    assert L.ls_filter3d_variance(10, fake, cams, 0, 0.2, 0.2, fake, fake, wsf, None) == 1  # no camera
    assert L.ls_filter3d_variance(10, fake, cams, 1, 0.2, 0.2, fake, ctypes.c_void_p(300), wsf, None) == 1
    assert L.ls_filter3d_apply(-1, fake, fake, fake, fake, fake, None) == 1
    assert L.ls_filter3d_apply_bwd(10, fake, None, fake, fake, fake, fake, fake, None) == 1
    assert L.ls_filter3d_apply(0, None, None, None, None, None, None) == 0
