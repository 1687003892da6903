"""GPU tests of the batched multi-camera render (ls_render_batch): every
camera's image equals the single-camera render bit for bit (same lists, same
per-pixel operation order) and the oracle within the image tolerance; the
CUDA-graph replay equals the eager call and follows in-place parameter
updates; the autotuner returns a measured candidate."""
import numpy as np
import pytest
import torch

import oracle
from paper_2411_12440_gb300 import raster, scenes
from paper_2411_12440_gb300.batch import Autotuner, BatchRenderer
from tests.gpu_helpers import assert_image_parity

pytestmark = pytest.mark.gpu


def _scene_and_cams(n=20_000, n_cams=5, seed=2):
    scene = scenes.cluster_scene(n, seed, 3)
    cams = scenes.ring_cameras(n_cams, seed, w_range=(96, 333), h_range=(64, 250))
    return scene, cams


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 16)])
def test_batch_equals_single_camera_bitwise(tile):
    scene, cams = _scene_and_cams()
    sp = raster.Splats.from_scene(scene)
    P = raster.RenderParams(sh_degree=3, tile_w=tile[0], tile_h=tile[1], bg=(0.1, 0.2, 0.3))
    br = BatchRenderer(sp, cams, P)
    br.render_eager()
    torch.cuda.synchronize()
    br.check()
    for c, cam in enumerate(cams):
        rz = raster.Rasterizer(raster.RenderParams.from_dict(vars(P)))
        img, T, _ = rz.forward(sp, cam)
        assert torch.equal(br.image(c), img), c


def test_batch_matches_oracle():
    scene, cams = _scene_and_cams(n=8000, n_cams=3, seed=7)
    sp = raster.Splats.from_scene(scene)
    P = dict(sh_degree=3)
    br = BatchRenderer(sp, cams, raster.RenderParams.from_dict(P), blend_batch=64)
    br.render_eager()
    torch.cuda.synchronize()
    br.check()
    for c, cam in enumerate(cams):
        ref = oracle.render_scene(scene, cam, P)
        assert_image_parity(br.image(c).cpu().numpy(), ref)


def test_batch_graph_replay_follows_parameter_updates():
    scene, cams = _scene_and_cams(n=10_000, n_cams=4, seed=3)
    sp = raster.Splats.from_scene(scene)
    br = BatchRenderer(sp, cams, raster.RenderParams(sh_degree=3), blend_batch=128)
    br.plan()
    br.capture()
    br.render()
    torch.cuda.synchronize()
    a = br.images.clone()
    br.render_eager()
    torch.cuda.synchronize()
    assert torch.equal(a, br.images)
    # same buffers, new values: the replay renders the new scene
    with torch.no_grad():
        sp.opac.mul_(0.5)
        sp.means.add_(0.01)
    br.render()
    torch.cuda.synchronize()
    b = br.images.clone()
    br.render_eager()
    torch.cuda.synchronize()
    br.check()
    assert torch.equal(b, br.images)
    assert not torch.equal(a, b)


def test_batch_capacity_overflow_is_reported():
    scene, cams = _scene_and_cams(n=5000, n_cams=2, seed=5)
    sp = raster.Splats.from_scene(scene)
    br = BatchRenderer(sp, cams, raster.RenderParams(sh_degree=3))
    br.plan()
    br.render_eager()
    torch.cuda.synchronize()
    br.check()
    K = int(br.n_keys.item())
    assert 0 < K <= br.count_keys()
    br.plan(capacity=K - 1)
    br.render_eager()
    torch.cuda.synchronize()
    assert int(br.status.item()) == 3 and int(br.n_keys.item()) == K
    br.status.zero_()
    br.plan(capacity=K)
    br.render_eager()
    torch.cuda.synchronize()
    br.check()


def test_autotuner_picks_a_measured_candidate():
    scene, cams = _scene_and_cams(n=20_000, n_cams=4, seed=9)
    sp = raster.Splats.from_scene(scene)
    res = Autotuner(batches=(32, 128), reps=2).tune(sp, cams, raster.RenderParams(sh_degree=3))
    assert (res.tile[0], res.tile[1], res.blend_batch) in res.table
    assert res.ms == min(res.table.values())
    assert len(res.table) == 6


def test_batch_blend_only_reproduces_the_call():
    """ls_render_batch_blend re-runs the blending stage on what the last
    ls_render_batch left in the workspace: the same images bit for bit."""
    scene, cams = _scene_and_cams(n=8000, n_cams=3, seed=5)
    sp = raster.Splats.from_scene(scene)
    br = BatchRenderer(sp, cams, raster.RenderParams(sh_degree=3), blend_batch=64)
    br.render_eager()
    torch.cuda.synchronize()
    br.check()
    a = br.images.clone()
    br.images.zero_()
    br.blend_only()
    torch.cuda.synchronize()
    br.check()
    assert torch.equal(br.images, a)
