"""GPU tests of FrameGraph, a frame's boundary calls (ls_project,
ls_duplicate_sort, ls_render_fwd, ls_render_bwd) recorded in one CUDA graph:
a replay gives the eager frame's image bit for bit and its gradients up to
the order of the float atomics, follows in-place parameter updates (the key
count included), and a frame that outgrows the captured key capacity reports
LS_ERR_CAPACITY instead of writing past it.  The frame's kernels give the
same results launched plainly and with programmatic dependent launch."""
import numpy as np
import pytest
import torch

from paper_2411_12440_gb300 import raster, scenes
from tests.gpu_helpers import log_parity

pytestmark = pytest.mark.gpu


def _setup(n=12_000, seed=4, W=320, H=200):
    scene = scenes.cluster_scene(n, seed, 3)
    cam = scenes.ring_cameras(1, seed, w_range=(W, W + 1), h_range=(H, H + 1))[0]
    sp = raster.Splats.from_scene(scene)
    w, v = scenes.loss_weights(cam["height"], cam["width"], seed=seed + 1)
    return sp, cam, torch.from_numpy(w).cuda(), torch.from_numpy(v).cuda()


def _eager(sp, cam, gimg, gT, P):
    rz = raster.Rasterizer(P)
    img, T, st = rz.forward(sp, cam)
    g = rz.render_bwd(sp, cam, st, gimg, gT)
    torch.cuda.synchronize()
    rz.check_status("eager")
    return img, T, g, int(st["n_keys"].item())


def _rel(a, b):
    return float((a - b).norm() / max(float(b.norm()), 1e-30))


def test_frame_graph_replay_equals_eager_frame():
    sp, cam, gimg, gT = _setup()
    P = raster.RenderParams(sh_degree=3, bg=(0.1, 0.2, 0.3))
    img0, T0, g0, nk0 = _eager(sp, cam, gimg, gT, P)
    fg = raster.FrameGraph(raster.Rasterizer(P), sp, cam, gimg, gT)
    for _ in range(2):
        img, T = fg.replay()
        torch.cuda.synchronize()
        fg.rz.check_status("replay")
        assert torch.equal(img, img0) and torch.equal(T, T0)
        assert int(fg.n_keys.item()) == nk0
        rels = {k: _rel(fg.grads[k], g0[k]) for k in g0}
        log_parity("replay_vs_eager_grad_rel_l2", **rels)
        for k, r in rels.items():  # float atomics add in another order
            assert r < 1e-4, k


def test_frame_graph_follows_parameter_updates():
    sp, cam, gimg, gT = _setup(seed=6)
    P = raster.RenderParams(sh_degree=3)
    rz = raster.Rasterizer(P)
    _, tc = rz.project(sp, [cam], counts=True)
    rz.ensure_capacity(tc)
    rz.capacity *= 2  # room for the moved scene
    fg = raster.FrameGraph(rz, sp, cam, gimg, gT)
    fg.replay()
    torch.cuda.synchronize()
    before = fg.image.clone()
    gen = torch.Generator(device="cpu").manual_seed(1)
    with torch.no_grad():  # in place, as an optimiser step does
        sp.means += (0.05 * torch.randn(sp.means.shape, generator=gen)).cuda()
        sp.opac.mul_(0.9)
    fg.replay()
    torch.cuda.synchronize()
    rz.check_status("replay after update")
    assert not torch.equal(fg.image, before)
    img1, T1, g1, nk1 = _eager(sp, cam, gimg, gT, P)
    assert torch.equal(fg.image, img1) and torch.equal(fg.T, T1)
    assert int(fg.n_keys.item()) == nk1
    rels = {k: _rel(fg.grads[k], g1[k]) for k in g1}
    log_parity("replay_vs_eager_grad_rel_l2", **rels)
    for k, r in rels.items():
        assert r < 1e-4, k


def test_frame_graph_reports_capacity_overflow():
    sp, cam, gimg, gT = _setup(seed=8)
    P = raster.RenderParams(sh_degree=3)
    rz = raster.Rasterizer(P)
    _, _, st = rz.forward(sp, cam)
    nk = int(st["n_keys"].item())
    rz.capacity = nk  # exactly the keys of this frame
    fg = raster.FrameGraph(rz, sp, cam, gimg, gT)
    fg.replay()  # the outputs hold a frame only once the graph has run
    torch.cuda.synchronize()
    assert int(fg.n_keys.item()) == nk and int(rz.status.item()) == 0
    with torch.no_grad():  # every primitive three times wider: more tile keys
        sp.scales.mul_(3.0)
    fg.replay()
    torch.cuda.synchronize()
    s = int(rz.status.item())
    assert s == 3, s  # LS_ERR_CAPACITY
    assert int(fg.n_keys.item()) > nk


def test_dependent_launch_gives_the_plain_launch_results():
    from paper_2411_12440_gb300 import _native as N
    sp, cam, gimg, gT = _setup(seed=9)
    P = raster.RenderParams(sh_degree=3)
    outs = []
    try:
        for on in (0, 1):
            assert N.lib().ls_set_dependent_launch(on) == 0
            rz = raster.Rasterizer(P)
            img, T, st = rz.forward(sp, cam)
            g = rz.render_bwd(sp, cam, st, gimg, gT)
            torch.cuda.synchronize()
            rz.check_status("launch mode %d" % on)
            K = int(st["n_keys"].item())
            outs.append((img, T, st["vals"][:K].clone(), st["ranges"].clone(), g))
    finally:
        N.lib().ls_set_dependent_launch(1)
    (i0, t0, v0, r0, g0), (i1, t1, v1, r1, g1) = outs
    assert torch.equal(i0, i1) and torch.equal(t0, t1) and torch.equal(v0, v1) and torch.equal(r0, r1)
    rels = {k: _rel(g1[k], g0[k]) for k in g0}
    log_parity("dependent_vs_plain_launch_grad_rel_l2", **rels)
    for k, r in rels.items():
        assert r < 1e-4, k


def _bucket(m):
    """Quarter-octave bucket of a tile's work (its largest n_last)."""
    if m == 0:
        return 0
    lg = int(m).bit_length() - 1
    f = (m >> (lg - 2)) & 3 if lg >= 2 else (m << (2 - lg)) & 3
    return 1 + 4 * lg + f


def test_backward_tile_order_is_longest_first_and_changes_no_result():
    """ls_render_bwd with the ordered workspace: the order it builds is a
    permutation of the tiles, heaviest bucket first, each tile in the bucket
    of its largest n_last; the gradients equal the plain order's up to the
    order of the float atomics."""
    sp, cam, gimg, gT = _setup(n=20_000, seed=11, W=333, H=250)
    P = raster.RenderParams(sh_degree=3)
    res = {}
    for order in (False, True):
        rz = raster.Rasterizer(P)
        rz.bwd_tile_order = order
        img, T, st = rz.forward(sp, cam)
        g = rz.render_bwd(sp, cam, st, gimg, gT)
        torch.cuda.synchronize()
        rz.check_status("order %s" % order)
        res[order] = (g, rz, st)
    # float atomics add the per-tile contributions in another order; where a
    # gradient cancels across tiles that shows as ~1e-4 relative at full size
    rels = {k: _rel(res[True][0][k], res[False][0][k]) for k in res[False][0]}
    log_parity("ordered_vs_plain_grad_rel_l2", **rels)
    for k, r in rels.items():
        assert r < 1e-3, k
    g, rz, st = res[True]
    tx, ty = (cam["width"] + 15) // 16, (cam["height"] + 15) // 16
    tiles = tx * ty
    n = sp.n
    al = lambda b: (b + 255) // 256 * 256
    ws = rz._bufs["bwd_ws"]
    base = (ws.data_ptr() + 255) // 256 * 256 - ws.data_ptr()
    raw = ws[base:].cpu().numpy()
    o = al(n * 48) + al(4 * 132)
    bkt = raw[o:o + 4 * tiles].view(np.uint32)
    o += al(4 * tiles)
    order = raw[o:o + 4 * tiles].view(np.uint32)
    assert sorted(order.tolist()) == list(range(tiles))
    nl = st["n_last"].cpu().numpy()
    for t in range(tiles):
        y0, x0 = (t // tx) * 16, (t % tx) * 16
        assert bkt[t] == _bucket(int(nl[y0:y0 + 16, x0:x0 + 16].max())), t
    seq = bkt[order]
    assert np.all(seq[:-1] >= seq[1:])



def test_tile_order_entry_points():
    """ls_tile_order lists every tile once, heaviest bucket first (buckets of
    the largest n_last recomputed here); ls_blend_bwd_ordered with it gives
    ls_blend_bwd's 2D gradients up to the order of the float atomics."""
    sp, cam, gimg, gT = _setup(n=15_000, seed=13, W=300, H=200)
    P = raster.RenderParams(sh_degree=3)
    rz = raster.Rasterizer(P)
    img, T, st = rz.forward(sp, cam)
    order = rz.tile_order(cam, st["n_last"])
    g_plain = torch.zeros((sp.n, 12), dtype=torch.float32, device="cuda")
    g_ord = torch.zeros_like(g_plain)
    rz.blend_bwd(st["proj"], sp.n, cam, st["ranges"], st["vals"], T, st["n_last"], gimg, gT, g_plain)
    rz.blend_bwd_ordered(st["proj"], sp.n, cam, st["ranges"], order, st["vals"], T, st["n_last"], gimg, gT, g_ord)
    torch.cuda.synchronize()
    rz.check_status("ordered entry points")
    tx, ty = (cam["width"] + 15) // 16, (cam["height"] + 15) // 16
    o = order.cpu().numpy().astype(np.int64)
    assert sorted(o.tolist()) == list(range(tx * ty))
    nl = st["n_last"].cpu().numpy()
    b = np.array([_bucket(int(nl[(t // tx) * 16:(t // tx) * 16 + 16, (t % tx) * 16:(t % tx) * 16 + 16].max()))
                  for t in o])
    assert np.all(b[:-1] >= b[1:])
    r = _rel(g_ord, g_plain)
    log_parity("ordered_vs_plain_g2d_rel_l2", g2d=r)
    assert r < 1e-4
