"""GPU tests of learned termination: tile features and labels against the
oracle; the truncated render equals the plain render bit for bit whatever
the proposals (refuted tiles resume exactly), stays within its bound in the
lossy mode; and a network trained on plain renders sorts fewer keys than the
same pipeline without it (keep everything, or one global depth tuned on the
same training renders)."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2411_12440_gb300 import raster, scenes
from paper_2411_12440_gb300.learned import LearnedRenderer, TerminationMLP, tile_examples, train
from tests.gpu_helpers import pack_records

pytestmark = pytest.mark.gpu


def test_tile_features_match_oracle_histogram():
    W, H = 333, 211
    rec = scenes.random_records(4000, W, H, seed=31)
    proj, dkey = pack_records(rec)
    rz = raster.Rasterizer(raster.RenderParams())
    cam = scenes.identity_camera(W, H)
    x, total = rz.tile_features(proj, 4000, cam)
    torch.cuda.synchronize()
    foot = np.concatenate([rec["mean2d"], rec["ext"]], 1)
    counts, cov = oracle.tile_depth_hist(foot, dkey, oracle.records_to_proj(rec), W, H, 16, 16)
    assert np.array_equal(total.cpu().numpy(), counts)
    feat = x.float().cpu().numpy()
    assert np.allclose(feat[:, :32], np.log1p(cov), rtol=2e-3, atol=2e-3)
    assert not feat[:, 35:].any()
    # unit view directions of the tile centres (identity camera: the camera ray)
    d = feat[:, 32:35].astype(np.float64)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=2e-3)
    tx = np.arange(counts.shape[0]) % ((W + 15) // 16)
    ty = np.arange(counts.shape[0]) // ((W + 15) // 16)
    ray = np.stack([((tx + 0.5) * 16 - cam["cx"]) / cam["fx"], ((ty + 0.5) * 16 - cam["cy"]) / cam["fy"],
                    np.ones_like(tx, dtype=np.float64)], 1)
    ray /= np.linalg.norm(ray, axis=1, keepdims=True)
    assert np.abs(d - ray).max() < 2e-3


def test_tile_labels_match_oracle():
    scene, cams, _ = scenes.make_workload("plain_10k_256")
    cam = cams[0]
    P = dict(sh_degree=0)
    rz = raster.Rasterizer(raster.RenderParams.from_dict(P))
    sp = raster.Splats.from_scene(scene)
    image, T, state = rz.forward(sp, cam)
    labels = torch.zeros(256, dtype=torch.float32, device="cuda")
    rz.render_stats(state["proj"], scene.n, cam, state["ranges"], state["vals"], labels=labels)
    torch.cuda.synchronize()
    ref = oracle.render_scene(scene, cam, P)
    got = labels.cpu().numpy().astype(np.float64)
    exp = ref["labels"]
    per_tile = lambda a: a.reshape(16, 16, 16, 16).transpose(0, 2, 1, 3).reshape(256, -1)
    flagged_tiles = per_tile(ref["flags"]).any(1)
    # a tile whose list is empty (no support ellipse reaches it, although
    # support boxes may cover it) is labelled 0; the oracle, whose lists hold
    # the boxes, composites nothing there either
    rg = state["ranges"].cpu().numpy().reshape(-1, 2)
    empty = rg[:, 1] == rg[:, 0]
    assert (got[empty] == 0).all()
    assert (per_tile(ref["T"])[empty & ~flagged_tiles] == 1.0).all()
    ok = ~flagged_tiles & ~empty
    assert ok.sum() > 150
    assert np.array_equal(np.isinf(got[ok]), np.isinf(exp[ok]))
    fin = ok & ~np.isinf(exp)
    assert np.allclose(got[fin], exp[fin], rtol=1e-6)


def _cluster(n, seed, w=640, h=480):
    scene = scenes.cluster_scene(n, seed, 3)
    cam = scenes.ring_cameras(1, seed, w_range=(w, w), h_range=(h, h))[0]
    return scene, cam


@pytest.mark.parametrize("margin", [-3.0, 0.0, 3.0])
def test_learned_render_is_exact_for_any_proposal(margin):
    """Random network weights: whatever the proposals, refuted tiles resume
    and the image, T and n_last equal the plain render bit for bit."""
    scene, cam = _cluster(150_000, 5)
    sp = raster.Splats.from_scene(scene)
    P = raster.RenderParams(sh_degree=3)
    rz = raster.Rasterizer(raster.RenderParams(sh_degree=3))
    img0, T0, st0 = rz.forward(sp, cam)
    lr = LearnedRenderer(sp, cam, P)
    net = TerminationMLP(scenes.random_mlp_params(7))
    img, T = lr.render(net, margin=margin)
    torch.cuda.synchronize()
    lr.check()
    total, kept, held, refuted = lr.counters()
    assert torch.equal(img, img0) and torch.equal(T, T0)
    assert torch.equal(lr.n_last, st0["n_last"])
    assert total == int(st0["n_keys"].item())
    if margin == -3.0:
        assert refuted > 0 and held > 0
    # without the counters, records beyond their box's proposals are dropped
    # up front: the same image
    img, T = lr.render(net, margin=margin, stats=False)
    torch.cuda.synchronize()
    lr.check()
    assert torch.equal(img, img0) and torch.equal(T, T0)
    assert torch.equal(lr.n_last, st0["n_last"])


def test_learned_proposals_follow_the_tile_features():
    """The render's own coverage planes (accumulated in depth order) give the
    same features as the standalone tile features (accumulated in record
    order): the proposals are the network's output on them."""
    scene, cam = _cluster(150_000, 5)
    sp = raster.Splats.from_scene(scene)
    P = raster.RenderParams(sh_degree=3)
    rz = raster.Rasterizer(raster.RenderParams(sh_degree=3))
    lr = LearnedRenderer(sp, cam, P)
    net = TerminationMLP(scenes.random_mlp_params(7))
    lr.render(net, margin=0.5)
    proj, _ = rz.project(sp, [cam], counts=False)
    x, _ = rz.tile_features(proj, sp.n, cam)
    y = net.forward(x)
    torch.cuda.synchronize()
    lr.check()
    expect = torch.exp(y + 0.5)
    assert torch.allclose(lr.dstar, expect, rtol=1e-5, atol=0)


@pytest.mark.parametrize("dstar", [0.0, math.inf])
def test_learned_render_extremes(dstar):
    """Proposal 0 keeps nothing (every non-empty tile refuted and resumed);
    +inf keeps everything (nothing refuted): both equal the plain render."""
    scene, cam = _cluster(60_000, 6, 320, 240)
    sp = raster.Splats.from_scene(scene)
    rz = raster.Rasterizer(raster.RenderParams(sh_degree=3))
    img0, T0, st0 = rz.forward(sp, cam)
    lr = LearnedRenderer(sp, cam, raster.RenderParams(sh_degree=3))
    d = torch.full((lr.tiles,), dstar, dtype=torch.float32, device="cuda")
    img, T = lr.render(dstar_in=d)
    torch.cuda.synchronize()
    lr.check()
    total, kept, held, refuted = lr.counters()
    assert torch.equal(img, img0) and torch.equal(T, T0)
    if dstar == 0.0:
        assert kept == 0 and held == total
    else:
        assert kept == total and refuted == 0 and held == 0


def test_learned_lossy_mode_error_bound():
    """t_thr > t_min: each pixel within t_thr (max rgb + bg) of the plain one."""
    scene, cam = _cluster(150_000, 8)
    sp = raster.Splats.from_scene(scene)
    bg = (0.2, 0.4, 0.1)
    rz = raster.Rasterizer(raster.RenderParams(sh_degree=3, bg=bg))
    img0, T0, st0 = rz.forward(sp, cam)
    lr = LearnedRenderer(sp, cam, raster.RenderParams(sh_degree=3, bg=bg))
    net = TerminationMLP(scenes.random_mlp_params(9))
    t_thr = 3e-3
    img, T = lr.render(net, margin=-1.0, t_thr=t_thr)
    torch.cuda.synchronize()
    lr.check()
    maxrgb = float(raster.Splats.sh_from_device_layout(sp.sh, sp.n).abs().max().item()) * 4 + 1.0
    err = (img - img0).abs().max().item()
    assert err <= t_thr * (maxrgb + max(bg)) + 1e-5
    psnr = -10 * math.log10(max(float(((img - img0) ** 2).mean().item()), 1e-30))
    assert psnr >= 50.0


def _sorted_keys(lr, **kw):
    lr.render(**kw)
    torch.cuda.synchronize()
    lr.check()
    total, kept, held, refuted = lr.counters()
    return kept + held, refuted


def test_trained_network_gains_over_the_method_without_it():
    """Train on plain renders of dense cluster scenes (cameras on the ring,
    targets at t_thr = 1e-3), then compare keys sorted per frame on held-out
    views of a held-out scene: the trained network against keeping
    everything and against one global depth tuned on the same training
    views.  Every image stays within PSNR 50 dB of the plain render."""
    t_thr = 1e-3
    P = raster.RenderParams(sh_degree=3)
    rz = raster.Rasterizer(raster.RenderParams(sh_degree=3))
    rz_lab = raster.Rasterizer(raster.RenderParams(sh_degree=3, t_min=t_thr))
    views = dict(w_range=(400, 640), h_range=(300, 480))
    train_scenes = [raster.Splats.from_scene(scenes.cluster_scene(1_200_000, 100 + k, 3)) for k in range(3)]
    xs, ys = [], []
    for i in range(120):
        cam = scenes.ring_cameras(1, 1000 + i, **views)[0]
        x, y = tile_examples(rz_lab, train_scenes[i % 3], cam)
        xs.append(x)
        ys.append(y)
    x, y = torch.cat(xs), torch.cat(ys)
    net = TerminationMLP(seed=0)
    losses = train(net, x, y, steps=3000, batch=16384, lr=2e-3, under_weight=2.0, log_every=1000)
    assert losses[-1][1] < losses[0][1]
    tune_views = [(train_scenes[k % 3], scenes.ring_cameras(1, 1000 + k, **views)[0]) for k in range(3)]
    finite = torch.exp(y[y < math.log(64.0) - 1e-3]).float()
    qs = [float(torch.quantile(finite[:100000], q).item()) for q in (0.5, 0.7, 0.8, 0.9, 0.97)]

    def cost(kw_fn):
        s = 0
        for spx, cam in tune_views:
            lr = LearnedRenderer(spx, cam, P)
            s += _sorted_keys(lr, t_thr=t_thr, **kw_fn(lr))[0]
        return s

    margin = min((0.0, 0.2, 0.4, 0.6, 0.8), key=lambda m: cost(lambda lr: dict(mlp=net, margin=m)))
    const = min(qs, key=lambda c: cost(lambda lr: dict(dstar_in=torch.full((lr.tiles,), c, device="cuda"))))
    test_scene = raster.Splats.from_scene(scenes.cluster_scene(1_200_000, 777, 3))
    tot = dict(mlp=0, const=0, all=0)
    for i in range(6):
        cam = scenes.ring_cameras(1, 5000 + i, w_range=(512, 512), h_range=(384, 384))[0]
        img0, _, _ = rz.forward(test_scene, cam)
        lr = LearnedRenderer(test_scene, cam, P)
        for name, kw in (("mlp", dict(mlp=net, margin=margin)),
                         ("const", dict(dstar_in=torch.full((lr.tiles,), const, device="cuda"))),
                         ("all", dict(dstar_in=torch.full((lr.tiles,), math.inf, device="cuda")))):
            k, _ = _sorted_keys(lr, t_thr=t_thr, **kw)
            tot[name] += k
            mse = float(((lr.image - img0) ** 2).mean().item())
            assert mse == 0.0 or -10 * math.log10(mse) >= 50.0
    print("keys sorted over the held-out views:", tot, "margin", margin, "depth", const)
    assert tot["mlp"] < 0.75 * tot["all"], tot
    assert tot["mlp"] < tot["const"], tot
