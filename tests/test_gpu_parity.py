"""GPU parity: every stage of the CUDA path, called through the C ABI, against
the FP64 oracle on the same seeded inputs.

  duplicate + sort    bit-exact keys, record order and tile ranges
  projection          records within 1e-5 relative (binary32 vs FP64)
  forward blend       images within 1e-4 max abs on unflagged pixels
  backward            gradients within 1e-3 relative L2 per tensor
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2411_12440_gb300 import _native as N
from paper_2411_12440_gb300 import raster, scenes
from tests.gpu_helpers import (GRAD_TOL, assert_image_parity, conic_of, log_parity, pack_records, rel_l2,
                               unpack_proj)

pytestmark = pytest.mark.gpu

TILES = [(8, 8), (16, 16), (32, 16)]


def _dupsort(rz, proj, R, cams, cap):
    keys, vals, n_keys, ranges = rz.duplicate_sort(proj, R, cams, capacity=cap)
    torch.cuda.synchronize()
    K = int(n_keys.item())
    return keys[:K].cpu().numpy().view(np.uint32), vals[:K].cpu().numpy().view(np.uint32), \
        ranges.cpu().numpy().reshape(-1, 2), K


# ------------------------------------------------------------------ a2 + a3
# A record is listed in the tiles of its binary32 support box that its
# support ellipse reaches (a binary32 rule both sides compute with the same
# roundings), so lists, orders and ranges are compared bit for bit with the
# oracle.  Two more checks tie the rule to the method: the lists hold every
# tile the oracle finds, by brute force over pixel centres, to be reached by
# the (slightly shrunk) ellipse, and they are the support-box lists filtered.
def _touch(rec, dkey, W, H, tw, th, shrink=0.999):
    foot = np.concatenate([rec["mean2d"], rec["ext"]], 1)
    l00, l01, l11 = (rec["chol"][:, k].astype(np.float64) for k in range(3))
    conic = np.stack([l00 * l00, l00 * l01, l01 * l01 + l11 * l11], 1)
    return oracle.touch_pairs(foot, dkey, conic, rec["rho2"].astype(np.float64), W, H, tw, th, shrink)


def _oracle_lists(rec, dkey, W, H, tw, th, reach=True):
    foot = np.concatenate([rec["mean2d"], rec["ext"]], 1)
    if not reach:
        return oracle.dupsort_f32(foot, dkey, W, H, tw, th)
    return oracle.dupsort_f32(foot, dkey, W, H, tw, th, chol=rec["chol"], rho2=rec["rho2"])


def _check_reach(keys, vals, ok, ov, et, er):
    """GPU lists against the box lists (ok, ov) and the pairs (et, er) that
    must be present; returns the fraction of box pairs listed."""
    R1 = np.int64(max(int(ov.max()) if len(ov) else 0, int(vals.max()) if len(vals) else 0) + 1)
    gid = keys.astype(np.int64) * R1 + vals.astype(np.int64)
    bid = ok.astype(np.int64) * R1 + ov.astype(np.int64)
    mask = np.isin(bid, gid)
    assert np.array_equal(bid[mask], gid), "listed pairs are not the box lists filtered, in order"
    assert np.isin(et.astype(np.int64) * R1 + er.astype(np.int64), gid).all(), "a reached tile is missing"
    return mask.mean() if len(mask) else 1.0


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("R,W,H", [(1, 300, 200), (3001, 300, 200), (40_000, 1297, 840)])
def test_duplicate_sort_bitexact(tile, R, W, H):
    rec = scenes.random_records(R, W, H, seed=R + tile[0])
    proj, dkey = pack_records(rec)
    P = raster.RenderParams(tile_w=tile[0], tile_h=tile[1])
    rz = raster.Rasterizer(P)
    cam = scenes.identity_camera(W, H)
    ok, ov, orr = _oracle_lists(rec, dkey, W, H, tile[0], tile[1])
    bk, bv, _ = _oracle_lists(rec, dkey, W, H, tile[0], tile[1], reach=False)
    et, er = _touch(rec, dkey, W, H, tile[0], tile[1])
    keys, vals, ranges, K = _dupsort(rz, proj, R, [cam], cap=len(bk) + 17)
    rz.check_status()
    assert K == len(ok)
    assert np.array_equal(keys, ok)
    assert np.array_equal(vals, ov)
    assert np.array_equal(ranges, orr)
    frac = _check_reach(keys, vals, bk, bv, et, er)
    if R > 1000:
        assert frac < 0.95  # the box corners the ellipses miss are dropped


def test_duplicate_sort_ties_and_culled():
    """Many equal depths (ties broken by record id) and a third of the records culled."""
    W, H = 640, 360
    rec = scenes.random_records(20_000, W, H, seed=11, visible_frac=0.66)
    rec["depth"][:] = rec["depth"][:7].repeat(20_000 // 7 + 1)[:20_000]
    proj, dkey = pack_records(rec)
    rz = raster.Rasterizer(raster.RenderParams())
    ok, ov, orr = _oracle_lists(rec, dkey, W, H, 16, 16)
    keys, vals, ranges, K = _dupsort(rz, proj, 20_000, [scenes.identity_camera(W, H)], cap=len(ok))
    rz.check_status()
    assert K == len(ok) and np.array_equal(keys, ok) and np.array_equal(vals, ov) and np.array_equal(ranges, orr)


def test_duplicate_sort_empty_and_all_culled():
    rz = raster.Rasterizer(raster.RenderParams())
    cam = scenes.identity_camera(100, 60)
    rec = scenes.random_records(500, 100, 60, seed=2, visible_frac=0.0)
    proj, _ = pack_records(rec)
    keys, vals, ranges, K = _dupsort(rz, proj, 500, [cam], cap=1000)
    assert K == 0 and not ranges.any()
    keys, vals, ranges, K = _dupsort(rz, torch.zeros(4, device="cuda"), 0, [cam], cap=0)
    assert K == 0 and not ranges.any()
    rz.check_status()


def test_duplicate_sort_capacity_overflow_reports_and_recovers():
    W, H = 300, 200
    rec = scenes.random_records(2000, W, H, seed=5)
    proj, dkey = pack_records(rec)
    rz = raster.Rasterizer(raster.RenderParams())
    cam = scenes.identity_camera(W, H)
    ok, ov, orr = _oracle_lists(rec, dkey, W, H, 16, 16)
    _, _, ranges, K = _dupsort(rz, proj, 2000, [cam], cap=len(ok) - 1)
    assert K == len(ok)  # the true count is reported
    assert not ranges.any()
    assert int(rz.status.item()) == 3
    with pytest.raises(N.LsError):
        rz.check_status()
    rz.reset_status()
    keys, vals, ranges, K = _dupsort(rz, proj, 2000, [cam], cap=len(ok))
    rz.check_status()
    assert np.array_equal(keys, ok) and np.array_equal(vals, ov) and np.array_equal(ranges, orr)


def test_sort_wait_timeout_reported_and_recovers():
    """Failure detection of the bounded device-side waits: partition 0 of the
    last tile-sort pass is made to publish nothing, so the look-back of the
    partitions after it gives up after a short limit.  LS_ERR_TIMEOUT reaches
    the status word, every write stays inside the key range (a sentinel past
    K survives, ranges lie in [0, K]), and the next call with the default
    limit is bit-exact again."""
    W, H = 1297, 840
    R = 40_000
    rec = scenes.random_records(R, W, H, seed=44)
    proj, dkey = pack_records(rec)
    P = raster.RenderParams()
    cam = scenes.identity_camera(W, H)
    ok, ov, orr = _oracle_lists(rec, dkey, W, H, 16, 16)
    K = len(ok)
    assert K > 3 * 4608  # several partitions of 4608 keys in the tile sort
    cap = K + 4096
    tiles = raster.tiles_of(cam, P)
    L = N.lib()

    def call():
        keys = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
        vals = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
        n_keys = torch.zeros(1, dtype=torch.int64, device="cuda")
        ranges = torch.empty(2 * tiles, dtype=torch.int32, device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        wsb = L.ls_duplicate_sort_workspace(R, cap, tiles)
        ws = torch.empty(wsb + 256, dtype=torch.uint8, device="cuda")
        wp = (ws.data_ptr() + 255) // 256 * 256
        N.check(L.ls_duplicate_sort(R, raster._p(proj), raster.cam_array([cam]), 1, ctypes.byref(P.c()), cap,
                                    raster._p(keys), raster._p(vals), raster._p(n_keys), raster._p(ranges),
                                    ctypes.c_void_p(wp), wsb, raster._p(status), raster._stream()),
                "ls_duplicate_sort")
        torch.cuda.synchronize()
        return (keys.cpu().numpy().view(np.uint32), vals.cpu().numpy().view(np.uint32), int(n_keys.item()),
                ranges.cpu().numpy().reshape(-1, 2), int(status.item()))

    N.check(L.ls_debug_set_sort_wait(2000, 0), "ls_debug_set_sort_wait")
    try:
        keys, vals, nk, ranges, status = call()
    finally:
        N.check(L.ls_debug_set_sort_wait(0, -1), "ls_debug_set_sort_wait")
    assert status == 4, status  # LS_ERR_TIMEOUT
    assert nk == K
    assert (keys[K:] == np.uint32(0xFFFFFFF9)).all() and (vals[K:] == np.uint32(0xFFFFFFF9)).all()
    assert (ranges >= 0).all() and (ranges <= K).all() and (ranges[:, 0] <= ranges[:, 1]).all()
    keys, vals, nk, ranges, status = call()
    assert status == 0
    assert nk == K and np.array_equal(keys[:K], ok) and np.array_equal(vals[:K], ov) and np.array_equal(ranges, orr)


def test_duplicate_sort_multi_camera_global_tiles():
    """Records of several cameras of different sizes share one sort; tile ids
    are global (camera c's tiles after those of cameras 0..c-1)."""
    sizes = [(300, 200), (128, 96), (517, 211)]
    cams = [scenes.identity_camera(w, h) for w, h in sizes]
    n = 1500
    recs = [scenes.random_records(n, w, h, seed=40 + i) for i, (w, h) in enumerate(sizes)]
    allrec = {k: np.concatenate([r[k] for r in recs]) for k in recs[0]}
    proj, dkey = pack_records(allrec)
    rz = raster.Rasterizer(raster.RenderParams())
    base = 0
    exp_k, exp_v, exp_r = [], [], []
    # oracle per camera, then merge: global order is (global tile, depth, record id)
    for i, (w, h) in enumerate(sizes):
        k, v, r = _oracle_lists(recs[i], dkey[i * n:(i + 1) * n], w, h, 16, 16)
        exp_k.append(k + base)
        exp_v.append(v + i * n)
        exp_r.append(r)
        base += raster.tiles_of(cams[i], rz.params)
    ok, ov = np.concatenate(exp_k), np.concatenate(exp_v)
    keys, vals, ranges, K = _dupsort(rz, proj, 3 * n, cams, cap=len(ok))
    rz.check_status()
    assert np.array_equal(keys, ok) and np.array_equal(vals, ov)
    shifted, before = [], 0
    for k, r in zip(exp_k, exp_r):
        rr = r.copy()
        nz = rr[:, 1] > rr[:, 0]
        rr[nz] += before
        shifted.append(rr)
        before += len(k)
    assert np.array_equal(ranges, np.concatenate(shifted))


# ------------------------------------------------------------------ a1
def _proj_parity(scene, cam, P, rtol=1e-5):
    """Record fields against the oracle, relative to the field's scale
    (5 rtol), visibility, support boxes and the binary32 depth key."""
    rz = raster.Rasterizer(raster.RenderParams.from_dict(P))
    sp = raster.Splats.from_scene(scene)
    proj, tc = rz.project(sp, [cam])
    torch.cuda.synchronize()
    rec, foot, dkey = unpack_proj(proj, scene.n)
    ref, vis = oracle.project(scene, cam, P)
    gvis = dkey != 0xFFFFFFFF
    # visibility may differ only where a cull threshold is met to rounding
    diff = np.nonzero(gvis != vis)[0]
    assert len(diff) <= max(2, 1e-4 * scene.n), len(diff)
    m = gvis & vis
    cols = [(0, oracle.P_MX), (1, oracle.P_MY), (5, oracle.P_O), (6, oracle.P_RHO2), (7, oracle.P_DEPTH),
            (8, oracle.P_R), (9, oracle.P_G), (10, oracle.P_BL)]
    abc = conic_of(rec)
    errs = {}
    for k, oi in enumerate((oracle.P_A, oracle.P_B, oracle.P_C)):
        g, o = abc[m, k], ref[m, oi]
        # relative to the conic's size: the factor L is accurate entry-wise
        scale = np.maximum(np.abs(ref[m, oracle.P_A]), np.abs(ref[m, oracle.P_C]))
        errs["abc"[k]] = float((np.abs(g - o) / scale).max())
    names = ["mx", "my", "o", "rho2", "depth", "r", "g", "b"]
    for (gi, oi), nm in zip(cols, names):
        g, o = rec[m, gi].astype(np.float64), ref[m, oi]
        scale = np.maximum(np.abs(o), np.abs(ref[m][:, [oi]]).mean() * 1e-2 + 1e-6)
        errs[nm] = float((np.abs(g - o) / scale).max())
    log_parity("record_fields", **errs)
    # measured on GB300: at most 2.2e-5 for the conic and 2.5e-5 for SH3
    # colours (binary32 sums of 16 SH terms against FP64), so 5e-5
    for k in "abc":
        assert errs[k] < 5 * rtol, (k, errs[k])
    for nm in names:
        assert errs[nm] < 5 * rtol, (nm, errs[nm])
    assert np.allclose(foot[m, 2], ref[m, oracle.P_EX], rtol=1e-4)
    # sort key: the binary32 camera depth, a few ulp from the FP64 value
    assert (np.abs(dkey[m].view(np.float32) - ref[m, oracle.P_DEPTH]) <= 1e-6 * ref[m, oracle.P_DEPTH]).all()
    return rec, foot, dkey, ref, vis, tc.cpu().numpy()


def test_project_parity_box_sh0():
    scene, cams, _ = scenes.make_workload("plain_10k_256")
    _proj_parity(scene, cams[0], dict(sh_degree=0))


@pytest.mark.parametrize("aa", [0, 1])
def test_project_parity_clusters_sh3(aa):
    scene, cams, _ = scenes.make_workload("scene_1m_1297x840_aa", n=50_000)
    _proj_parity(scene, cams[0], dict(sh_degree=3, antialias=aa))


def test_project_tile_counts_match_oracle_rects():
    scene, cams, _ = scenes.make_workload("scene_1m_1297x840_aa", n=20_000)
    cam = cams[0]
    rec, foot, dkey, ref, vis, tc = _proj_parity(scene, cam, dict(sh_degree=3))
    bad = 0
    for i in range(scene.n):
        if dkey[i] == 0xFFFFFFFF:
            assert tc[i] == 0
            continue
        r = oracle.rect(*foot[i].astype(np.float64).tolist(), cam["width"], cam["height"], True)
        cnt = 0 if r is None else (r[1] // 16 - r[0] // 16 + 1) * (r[3] // 16 - r[2] // 16 + 1)
        bad += cnt != tc[i]
    assert bad == 0


# ------------------------------------------------------------------ a4
@pytest.mark.parametrize("tile", TILES)
def test_render_records_parity(tile):
    """Blend of random records alone: same binary32 lists on both sides."""
    W, H = 333, 211
    rec = scenes.random_records(3000, W, H, seed=21, max_ext=25)
    proj, dkey = pack_records(rec)
    P = dict(tile_w=tile[0], tile_h=tile[1], bg=(0.2, 0.1, 0.3))
    rz = raster.Rasterizer(raster.RenderParams.from_dict(P))
    cam = scenes.identity_camera(W, H)
    rz.capacity = 3000 * 400
    keys, vals, n_keys, ranges = rz.duplicate_sort(proj, 3000, [cam])
    image, T, n_last = rz.render_fwd(proj, 3000, cam, ranges, vals)
    torch.cuda.synchronize()
    rz.check_status()
    ref = oracle.render(oracle.records_to_proj(rec), rec["visible"], W, H, P, rule_f32=True, dkey=dkey)
    assert_image_parity(image.cpu().numpy(), ref)
    ok = ~ref["flags"]
    assert np.abs(T.cpu().numpy() - ref["T"])[ok].max() < 1e-4
    # n_last indexes the pixel's own tile list; the record it points at is
    # the oracle's last composited record
    nl = n_last.cpu().numpy()
    rg = ranges.cpu().numpy().reshape(-1, 2)
    py, px = np.nonzero(nl > 0)
    tid = (py // tile[1]) * ((W + tile[0] - 1) // tile[0]) + px // tile[0]
    last = np.full(nl.shape, -1, dtype=np.int64)
    last[py, px] = vals.cpu().numpy().view(np.uint32)[rg[tid, 0] + nl[py, px] - 1]
    exp = np.where(ref["n_last"] > 0, ref["last_id"], -1)
    assert (last == exp)[ok].mean() > 0.9999


def _render_gpu(scene, cam, P):
    rz = raster.Rasterizer(raster.RenderParams.from_dict(P))
    sp = raster.Splats.from_scene(scene)
    image, T, state = rz.forward(sp, cam)
    torch.cuda.synchronize()
    rz.check_status()
    return rz, sp, image, T, state


@pytest.mark.parametrize("P", [dict(), dict(bg=(0.3, 0.6, 0.9)), dict(eps2d=0.0), dict(antialias=1)],
                         ids=["default", "bg", "noeps", "aa"])
def test_render_scene_parity_plain_10k(P):
    scene, cams, _ = scenes.make_workload("plain_10k_256")
    P = dict(P, sh_degree=0)
    _, _, image, T, _ = _render_gpu(scene, cams[0], P)
    ref = oracle.render_scene(scene, cams[0], P)
    assert_image_parity(image.cpu().numpy(), ref)


def test_render_images_independent_of_tile_shape():
    """Same per-pixel operation order for every tile shape: bitwise equal."""
    scene, cams, _ = scenes.make_workload("plain_10k_256")
    imgs = []
    for tw, th in TILES:
        _, _, image, T, _ = _render_gpu(scene, cams[0], dict(sh_degree=0, tile_w=tw, tile_h=th))
        imgs.append(image.cpu().numpy())
    assert np.array_equal(imgs[0], imgs[1]) and np.array_equal(imgs[1], imgs[2])


@pytest.mark.parametrize("kid,lam", [(1, 1.0), (2, 1.0), (3, 2.5), (4, 6.0)])
def test_render_kernel_family_parity(kid, lam):
    scene, cams, _ = scenes.make_workload("plain_10k_256", n=4000)
    P = dict(sh_degree=0, kernel=kid, lam=lam)
    _, _, image, T, _ = _render_gpu(scene, cams[0], P)
    ref = oracle.render_scene(scene, cams[0], P)
    assert_image_parity(image.cpu().numpy(), ref)


def test_render_stats_counts_match_oracle():
    """Work units of the tile method: composited pairs equal the oracle's up
    to threshold flips; evaluated pairs are bounded by the oracle's."""
    scene, cams, _ = scenes.make_workload("plain_10k_256")
    cam = cams[0]
    rz, sp, image, T, state = _render_gpu(scene, cam, dict(sh_degree=0))
    img2, T2, nl2, n_eval, n_contrib = rz.render_stats(state["proj"], scene.n, cam, state["ranges"], state["vals"])
    assert torch.equal(img2, image) and torch.equal(T2, T)
    ref = oracle.render_scene(scene, cam, dict(sh_degree=0))
    assert abs(n_contrib - ref["n_contrib"]) <= ref["flags"].sum()
    # the oracle's lists hold every support-box tile, the GPU's only those the
    # support ellipse reaches: fewer pairs are evaluated, never fewer composited
    assert n_contrib <= n_eval <= ref["n_eval"] * (1 + 1e-3)


# ------------------------------------------------------------------ a5
def test_blend_bwd_records_parity():
    W, H = 200, 136
    rec = scenes.random_records(1500, W, H, seed=8, max_ext=20)
    proj, dkey = pack_records(rec)
    P = dict(bg=(0.1, 0.5, 0.2))
    rz = raster.Rasterizer(raster.RenderParams.from_dict(P))
    cam = scenes.identity_camera(W, H)
    rz.capacity = 1500 * 200
    keys, vals, n_keys, ranges = rz.duplicate_sort(proj, 1500, [cam])
    image, T, n_last = rz.render_fwd(proj, 1500, cam, ranges, vals)
    w, v = scenes.loss_weights(H, W, seed=3)
    g2d = torch.zeros((1500, 12), device="cuda")
    c = raster.cam_struct(cam)
    wd, vd = torch.from_numpy(w).cuda(), torch.from_numpy(v).cuda()  # alive until the kernel has run
    N.check(N.lib().ls_blend_bwd(raster._p(proj), 1500, ctypes.byref(c), ctypes.byref(rz.params.c()),
                                 raster._p(ranges), raster._p(vals), raster._p(T), raster._p(n_last), raster._p(wd),
                                 raster._p(vd), raster._p(g2d), raster._p(rz.status), raster._stream()),
            "ls_blend_bwd")
    torch.cuda.synchronize()
    rz.check_status()
    ref = oracle.render_bwd(oracle.records_to_proj(rec), rec["visible"], W, H, w.astype(np.float64),
                            v.astype(np.float64), P, rule_f32=True, dkey=dkey)
    g = g2d.cpu().numpy()
    cols = [0, 1, 2, 3, 4, 5, 6, 7, 8]
    for j, gc in enumerate(cols):
        assert rel_l2(g[:, gc], ref[:, j]) < GRAD_TOL, (j, rel_l2(g[:, gc], ref[:, j]))


CASES_BWD = [
    ("plain", "plain_10k_256", None, dict(sh_degree=0)),
    ("bg_aa", "plain_10k_256", None, dict(sh_degree=0, antialias=1, bg=(0.5, 0.2, 0.7))),
    ("ags", "plain_10k_256", None, dict(sh_degree=0, ags=1)),
    ("ags_aligned", "plain_10k_256", None, dict(sh_degree=0, ags=2)),
    ("sh3_clusters", "scene_1m_1297x840_aa", 30_000, dict(sh_degree=3, antialias=1)),
    # the kernel family of Appendix B (Eq. 21-24) with its alignment factors
    ("gaussian", "plain_10k_256", 4000, dict(sh_degree=0, kernel=1, lam=1.0)),
    ("laplacian", "plain_10k_256", 4000, dict(sh_degree=0, kernel=2, lam=1.0)),
    ("cosine", "plain_10k_256", 4000, dict(sh_degree=0, kernel=3, lam=2.5)),
    ("quadratic", "plain_10k_256", 4000, dict(sh_degree=0, kernel=4, lam=6.0)),
    ("gaussian_sh3_aa", "scene_1m_1297x840_aa", 20_000, dict(sh_degree=3, antialias=1, kernel=1, lam=1.0)),
]


def _masked_weights(scene, cam, P, seed):
    """Loss weights with the pixels the oracle flags (a pair within 1e-5 of
    alpha_min, T within 1e-9 of T_min, alpha within 1e-6 of the clamp) set
    to zero: there binary32 and FP64 may take different skip/stop decisions,
    a jump of the forward, so the adjoints are compared on the rest."""
    w, v = scenes.loss_weights(cam["height"], cam["width"], seed=seed)
    flags = oracle.render_scene(scene, cam, P)["flags"]
    w[flags] = 0.0
    v[flags] = 0.0
    return w, v


@pytest.mark.parametrize("name,wl,n,P", CASES_BWD, ids=[c[0] for c in CASES_BWD])
def test_render_bwd_parity(name, wl, n, P):
    scene, cams, _ = scenes.make_workload(wl, n=n)
    cam = cams[0]
    rz, sp, image, T, state = _render_gpu(scene, cam, P)
    w, v = _masked_weights(scene, cam, P, seed=4)
    g = rz.render_bwd(sp, cam, state, torch.from_numpy(w).cuda(), torch.from_numpy(v).cuda(), want_g2d=True)
    torch.cuda.synchronize()
    rz.check_status()
    ref = oracle.scene_grads(scene, cam, w.astype(np.float64), v.astype(np.float64), P)
    n = scene.n
    got = dict(means=g["means"].cpu().numpy(), scales=g["scales"].cpu().numpy(), quats=g["quats"].cpu().numpy(),
               opac=g["opac"].cpu().numpy(), sh=raster.Splats.sh_from_device_layout(g["sh"], n).cpu().numpy())
    errs = {k: rel_l2(got[k], ref[k]) for k in ("means", "scales", "quats", "opac", "sh")}
    log_parity("grad_rel_l2", **errs)
    for k, e in errs.items():
        assert e < GRAD_TOL, (k, e)


def test_autograd_function_matches_direct_backward():
    scene, cams, _ = scenes.make_workload("plain_10k_256", n=3000)
    cam = cams[0]
    rz = raster.Rasterizer(raster.RenderParams(sh_degree=0))
    sp = raster.Splats.from_scene(scene)
    for t in sp.tensors():
        t.requires_grad_(True)
    image, T = raster.render(sp, cam, rz)
    w, v = scenes.loss_weights(cam["height"], cam["width"], seed=6)
    loss = (image * torch.from_numpy(w).cuda()).sum() + (T * torch.from_numpy(v).cuda()).sum()
    loss.backward()
    ref = oracle.scene_grads(scene, cam, w.astype(np.float64), v.astype(np.float64), dict(sh_degree=0))
    assert rel_l2(sp.means.grad.cpu().numpy(), ref["means"]) < GRAD_TOL
    assert rel_l2(sp.opac.grad.cpu().numpy(), ref["opac"]) < GRAD_TOL
    sh = raster.Splats.sh_from_device_layout(sp.sh.grad, scene.n).cpu().numpy()
    assert rel_l2(sh, ref["sh"]) < GRAD_TOL


# ------------------------------------------------------------------ full size, sampled
@pytest.mark.parametrize("wl,window", [("scene_1m_1297x840_aa", (600, 728, 380, 476)),
                                       ("diff_3m_1080p", (900, 1028, 500, 580))])
def test_full_size_forward_window(wl, window):
    """Full-size scenes in the launch configuration the benchmark times,
    checked on a pixel window the oracle composites in seconds."""
    scene, cams, extra = scenes.make_workload(wl)
    cam = cams[0]
    P = dict(sh_degree=3, antialias=int(extra["antialias"]))
    _, _, image, T, state = _render_gpu(scene, cam, P)
    oracle.set_threads(8)
    ref = oracle.render_scene(scene, cam, P, window=window)
    assert_image_parity(image.cpu().numpy(), ref, region=window)
    x0, x1, y0, y1 = window
    ok = ~ref["flags"][y0:y1, x0:x1]
    assert np.abs(T.cpu().numpy()[y0:y1, x0:x1] - ref["T"][y0:y1, x0:x1])[ok].max() < 1e-4


def test_full_size_backward_window():
    """The benchmarked frame (3M primitives, SH3, 1920x1080, 16x16 tiles) in
    the launch configuration the benchmark times, backward: the loss weights
    are zero outside a 64x64 window (and on the pixels the oracle flags), so
    the oracle's adjoint of that window is exact at full size.  Long lists,
    per-warp start points and vector atomics from every tile a large record
    reaches are all exercised.  2D record gradients and the 3D gradients of
    every primitive (zero for those that miss the window) within 1e-3
    relative L2."""
    scene, cams, extra = scenes.make_workload("diff_3m_1080p")
    cam = cams[0]
    H, W = cam["height"], cam["width"]
    P = dict(sh_degree=3, antialias=int(extra["antialias"]))
    rz, sp, image, T, state = _render_gpu(scene, cam, P)
    window = (896, 960, 512, 576)
    x0, x1, y0, y1 = window
    oracle.set_threads(8)
    ref_f = oracle.render_scene(scene, cam, P, window=window)
    w, v = scenes.loss_weights(H, W, seed=9)
    keep = np.zeros((H, W), bool)
    keep[y0:y1, x0:x1] = True
    keep &= ~ref_f["flags"]
    w[~keep] = 0.0
    v[~keep] = 0.0
    g = rz.render_bwd(sp, cam, state, torch.from_numpy(w).cuda(), torch.from_numpy(v).cuda(), want_g2d=True)
    torch.cuda.synchronize()
    rz.check_status()
    g2d_ref = oracle.render_bwd(ref_f["proj"], ref_f["vis"], W, H, w.astype(np.float64), v.astype(np.float64), P,
                                window=window)
    touched = np.nonzero(np.abs(g2d_ref).sum(1) > 0)[0]
    assert len(touched) > 100  # ~200 primitives composite into the window before its pixels stop
    g2d = g["g2d"].cpu().numpy()
    errs = {"g2d_col%d" % j: rel_l2(g2d[:, j], g2d_ref[:, j]) for j in range(9)}
    # 3D gradients: the oracle's chain rule on the primitives the window
    # reaches; every other primitive has a zero 2D gradient on both sides
    sub = scene.subset(touched)
    ref3 = oracle.project_bwd(sub, cam, g2d_ref[touched], P)
    n = scene.n
    got = dict(means=g["means"].cpu().numpy(), scales=g["scales"].cpu().numpy(), quats=g["quats"].cpu().numpy(),
               opac=g["opac"].cpu().numpy(), sh=raster.Splats.sh_from_device_layout(g["sh"], n).cpu().numpy())
    rest = np.ones(n, bool)
    rest[touched] = False
    for k in ("means", "scales", "quats", "opac", "sh"):
        errs[k] = rel_l2(got[k][touched], ref3[k])
        assert not got[k][rest].any(), k
    log_parity("full_size_grad_rel_l2", touched=int(len(touched)), **errs)
    for k, e in errs.items():
        assert e < GRAD_TOL, (k, e)
