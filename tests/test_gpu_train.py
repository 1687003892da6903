"""GPU parity of the training-side consumers of the backward against the
FP64 references of oracle/train.py: the 6:2:2 image loss (L1, L2, SSIM)
with its gradient, and the Adam step in each parameter space."""
import numpy as np
import pytest
import torch

from oracle import train
from paper_2411_12440_gb300 import training
from tests.gpu_helpers import log_parity, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("H,W", [(1, 1), (37, 53), (256, 256), (1080, 1920)])
def test_image_loss_matches_oracle(H, W):
    r = np.random.default_rng(H + W)
    y = r.random((H, W, 3)).astype(np.float32)
    x = np.clip(y + 0.1 * r.standard_normal((H, W, 3)), 0, 1).astype(np.float32)
    L, g, parts = train.loss622(x.astype(np.float64), y.astype(np.float64))
    loss = training.ImageLoss(H, W)
    gx = torch.empty((H, W, 3), device="cuda")
    out = loss(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), gx)
    torch.cuda.synchronize()
    o = out.cpu().numpy().astype(np.float64)
    e_grad = rel_l2(gx.cpu().numpy(), g)
    log_parity("loss622", total=float(abs(o[0] - L) / L), l1=float(abs(o[1] - parts["l1"]) / parts["l1"]),
               l2=float(abs(o[2] - parts["l2"]) / parts["l2"]), ssim=float(abs(o[3] - parts["ssim"])), grad=e_grad)
    assert o[0] == pytest.approx(L, rel=1e-5)
    assert o[1] == pytest.approx(parts["l1"], rel=1e-5)
    assert o[2] == pytest.approx(parts["l2"], rel=1e-5)
    assert o[3] == pytest.approx(parts["ssim"], abs=1e-5)
    assert e_grad < 1e-4


def test_image_loss_of_identical_images_is_zero():
    y = torch.rand((64, 80, 3), device="cuda")
    g = torch.full((64, 80, 3), 7.0, device="cuda")
    out = training.ImageLoss(64, 80)(y, y.clone(), g)
    torch.cuda.synchronize()
    assert abs(float(out[0])) < 1e-6 and abs(float(out[3]) - 1.0) < 1e-6
    assert float(g.abs().max()) < 1e-7


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_adam_matches_oracle(mode):
    r = np.random.default_rng(mode)
    n = 100_003
    p = r.uniform(0.05, 0.95, n).astype(np.float32)
    pt = torch.from_numpy(p).cuda()
    m1 = torch.zeros(n, device="cuda")
    m2 = torch.zeros(n, device="cuda")
    pr, mr, vr = p.astype(np.float64), np.zeros(n), np.zeros(n)
    for step in range(1, 4):
        g = r.standard_normal(n).astype(np.float32)
        training.adam_(pt, torch.from_numpy(g).cuda(), m1, m2, step, 1e-3, mode=mode)
        pr, mr, vr = train.adam_step(pr, g.astype(np.float64), mr, vr, step, 1e-3, eps=1e-15, mode=mode)
    torch.cuda.synchronize()
    err = np.abs(pt.cpu().numpy() - pr).max()
    log_parity("adam", mode=mode, max_abs=float(err))
    assert err < 2e-6


def _rand_views(R, W, H, seed):
    from paper_2411_12440_gb300 import scenes
    from tests.gpu_helpers import pack_records
    rec = scenes.random_records(R, W, H, seed=seed, visible_frac=0.8)
    rec["mean2d"][: R // 10] -= 2 * max(W, H)  # some boxes entirely off the image
    proj, dkey = pack_records(rec)
    foot = np.concatenate([rec["mean2d"], rec["ext"]], 1).astype(np.float32)
    return proj, foot, dkey


def test_densify_statistics_match_oracle_bitwise():
    """Two views accumulated on the GPU and by the binary32 reference: the
    same bits (every operation is rounded once on both sides)."""
    from paper_2411_12440_gb300 import scenes
    R, W, H = 50_000, 640, 360
    st = training.DensifyStats(R)
    a, c, m = np.zeros(R, np.float32), np.zeros(R, np.int32), np.zeros(R, np.float32)
    r = np.random.default_rng(9)
    for v in range(2):
        proj, foot, dkey = _rand_views(R, W, H, seed=20 + v)
        g2d = (r.standard_normal((R, 12)) * 1e-5).astype(np.float32)
        st.accumulate(torch.from_numpy(g2d).cuda(), proj, scenes.identity_camera(W, H), n_cams=1)
        a, c, m = train.densify_accumulate(g2d, foot, dkey, W, H, 1, a, c, m)
    torch.cuda.synchronize()
    assert np.array_equal(st.grad_accum.cpu().numpy().view(np.uint32), a.view(np.uint32))
    assert np.array_equal(st.count.cpu().numpy(), c)
    assert np.array_equal(st.max_radius.cpu().numpy().view(np.uint32), m.view(np.uint32))
    assert 0 < (c > 0).sum() < R


@pytest.mark.parametrize("rules", [(False, False), (True, True)])
def test_densify_decision_matches_oracle_bitwise(rules):
    from paper_2411_12440_gb300 import raster
    r = np.random.default_rng(11)
    n = 100_000
    accum = (r.random(n) * 6e-4).astype(np.float32)
    count = r.integers(0, 4, n).astype(np.int32)
    rad = (r.random(n) * 0.3).astype(np.float32)
    scales = (r.random((n, 3)) ** 3 * 0.1).astype(np.float32)
    opac = r.random(n).astype(np.float32)
    extent = 4.0
    want = train.densify_decide(accum, count, rad, scales, opac, extent, train.DENSIFY_3DLS, *rules)
    st = training.DensifyStats(n)
    st.grad_accum.copy_(torch.from_numpy(accum))
    st.count.copy_(torch.from_numpy(count))
    st.max_radius.copy_(torch.from_numpy(rad))
    sp = raster.Splats(torch.zeros((n, 3), device="cuda"), torch.from_numpy(scales).cuda(),
                       torch.zeros((n, 4), device="cuda"), torch.from_numpy(opac).cuda(), torch.zeros((3, n), device="cuda"), 0)
    flags, counts = st.decide(sp, extent, training.DENSIFY_3DLS, *rules)
    torch.cuda.synchronize()
    got = flags.cpu().numpy()
    assert np.array_equal(got, want)
    assert counts.cpu().tolist() == [int(((want >> b) & 1).sum()) for b in range(3)]
    assert all(0 < int(((want >> b) & 1).sum()) < n for b in range(3))
