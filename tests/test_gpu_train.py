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
