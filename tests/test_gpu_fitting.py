"""Pattern fits of Sec. 5.1 (Fig. 5) on the GPU: the training loop built
from the library's own forward, 6:2:2 loss, backward and Adam lowers the
loss, the end-to-end gradient of that loss matches the oracle's, and the
kernels of the family are reported side by side on the same budget."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import train
from paper_2411_12440_gb300 import fitting, raster, training
from tests.gpu_helpers import GRAD_TOL, log_parity, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", fitting.PATTERNS)
def test_fit_lowers_the_loss(kind):
    out = fitting.fit(kind, 4, "linear", size=128, n_side=24, steps=150)
    first, last = out["loss_curve"][0][1], out["loss"]
    log_parity("fit_" + kind, first=first, last=last, psnr=out["psnr_db"])
    assert last < 0.5 * first
    assert out["psnr_db"] > 12.0


def test_loss_gradient_end_to_end_matches_oracle():
    """GPU render -> 6:2:2 loss gradient -> ls_render_bwd, against the oracle's
    render -> FP64 loss gradient -> adjoint, on a fitting scene (pixels the
    oracle flags weighted by zero)."""
    scene, cam = fitting.init_scene(16, 64, seed=3)
    target = fitting.pattern("checkerboard", 4, 64)
    P = dict(sh_degree=0)
    rz = raster.Rasterizer(raster.RenderParams(sh_degree=0))
    sp = raster.Splats.from_scene(scene)
    image, T, state = rz.forward(sp, cam)
    ref = oracle.render_scene(scene, cam, P)
    _, g_ref, _ = train.loss622(ref["image"], target.astype(np.float64))
    g_ref[ref["flags"]] = 0.0
    gimg = torch.empty((64, 64, 3), device="cuda")
    training.ImageLoss(64, 64)(image, torch.from_numpy(target).cuda(), gimg)
    gi = gimg.cpu().numpy()
    e_img = rel_l2(gi[~ref["flags"]], g_ref[~ref["flags"]])
    gi[ref["flags"]] = 0.0
    g = rz.render_bwd(sp, cam, state, torch.from_numpy(gi).cuda(), None)
    torch.cuda.synchronize()
    gr = oracle.scene_grads(scene, cam, g_ref, np.zeros((64, 64)), P)
    errs = dict(dimage=e_img, means=rel_l2(g["means"].cpu().numpy(), gr["means"]),
                scales=rel_l2(g["scales"].cpu().numpy(), gr["scales"]),
                opac=rel_l2(g["opac"].cpu().numpy(), gr["opac"]),
                sh=rel_l2(raster.Splats.sh_from_device_layout(g["sh"], sp.n).cpu().numpy(), gr["sh"]))
    log_parity("fit_step_grad_rel_l2", **errs)
    for k, e in errs.items():
        assert e < GRAD_TOL, (k, e)


def test_kernels_reported_side_by_side():
    t = fitting.sweep(patterns=("stripes",), freqs=(16,), kernels=("linear", "gaussian"), size=128, n_side=24,
                      steps=100)
    row = t["stripes/16"]
    assert set(row) == {"linear", "gaussian"}
    for k, r in row.items():
        assert math.isfinite(r["psnr_db"]) and r["steps"] == 100 and r["prims"] == 24 * 24
    log_parity("fit_stripes16", linear=row["linear"]["psnr_db"], gaussian=row["gaussian"]["psnr_db"])
