"""The anti-aliased variant (Sec. 4.1, 3DLS+AA): the 3D smoothing filter's
variances, filtered parameters and chain rule against the FP64 reference
(oracle/train.py), and a full render with both filters (3D and the 2D
eps2d dilation with opacity compensation) against the oracle, forward and
backward."""
import numpy as np
import pytest
import torch

import oracle
from oracle import train
from paper_2411_12440_gb300 import antialias, raster, scenes
from tests.gpu_helpers import GRAD_TOL, assert_image_parity, log_parity, rel_l2

pytestmark = pytest.mark.gpu


def _ring(k, size=(640, 480)):
    cams = []
    for a in np.linspace(0, 2 * np.pi, k, endpoint=False):
        eye = np.array([4.0 * np.cos(a), 0.3, 4.0 * np.sin(a)])
        cams.append(scenes.look_at_camera(eye, np.zeros(3), size[0], size[1]))
    return cams


def test_filter_variance_matches_oracle():
    scene, _, _ = scenes.make_workload("scene_1m_1297x840_aa", n=200_000)
    cams = _ring(8)
    sp = raster.Splats.from_scene(scene)
    f = antialias.Filter3D(sp, cams)
    torch.cuda.synchronize()
    got = f.var.cpu().numpy().astype(np.float64)
    want = train.filter3d_variance(scene.means.astype(np.float64), cams)
    rel = np.abs(got - want) / want
    bad = rel > 1e-5
    log_parity("filter3d_var", max_rel_agreeing=float(rel[~bad].max()), disagreeing_frac=float(bad.mean()),
               unseen_frac=float((want == want.max()).mean()))
    # a centre within rounding of a frustum edge may pick another camera
    assert bad.mean() < 1e-4
    assert rel[~bad].max() < 1e-5


def test_filter_apply_and_chain_rule_match_oracle():
    r = np.random.default_rng(2)
    n = 100_000
    s = (r.random((n, 3)) * 0.05 + 1e-3).astype(np.float32)
    o = r.random(n).astype(np.float32)
    v = (r.random(n) * 1e-3).astype(np.float32)
    gs_, go_ = r.standard_normal((n, 3)).astype(np.float32), r.standard_normal(n).astype(np.float32)
    sp = raster.Splats(torch.zeros((n, 3), device="cuda"), torch.from_numpy(s).cuda(),
                       torch.zeros((n, 4), device="cuda"), torch.from_numpy(o).cuda(), torch.zeros((3, n), device="cuda"),
                       0)
    f = antialias.Filter3D.__new__(antialias.Filter3D)
    f.n = n
    f.var = torch.from_numpy(v).cuda()
    spf = f.apply(sp)
    gs, go = f.backward(sp, torch.from_numpy(gs_).cuda(), torch.from_numpy(go_).cuda())
    torch.cuda.synchronize()
    se, oe = train.filter3d_apply(s, o, v)
    ws, wo = train.filter3d_apply_bwd(s, o, v, gs_, go_)
    errs = dict(scales=rel_l2(spf.scales.cpu().numpy(), se), opac=rel_l2(spf.opac.cpu().numpy(), oe),
                g_scales=rel_l2(gs.cpu().numpy(), ws), g_opac=rel_l2(go.cpu().numpy(), wo))
    log_parity("filter3d_apply", **errs)
    for k, e in errs.items():
        assert e < 1e-6, (k, e)


def test_full_aa_variant_render_matches_oracle():
    """3D filter from 8 ring cameras, then the render of one of them with the
    2D filter on: image and gradients of the unfiltered parameters."""
    scene, _, _ = scenes.make_workload("scene_1m_1297x840_aa", n=20_000)
    cams = _ring(8)
    cam = cams[3]
    P = dict(sh_degree=3, antialias=1)
    sp = raster.Splats.from_scene(scene)
    f = antialias.Filter3D(sp, cams)
    spf = f.apply(sp)
    rz = raster.Rasterizer(raster.RenderParams.from_dict(P))
    image, T, state = rz.forward(spf, cam)
    torch.cuda.synchronize()
    rz.check_status()
    var = f.var.cpu().numpy().astype(np.float64)
    se, oe = train.filter3d_apply(scene.scales, scene.opac, var)
    filt = scenes.Scene(scene.means, se.astype(np.float32), scene.quats, oe.astype(np.float32), scene.sh,
                        scene.sh_degree)
    ref = oracle.render_scene(filt, cam, P)
    assert_image_parity(image.cpu().numpy(), ref)
    w, v = scenes.loss_weights(cam["height"], cam["width"], seed=5)
    w[ref["flags"]] = 0.0
    v[ref["flags"]] = 0.0
    g = rz.render_bwd(spf, cam, state, torch.from_numpy(w).cuda(), torch.from_numpy(v).cuda())
    gs, go = f.backward(sp, g["scales"], g["opac"])
    torch.cuda.synchronize()
    gr = oracle.scene_grads(filt, cam, w.astype(np.float64), v.astype(np.float64), P)
    ws, wo = train.filter3d_apply_bwd(scene.scales, scene.opac, var, gr["scales"], gr["opac"])
    errs = dict(means=rel_l2(g["means"].cpu().numpy(), gr["means"]), scales=rel_l2(gs.cpu().numpy(), ws),
                opac=rel_l2(go.cpu().numpy(), wo))
    log_parity("aa_variant_grad_rel_l2", **errs)
    for k, e in errs.items():
        assert e < GRAD_TOL, (k, e)
