"""Pins of the FP64 training-loss and optimiser reference (oracle/train.py)
against what the definitions fix: SSIM of an image with itself, closed forms
for constant images and linear ramps, symmetry, the L1/L2 means, finite
differences of the whole loss, and Adam's first step."""
import math

import numpy as np
import pytest

from oracle import train


def test_window_is_a_normalised_gaussian():
    g = train.gauss_window()
    assert len(g) == 11 and g.sum() == pytest.approx(1.0, abs=1e-15)
    assert g[5] / g[6] == pytest.approx(math.exp(1 / 4.5), rel=1e-14)
    assert np.allclose(g, g[::-1], atol=0)


def test_ssim_of_an_image_with_itself_is_one():
    x = np.random.default_rng(0).random((20, 17, 3))
    s, _ = train.ssim_map(x, x)
    assert np.allclose(s, 1.0, atol=1e-12)
    L, g, parts = train.loss622(x, x)
    assert L == pytest.approx(0.0, abs=1e-12) and np.abs(g).max() < 1e-12


def test_ssim_constant_images_closed_form():
    """x = a, y = b everywhere: away from the border the local variances
    vanish, so SSIM = (2ab + C1) / (a^2 + b^2 + C1)."""
    a, b = 0.3, 0.7
    x = np.full((30, 30, 1), a)
    y = np.full((30, 30, 1), b)
    s, _ = train.ssim_map(x, y)
    want = (2 * a * b + train.C1) / (a * a + b * b + train.C1)
    assert np.allclose(s[5:-5, 5:-5], want, rtol=1e-12)


def test_ssim_linear_ramp_closed_form():
    """x = a, y = b + k (i - i0) along rows: away from the border the window
    keeps linear functions (mean b + k (i - i0)), the variance of y is k^2 V
    with V the window's second moment, and the covariance is 0, so
    SSIM = (2 a my + C1) / (a^2 + my^2 + C1) * C2 / (k^2 V + C2)."""
    a, b, k = 0.4, 0.5, 0.02
    H, W = 40, 24
    i = np.arange(H, dtype=np.float64)[:, None, None]
    x = np.full((H, W, 1), a)
    y = (b + k * (i - 20)) * np.ones((H, W, 1))
    s, t = train.ssim_map(x, y)
    g = train.gauss_window()
    V = float((g * (np.arange(11) - 5.0) ** 2).sum())
    my = b + k * (i - 20)
    want = (2 * a * my + train.C1) / (a * a + my * my + train.C1) * train.C2 / (k * k * V + train.C2)
    want = np.broadcast_to(want, s.shape)
    assert np.allclose(s[5:-5, 5:-5], want[5:-5, 5:-5], rtol=1e-10)


def test_ssim_is_symmetric():
    r = np.random.default_rng(1)
    x, y = r.random((12, 14, 3)), r.random((12, 14, 3))
    assert np.allclose(train.ssim_map(x, y)[0], train.ssim_map(y, x)[0], rtol=1e-13)


def test_l1_l2_terms():
    x = np.zeros((2, 3, 1))
    y = np.zeros((2, 3, 1))
    y[0, 0, 0] = 0.5
    y[1, 2, 0] = -0.25
    _, _, p = train.loss622(x, y)
    assert p["l1"] == pytest.approx(0.75 / 6) and p["l2"] == pytest.approx((0.25 + 0.0625) / 6)


def test_loss_gradient_finite_differences():
    r = np.random.default_rng(2)
    H, W = 9, 13
    y = r.random((H, W, 3))
    # differences bounded away from 0 so the L1 kink is never crossed
    x = np.clip(y + np.where(r.random((H, W, 3)) < 0.5, -1, 1) * (0.05 + 0.2 * r.random((H, W, 3))), -0.5, 1.5)
    L, g, _ = train.loss622(x, y)
    h = 1e-6
    for idx in [(0, 0, 0), (4, 6, 1), (8, 12, 2), (3, 0, 2), (0, 7, 0), (6, 11, 1)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (train.loss622(xp, y)[0] - train.loss622(xm, y)[0]) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=1e-6, abs=1e-11), idx


def test_adam_first_step_moves_by_lr():
    """Bias correction makes the first step -lr sign(g) (|g| >> eps), in the
    unconstrained space of each mode."""
    p = np.array([0.5, 2.0, -1.0])
    g = np.array([3.0, -0.1, 1e-3])
    z = np.zeros(3)
    p1, m, v = train.adam_step(p, g, z, z, 1, 0.01)
    assert np.allclose(p1, p - 0.01 * np.sign(g), rtol=1e-12)
    s = np.array([0.5, 2.0, 0.1])
    s1, _, _ = train.adam_step(s, g, z, z, 1, 0.01, mode=1)
    assert np.allclose(np.log(s1), np.log(s) - 0.01 * np.sign(g), rtol=1e-12)
    o = np.array([0.5, 0.9, 0.1])
    o1, _, _ = train.adam_step(o, g, z, z, 1, 0.01, mode=2)
    lo = np.log(o / (1 - o))
    assert np.allclose(np.log(o1 / (1 - o1)), lo - 0.01 * np.sign(g), rtol=1e-9, atol=1e-12)


def test_densify_accumulate_closed_form():
    """Two primitives in a 200 x 100 view, one culled and one whose box lies
    outside the image: only the first counts; its NDC gradient norm is
    |(gx W/2, gy H/2)| = |(3e-6 * 100, -4e-6 * 50)|."""
    g2d = np.array([[3e-6, -4e-6], [1.0, 1.0], [1.0, 1.0]], np.float32)
    foot = np.array([[50, 50, 10, 20], [50, 50, 10, 10], [-30, 50, 5, 5]], np.float32)
    dkey = np.array([0x40000000, 0xFFFFFFFF, 0x40000000], np.uint32)
    a, c, r = train.densify_accumulate(g2d, foot, dkey, 200, 100, 1, np.zeros(3), np.zeros(3), np.zeros(3))
    assert a[0] == pytest.approx(math.hypot(3e-6 * 100, 4e-6 * 50), rel=1e-6) and a[1] == 0 and a[2] == 0
    assert list(c) == [1, 0, 0] and r[0] == pytest.approx(20 / 200) and r[1] == 0
    a2, c2, r2 = train.densify_accumulate(g2d, foot, dkey, 200, 100, 2, a, c, r)
    assert a2[0] == pytest.approx(3 * a[0], rel=1e-6) and c2[0] == 2


def test_densify_decide_rules():
    """The thresholds of the appendix table (3DLS row) on hand-made cases."""
    th = train.DENSIFY_3DLS
    ext = 10.0
    #            grad high, small   grad high, large   grad low         faint          huge 3D
    accum = np.array([3e-4, 3e-4, 1e-4, 0.0, 0.0], np.float32)
    count = np.array([1, 1, 1, 0, 1], np.int32)
    scales = np.array([[0.05, 0.01, 0.01], [0.07, 0.01, 0.01], [0.01] * 3, [0.01] * 3, [5.0, 1, 1]], np.float32)
    opac = np.array([0.5, 0.5, 0.5, 0.02, 0.5], np.float32)
    rad = np.array([0.0, 0.0, 0.2, 0.0, 0.0], np.float32)
    f = train.densify_decide(accum, count, rad, scales, opac, ext, th)
    assert list(f) == [1, 2, 0, 4, 0]  # 0.05 <= 0.006 * 10 < 0.07
    f = train.densify_decide(accum, count, rad, scales, opac, ext, th, use_scale2d=True, use_prune_scale3d=True)
    assert list(f) == [1, 2, 2 | 4, 4, 4]  # radius 0.2 > 0.05 (split) and > 0.15 (prune); 5 > 0.4 * 10
    # the 3DGS row of the same table grows at 0.01 * extent instead
    f = train.densify_decide(accum, count, rad, scales, opac, ext, train.DENSIFY_3DGS)
    assert list(f) == [1, 1, 0, 0, 0]  # 0.07 <= 0.1; opacity 0.02 >= 0.005


def _cam(fx, W=200, H=100, vm=None):
    from paper_2411_12440_gb300 import scenes
    return scenes.camera(np.eye(4) if vm is None else vm, fx, fx, W / 2, H / 2, W, H)


def test_filter3d_variance_closed_forms():
    """On the axis at depth z: v = 0.2 (z / fx)^2; two cameras: the nearer /
    longer-focal one decides; outside every frustum: the largest v."""
    means = np.array([[0.0, 0.0, 4.0], [0.0, 0.0, 2.0], [100.0, 0.0, 1.0]])
    v = train.filter3d_variance(means, [_cam(100.0)])
    assert v[0] == pytest.approx(0.2 * (4 / 100) ** 2) and v[1] == pytest.approx(0.2 * (2 / 100) ** 2)
    assert v[2] == pytest.approx(v[0])  # x = 100 * 100 + 100 is far outside: takes the largest
    v2 = train.filter3d_variance(means, [_cam(100.0), _cam(300.0)])
    assert v2[0] == pytest.approx(0.2 * (4 / 300) ** 2)
    # the 1.15 margin: a centre at x = 1.1 W is seen, at 1.2 W it is not
    m = np.array([[(1.1 * 200 - 100) * 4 / 100, 0, 4.0], [(1.2 * 200 - 100) * 4 / 100, 0, 4.0], [0, 0, 8.0]])
    v3 = train.filter3d_variance(m, [_cam(100.0)])
    assert v3[0] == pytest.approx(0.2 * 0.04 ** 2) and v3[1] == pytest.approx(v3[2]) == pytest.approx(0.2 * 0.08 ** 2)


def test_filter3d_keeps_opacity_times_volume():
    """o sqrt(det Sigma) = o prod(scales) is what the filter keeps."""
    r = np.random.default_rng(4)
    s = r.random((50, 3)) * 0.1 + 1e-3
    o = r.random(50)
    v = r.random(50) * 1e-3
    se, oe = train.filter3d_apply(s, o, v)
    assert np.allclose(oe * se.prod(1), o * s.prod(1), rtol=1e-13)
    assert np.allclose(se ** 2 - s ** 2, v[:, None], rtol=1e-12, atol=1e-18)
    se0, oe0 = train.filter3d_apply(s, o, np.zeros(50))
    assert np.array_equal(se0, s) and np.allclose(oe0, o, rtol=1e-15)


def test_filter3d_gradient_finite_differences():
    r = np.random.default_rng(5)
    s = r.random((6, 3)) * 0.1 + 0.01
    o = r.random(6)
    v = r.random(6) * 1e-3
    ws, wo = r.standard_normal((6, 3)), r.standard_normal(6)
    f = lambda s_, o_: (train.filter3d_apply(s_, o_, v)[0] * ws).sum() + (train.filter3d_apply(s_, o_, v)[1] * wo).sum()
    g_s, g_o = train.filter3d_apply_bwd(s, o, v, ws, wo)
    h = 1e-7
    for i in range(6):
        for k in range(3):
            sp, sm = s.copy(), s.copy()
            sp[i, k] += h
            sm[i, k] -= h
            assert g_s[i, k] == pytest.approx((f(sp, o) - f(sm, o)) / (2 * h), rel=1e-6, abs=1e-9)
        op, om = o.copy(), o.copy()
        op[i] += h
        om[i] -= h
        assert g_o[i] == pytest.approx((f(s, op) - f(s, om)) / (2 * h), rel=1e-6, abs=1e-9)
