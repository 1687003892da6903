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
