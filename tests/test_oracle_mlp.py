"""Pins of the FP64 termination-MLP reference: its gradient against central
finite differences of its own real-valued forward, the asymmetric loss on a
hand-computed case, and Adam's first step against its closed form."""
import numpy as np
import pytest

from oracle import mlp
from paper_2411_12440_gb300 import scenes


def test_gradient_matches_finite_differences():
    p = scenes.random_mlp_params(1)
    x, t = scenes.random_mlp_batch(40, 2)
    x = x.astype(np.float64)
    loss, g = mlp.loss_and_grad(x, p, t, 3.0, fp16=False)
    h = 1e-6
    fd = np.zeros_like(p)
    for j in range(mlp.NPARAM):
        pp = p.copy()
        pp[j] += h
        lp, _ = mlp.loss_and_grad(x, pp, t, 3.0, fp16=False)
        pp[j] -= 2 * h
        lm, _ = mlp.loss_and_grad(x, pp, t, 3.0, fp16=False)
        fd[j] = (lp - lm) / (2 * h)
    for name in ("w1t", "b1", "w2t", "b2", "w3", "b3"):
        a, b = mlp.OFF[name], list(mlp.OFF.values())[list(mlp.OFF).index(name) + 1] if name != "b3" else mlp.NPARAM
        rel = np.linalg.norm(g[a:b] - fd[a:b]) / max(np.linalg.norm(fd[a:b]), 1e-30)
        assert rel < 1e-6, (name, rel)


def test_asymmetric_loss_hand_computed():
    """Two rows with a zero network except b3 = 1: y = 1 for both; targets
    0 and 3 give errors +1 and -2, weights 1 and u: loss = (1 + 4u) / 2."""
    p = np.zeros(mlp.NPARAM)
    p[mlp.OFF["b3"]] = 1.0
    x = np.zeros((2, 48))
    loss, g = mlp.loss_and_grad(x, p, np.array([0.0, 3.0]), 2.5, fp16=False)
    assert loss == pytest.approx((1 + 4 * 2.5) / 2)
    assert g[mlp.OFF["b3"]] == pytest.approx((2 * 1 + 2 * 2.5 * -2) / 2)


def test_adam_first_step_closed_form():
    """At step 1 the bias-corrected moments are g and g^2, so every
    parameter moves by -lr g / (|g| + eps)."""
    rng = np.random.default_rng(3)
    p0 = rng.normal(size=mlp.NPARAM)
    g = rng.normal(size=mlp.NPARAM)
    lr, eps = 1e-3, 1e-8
    p1, m1, m2 = mlp.adam(1, lr, 0.9, 0.999, eps, p0, g, np.zeros_like(p0), np.zeros_like(p0))
    assert np.allclose(p1 - p0, -lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-15)
    assert np.allclose(m1, 0.1 * g) and np.allclose(m2, 0.001 * g * g)
