"""FP64 reference of the training-side consumers of the rasterizer's
backward (test infrastructure only: imported by tests/, never by the
product path).

  * loss622     the training loss of the appendix "Loss Functions":
                L = 0.6 L1 + 0.2 L2 + 0.2 (1 - SSIM) over an image pair,
                with its gradient with respect to the rendered image.
  * adam_step   one Adam update of a parameter tensor (the optimiser of the
                pattern-fitting experiment of Sec. 5.1, Fig. 5).

Readings where the paper is silent (SSIM is only named): the SSIM of Wang
et al. 2004 as 3DGS computes it -- per colour channel, an 11 x 11 Gaussian
window of standard deviation 1.5 (normalised to sum 1), zero padding at the
image border, C1 = 0.01^2 and C2 = 0.03^2 for values in [0, 1], the map
averaged over every pixel and channel.  The L1 term's derivative at a zero
difference is taken as 0.  N in the L1 and L2 means counts pixels times
channels.

Pinned in tests/test_oracle_train.py by SSIM(x, x) = 1, closed forms for
constant images (C1) and linear ramps (C2 and the window's second moment),
symmetry, the L1/L2 definitions, and central finite differences of the
whole loss.
"""
import numpy as np
from scipy.ndimage import correlate1d

SSIM_SIZE = 11
SSIM_SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2
WEIGHTS = (0.6, 0.2, 0.2)  # L1, L2, SSIM (the appendix's 6:2:2)


def gauss_window(size=SSIM_SIZE, sigma=SSIM_SIGMA):
    """1D Gaussian taps exp(-k^2 / (2 sigma^2)), k = -size//2 .. size//2,
    normalised to sum 1 (the 2D window is their outer product)."""
    k = np.arange(size, dtype=np.float64) - size // 2
    g = np.exp(-k * k / (2.0 * sigma * sigma))
    return g / g.sum()


def blur(img):
    """Correlation of [H, W, ...] with the 2D window, zero outside the image."""
    g = gauss_window()
    t = correlate1d(np.asarray(img, np.float64), g, axis=0, mode="constant", cval=0.0)
    return correlate1d(t, g, axis=1, mode="constant", cval=0.0)


def ssim_map(x, y):
    """Per-pixel, per-channel SSIM of [H, W, C] images and its parts."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    mx, my = blur(x), blur(y)
    sxx = blur(x * x) - mx * mx
    syy = blur(y * y) - my * my
    sxy = blur(x * y) - mx * my
    a1 = 2.0 * mx * my + C1
    a2 = 2.0 * sxy + C2
    b1 = mx * mx + my * my + C1
    b2 = sxx + syy + C2
    s = a1 * a2 / (b1 * b2)
    return s, dict(mx=mx, my=my, sxx=sxx, syy=syy, sxy=sxy, a1=a1, a2=a2, b1=b1, b2=b2)


def loss622(x, y, weights=WEIGHTS):
    """(L, dL/dx, parts) for rendered x and target y, [H, W, C]."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    wl1, wl2, wss = weights
    n = x.size
    d = x - y
    l1 = np.abs(d).mean()
    l2 = (d * d).mean()
    s, t = ssim_map(x, y)
    ssim = s.mean()
    loss = wl1 * l1 + wl2 * l2 + wss * (1.0 - ssim)
    # d SSIM(q) with respect to the local statistics at q, mx, sxx and sxy
    # taken as independent; then through mx = G x, sxx = G x^2 - mx^2,
    # sxy = G xy - mx my back to every pixel p under the window at q
    ds_dmx = 2.0 * t["my"] * t["a2"] / (t["b1"] * t["b2"]) - s * 2.0 * t["mx"] / t["b1"]
    ds_dsxx = -s / t["b2"]
    ds_dsxy = 2.0 * t["a1"] / (t["b1"] * t["b2"])
    pm = ds_dmx - 2.0 * t["mx"] * ds_dsxx - t["my"] * ds_dsxy
    dssim = blur(pm) + 2.0 * x * blur(ds_dsxx) + y * blur(ds_dsxy)
    grad = (wl1 * np.sign(d) + wl2 * 2.0 * d - wss * dssim) / n
    return loss, grad, dict(l1=l1, l2=l2, ssim=ssim)


def adam_step(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-15, mode=0):
    """One bias-corrected Adam step (step >= 1) in the unconstrained space of
    the parameter: mode 0 p itself, mode 1 log p (p > 0, gradient p g),
    mode 2 logit p (0 < p < 1, gradient p (1 - p) g).  Returns (p, m, v)."""
    p = np.asarray(p, np.float64)
    g = np.asarray(g, np.float64)
    if mode == 1:
        u, gu = np.log(p), g * p
    elif mode == 2:
        u, gu = np.log(p / (1.0 - p)), g * p * (1.0 - p)
    else:
        u, gu = p, g
    m = b1 * m + (1.0 - b1) * gu
    v = b2 * v + (1.0 - b2) * gu * gu
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    u = u - lr * mh / (np.sqrt(vh) + eps)
    if mode == 1:
        p = np.exp(u)
    elif mode == 2:
        p = 1.0 / (1.0 + np.exp(-u))
    else:
        p = u
    return p, m, v
