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


# ------------------------------------------------------------------ densification statistics
# The appendix's densification table gives six thresholds (tau_grad, tau_s2g,
# tau_s3g, tau_s2p, tau_s3p, tau_op) and says the method is built on gsplat
# v1.3, whose default strategy they parametrise.  Reading of how they apply:
#   per step and view, every primitive whose support box meets the image adds
#   the norm of its screen-mean gradient in normalised device units,
#   |(dL/dmx W / 2 n_cams, dL/dmy H / 2 n_cams)|, to its accumulator, counts
#   the view, and keeps the largest support radius max(ex, ey) / max(W, H);
#   at a refinement step, with g = accumulator / max(count, 1):
#     grow   = g > tau_grad
#     small  = max(scale) <= tau_s3g * extent
#     duplicate = grow and small;  split = grow and not small
#                 (or radius > tau_s2g when the 2D rules are on)
#     prune  = opacity < tau_op (or max(scale) > tau_s3p * extent when the
#              3D-scale prune is on, or radius > tau_s2p with the 2D rules).
# Everything is evaluated in binary32 with each operation rounded once, the
# precision the GPU kernels use, so the integer decisions can be compared
# bit for bit.
DENSIFY_3DLS = dict(grad2d=0.0002, grow_scale2d=0.05, grow_scale3d=0.006, prune_scale2d=0.15,
                    prune_scale3d=0.4, prune_opacity=0.025)
DENSIFY_3DGS = dict(grad2d=0.0002, grow_scale2d=0.05, grow_scale3d=0.01, prune_scale2d=0.15,
                    prune_scale3d=0.1, prune_opacity=0.005)

F = np.float32


def densify_accumulate(g2d, foot, dkey, width, height, n_cams, accum, count, max_radius):
    """One view's contribution (binary32).  g2d [n][>=2] (screen-mean
    gradient in pixels), foot [n][4] (mx, my, ex, ey), dkey [n] (0xFFFFFFFF
    when culled); accum, count, max_radius updated and returned."""
    accum = np.array(accum, F)
    count = np.array(count, np.int32)
    max_radius = np.array(max_radius, F)
    W, H = int(width), int(height)
    sx = F(F(W) * F(0.5)) * F(n_cams)
    sy = F(F(H) * F(0.5)) * F(n_cams)
    inv = F(1.0) / F(max(W, H))
    for i in range(len(accum)):
        if int(dkey[i]) == 0xFFFFFFFF:
            continue
        mx, my, ex, ey = (F(v) for v in foot[i])
        # the support box meets a pixel centre of the image (the binary32 tile rule)
        xl, xh = np.ceil(F(F(mx - ex) - F(0.5))), np.floor(F(F(mx + ex) - F(0.5)))
        yl, yh = np.ceil(F(F(my - ey) - F(0.5))), np.floor(F(F(my + ey) - F(0.5)))
        if not (xl <= xh and yl <= yh) or xh < 0 or yh < 0 or xl > W - 1 or yl > H - 1:
            continue
        gx = F(F(g2d[i][0]) * sx)
        gy = F(F(g2d[i][1]) * sy)
        nrm = F(np.sqrt(F(F(gx * gx) + F(gy * gy))))
        accum[i] = F(accum[i] + nrm)
        count[i] += 1
        max_radius[i] = max(max_radius[i], F(max(ex, ey) * inv))
    return accum, count, max_radius


def densify_decide(accum, count, max_radius, scales, opac, extent, th, use_scale2d=False, use_prune_scale3d=False):
    """Flags per primitive: bit 0 duplicate, bit 1 split, bit 2 prune."""
    accum = np.asarray(accum, F)
    count = np.asarray(count, np.int32)
    g = (accum / np.maximum(count, 1).astype(F)).astype(F)
    smax = np.asarray(scales, F).max(axis=1)
    ext = F(extent)
    grow = g > F(th["grad2d"])
    small = smax <= F(F(th["grow_scale3d"]) * ext)
    dup = grow & small
    split = grow & ~small
    if use_scale2d:
        split |= np.asarray(max_radius, F) > F(th["grow_scale2d"])
    prune = np.asarray(opac, F) < F(th["prune_opacity"])
    if use_prune_scale3d:
        prune |= smax > F(F(th["prune_scale3d"]) * ext)
    if use_scale2d:
        prune |= np.asarray(max_radius, F) > F(th["prune_scale2d"])
    return (dup.astype(np.uint8) | (split.astype(np.uint8) << 1) | (prune.astype(np.uint8) << 2))


# ------------------------------------------------------------------ 3D smoothing filter
# Sec. 4.1 evaluates a 3DLS+AA variant with "the technique from
# Mip-Splatting": its 2D filter is the eps2d dilation with opacity
# compensation of the projection; its 3D smoothing filter, read here, bounds
# the frequency of each primitive by the highest sampling rate any camera
# gives it: nu_i = max over cameras that see its centre of fx / z (z its
# camera depth, > near; "sees": the projected centre within 1.15x the image,
# i.e. x in [-0.15 W, 1.15 W], y in [-0.15 H, 1.15 H]), and adds the
# variance s^2 / nu_i^2 (s^2 = 0.2) to all three axes: the covariance
# R diag(scale^2) R^T becomes R diag(scale^2 + v) R^T, so the scales become
# sqrt(scale^2 + v) and the opacity o prod_k scale_k / sqrt(scale_k^2 + v)
# keeps o sqrt(det Sigma).  A primitive no camera sees takes the largest
# variance of the others.
FILTER3D_S2 = 0.2


def filter3d_variance(means, cams, near=0.2, s2=FILTER3D_S2):
    """[n] variance of the 3D filter (FP64)."""
    means = np.asarray(means, np.float64)
    n = len(means)
    best = np.zeros(n)  # highest sampling rate seen, 0 = none
    for cam in cams:
        V = np.asarray(cam["viewmat"], np.float64).reshape(4, 4)
        t = means @ V[:3, :3].T + V[:3, 3]
        z = t[:, 2]
        ok = z > near
        zs = np.where(ok, z, 1.0)
        x = cam["fx"] * t[:, 0] / zs + cam["cx"]
        y = cam["fy"] * t[:, 1] / zs + cam["cy"]
        W, H = cam["width"], cam["height"]
        ok &= (x >= -0.15 * W) & (x <= 1.15 * W) & (y >= -0.15 * H) & (y <= 1.15 * H)
        best = np.where(ok, np.maximum(best, cam["fx"] / zs), best)
    seen = best > 0
    var = np.zeros(n)
    var[seen] = s2 / best[seen] ** 2
    if (~seen).any():
        var[~seen] = var[seen].max() if seen.any() else 0.0
    return var


def filter3d_apply(scales, opac, var):
    """Scales and opacities after the 3D filter (FP64)."""
    s = np.asarray(scales, np.float64)
    v = np.asarray(var, np.float64)[:, None]
    se = np.sqrt(s * s + v)
    return se, np.asarray(opac, np.float64) * np.prod(s / se, axis=1)


def filter3d_apply_bwd(scales, opac, var, g_se, g_oe):
    """Gradients with respect to the unfiltered scales and opacities."""
    s = np.asarray(scales, np.float64)
    v = np.asarray(var, np.float64)[:, None]
    se2 = s * s + v
    se = np.sqrt(se2)
    ratio = np.prod(s / se, axis=1)
    oe = np.asarray(opac, np.float64) * ratio
    g_s = np.asarray(g_se, np.float64) * s / se + (np.asarray(g_oe, np.float64) * oe)[:, None] * v / (s * se2)
    g_o = np.asarray(g_oe, np.float64) * ratio
    return g_s, g_o
