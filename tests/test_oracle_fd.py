"""The oracle's adjoint against central finite differences of its own FP64
forward (Eq. 6 with the kernel of Eq. 12, projection of Eq. 1-4), and the
AGS scaling of Eq. 13-14 against its closed form.

Scenes are rejected when a pixel/primitive pair sits within a margin of a
kink or jump of the forward (support edge, alpha threshold, centre cone
point), so the difference quotient measures the derivative.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2411_12440_gb300 import scenes

# FP64 rounding of a loss of size ~10 gives ~1e-8 absolute error at this step,
# while perturbed distances move by ~1e-6, well inside the 2e-5 kink margins.
H_STEP = 1e-7
MARGIN = 2e-5


def _fd_scene(seed, deg, n=64, size=32, f=40.0, rho_typ=2.48):
    s = scenes.box_scene(n, seed, deg)
    # overlapping footprints in a 32x32 view, of similar pixel size whatever
    # the kernel's support radius rho_typ (in units of the 2D std)
    s.scales = s.scales * (15.0 / rho_typ)
    s = scenes.Scene(*(a.astype(np.float64) for a in (s.means, s.scales, s.quats, s.opac, s.sh)), deg)
    cam = scenes.camera(np.eye(4), f, f, size / 2 + 0.13, size / 2 - 0.21, size, size)
    return s, cam


def _pair_margins(proj, vis, W, H):
    """Smallest distance, over all pixel/primitive pairs of visible primitives,
    of D to the support end rho (where alpha crosses alpha_min, or the
    kernel's own end when alpha_min = 0) and to the centre cone point D = 0."""
    ys, xs = np.mgrid[0:H, 0:W] + 0.5
    m_support, m_centre = np.inf, np.inf
    for i in np.nonzero(vis)[0]:
        p = proj[i]
        dx, dy = xs - p[oracle.P_MX], ys - p[oracle.P_MY]
        q = p[oracle.P_A] * dx * dx + 2 * p[oracle.P_B] * dx * dy + p[oracle.P_C] * dy * dy
        D = np.sqrt(np.maximum(q, 0))
        m_support = min(m_support, np.abs(D - np.sqrt(p[oracle.P_RHO2])).min())
        m_centre = min(m_centre, D.min())
    return m_support, m_centre


def _loss(scene, cam, P, w, v):
    out = oracle.render_scene(scene, cam, P)
    return float((out["image"] * w).sum() + (out["T"] * v).sum())


def _pick_scene(deg, P, seeds):
    rho_typ = P.get("lam", 2.5) * oracle.kernel_support(P.get("kernel", 0), 0.5, 1 / 255)
    for seed in seeds:
        s, cam = _fd_scene(seed, deg, rho_typ=rho_typ)
        Pd = dict(P, sh_degree=deg)
        proj, vis = oracle.project(s, cam, Pd)
        out = oracle.render(proj, vis, cam["width"], cam["height"], Pd)
        m_sup, m_cen = _pair_margins(proj, vis, cam["width"], cam["height"])
        # keep every pair off the support jump and the cone point, and T well
        # above T_min so no stop decision can flip
        ok = m_sup > MARGIN and m_cen > MARGIN and out["T"].min() > 2e-3
        if ok:
            return s, cam, Pd
    raise RuntimeError("no kink-free scene among the seeds")


CASES = [
    ("smooth_sh0", 0, dict(alpha_min=0.0, t_min=0.0, eps2d=0.3)),
    ("default_sh0", 0, dict()),
    ("default_sh3_aa", 3, dict(antialias=1)),
    ("smooth_sh1_noeps", 1, dict(alpha_min=0.0, t_min=0.0, eps2d=0.0)),
    # kernel family of Appendix B with the alignment factors it states
    ("default_gaussian", 0, dict(kernel=1, lam=1.0)),
    ("default_laplacian", 0, dict(kernel=2, lam=1.0)),
    ("default_cosine", 0, dict(kernel=3, lam=2.5)),
    ("default_quadratic", 0, dict(kernel=4, lam=6.0)),
    ("default_ags_is_not_a_gradient_so_off", 0, dict(ags=0, bg=(0.3, 0.6, 0.1))),
]


@pytest.mark.parametrize("name,deg,P", CASES, ids=[c[0] for c in CASES])
def test_adjoint_matches_finite_differences(name, deg, P):
    s, cam, Pd = _pick_scene(deg, P, range(10, 60))
    w, v = scenes.loss_weights(cam["height"], cam["width"], seed=99)
    w, v = w.astype(np.float64), v.astype(np.float64)
    g = oracle.scene_grads(s, cam, w, v, Pd)
    for field in ("means", "scales", "quats", "opac", "sh"):
        arr = getattr(s, field)
        fd = np.zeros_like(arr)
        flat = arr.reshape(-1)
        fdf = fd.reshape(-1)
        for j in range(flat.size):
            x0 = flat[j]
            flat[j] = x0 + H_STEP
            lp = _loss(s, cam, Pd, w, v)
            flat[j] = x0 - H_STEP
            lm = _loss(s, cam, Pd, w, v)
            flat[j] = x0
            fdf[j] = (lp - lm) / (2 * H_STEP)
        ad = g[field].reshape(fd.shape)
        rel = np.linalg.norm(ad - fd) / max(np.linalg.norm(fd), 1e-30)
        assert np.linalg.norm(fd) > 0, field
        assert rel < 1e-5, (field, rel)


def test_blend_adjoint_matches_finite_differences_2d():
    """d/d(mx, my, a, b, c, o_eff, rgb) of the composite, lists held fixed."""
    s, cam, Pd = _pick_scene(0, dict(), range(70, 120))
    W, H = cam["width"], cam["height"]
    proj, vis = oracle.project(s, cam, Pd)
    w, v = scenes.loss_weights(H, W, seed=5)
    w, v = w.astype(np.float64), v.astype(np.float64)
    g2d = oracle.render_bwd(proj, vis, W, H, w, v, Pd)
    cols = [oracle.P_MX, oracle.P_MY, oracle.P_A, oracle.P_B, oracle.P_C, oracle.P_O, oracle.P_R, oracle.P_G,
            oracle.P_BL]

    def L(pp):
        o = oracle.render(pp, vis, W, H, Pd)
        return (o["image"] * w).sum() + (o["T"] * v).sum()

    fd = np.zeros_like(g2d)
    for i in np.nonzero(vis)[0]:
        for j, c in enumerate(cols):
            pp = proj.copy()
            h = H_STEP * max(1.0, abs(proj[i, c]))
            pp[i, c] += h
            lp = L(pp)
            pp[i, c] -= 2 * h
            lm = L(pp)
            fd[i, j] = (lp - lm) / (2 * h)
    for j in range(9):
        rel = np.linalg.norm(g2d[:, j] - fd[:, j]) / max(np.linalg.norm(fd[:, j]), 1e-30)
        assert rel < 1e-5, (j, rel)


@pytest.mark.parametrize("ags", [1, 2])
def test_ags_scaling_closed_form(ags):
    """Eq. 13-14 on one primitive and one pixel: the geometric gradients are
    scaled by w(D) = exp(-D^2) (exp(-(D/lambda)^2) for the aligned reading),
    opacity and colour gradients are unchanged."""
    z, f, eps = 4.0, 100.0, 0.3
    sc = float(np.float32(0.2))
    sh = np.zeros((1, 1, 3))
    sh[0, 0] = scenes.dc_for_colour(np.array([0.9, 0.4, 0.1]))
    s = scenes.Scene(np.array([[0.0, 0.0, z]]), np.array([[sc, sc, sc]]), np.array([[1.0, 0, 0, 0]]),
                     np.array([0.7]), sh, 0)
    cam = scenes.camera(np.eye(4), f, f, 24.5, 24.5, 48, 48)
    sigma = math.sqrt((f * sc / z) ** 2 + eps)
    proj, vis = oracle.project(s, cam)
    for k, dy in ((3, 1), (5, 2), (8, 0)):
        gC = np.zeros((48, 48, 3))
        gC[24 + dy, 24 + k] = (0.3, -0.7, 0.5)
        gT = np.zeros((48, 48))
        gT[24 + dy, 24 + k] = 0.4
        g0 = oracle.render_bwd(proj, vis, 48, 48, gC, gT, dict())
        g1 = oracle.render_bwd(proj, vis, 48, 48, gC, gT, dict(ags=ags))
        D = math.hypot(k, dy) / sigma
        wgt = math.exp(-D * D) if ags == 1 else math.exp(-(D / 2.5) ** 2)
        assert np.allclose(g1[0, :5], g0[0, :5] * wgt, rtol=1e-12, atol=1e-300)
        assert np.abs(g0[0, :2]).max() > 0
        assert np.array_equal(g1[0, 5:], g0[0, 5:])
