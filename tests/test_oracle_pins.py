"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper's equations fix (tests/golden), closed forms, textbook identities,
brute force and invariants.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2411_12440_gb300 import scenes

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_table(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split()[:4])
    return rows


# ------------------------------------------------------------------ kernels
def test_kernel_values_fixed_by_paper():
    """Eq. 9, 21-25: the attenuation functions at points the formulas fix."""
    for kid, name, x, fx in _read_table("paper_kernel_values.txt"):
        assert oracle.kernel_f(int(kid), float(x)) == pytest.approx(float(fx), abs=1e-15), (name, x)


def test_kernel_integrals_closed_form():
    """Radial integral of f(r / lambda) over the plane for each kernel, at the
    paper's alignment factors (Appendix B): linear pi l^2/3, cosine
    pi l^2 (1/2 - 2/pi^2), quadratic pi l^2/2, laplacian 2 pi l^2."""
    closed = {0: lambda l: math.pi * l * l / 3.0,
              3: lambda l: math.pi * l * l * (0.5 - 2.0 / math.pi ** 2),
              4: lambda l: math.pi * l * l / 2.0,
              2: lambda l: 2.0 * math.pi * l * l}
    for kid, name, lam, _ in _read_table("paper_alignment.txt"):
        kid, lam = int(kid), float(lam)
        rmax = lam * (40.0 if kid == 2 else 1.0)
        r = np.linspace(0.0, rmax, 400001)
        f = np.array([oracle.kernel_f(kid, x) for x in (r / lam)[::50]])
        rr = r[::50]
        integ = np.trapezoid(f * 2 * math.pi * rr, rr)
        assert integ == pytest.approx(closed[kid](lam), rel=1e-5), name


def test_linear_kernel_alignment_closed_form():
    """Eq. 12 with lambda = 2.5: L(0) = 1, L(lambda/2) = 1/2, L(lambda) = 0."""
    lam = 2.5
    assert oracle.kernel_f(0, 0.0 / lam) == 1.0
    assert oracle.kernel_f(0, (lam / 2) / lam) == 0.5
    assert oracle.kernel_f(0, lam / lam) == 0.0
    assert oracle.kernel_f(0, 3.0 / lam) == 0.0


@pytest.mark.parametrize("kid", [0, 1, 2, 3, 4])
def test_kernel_support_is_alpha_threshold(kid):
    """The support radius x_s is where o f(x_s) = alpha_min."""
    for o in (0.05, 0.3, 0.999):
        xs = oracle.kernel_support(kid, o, 1.0 / 255.0)
        assert o * oracle.kernel_f(kid, xs) == pytest.approx(1.0 / 255.0, rel=1e-9)
        assert o * oracle.kernel_f(kid, xs * 1.001) < 1.0 / 255.0


# ------------------------------------------------------------------ SH basis
def _sphere_quadrature(nz=12, nphi=24):
    z, wz = np.polynomial.legendre.leggauss(nz)
    phi = (np.arange(nphi) + 0.5) * 2 * math.pi / nphi
    Z, PHI = np.meshgrid(z, phi, indexing="ij")
    W = np.outer(wz, np.full(nphi, 2 * math.pi / nphi))
    s = np.sqrt(1 - Z ** 2)
    dirs = np.stack([s * np.cos(PHI), s * np.sin(PHI), Z], -1).reshape(-1, 3)
    return dirs, W.reshape(-1)


def test_sh_orthonormal():
    """Real SH up to degree 3 are orthonormal on the sphere (exact quadrature)."""
    dirs, w = _sphere_quadrature()
    Y = oracle.sh_basis(dirs, 3)
    G = (Y * w[:, None]).T @ Y
    assert np.abs(G - np.eye(16)).max() < 1e-12


def test_sh_addition_theorem_and_sign_convention():
    """sum_m Y_lm(u)^2 = (2l+1)/(4 pi) for every unit u (addition theorem);
    Y_l0(z-axis) = sqrt((2l+1)/(4 pi)); with the Condon-Shortley phase
    Y_11(x-axis) = -sqrt(3/(4 pi)) and Y_1,-1(y-axis) = -sqrt(3/(4 pi))."""
    rng = np.random.default_rng(5)
    u = rng.standard_normal((50, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    Y = oracle.sh_basis(u, 3)
    for l in range(4):
        s = (Y[:, l * l:(l + 1) * (l + 1)] ** 2).sum(1)
        assert np.allclose(s, (2 * l + 1) / (4 * math.pi), atol=1e-13)
    Yz = oracle.sh_basis(np.array([[0.0, 0.0, 1.0]]), 3)[0]
    for l in range(4):
        assert Yz[l * l + l] == pytest.approx(math.sqrt((2 * l + 1) / (4 * math.pi)), abs=1e-14)
    c1 = math.sqrt(3 / (4 * math.pi))
    assert oracle.sh_basis(np.array([[1.0, 0.0, 0.0]]), 1)[0][3] == pytest.approx(-c1, abs=1e-15)
    assert oracle.sh_basis(np.array([[0.0, 1.0, 0.0]]), 1)[0][1] == pytest.approx(-c1, abs=1e-15)


# ------------------------------------------------------------------ projection
def _f(x):
    """The value a float32 input actually holds."""
    return float(np.float32(x))


def _one(mu, s, q, o=0.8, colour=(0.2, 0.5, 0.9), deg=0):
    k = (deg + 1) ** 2
    sh = np.zeros((1, k, 3), np.float32)
    sh[0, 0] = scenes.dc_for_colour(np.array(colour))
    return scenes.Scene(np.array([mu], np.float32), np.array([s], np.float32), np.array([q], np.float32),
                        np.array([o], np.float32), sh, deg)


def _cam(w=64, h=64, f=100.0, cx=None, cy=None, vm=None):
    return scenes.camera(np.eye(4) if vm is None else vm, f, f, w / 2 if cx is None else cx,
                         h / 2 if cy is None else cy, w, h)


def test_projection_isotropic_on_axis():
    """Isotropic scale s at depth z on the optical axis: Sigma_2D = (f s / z)^2 I
    (Eq. 3-4), centre at the principal point, conic = 1 / (Sigma_2D + eps)."""
    s, z, f, eps = _f(0.05), 3.0, 100.0, 0.3
    sc = _one((0, 0, z), (s, s, s), (1, 0, 0, 0))
    proj, vis = oracle.project(sc, _cam(f=f), dict(eps2d=eps))
    p = proj[0]
    var = (f * s / z) ** 2 + eps
    assert vis[0]
    assert p[oracle.P_MX] == pytest.approx(32.0, abs=1e-12) and p[oracle.P_MY] == pytest.approx(32.0, abs=1e-12)
    assert p[oracle.P_SXX] == pytest.approx(var, rel=1e-12) and p[oracle.P_SYY] == pytest.approx(var, rel=1e-12)
    assert abs(p[oracle.P_SXY]) < 1e-15
    assert p[oracle.P_A] == pytest.approx(1 / var, rel=1e-12) and p[oracle.P_C] == pytest.approx(1 / var, rel=1e-12)
    assert p[oracle.P_DEPTH] == pytest.approx(z)
    assert p[oracle.P_R:oracle.P_BL + 1] == pytest.approx([0.2, 0.5, 0.9], abs=1e-7)
    rho = 2.5 * (1 - (1 / 255) / _f(0.8))
    assert p[oracle.P_RHO2] == pytest.approx(rho * rho, rel=1e-6)
    assert p[oracle.P_EX] == pytest.approx(rho * math.sqrt(var), rel=1e-6)


def test_projection_rotated_anisotropic():
    """Rotation by theta about the optical axis, scales (s1, s2, s3), centre on
    the axis: Sigma_2D = (f/z)^2 R2 diag(s1^2, s2^2) R2^T."""
    th, z, f = 0.7, 4.0, 120.0
    s1, s2, s3 = _f(0.08), _f(0.02), _f(0.05)
    q = (_f(math.cos(th / 2)), 0.0, 0.0, _f(math.sin(th / 2)))
    qn = math.hypot(q[0], q[3])
    th = 2 * math.atan2(q[3] / qn, q[0] / qn)
    sc = _one((0, 0, z), (s1, s2, s3), q)
    proj, _ = oracle.project(sc, _cam(f=f), dict(eps2d=0.0))
    R2 = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    S = (f / z) ** 2 * R2 @ np.diag([s1 * s1, s2 * s2]) @ R2.T
    p = proj[0]
    assert p[oracle.P_SXX] == pytest.approx(S[0, 0], rel=1e-6)
    assert p[oracle.P_SXY] == pytest.approx(S[0, 1], rel=1e-6)
    assert p[oracle.P_SYY] == pytest.approx(S[1, 1], rel=1e-6)


# ------------------------------------------------------------------ anti-aliasing compensation
# Sec. 4.1 names the Mip-Splatting anti-aliasing; its 2D filter dilates the
# screen covariance by eps2d I and scales the opacity by
# sqrt(det Sigma_2D / det(Sigma_2D + eps2d I)), so that the footprint keeps
# the integral it had before the dilation.  The pins below fix that factor
# from outside the oracle: its value at eps2d = 0, two closed forms, and the
# integral it preserves.
def test_aa_eps_zero_is_plain_bitwise():
    """With eps2d = 0 the dilated and the plain covariance are the same
    numbers, so the factor is exactly 1: AA on gives the AA-off records bit
    for bit."""
    s = scenes.box_scene(300, 3, sh_degree=1)
    cam = scenes.identity_camera(128, 96)
    p0, v0 = oracle.project(s, cam, dict(eps2d=0.0, antialias=0))
    p1, v1 = oracle.project(s, cam, dict(eps2d=0.0, antialias=1))
    assert v0.sum() > 100 and np.array_equal(v0, v1)
    assert np.array_equal(p0, p1)


@pytest.mark.parametrize("eps", [0.05, 0.3, 2.0])
def test_aa_isotropic_on_axis_closed_form(eps):
    """Isotropic s at depth z on the axis: Sigma_2D = v I with v = (f s / z)^2,
    so the factor is sqrt(v^2 / (v + eps)^2) = v / (v + eps)."""
    s, z, f, o = _f(0.02), 3.0, 100.0, _f(0.9)
    sc = _one((0, 0, z), (s, s, s), (1, 0, 0, 0), o=o)
    v = (f * s / z) ** 2
    p_on = oracle.project(sc, _cam(f=f), dict(eps2d=eps, antialias=1))[0][0]
    p_off = oracle.project(sc, _cam(f=f), dict(eps2d=eps, antialias=0))[0][0]
    assert p_off[oracle.P_O] == pytest.approx(o, abs=0)
    assert p_on[oracle.P_O] == pytest.approx(o * v / (v + eps), rel=1e-12)
    # the support radius follows the compensated opacity (Eq. 12, alpha_min)
    rho = 2.5 * (1 - (1 / 255) / (o * v / (v + eps)))
    assert p_on[oracle.P_RHO2] == pytest.approx(rho * rho, rel=1e-10)


@pytest.mark.parametrize("th", [0.0, 0.7, 2.1])
def test_aa_rotated_anisotropic_det_ratio(th):
    """Scales (s1, s2) rotated by th about the axis: Sigma_2D has eigenvalues
    a = (f s1 / z)^2 and b = (f s2 / z)^2 whatever th, so the factor is
    sqrt(a b / ((a + eps)(b + eps)))."""
    z, f, eps, o = 4.0, 120.0, 0.3, _f(0.6)
    s1, s2, s3 = _f(0.08), _f(0.01), _f(0.05)
    q = (_f(math.cos(th / 2)), 0.0, 0.0, _f(math.sin(th / 2)))
    sc = _one((0, 0, z), (s1, s2, s3), q, o=o)
    p = oracle.project(sc, _cam(f=f), dict(eps2d=eps, antialias=1))[0][0]
    a, b = (f * s1 / z) ** 2, (f * s2 / z) ** 2
    assert p[oracle.P_O] == pytest.approx(o * math.sqrt(a * b / ((a + eps) * (b + eps))), rel=1e-6)


def test_aa_preserves_the_footprint_integral():
    """What the compensation is for: the image-plane integral of alpha,
    o_eff * (pi lambda^2 / 3) * sqrt(det Sigma_d) for the linear kernel, does
    not change with eps2d; it is o (pi lambda^2 / 3) sqrt(det Sigma_2D).
    Checked on the rendered alpha = 1 - T of one primitive (no alpha_min cut,
    alpha below the clamp), summed over unit pixels."""
    s1, s2, z, f, o = _f(0.3), _f(0.12), 4.0, 100.0, _f(0.5)
    th = 0.4
    q = (_f(math.cos(th / 2)), 0.0, 0.0, _f(math.sin(th / 2)))
    sc = _one((0, 0, z), (s1, s2, s1), q, o=o)
    cam = _cam(w=160, h=160, f=f, cx=80.25, cy=79.6)
    a, b = (f * s1 / z) ** 2, (f * s2 / z) ** 2
    want = o * (math.pi * 2.5 ** 2 / 3.0) * math.sqrt(a * b)
    sums = []
    for eps in (0.0, 0.3, 1.0, 4.0):
        out = oracle.render_scene(sc, cam, dict(eps2d=eps, antialias=1, alpha_min=0.0))
        sums.append((1.0 - out["T"]).sum())
    assert sums == pytest.approx([want] * 4, rel=2e-3)
    # without the compensation the integral grows with the dilation
    plain = (1.0 - oracle.render_scene(sc, cam, dict(eps2d=4.0, antialias=0, alpha_min=0.0))["T"]).sum()
    assert plain > 1.2 * want


def test_projection_off_axis_jacobian():
    """Isotropic s at (x0, 0, z): J = [[f/z, 0, -f x0/z^2], [0, f/z, 0]] so
    Sigma_2D = s^2 J J^T, centre at (f x0 / z + cx, cy)."""
    s, x0, z, f = _f(0.03), _f(0.6), 3.0, 90.0
    sc = _one((x0, 0, z), (s, s, s), (1, 0, 0, 0))
    proj, _ = oracle.project(sc, _cam(f=f), dict(eps2d=0.0))
    p = proj[0]
    assert p[oracle.P_SXX] == pytest.approx(s * s * ((f / z) ** 2 + (f * x0 / z ** 2) ** 2), rel=1e-6)
    assert p[oracle.P_SYY] == pytest.approx(s * s * (f / z) ** 2, rel=1e-6)
    assert abs(p[oracle.P_SXY]) < 1e-12
    assert p[oracle.P_MX] == pytest.approx(f * x0 / z + 32.0, rel=1e-6)


def test_projection_invariances():
    """q, -q and -2q give the same record; moving the camera and the scene by
    the same rigid motion changes nothing."""
    s = scenes.box_scene(200, 0, sh_degree=3)  # view-dependent colour too
    cam = scenes.identity_camera(256, 256)
    p0, v0 = oracle.project(s, cam)
    s2 = s.subset(np.arange(s.n))
    s2.quats = -2.0 * s2.quats  # exact in binary32
    p1, v1 = oracle.project(s2, cam)
    assert (v0 == v1).all()
    assert np.allclose(p0, p1, rtol=1e-12, atol=1e-12)
    # rigid motion G applied to the world: mu -> G mu, camera W -> W G^-1
    th = 0.3
    Rg = np.array([[math.cos(th), 0, math.sin(th)], [0, 1, 0], [-math.sin(th), 0, math.cos(th)]])
    tg = np.array([0.3, -0.2, 1.0])
    s3 = s.subset(np.arange(s.n))
    s3.means = (s.means.astype(np.float64) @ Rg.T + tg).astype(np.float32)
    # quaternion of Rg composed with each primitive rotation
    qg = np.array([math.cos(th / 2), 0, math.sin(th / 2), 0])

    def qmul(a, b):
        w1, x1, y1, z1 = a
        w2, x2, y2, z2 = b.T
        return np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                         w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], 1)

    s3.quats = qmul(qg, s.quats.astype(np.float64)).astype(np.float32)
    G = np.eye(4)
    G[:3, :3] = Rg
    G[:3, 3] = tg
    cam3 = dict(cam)
    cam3["viewmat"] = (np.asarray(cam["viewmat"], np.float64) @ np.linalg.inv(G)).astype(np.float32)
    p3, v3 = oracle.project(s3, cam3)
    m = v0 & v3
    assert m.sum() > 0.9 * v0.sum()
    # geometry is invariant (float32 rounding of the moved inputs bounds the
    # agreement); SH colour lives in the world frame, so only a translation
    # leaves it unchanged
    assert np.allclose(p0[m][:, :oracle.P_DEPTH + 1], p3[m][:, :oracle.P_DEPTH + 1], rtol=2e-4, atol=2e-3)
    s4 = s.subset(np.arange(s.n))
    s4.means = (s.means.astype(np.float64) + tg).astype(np.float32)
    T4 = np.eye(4)
    T4[:3, 3] = tg
    cam4 = dict(cam)
    cam4["viewmat"] = (np.asarray(cam["viewmat"], np.float64) @ np.linalg.inv(T4)).astype(np.float32)
    p4, v4 = oracle.project(s4, cam4)
    m = v0 & v4
    assert m.sum() > 0.9 * v0.sum()
    assert np.allclose(p0[m][:, :oracle.P_BL + 1], p4[m][:, :oracle.P_BL + 1], rtol=2e-4, atol=2e-3)


# ------------------------------------------------------------------ compositing
def test_single_primitive_closed_form():
    """One isotropic primitive whose centre sits on a pixel centre: at the
    pixel k to the right, D = k / sigma, alpha = o (1 - D/lambda), so
    C = rgb alpha + (1 - alpha) bg and T = 1 - alpha (Eq. 6, Eq. 12)."""
    s, z, f, eps, o = _f(0.2), 4.0, 100.0, 0.3, _f(0.7)
    sc = _one((0, 0, z), (s, s, s), (1, 0, 0, 0), o=o, colour=(0.9, 0.4, 0.1))
    cam = _cam(w=48, h=48, f=f, cx=24.5, cy=24.5)
    bg = (0.1, 0.2, 0.3)
    out = oracle.render_scene(sc, cam, dict(bg=bg))
    sigma = math.sqrt((f * s / z) ** 2 + eps)
    for k in range(0, 14):
        D = k / sigma
        a = o * max(0.0, 1 - D / 2.5)
        if a < 1 / 255:
            a = 0.0
        px = out["image"][24, 24 + k]
        assert out["T"][24, 24 + k] == pytest.approx(1 - a, abs=1e-12)
        assert px == pytest.approx(np.array([0.9, 0.4, 0.1]) * a + (1 - a) * np.array(bg), abs=1e-7)


def test_two_primitives_front_to_back():
    """Two overlapping primitives: C = c1 a1 + c2 a2 (1 - a1) with the nearer
    one first whatever the id order (Eq. 6)."""
    far = _one((0, 0, 5.0), (0.3, 0.3, 0.3), (1, 0, 0, 0), o=0.6, colour=(1, 0, 0))
    near = _one((0, 0, 3.0), (0.2, 0.2, 0.2), (1, 0, 0, 0), o=0.5, colour=(0, 0, 1))
    sc = scenes.Scene(np.concatenate([far.means, near.means]), np.concatenate([far.scales, near.scales]),
                      np.concatenate([far.quats, near.quats]), np.concatenate([far.opac, near.opac]),
                      np.concatenate([far.sh, near.sh]), 0)
    cam = _cam(w=32, h=32, f=100.0, cx=16.5, cy=16.5)
    out = oracle.render_scene(sc, cam)
    p = out["image"][16, 16]  # both centres project here: D = 0 for both
    a1, a2 = 0.5, _f(0.6)
    assert p == pytest.approx(np.array([0, 0, 1]) * a1 + np.array([1, 0, 0]) * a2 * (1 - a1), abs=1e-7)
    assert out["T"][16, 16] == pytest.approx((1 - a1) * (1 - a2), abs=1e-12)
    assert out["last_id"][16, 16] == 0 and out["n_last"][16, 16] == 2


@pytest.mark.parametrize("tile", [(8, 8), (16, 16), (32, 16)])
def test_tiled_equals_bruteforce_bitwise(tile):
    """Tiles and the sort only accelerate: tiled == per-pixel compositing of
    all primitives in (depth, id) order, bit for bit in FP64, for every tile
    shape; the image does not depend on the tile shape."""
    s, cams, _ = scenes.make_workload("plain_10k_256", n=1500)
    cam = cams[0]
    P = dict(tile_w=tile[0], tile_h=tile[1], bg=(0.3, 0.1, 0.2))
    proj, vis = oracle.project(s, cam, P)
    t = oracle.render(proj, vis, cam["width"], cam["height"], P)
    b = oracle.render(proj, vis, cam["width"], cam["height"], P, brute=True)
    assert np.array_equal(t["image"], b["image"])
    assert np.array_equal(t["T"], b["T"])
    assert np.array_equal(t["last_id"], b["last_id"])
    ref = oracle.render(proj, vis, cam["width"], cam["height"], dict(P, tile_w=16, tile_h=16))
    assert np.array_equal(t["image"], ref["image"])


def test_compact_support_and_rect_cover():
    """No pixel outside a primitive's rho-ellipse gets alpha >= alpha_min and
    every such pixel lies inside the primitive's FP64 rectangle."""
    s, cams, _ = scenes.make_workload("plain_10k_256", n=300)
    cam = cams[0]
    W, H = cam["width"], cam["height"]
    proj, vis = oracle.project(s, cam)
    ys, xs = np.mgrid[0:H, 0:W] + 0.5
    for i in np.nonzero(vis)[0][:120]:
        p = proj[i]
        dx, dy = xs - p[oracle.P_MX], ys - p[oracle.P_MY]
        # Mahalanobis distance from the 2x2 covariance (not the conic)
        Sd = np.array([[p[oracle.P_SXX], p[oracle.P_SXY]], [p[oracle.P_SXY], p[oracle.P_SYY]]])
        Si = np.linalg.inv(Sd)
        D = np.sqrt(Si[0, 0] * dx * dx + 2 * Si[0, 1] * dx * dy + Si[1, 1] * dy * dy)
        alpha = p[oracle.P_O] * np.maximum(0, 1 - D / 2.5)
        inside = alpha >= 1 / 255 + 1e-9
        r = oracle.rect(p[oracle.P_MX], p[oracle.P_MY], p[oracle.P_EX], p[oracle.P_EY], W, H, False)
        if r is None:
            assert not inside.any()
            continue
        x0, x1, y0, y1 = r
        mask = np.zeros_like(inside)
        mask[y0:y1 + 1, x0:x1 + 1] = True
        assert not (inside & ~mask).any()
        assert (D[inside] <= math.sqrt(p[oracle.P_RHO2]) + 1e-9).all()


def test_blend_invariants():
    """T is in [T_min, 1]; colour is bounded by (1 - T) max rgb + T bg;
    transmittance does not increase as primitives are added in front."""
    s, cams, _ = scenes.make_workload("plain_10k_256", n=3000)
    cam = cams[0]
    bg = (0.2, 0.3, 0.4)
    out = oracle.render_scene(s, cam, dict(bg=bg))
    T = out["T"]
    assert T.min() >= 1e-4 and T.max() <= 1.0
    maxrgb = out["proj"][out["vis"]][:, oracle.P_R:oracle.P_BL + 1].max()
    bound = (1 - T)[..., None] * maxrgb + T[..., None] * np.array(bg)
    assert (out["image"] <= bound + 1e-12).all()
    # adding primitives can only lower T, except where the T_min stop ended
    # the fuller list early, which bounds T by T_min / (1 - alpha_max)
    s2 = s.subset(np.arange(2000))
    out2 = oracle.render_scene(s2, cam, dict(bg=bg))
    assert ((T <= out2["T"] + 1e-12) | (T < 1e-4 / (1 - 0.999))).all()


def test_rect_f32_agrees_with_f64_away_from_boundaries():
    """The binary32 tile rule gives the FP64 rectangle unless a bound of the
    FP64 rule lies within 1e-3 px of an integer."""
    rng = np.random.default_rng(7)
    W, H = 300, 200
    bad = 0
    for _ in range(3000):
        mx, my = rng.uniform(-40, 340), rng.uniform(-40, 240)
        ex, ey = np.exp(rng.uniform(-1, 4, 2))
        mx, my, ex, ey = [float(np.float32(v)) for v in (mx, my, ex, ey)]
        bounds = [mx - ex - 0.5, mx + ex - 0.5, my - ey - 0.5, my + ey - 0.5]
        near = any(abs(b - round(b)) < 1e-3 for b in bounds)
        r64 = oracle.rect(mx, my, ex, ey, W, H, False)
        r32 = oracle.rect(mx, my, ex, ey, W, H, True)
        if not near:
            assert r64 == r32
        else:
            bad += 1
    assert bad < 30


def test_dupsort_f32_structure():
    """Duplication + sort of random binary32 footprints: every record appears
    once in each tile its rectangle covers, tiles ascend, (depth bits, id)
    ascend inside a tile, ranges delimit the tiles."""
    W, H, TW, TH = 200, 120, 16, 16
    rec = scenes.random_records(400, W, H, seed=3)
    foot = np.concatenate([rec["mean2d"], rec["ext"]], 1)
    dkey = oracle.depth_keys(rec)
    keys, vals, ranges = oracle.dupsort_f32(foot, dkey, W, H, TW, TH)
    tx_n = (W + TW - 1) // TW
    expect = set()
    for r in range(400):
        if not rec["visible"][r]:
            continue
        rc = oracle.rect(*foot[r].tolist(), W, H, True)
        if rc is None:
            continue
        for ty in range(rc[2] // TH, rc[3] // TH + 1):
            for tx in range(rc[0] // TW, rc[1] // TW + 1):
                expect.add((ty * tx_n + tx, r))
    got = list(zip(keys.tolist(), vals.tolist()))
    assert len(got) == len(set(got)) == len(expect) and set(got) == expect
    order = [(k, int(dkey[v]), v) for k, v in got]
    assert order == sorted(order)
    for t in range(ranges.shape[0]):
        a, b = ranges[t]
        assert (keys[a:b] == t).all()
        assert b - a == int((keys == t).sum())


def test_view_direction_convention():
    """Colour reads the SH at the unit vector from the camera centre to the
    primitive: with only the z-term (l=1, m=0) set, a primitive straight
    ahead of a camera at the origin gets 0.5 + c sqrt(3/(4 pi)); moved behind
    a camera looking along -z it gets 0.5 - c sqrt(3/(4 pi))."""
    c = 0.3
    sh = np.zeros((1, 4, 3), np.float32)
    sh[0, 2, :] = c
    sc = scenes.Scene(np.array([[0, 0, 3.0]], np.float32), np.full((1, 3), 0.05, np.float32),
                      np.array([[1, 0, 0, 0]], np.float32), np.array([0.5], np.float32), sh, 1)
    proj, vis = oracle.project(sc, _cam(), dict(sh_degree=1))
    expect = 0.5 + float(np.float32(c)) * math.sqrt(3 / (4 * math.pi))
    assert proj[0, oracle.P_R:oracle.P_BL + 1] == pytest.approx([expect] * 3, abs=1e-12)
    # camera at (0, 0, 6) looking back towards -z (180 deg about y)
    vm = np.diag([-1.0, 1.0, -1.0, 1.0])
    vm[2, 3] = 6.0
    proj, vis = oracle.project(sc, _cam(vm=vm), dict(sh_degree=1))
    assert vis[0]
    expect = 0.5 - float(np.float32(c)) * math.sqrt(3 / (4 * math.pi))
    assert proj[0, oracle.P_R:oracle.P_BL + 1] == pytest.approx([expect] * 3, abs=1e-12)


def test_tile_termination_labels_closed_form():
    """One 16x16 tile covered by two large primitives (depths 2 and 3): with
    T_min = 0.9 every pixel stops at the first entry, so the tile's label is
    2.0; with T_min = 0 no pixel stops, so it is +inf; an empty view gives 0."""
    s = scenes.Scene(np.array([[0, 0, 2.0], [0, 0, 3.0]], np.float32), np.full((2, 3), 1.0, np.float32),
                     np.array([[1, 0, 0, 0]] * 2, np.float32), np.array([0.9, 0.9], np.float32),
                     np.zeros((2, 1, 3), np.float32), 0)
    cam = scenes.camera(np.eye(4), 20.0, 20.0, 8.0, 8.0, 16, 16)
    out = oracle.render_scene(s, cam, dict(t_min=0.9))
    assert out["labels"].tolist() == [pytest.approx(2.0)]
    out = oracle.render_scene(s, cam, dict(t_min=0.0))
    assert out["labels"].tolist() == [np.inf]
    far = s.subset([0])
    far.means = np.array([[50.0, 0, 2.0]], np.float32)  # off screen
    assert oracle.render_scene(far, cam)["labels"].tolist() == [0.0]


def test_tile_depth_hist_brute_force():
    """Counts of random footprints against a direct count with numpy; the
    coverage is cumulative over bins and conserves each record's weight:
    summed over tiles, the last bin equals sum_r w_r (tiles in r's box)."""
    W, H, TW, TH = 160, 96, 16, 16
    rec = scenes.random_records(500, W, H, seed=12)
    foot = np.concatenate([rec["mean2d"], rec["ext"]], 1)
    dkey = oracle.depth_keys(rec)
    proj = oracle.records_to_proj(rec)
    counts, cov = oracle.tile_depth_hist(foot, dkey, proj, W, H, TW, TH)
    exp = np.zeros_like(counts)
    tx_n = (W + TW - 1) // TW
    total_w = 0.0
    for r in range(500):
        if not rec["visible"][r]:
            continue
        rc = oracle.rect(*foot[r].astype(np.float64).tolist(), W, H, True)
        if rc is None:
            continue
        n_t = (rc[1] // TW - rc[0] // TW + 1) * (rc[3] // TH - rc[2] // TH + 1)
        for ty in range(rc[2] // TH, rc[3] // TH + 1):
            for tx in range(rc[0] // TW, rc[1] // TW + 1):
                exp[ty * tx_n + tx] += 1
        l00, l01, l11 = (float(v) for v in rec["chol"][r])
        ellipse = math.pi * float(rec["rho2"][r]) / (l00 * l11)   # det A = (l00 l11)^2
        total_w += n_t * float(rec["opac"][r]) / 3.0 * min(1.0, ellipse / (n_t * TW * TH))
    assert np.array_equal(counts, exp) and counts.sum() > 0
    assert (np.diff(cov, axis=1) >= 0).all()
    assert cov[:, -1].sum() == pytest.approx(total_w, rel=1e-9)


@pytest.mark.parametrize("tw,th", [(16, 16), (8, 8), (32, 16)])
def test_touch_pairs_are_the_tiles_holding_support_pixels(tw, th):
    """The pairs every tile list must hold: brute force over every pixel of
    the image — a tile is reached iff one of its pixel centres lies in the
    (shrunk) support ellipse — and they are a subset of the box lists."""
    W, H = 70, 45
    rec = scenes.random_records(150, W, H, seed=9, max_ext=25.0)
    dkey = np.where(rec["visible"], rec["depth"].view(np.uint32), np.uint32(0xFFFFFFFF)).astype(np.uint32)
    foot = np.concatenate([rec["mean2d"], rec["ext"]], 1)
    l00, l01, l11 = (rec["chol"][:, k].astype(np.float64) for k in range(3))
    conic = np.stack([l00 * l00, l00 * l01, l01 * l01 + l11 * l11], 1)
    rho2 = rec["rho2"].astype(np.float64)
    shrink = 0.9
    t, r = oracle.touch_pairs(foot, dkey, conic, rho2, W, H, tw, th, shrink)
    ok, ov, _ = oracle.dupsort_f32(foot, dkey, W, H, tw, th)
    R1 = 151
    assert np.isin(t.astype(np.int64) * R1 + r, ok.astype(np.int64) * R1 + ov).all()
    px, py = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    tiles_x = (W + tw - 1) // tw
    exp = set()
    for i in range(150):
        if dkey[i] == 0xFFFFFFFF or oracle.rect(foot[i, 0], foot[i, 1], foot[i, 2], foot[i, 3], W, H, True) is None:
            continue
        x0, x1, y0, y1 = oracle.rect(foot[i, 0], foot[i, 1], foot[i, 2], foot[i, 3], W, H, True)
        dx, dy = px - np.float64(foot[i, 0]), py - np.float64(foot[i, 1])
        q = conic[i, 0] * dx * dx + 2 * conic[i, 1] * dx * dy + conic[i, 2] * dy * dy
        inside = (q <= shrink * rho2[i])
        inside[:, :x0] = False
        inside[:, x1 + 1:] = False
        inside[:y0, :] = False
        inside[y1 + 1:, :] = False
        ys, xs = np.nonzero(inside)
        for tt in set(((ys // th) * tiles_x + xs // tw).tolist()):
            exp.add((tt, i))
    got = set(zip(t.tolist(), r.tolist()))
    assert got == exp
    assert 0 < len(got) < len(ok)


@pytest.mark.parametrize("tw,th", [(16, 16), (8, 8), (32, 16)])
def test_reach_lists_between_touched_pairs_and_boxes(tw, th):
    """The binary32 reach rule of the tile lists is conservative and tight:
    its lists hold every pair whose tile has a pixel centre in the support
    ellipse (brute force, FP64), lie inside the support-box lists in the same
    order, and drop box corners the ellipses miss."""
    W, H = 300, 200
    rec = scenes.random_records(3000, W, H, seed=17, max_ext=40.0)
    dkey = np.where(rec["visible"], rec["depth"].view(np.uint32), np.uint32(0xFFFFFFFF)).astype(np.uint32)
    foot = np.concatenate([rec["mean2d"], rec["ext"]], 1)
    k, v, _ = oracle.dupsort_f32(foot, dkey, W, H, tw, th, chol=rec["chol"], rho2=rec["rho2"])
    bk, bv, _ = oracle.dupsort_f32(foot, dkey, W, H, tw, th)
    l00, l01, l11 = (rec["chol"][:, i].astype(np.float64) for i in range(3))
    conic = np.stack([l00 * l00, l00 * l01, l01 * l01 + l11 * l11], 1)
    t, r = oracle.touch_pairs(foot, dkey, conic, rec["rho2"].astype(np.float64), W, H, tw, th, 1.0)
    R1 = np.int64(3001)
    gid = k.astype(np.int64) * R1 + v
    bid = bk.astype(np.int64) * R1 + bv
    mask = np.isin(bid, gid)
    assert np.array_equal(bid[mask], gid)
    assert np.isin(t.astype(np.int64) * R1 + r, gid).all()
    assert len(t) <= len(k) < 0.95 * len(bk)
    # tight: boxes of one or two tiles are taken whole and the test is against
    # the rectangle of pixel centres, yet the lists stay near the pixel-exact set
    assert len(k) < 1.25 * len(t)


def test_tile_mask_sample_equals_full_render_on_its_tiles():
    """The timing sample of the CPU baseline composites a subset of tiles: on
    those tiles it is the full render bit for bit (image, T and adjoint
    terms), and it leaves the other tiles untouched."""
    s, cams, _ = scenes.make_workload("plain_10k_256", n=1200)
    cam = cams[0]
    W, H = cam["width"], cam["height"]
    P = dict(bg=(0.2, 0.3, 0.1))
    proj, vis = oracle.project(s, cam, P)
    tiles = (W // 16) * (H // 16)
    mask = np.random.default_rng(3).random(tiles) < 0.25
    full = oracle.render(proj, vis, W, H, P)
    part = oracle.render(proj, vis, W, H, P, tile_mask=mask)
    pix = np.repeat(np.repeat(mask.reshape(H // 16, W // 16), 16, 0), 16, 1)
    assert np.array_equal(part["image"][pix], full["image"][pix])
    assert np.array_equal(part["T"][pix], full["T"][pix])
    assert not part["image"][~pix].any() and not part["T"][~pix].any()
    gC = np.random.default_rng(4).standard_normal((H, W, 3))
    gT = np.random.default_rng(5).standard_normal((H, W))
    g_part = oracle.render_bwd(proj, vis, W, H, gC, gT, P, tile_mask=mask)
    g_win = oracle.render_bwd(proj, vis, W, H, gC * pix[..., None], gT * pix, P)
    assert np.allclose(g_part, g_win, rtol=1e-12, atol=1e-12)
