"""Seeded synthetic scenes and cameras for the linear-splatting rasterizer.

This module only draws random inputs; it holds none of the renderer's
arithmetic, so both the FP64 oracle (tests) and the CUDA path read the very
same arrays.  Every scene is a set of 3D primitives parameterised as in
Sec. 3.1, Eq. 1-2 (mean, per-axis scale, rotation quaternion, opacity) plus
view-dependent colour as real spherical-harmonic coefficients.

The paper trains on Mip-NeRF360, Tanks&Temples and Deep Blending (Sec. 4.1);
those datasets are not available, so the recipes below stand in for them with
the primitive counts, resolutions and value distributions of the workloads the
rasterizer is measured on (Table 3 reports about 3.35M primitives per scene).

Layouts (float32, C-contiguous):
  means  [N, 3]      world-space centres
  scales [N, 3]      activated (positive) per-axis scales
  quats  [N, 4]      (w, x, y, z), not normalised
  opac   [N]         activated opacity in (0, 1)
  sh     [N, K, 3]   K = (deg+1)^2 coefficients per colour channel
Cameras: dict(viewmat [4, 4] row-major world->camera, fx, fy, cx, cy, width,
height), OpenCV axes (x right, y down, z forward).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SH_Y00 = 0.28209479177387814  # 1 / (2 sqrt(pi)): the constant degree-0 basis value


@dataclasses.dataclass
class Scene:
    means: np.ndarray
    scales: np.ndarray
    quats: np.ndarray
    opac: np.ndarray
    sh: np.ndarray
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(self.means[idx].copy(), self.scales[idx].copy(), self.quats[idx].copy(),
                     self.opac[idx].copy(), self.sh[idx].copy(), self.sh_degree)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def random_quats(rng, n):
    """Uniform rotations: a normalised 4D Gaussian is uniform on S^3."""
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def dc_for_colour(colour):
    """Degree-0 coefficient whose constant basis term adds `colour - 0.5`."""
    return (colour - 0.5) / SH_Y00


def camera(viewmat, fx, fy, cx, cy, width, height):
    return dict(viewmat=np.ascontiguousarray(viewmat, dtype=np.float32), fx=float(fx), fy=float(fy),
                cx=float(cx), cy=float(cy), width=int(width), height=int(height))


def identity_camera(width, height, hfov_deg=60.0):
    fx = (width / 2.0) / math.tan(math.radians(hfov_deg) / 2.0)
    return camera(np.eye(4), fx, fx, width / 2.0, height / 2.0, width, height)


def look_at_camera(eye, target, width, height, hfov_deg=60.0):
    """World->camera matrix of a pinhole at `eye` looking at `target`, world +y up."""
    eye = np.asarray(eye, dtype=np.float64)
    fwd = np.asarray(target, dtype=np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    down_hint = np.array([0.0, -1.0, 0.0])
    right = np.cross(down_hint, fwd)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    rot = np.stack([right, down, fwd], axis=0)
    vm = np.eye(4)
    vm[:3, :3] = rot
    vm[:3, 3] = -rot @ eye
    fx = (width / 2.0) / math.tan(math.radians(hfov_deg) / 2.0)
    return camera(vm, fx, fx, width / 2.0, height / 2.0, width, height)


# --------------------------------------------------------------------------
# Scene recipes
# --------------------------------------------------------------------------

def box_scene(n, seed, sh_degree=0):
    """Plain fwd+bwd recipe: means uniform in [-1,1]x[-1,1]x[2,6] in front of an
    identity camera, scales log-uniform [0.005, 0.05], uniform rotations,
    opacities U[0.05, 0.95], colours U[0, 1] stored as the DC coefficient."""
    rng = np.random.default_rng(seed)
    means = np.empty((n, 3))
    means[:, 0] = rng.uniform(-1, 1, n)
    means[:, 1] = rng.uniform(-1, 1, n)
    means[:, 2] = rng.uniform(2, 6, n)
    scales = np.exp(rng.uniform(math.log(0.005), math.log(0.05), (n, 3)))
    quats = random_quats(rng, n)
    opac = rng.uniform(0.05, 0.95, n)
    k = (sh_degree + 1) ** 2
    sh = np.zeros((n, k, 3))
    sh[:, 0, :] = dc_for_colour(rng.uniform(0, 1, (n, 3)))
    if k > 1:
        sh[:, 1:, :] = rng.normal(0, 0.2, (n, k - 1, 3))
    return Scene(_f32(means), _f32(scales), _f32(quats), _f32(opac), _f32(sh), sh_degree)


def cluster_scene(n, seed, sh_degree=3, n_clusters=64, bg_frac=0.10):
    """Scene-scale recipe: 90% of the means from 64 anisotropic Gaussian
    clusters (Dirichlet(1) weights, centres uniform in a ball of radius 3,
    random rotations, axis std log-uniform [0.05, 0.5]), 10% uniform on the
    sphere of radius 20; scales log-normal(ln 0.01, 1); opacities Beta(2, 2);
    SH coefficients N(0, 0.2) with the DC colour U[0, 1]."""
    rng = np.random.default_rng(seed)
    n_bg = int(round(n * bg_frac))
    n_cl = n - n_bg
    w = rng.dirichlet(np.ones(n_clusters))
    d = rng.standard_normal((n_clusters, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    centres = d * (3.0 * rng.uniform(0, 1, (n_clusters, 1)) ** (1.0 / 3.0))
    cq = random_quats(rng, n_clusters)
    stds = np.exp(rng.uniform(math.log(0.05), math.log(0.5), (n_clusters, 3)))
    crot = _quat_to_rotmat_np(cq)
    lab = rng.choice(n_clusters, size=n_cl, p=w)
    z = rng.standard_normal((n_cl, 3)) * stds[lab]
    pts = centres[lab] + np.einsum("nij,nj->ni", crot[lab], z)
    bgd = rng.standard_normal((n_bg, 3))
    bgd /= np.linalg.norm(bgd, axis=1, keepdims=True)
    means = np.concatenate([pts, 20.0 * bgd], axis=0)
    perm = rng.permutation(n)
    means = means[perm]
    scales = rng.lognormal(math.log(0.01), 1.0, (n, 3))
    quats = random_quats(rng, n)
    opac = rng.beta(2.0, 2.0, n)
    k = (sh_degree + 1) ** 2
    sh = np.empty((n, k, 3), dtype=np.float32)
    sh[:, 0, :] = dc_for_colour(rng.uniform(0, 1, (n, 3)))
    if k > 1:
        sh[:, 1:, :] = rng.normal(0, 0.2, (n, k - 1, 3)).astype(np.float32)
    return Scene(_f32(means), _f32(scales), _f32(quats), _f32(opac), sh, sh_degree)


def _quat_to_rotmat_np(q):
    """Rotation matrices used only to orient the synthetic clusters."""
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], axis=1)


def ring_cameras(n_cams, seed, radius=4.0, w_range=(400, 1600), h_range=(300, 1060), hfov_deg=60.0):
    """Cameras of uneven resolution on a ring around the origin, looking at it."""
    rng = np.random.default_rng(seed)
    cams = []
    for _ in range(n_cams):
        wdt = int(rng.integers(w_range[0], w_range[1] + 1))
        hgt = int(rng.integers(h_range[0], h_range[1] + 1))
        ang = rng.uniform(0, 2 * math.pi)
        y = rng.uniform(-0.5, 0.5)
        eye = (radius * math.cos(ang), y, radius * math.sin(ang))
        cams.append(look_at_camera(eye, (0.0, 0.0, 0.0), wdt, hgt, hfov_deg))
    return cams


def scene_camera(width, height):
    """The single camera of the scene-scale workloads: at (4, 0.5, 0), 60 deg hfov."""
    return look_at_camera((4.0, 0.5, 0.0), (0.0, 0.0, 0.0), width, height)


# --------------------------------------------------------------------------
# The five workloads
# --------------------------------------------------------------------------

WORKLOADS = {
    "plain_10k_256": "10k box primitives, 256x256, SH0, fwd+bwd",
    "scene_1m_1297x840_aa": "1M cluster primitives, SH3, 1297x840, anti-aliased, fwd+bwd",
    "batch_3m_64cams": "3M cluster primitives, SH3, 64 ring cameras 400x300..1600x1060, fwd",
    "diff_3m_1080p": "3M cluster primitives, SH3, 1920x1080, fwd+bwd",
    "learned_5m_1080p": "5M cluster primitives, SH3, 1920x1080, learned termination",
}


def make_workload(name, n=None, seed=None):
    """Returns (scene, [cameras], extra) for a named workload; `n` overrides the
    primitive count for reduced-size parity cases with the same recipe."""
    if name == "plain_10k_256":
        s = box_scene(n or 10_000, 0 if seed is None else seed, 0)
        return s, [identity_camera(256, 256)], dict(antialias=False)
    if name == "scene_1m_1297x840_aa":
        s = cluster_scene(n or 1_000_000, 1 if seed is None else seed, 3)
        return s, [scene_camera(1297, 840)], dict(antialias=True)
    if name == "batch_3m_64cams":
        s = cluster_scene(n or 3_000_000, 2 if seed is None else seed, 3)
        return s, ring_cameras(64, 2 if seed is None else seed), dict(antialias=False)
    if name == "diff_3m_1080p":
        s = cluster_scene(n or 3_000_000, 3 if seed is None else seed, 3)
        return s, [scene_camera(1920, 1080)], dict(antialias=False)
    if name == "learned_5m_1080p":
        s = cluster_scene(n or 5_000_000, 4 if seed is None else seed, 3)
        return s, ring_cameras(1, 4 if seed is None else seed, w_range=(1920, 1920),
                               h_range=(1080, 1080)), dict(antialias=False)
    raise KeyError(name)


# --------------------------------------------------------------------------
# Random projected records (inputs of the duplicate/sort and blend stages
# on their own) and random loss weights.
# --------------------------------------------------------------------------

def random_records(n, width, height, seed, visible_frac=0.9, max_ext=40.0):
    """Random screen-space footprints, all float32: centre, half extents of
    the support box, the upper-triangular factor (l00, l01, l11) of an
    ellipse's inverse covariance, effective opacity, squared cutoff, depth
    and colour.  The ellipse has axis std (ex, ey) / 2.5 and correlation
    cc, so a cutoff up to 2.5 stays inside the box.  Depths come from a
    small set of values so ties are frequent."""
    rng = np.random.default_rng(seed)
    mx = rng.uniform(-0.2 * width, 1.2 * width, n)
    my = rng.uniform(-0.2 * height, 1.2 * height, n)
    ex = np.exp(rng.uniform(math.log(0.3), math.log(max_ext), n))
    ey = np.exp(rng.uniform(math.log(0.3), math.log(max_ext), n))
    sx = ex / 2.5
    sy = ey / 2.5
    rho = rng.uniform(0.4, 1.0, n)
    cc = rng.uniform(-0.9, 0.9, n)
    sq = np.sqrt(1 - cc * cc)
    chol = np.stack([1.0 / (sx * sq), -cc / (sy * sq), 1.0 / sy], 1)
    o = rng.uniform(0.05, 0.99, n)
    depth = rng.choice(np.linspace(0.5, 50.0, 997), size=n)
    rgb = rng.uniform(0, 1, (n, 3))
    vis = rng.uniform(0, 1, n) < visible_frac
    return dict(mean2d=_f32(np.stack([mx, my], 1)), ext=_f32(np.stack([ex, ey], 1)), chol=_f32(chol),
                opac=_f32(o), rho2=_f32((2.5 * rho) ** 2), depth=_f32(depth), rgb=_f32(rgb), visible=vis)


def loss_weights(height, width, seed):
    """Seeded weights w [H, W, 3] and v [H, W] of the test loss <w, C> + <v, T>."""
    rng = np.random.default_rng(seed)
    return _f32(rng.standard_normal((height, width, 3))), _f32(rng.standard_normal((height, width)))


def random_mlp_params(seed, n_param=7361, n_in=48, hid=64, features=35):
    """Random packed parameters of the 48 -> 64 -> 64 -> 1 termination MLP
    (w1t [64][48] | b1 | w2t [64][64] | b2 | w3 | b3) and nothing else."""
    rng = np.random.default_rng(seed)
    p = np.zeros(n_param)
    o = 0
    p[o:o + hid * n_in] = rng.normal(0, np.sqrt(2.0 / features), hid * n_in)
    o += hid * n_in
    p[o:o + hid] = rng.normal(0, 0.05, hid)
    o += hid
    p[o:o + hid * hid] = rng.normal(0, np.sqrt(2.0 / hid), hid * hid)
    o += hid * hid
    p[o:o + hid] = rng.normal(0, 0.05, hid)
    o += hid
    p[o:o + hid] = rng.normal(0, np.sqrt(1.0 / hid), hid)
    o += hid
    p[o] = 0.3
    return p


def random_mlp_batch(m, seed, n_in=48, features=35):
    """Random feature rows (half precision, zero past `features`) and targets."""
    rng = np.random.default_rng(seed)
    x = np.zeros((m, n_in), np.float16)
    x[:, :features] = rng.uniform(-1.0, 2.0, (m, features)).astype(np.float16)
    t = rng.normal(1.0, 0.7, m)
    return x, t
