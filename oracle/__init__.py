"""FP64 CPU oracle for the linear-splatting rasterizer.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the package smoke check and
by the benchmark's CPU-baseline leg, never by the product path.  It shares no
code with the CUDA implementation; both read the same seeded inputs.

Functions follow the paper's definitions (Sec. 3.1 Eq. 1-6, Sec. 3.2 Eq. 7-11,
Sec. 3.3 Eq. 12-14, Appendix B Eq. 19-26); the readings where the paper is
silent are listed at the top of lso.cpp.  Parity is pinned by tests in
tests/test_oracle_*.py (closed forms, brute force, invariants, finite
differences), the anti-aliasing opacity compensation included (its value at
eps2d = 0, closed forms for isotropic and rotated anisotropic footprints, and
the footprint integral it preserves).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lso.cpp")
_LIB = os.path.join(_HERE, "liblso.so")
_lib = None

NP = 16
P_MX, P_MY, P_A, P_B, P_C, P_O, P_RHO2, P_DEPTH, P_R, P_G, P_BL, P_EX, P_EY, P_SXX, P_SXY, P_SYY = range(16)

DEFAULTS = dict(lam=2.5, kernel=0, ags=0, antialias=0, eps2d=0.3, alpha_min=1.0 / 255.0, alpha_max=0.999,
                t_min=1e-4, tile_w=16, tile_h=16, bg=(0.0, 0.0, 0.0), near=0.2, far=1e4, sh_degree=0)


def build(force=False):
    """Compile liblso.so with g++ (-ffp-contract=off keeps the binary32 tile
    rule free of fused multiply-adds on every host)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        L.lso_project.restype = ctypes.c_int
        L.lso_render.restype = ctypes.c_int
        L.lso_render_bwd.restype = ctypes.c_int
        L.lso_project_bwd.restype = ctypes.c_int
        L.lso_dupsort_f32.restype = ctypes.c_longlong
        L.lso_touch_pairs.restype = ctypes.c_longlong
        L.lso_kernel_f.restype = ctypes.c_double
        L.lso_kernel_f.argtypes = [ctypes.c_int, ctypes.c_double]
        L.lso_kernel_support.restype = ctypes.c_double
        L.lso_kernel_support.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.lso_rect.restype = ctypes.c_int
        L.lso_rect.argtypes = [ctypes.c_double] * 4 + [ctypes.c_int] * 3 + [ctypes.POINTER(ctypes.c_int)]
        del dp
        _lib = L
    return _lib


def set_threads(n):
    lib().lso_set_threads(int(n))


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def params_array(params=None):
    P = dict(DEFAULTS)
    if params:
        P.update(params)
    bg = P["bg"]
    return np.array([P["lam"], P["kernel"], P["ags"], P["antialias"], P["eps2d"], P["alpha_min"], P["alpha_max"],
                     P["t_min"], P["tile_w"], P["tile_h"], bg[0], bg[1], bg[2], P["near"], P["far"],
                     P["sh_degree"]], dtype=np.float64)


def cam_array(cam):
    vm = np.asarray(cam["viewmat"], dtype=np.float64).reshape(16)
    return np.concatenate([vm, [cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["width"], cam["height"]]]).astype(
        np.float64)


def project(scene, cam, params=None):
    """Projected records [n, NP] (FP64) and visibility [n] of a scene."""
    P = dict(params or {})
    P.setdefault("sh_degree", scene.sh_degree)
    n = scene.n
    out = np.zeros((n, NP))
    vis = np.zeros(n, dtype=np.uint8)
    lib().lso_project(ctypes.c_int(n), _p(_d(scene.means)), _p(_d(scene.scales)), _p(_d(scene.quats)),
                      _p(_d(scene.opac)), _p(_d(scene.sh)), _p(cam_array(cam)), _p(params_array(P)), _p(out),
                      _p(vis))
    return out, vis.astype(bool)


def _window(window):
    if window is None:
        return ctypes.c_void_p(0), None
    w = np.ascontiguousarray(window, dtype=np.int32)
    return _p(w), w


def _mask(tile_mask):
    if tile_mask is None:
        return ctypes.c_void_p(0), None
    m = np.ascontiguousarray(tile_mask, dtype=np.uint8)
    return _p(m), m


def render(proj, vis, width, height, params=None, rule_f32=False, dkey=None, brute=False, window=None,
           tile_mask=None):
    """Front-to-back composite (Eq. 6) of projected records; `window` =
    (x0, x1, y0, y1) restricts it to those pixels (others stay zero), and
    `tile_mask` [tiles] to the tiles where it is set.  Also returns per-tile
    termination depths `labels` (tiled mode)."""
    n = proj.shape[0]
    proj = _d(proj)
    vis8 = np.ascontiguousarray(vis, dtype=np.uint8)
    img = np.zeros((height, width, 3))
    T = np.zeros((height, width))
    n_last = np.zeros((height, width), dtype=np.int32)
    last_id = np.zeros((height, width), dtype=np.int32)
    flags = np.zeros((height, width), dtype=np.uint8)
    stats = np.zeros(2, dtype=np.int64)
    dk = None if dkey is None else np.ascontiguousarray(dkey, dtype=np.uint32)
    wp, _keep = _window(window)
    mp, _mkeep = _mask(tile_mask)
    Pd = dict(DEFAULTS)
    Pd.update(params or {})
    tiles = ((width + Pd["tile_w"] - 1) // Pd["tile_w"]) * ((height + Pd["tile_h"] - 1) // Pd["tile_h"])
    labels = np.zeros(tiles)
    lib().lso_render(ctypes.c_int(n), _p(proj), _p(vis8), ctypes.c_int(width), ctypes.c_int(height),
                     _p(params_array(params)), ctypes.c_int(int(rule_f32)),
                     _p(dk) if dk is not None else ctypes.c_void_p(0), ctypes.c_int(int(brute)), _p(img), _p(T),
                     _p(n_last), _p(last_id), _p(flags), _p(stats), wp, _p(labels), mp)
    return dict(image=img, T=T, n_last=n_last, last_id=last_id, flags=flags.astype(bool), n_eval=int(stats[0]),
                n_contrib=int(stats[1]), labels=labels)


def tile_depth_hist(foot, dkey, proj, width, height, tile_w, tile_h):
    """Per-tile inputs of the termination network: (counts [tiles], cumulative
    coverage [tiles, 32]) of binary32 footprints; proj [R, NP] supplies each
    record's opacity, squared support radius and conic."""
    R = foot.shape[0]
    tiles = ((width + tile_w - 1) // tile_w) * ((height + tile_h - 1) // tile_h)
    counts = np.zeros(tiles, dtype=np.int32)
    cov = np.zeros((tiles, 32))
    lib().lso_tile_depth_hist(ctypes.c_longlong(R), _p(np.ascontiguousarray(foot, np.float32)),
                              _p(np.ascontiguousarray(dkey, np.uint32)), _p(_d(proj)), ctypes.c_int(width),
                              ctypes.c_int(height), ctypes.c_int(tile_w), ctypes.c_int(tile_h), _p(counts), _p(cov))
    return counts, cov


def render_bwd(proj, vis, width, height, gC, gT, params=None, rule_f32=False, dkey=None, window=None,
               tile_mask=None):
    """Adjoint of `render` with respect to (mx, my, a, b, c, o_eff, r, g, b);
    with `window` (`tile_mask`) only those pixels' (tiles') terms are summed."""
    n = proj.shape[0]
    g2d = np.zeros((n, 9))
    dk = None if dkey is None else np.ascontiguousarray(dkey, dtype=np.uint32)
    wp, _keep = _window(window)
    mp, _mkeep = _mask(tile_mask)
    lib().lso_render_bwd(ctypes.c_int(n), _p(_d(proj)), _p(np.ascontiguousarray(vis, dtype=np.uint8)),
                         ctypes.c_int(width), ctypes.c_int(height), _p(params_array(params)),
                         ctypes.c_int(int(rule_f32)), _p(dk) if dk is not None else ctypes.c_void_p(0),
                         _p(_d(gC)), _p(_d(gT)), _p(g2d), wp, mp)
    return g2d


def project_bwd(scene, cam, g2d, params=None):
    """Gradients of the 3D parameters from g2d (forward-mode dual numbers)."""
    P = dict(params or {})
    P.setdefault("sh_degree", scene.sh_degree)
    n = scene.n
    K = (scene.sh_degree + 1) ** 2
    gm = np.zeros((n, 3))
    gs = np.zeros((n, 3))
    gq = np.zeros((n, 4))
    go = np.zeros(n)
    gsh = np.zeros((n, K, 3))
    lib().lso_project_bwd(ctypes.c_int(n), _p(_d(scene.means)), _p(_d(scene.scales)), _p(_d(scene.quats)),
                          _p(_d(scene.opac)), _p(_d(scene.sh)), _p(cam_array(cam)), _p(params_array(P)),
                          _p(_d(g2d)), _p(gm), _p(gs), _p(gq), _p(go), _p(gsh))
    return dict(means=gm, scales=gs, quats=gq, opac=go, sh=gsh)


def render_scene(scene, cam, params=None, brute=False, window=None):
    P = dict(params or {})
    P.setdefault("sh_degree", scene.sh_degree)
    proj, vis = project(scene, cam, P)
    out = render(proj, vis, cam["width"], cam["height"], P, brute=brute, window=window)
    out["proj"] = proj
    out["vis"] = vis
    return out


def scene_grads(scene, cam, gC, gT, params=None, window=None):
    """Full adjoint: d/d(3D parameters) of <gC, C> + <gT, T> (pixels of
    `window` only, when given)."""
    P = dict(params or {})
    P.setdefault("sh_degree", scene.sh_degree)
    proj, vis = project(scene, cam, P)
    g2d = render_bwd(proj, vis, cam["width"], cam["height"], gC, gT, P, window=window)
    g = project_bwd(scene, cam, g2d, P)
    g["g2d"] = g2d
    return g


def dupsort_f32(foot, dkey, width, height, tile_w, tile_h, cap=None, chol=None, rho2=None):
    """Duplicate + stable sort of binary32 footprints: (keys, vals, ranges).
    Without chol every support-box tile is listed; with chol [R][3] = l00 l01
    l11 and rho2 [R] (binary32) only the tiles the support ellipse reaches."""
    R = foot.shape[0]
    foot = np.ascontiguousarray(foot, dtype=np.float32)
    dkey = np.ascontiguousarray(dkey, dtype=np.uint32)
    tiles = ((width + tile_w - 1) // tile_w) * ((height + tile_h - 1) // tile_h)
    ranges = np.zeros(2 * tiles, dtype=np.int32)
    # upper bound on K: every record covering every tile
    if cap is None:
        cap = min(int(R) * tiles, 50_000_000)
    keys = np.zeros(cap, dtype=np.uint32)
    vals = np.zeros(cap, dtype=np.uint32)
    if chol is not None:
        chol = np.ascontiguousarray(chol, dtype=np.float32)
        rho2 = np.ascontiguousarray(rho2, dtype=np.float32)
    K = lib().lso_dupsort_f32(ctypes.c_longlong(R), _p(foot), _p(dkey), _p(chol) if chol is not None else None,
                              _p(rho2) if chol is not None else None, ctypes.c_int(width), ctypes.c_int(height),
                              ctypes.c_int(tile_w), ctypes.c_int(tile_h), ctypes.c_longlong(cap), _p(keys), _p(vals),
                              _p(ranges))
    if K < 0:
        raise RuntimeError("oracle dupsort capacity exceeded")
    return keys[:K].copy(), vals[:K].copy(), ranges.reshape(-1, 2)


def touch_pairs(foot, dkey, conic, rho2, width, height, tile_w, tile_h, shrink=1.0):
    """(tile, record) pairs whose tile holds a pixel centre inside the
    record's support ellipse scaled by `shrink` (FP64 brute force), within
    its binary32 support box; sorted by (tile, record)."""
    R = foot.shape[0]
    foot = np.ascontiguousarray(foot, dtype=np.float32)
    dkey = np.ascontiguousarray(dkey, dtype=np.uint32)
    conic = np.ascontiguousarray(conic, dtype=np.float64)
    rho2 = np.ascontiguousarray(rho2, dtype=np.float64)
    args = (ctypes.c_longlong(R), _p(foot), _p(dkey), _p(conic), _p(rho2), ctypes.c_int(width), ctypes.c_int(height),
            ctypes.c_int(tile_w), ctypes.c_int(tile_h), ctypes.c_double(shrink))
    n = lib().lso_touch_pairs(*args, ctypes.c_longlong(0), None, None)
    t = np.zeros(max(n, 1), dtype=np.uint32)
    r = np.zeros(max(n, 1), dtype=np.uint32)
    lib().lso_touch_pairs(*args, ctypes.c_longlong(n), _p(t), _p(r))
    order = np.lexsort((r[:n], t[:n]))
    return t[:n][order], r[:n][order]


def rect(mx, my, ex, ey, width, height, f32):
    out = (ctypes.c_int * 4)()
    ok = lib().lso_rect(mx, my, ex, ey, width, height, int(f32), out)
    return (list(out) if ok else None)


def sh_basis(dirs, deg=3):
    dirs = _d(dirs)
    m = dirs.shape[0]
    out = np.zeros((m, 16))
    lib().lso_sh_basis(ctypes.c_int(m), ctypes.c_int(deg), _p(dirs), _p(out))
    return out


def kernel_f(k, x):
    return lib().lso_kernel_f(int(k), float(x))


def kernel_support(k, o, amin):
    return lib().lso_kernel_support(int(k), float(o), float(amin))


def records_to_proj(rec):
    """Random binary32 records (scenes.random_records) in the FP64 NP layout."""
    n = rec["opac"].shape[0]
    p = np.zeros((n, NP))
    p[:, P_MX] = rec["mean2d"][:, 0]
    p[:, P_MY] = rec["mean2d"][:, 1]
    # inverse covariance A = L^T L of the stored factor L = [[l00, l01], [0, l11]]
    l00, l01, l11 = (rec["chol"][:, k].astype(np.float64) for k in range(3))
    p[:, P_A] = l00 * l00
    p[:, P_B] = l00 * l01
    p[:, P_C] = l01 * l01 + l11 * l11
    p[:, P_O] = rec["opac"]
    p[:, P_RHO2] = rec["rho2"]
    p[:, P_DEPTH] = rec["depth"]
    p[:, P_R:P_BL + 1] = rec["rgb"]
    p[:, P_EX] = rec["ext"][:, 0]
    p[:, P_EY] = rec["ext"][:, 1]
    return p


def depth_keys(rec):
    """Sort bits of random records: binary32 depth bits, 0xFFFFFFFF if hidden."""
    d = np.ascontiguousarray(rec["depth"], dtype=np.float32).view(np.uint32).copy()
    d[~rec["visible"]] = 0xFFFFFFFF
    return d
