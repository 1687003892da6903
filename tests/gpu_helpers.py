"""Shared helpers of the GPU parity tests (packing inputs in the ABI layout,
comparison rules).  The comparison rules follow the parity bar: tile lists
and orders bit-exact; images within 1e-4 max abs on pixels the oracle does
not flag as near a threshold; gradients within 1e-3 relative L2."""
import os

import numpy as np
import torch

IMG_TOL = 1e-4
GRAD_TOL = 1e-3

# Measured parity figures of this session (printed at the end of the run by
# tests/conftest.py): (test, what, {figure: value}).
PARITY_LOG = []


def log_parity(what, **figures):
    test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0].split("::")[-1]
    PARITY_LOG.append((test, what, figures))


def pack_records(rec, device="cuda"):
    """Random binary32 records -> the projected-record buffer of include/ls.h:
    rec [R][12] | foot [R][4] | dkey [R]."""
    R = rec["opac"].shape[0]
    r12 = np.zeros((R, 12), np.float32)
    r12[:, 0:2] = rec["mean2d"]
    r12[:, 2] = rec["chol"][:, 0]
    r12[:, 3] = rec["chol"][:, 1]
    r12[:, 4] = rec["chol"][:, 2]
    r12[:, 5] = rec["opac"]
    r12[:, 6] = rec["rho2"]
    r12[:, 7] = rec["depth"]
    r12[:, 8:11] = rec["rgb"]
    foot = np.concatenate([rec["mean2d"], rec["ext"]], 1).astype(np.float32)
    dkey = np.ascontiguousarray(rec["depth"], np.float32).view(np.uint32).copy()
    dkey[~rec["visible"]] = 0xFFFFFFFF
    buf = np.concatenate([r12.reshape(-1).view(np.uint8), foot.reshape(-1).view(np.uint8),
                          dkey.view(np.uint8)])
    t = torch.from_numpy(buf.view(np.float32).copy()).to(device)
    return t, dkey


def unpack_proj(proj, R):
    """Device projected-record buffer -> numpy planes."""
    a = proj.detach().cpu().numpy().view(np.uint8)
    rec = a[:48 * R].view(np.float32).reshape(R, 12)
    foot = a[48 * R:64 * R].view(np.float32).reshape(R, 4)
    dkey = a[64 * R:68 * R].view(np.uint32)
    return rec, foot, dkey


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def assert_image_parity(img, ref, region=None, tol=IMG_TOL, max_mismatch_frac=1e-4):
    """img (GPU, float32) against the oracle output dict: max abs error
    <= tol on pixels the oracle does not flag; the pixels beyond tol (a
    skip/stop decision that binary32 and FP64 took differently: a pair
    within 1e-5 of alpha_min, T within 1e-9 of T_min, alpha within 1e-6 of
    the clamp) must all be flagged ones, at most max_mismatch_frac of the
    region (at least one pixel allowed), each within 1/255 + tol (one pair
    of alpha ~ alpha_min added or dropped)."""
    img = np.asarray(img, np.float64)
    flags = ref["flags"]
    if region is not None:
        x0, x1, y0, y1 = region
        img = img[y0:y1, x0:x1]
        refi = ref["image"][y0:y1, x0:x1]
        flags = flags[y0:y1, x0:x1]
    else:
        refi = ref["image"]
    err = np.abs(img - refi).max(-1)
    ok = ~flags
    nflag = int(flags.sum())
    mism = err > tol
    log_parity("image", pixels=int(flags.size), max_err_unflagged=float(err[ok].max()) if ok.any() else 0.0,
               flagged_frac=nflag / flags.size, mismatched_frac=float(mism.mean()),
               max_err_flagged=float(err[flags].max()) if nflag else 0.0)
    assert err[ok].max() <= tol, "max abs error %.3g on unflagged pixels" % err[ok].max()
    assert int(mism.sum()) <= max(1, max_mismatch_frac * flags.size), "%d pixels beyond tol" % int(mism.sum())
    if mism.any():
        assert err[mism].max() <= 1 / 255 + tol, err[mism].max()
    return float(err[ok].max()), nflag


def conic_of(rec12):
    """(a, b, c) of A = L^T L from the stored factor (l00, l01, l11), FP64."""
    l00, l01, l11 = (rec12[:, k].astype(np.float64) for k in (2, 3, 4))
    return np.stack([l00 * l00, l00 * l01, l01 * l01 + l11 * l11], 1)
