"""ctypes binding of the FP64 CPU oracle (test infrastructure only; see kb_oracle.c).

Arrays are numpy.  Image inputs are the float32 arrays the synthetic generator writes; psi/phi
inputs of the search are widened to float64 (exactly, when they are float32), so the oracle
evaluates the same values the CUDA path reads.  Results are float64 (int32 for counts and
indices, uint32 for kept-epoch masks).
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        _LIB = C.CDLL(_build.build())
        d, i, f = C.c_double, C.c_int, C.c_float
        p = C.c_void_p
        _LIB.kbo_erfinv.restype = d
        _LIB.kbo_erfinv.argtypes = [d]
        _LIB.kbo_sigma_g_coeff.restype = d
        _LIB.kbo_sigma_g_coeff.argtypes = [d, d]
        _LIB.kbo_percentile_sorted.restype = d
        _LIB.kbo_percentile_sorted.argtypes = [p, i, d]
        _LIB.kbo_sigma_g_clip.restype = i
        _LIB.kbo_sigma_g_clip.argtypes = [p, i, d, d, d, d, p, p, p]
        _LIB.kbo_track_offsets.restype = None
        _LIB.kbo_track_offsets.argtypes = [p, i, p, p, i, p, p]
        _LIB.kbo_psi_phi.restype = None
        _LIB.kbo_psi_phi.argtypes = [p, p, p, p, i, i, i, i, p, p]
        _LIB.kbo_psi_phi_at.restype = None
        _LIB.kbo_psi_phi_at.argtypes = [p, p, p, p, i, i, i, i, p, i, p, p]
        _LIB.kbo_eval_one.restype = i
        _LIB.kbo_eval_one.argtypes = [p, p, p, i, i, i, i, i, f, f, i, i, d, d, d, d, i,
                                      p, p, p, p, p]
        _LIB.kbo_clip_margin.restype = d
        _LIB.kbo_clip_margin.argtypes = [p, p, p, i, i, i, i, i, f, f, i, i, d, d, d, d, i]
        _LIB.kbo_stage_counts.restype = i
        _LIB.kbo_stage_counts.argtypes = [p, p, p, i, i, i, p, p, i, d, i, i, d, d, d, d, i,
                                          i, i, i, i, p]
        _LIB.kbo_search.restype = i
        _LIB.kbo_search.argtypes = [p, p, p, i, i, i, p, p, i, i, d, i, i, d, d, d, d, i,
                                    i, i, i, i, p, p, p, p, p, p]
        _LIB.kbo_stamps.restype = i
        _LIB.kbo_stamps.argtypes = [p, p, p, p, i, i, i, p, p, p, p, p, i, i, p, p]
        _LIB.kbo_traj_eval_subpixel.restype = i
        _LIB.kbo_traj_eval_subpixel.argtypes = [p, p, p, i, i, i, p, d, d, d, d, p, p, p]
        _LIB.kbo_traj_vjp.restype = i
        _LIB.kbo_traj_vjp.argtypes = [p, p, p, i, i, i, p, d, d, d, d, d, d, p, p, p]
        _LIB.kbo_set_threads.restype = None
        _LIB.kbo_set_threads.argtypes = [i]
        _LIB.kbo_get_threads.restype = i
        _LIB.kbo_get_threads.argtypes = []
        _LIB.kbo_cluster.restype = None
        _LIB.kbo_cluster.argtypes = [p, p, p, p, p, i, d, d, p, p]
        _LIB.kbo_stamp_moments.restype = i
        _LIB.kbo_stamp_moments.argtypes = [p, i, p, p]
        _LIB.kbo_refine_adam.restype = i
        _LIB.kbo_refine_adam.argtypes = [p, p, p, i, i, i, p, p, i, d, d, d, d, d, p, p]
    return _LIB


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def erfinv(y):
    return lib().kbo_erfinv(float(y))


def sigma_g_coeff(q_lo=0.25, q_hi=0.75):
    return lib().kbo_sigma_g_coeff(float(q_lo), float(q_hi))


def percentile(values, q):
    s = np.sort(_f64(values))
    return lib().kbo_percentile_sorted(_ptr(s), len(s), float(q))


def sigma_g_clip(values, q_lo=0.25, q_mid=0.5, q_hi=0.75, n_sigma=2.0):
    """Returns (keep bool array, median, sigma_G)."""
    a = _f64(values)
    keep = np.zeros(len(a), dtype=np.uint8)
    med, sg = C.c_double(0), C.c_double(0)
    lib().kbo_sigma_g_clip(_ptr(a), len(a), q_lo, q_mid, q_hi, n_sigma, _ptr(keep),
                           C.byref(med), C.byref(sg))
    return keep.astype(bool), med.value, sg.value


def track_offsets(times, vx, vy):
    times = _f64(times)
    vx, vy = _f32(vx), _f32(vy)
    n, T = len(vx), len(times)
    ox = np.zeros((n, T), np.int32)
    oy = np.zeros((n, T), np.int32)
    lib().kbo_track_offsets(_ptr(times), T, _ptr(vx), _ptr(vy), n, _ptr(ox), _ptr(oy))
    return ox, oy


def _mask_u8(mask, shape):
    if mask is None:
        return None
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    assert m.shape == shape
    return m


def psi_phi(img, var, mask, psf):
    """psi, phi (float64, [T][H][W]) of R0 from float32 img/var [T][H][W] and psf [T][k][k]."""
    img, var, psf = _f32(img), _f32(var), _f32(psf)
    T, H, W = img.shape
    k = psf.shape[-1]
    m = _mask_u8(mask, img.shape)
    psi = np.zeros((T, H, W), np.float64)
    phi = np.zeros((T, H, W), np.float64)
    lib().kbo_psi_phi(_ptr(img), _ptr(var), _ptr(m), _ptr(psf), T, H, W, k, _ptr(psi), _ptr(phi))
    return psi, phi


def psi_phi_at(img, var, mask, psf, tyx):
    """psi, phi at sample pixels tyx (int [n][3] of t, y, x)."""
    img, var, psf = _f32(img), _f32(var), _f32(psf)
    T, H, W = img.shape
    k = psf.shape[-1]
    m = _mask_u8(mask, img.shape)
    tyx = np.ascontiguousarray(tyx, dtype=np.int32)
    n = len(tyx)
    psi = np.zeros(n, np.float64)
    phi = np.zeros(n, np.float64)
    lib().kbo_psi_phi_at(_ptr(img), _ptr(var), _ptr(m), _ptr(psf), T, H, W, k, _ptr(tyx), n,
                         _ptr(psi), _ptr(phi))
    return psi, phi


def window_inputs(img, var, mask, psf, times, vx, vy, window):
    """The oracle's psi/phi (FP64) on the part of the image the tracks of the start pixels in
    `window` = (x_lo, x_hi, y_lo, y_hi) can reach, and that window in the crop's coordinates.

    The crop is the bounding box of every track position of every window pixel, clipped to the
    image, so a position inside the image lies in the crop and one outside the image lies outside
    it: an oracle search of the crop over the shifted window gives the results of a search of the
    whole image over `window`.  psi/phi are formed on the crop widened by the PSF radius (clipped
    to the image), so every value kept equals the whole-image value.  Returns
    (psi, phi, window_in_crop, (x0, y0) of the crop)."""
    img, var, psf = _f32(img), _f32(var), _f32(psf)
    T, H, W = img.shape
    x_lo, x_hi, y_lo, y_hi = (int(v) for v in window)
    ox, oy = track_offsets(times, vx, vy)
    xa, xb = max(0, x_lo + int(ox.min())), min(W, x_hi - 1 + int(ox.max()) + 1)
    ya, yb = max(0, y_lo + int(oy.min())), min(H, y_hi - 1 + int(oy.max()) + 1)
    r = psf.shape[-1] // 2
    xa2, xb2, ya2, yb2 = max(0, xa - r), min(W, xb + r), max(0, ya - r), min(H, yb + r)
    sub = (slice(None), slice(ya2, yb2), slice(xa2, xb2))
    m = None if mask is None else np.ascontiguousarray(mask[sub])
    psi, phi = psi_phi(img[sub], var[sub], m, psf)
    inner = (slice(None), slice(ya - ya2, yb - ya2), slice(xa - xa2, xb - xa2))
    psi = np.ascontiguousarray(psi[inner])
    phi = np.ascontiguousarray(phi[inner])
    return psi, phi, (x_lo - xa, x_hi - xa, y_lo - ya, y_hi - ya), (xa, ya)


DEFAULTS = dict(k=1, lh_min=7.0, min_obs=1, clip=1, q_lo=0.25, q_mid=0.5, q_hi=0.75,
                n_sigma=2.0, clip_on=0)


def _params(p):
    q = dict(DEFAULTS)
    if p:
        q.update(p)
    # The CUDA path receives float32 parameters; the oracle uses the same values, widened.
    for key in ("lh_min", "q_lo", "q_mid", "q_hi", "n_sigma"):
        q[key] = float(np.float32(q[key]))
    return q


def eval_one(psi, phi, times, x0, y0, vx, vy, params=None):
    """Single integer-pixel trajectory (Section 4.1's single-trajectory variant)."""
    q = _params(params)
    psi, phi, times = _f64(psi), _f64(phi), _f64(times)
    T, H, W = psi.shape
    lh, fl = C.c_double(0), C.c_double(0)
    nv, nk = C.c_int32(0), C.c_int32(0)
    mask = np.zeros((T + 31) // 32, np.uint32)
    ok = lib().kbo_eval_one(_ptr(psi), _ptr(phi), _ptr(times), T, H, W, int(x0), int(y0),
                            float(vx), float(vy), q["min_obs"], q["clip"], q["q_lo"], q["q_mid"],
                            q["q_hi"], q["n_sigma"], q["clip_on"], C.byref(lh), C.byref(fl),
                            C.byref(nv), C.byref(nk), _ptr(mask))
    return dict(ok=bool(ok), lh=lh.value, flux=fl.value, nvalid=nv.value, nkept=nk.value,
                mask=mask)


def clip_margin(psi, phi, times, x0, y0, vx, vy, params=None):
    """Closest approach of one trajectory's lightcurve to its clip bounds in units of
    max(sigma_G, |median|, 1e-30) (reading R6; +inf when no clip decision is taken)."""
    q = _params(params)
    psi, phi, times = _f64(psi), _f64(phi), _f64(times)
    T, H, W = psi.shape
    return lib().kbo_clip_margin(_ptr(psi), _ptr(phi), _ptr(times), T, H, W, int(x0), int(y0),
                                 float(vx), float(vy), q["min_obs"], q["clip"], q["q_lo"],
                                 q["q_mid"], q["q_hi"], q["n_sigma"], q["clip_on"])


def stage_counts(psi, phi, times, vx, vy, params=None, window=None):
    """Stage counts over every pair of the window: (n_valid >= min_obs, LH' >= lh_min after the
    clip, sum of n_kept and sum of n_valid over the latter)."""
    q = _params(params)
    psi, phi, times = _f64(psi), _f64(phi), _f64(times)
    vx, vy = _f32(vx), _f32(vy)
    T, H, W = psi.shape
    x_lo, x_hi, y_lo, y_hi = (int(v) for v in (window or (0, W, 0, H)))
    out = np.zeros(4, np.uint64)
    rc = lib().kbo_stage_counts(_ptr(psi), _ptr(phi), _ptr(times), T, H, W, _ptr(vx), _ptr(vy),
                                len(vx), q["lh_min"], q["min_obs"], q["clip"], q["q_lo"],
                                q["q_mid"], q["q_hi"], q["n_sigma"], q["clip_on"], x_lo, x_hi,
                                y_lo, y_hi, _ptr(out))
    if rc != 0:
        raise ValueError("oracle stage_counts rejected its arguments")
    return tuple(int(v) for v in out)


def search(psi, phi, times, vx, vy, params=None, window=None):
    """Exhaustive search over the start-pixel window (x_lo, x_hi, y_lo, y_hi).

    Returns a dict of arrays shaped [wy][wx][K] (mask [wy][wx][K][ceil(T/32)])."""
    q = _params(params)
    psi, phi, times = _f64(psi), _f64(phi), _f64(times)
    vx, vy = _f32(vx), _f32(vy)
    T, H, W = psi.shape
    if window is None:
        window = (0, W, 0, H)
    x_lo, x_hi, y_lo, y_hi = (int(v) for v in window)
    K = int(q["k"])
    wy, wx = y_hi - y_lo, x_hi - x_lo
    mw = (T + 31) // 32
    out = dict(lh=np.zeros((wy, wx, K)), flux=np.zeros((wy, wx, K)),
               idx=np.zeros((wy, wx, K), np.int32), nvalid=np.zeros((wy, wx, K), np.int32),
               nkept=np.zeros((wy, wx, K), np.int32), mask=np.zeros((wy, wx, K, mw), np.uint32))
    rc = lib().kbo_search(_ptr(psi), _ptr(phi), _ptr(times), T, H, W, _ptr(vx), _ptr(vy), len(vx),
                          K, q["lh_min"], q["min_obs"], q["clip"], q["q_lo"], q["q_mid"],
                          q["q_hi"], q["n_sigma"], q["clip_on"], x_lo, x_hi, y_lo, y_hi,
                          _ptr(out["lh"]), _ptr(out["flux"]), _ptr(out["idx"]),
                          _ptr(out["nvalid"]), _ptr(out["nkept"]), _ptr(out["mask"]))
    if rc != 0:
        raise ValueError("oracle search rejected its arguments")
    return out


def stamps(img, var, mask, times, x0, y0, vx, vy, radius=10, keep_mask=None):
    """Mean and median coadded stamps [n][2r+1][2r+1] (Section 3.3)."""
    img, var, times = _f32(img), _f32(var), _f64(times)
    T, H, W = img.shape
    m = _mask_u8(mask, img.shape)
    x0 = np.ascontiguousarray(x0, np.int32)
    y0 = np.ascontiguousarray(y0, np.int32)
    vx, vy = _f32(vx), _f32(vy)
    n = len(x0)
    side = 2 * radius + 1
    km = None if keep_mask is None else np.ascontiguousarray(keep_mask, np.uint32)
    mean = np.zeros((n, side, side))
    med = np.zeros((n, side, side))
    lib().kbo_stamps(_ptr(img), _ptr(var), _ptr(m), _ptr(times), T, H, W, _ptr(x0), _ptr(y0),
                     _ptr(vx), _ptr(vy), _ptr(km), n, radius, _ptr(mean), _ptr(med))
    return mean, med


def traj_eval_subpixel(psi, phi, times, keep, x0, y0, vx, vy, grad=True):
    """Bilinear sub-pixel L, alpha and dL/d(x0, y0, vx, vy) over the fixed kept epochs."""
    psi, phi, times = _f64(psi), _f64(phi), _f64(times)
    T, H, W = psi.shape
    keep = np.ascontiguousarray(keep, np.uint32)
    lh, fl = C.c_double(0), C.c_double(0)
    g = np.zeros(4)
    lib().kbo_traj_eval_subpixel(_ptr(psi), _ptr(phi), _ptr(times), T, H, W, _ptr(keep),
                                 float(x0), float(y0), float(vx), float(vy), C.byref(lh),
                                 C.byref(fl), _ptr(g) if grad else None)
    return lh.value, fl.value, g


def traj_vjp(psi, phi, times, keep, x0, y0, vx, vy, gL=1.0, gA=0.0, images=True):
    """gL dL/d. + gA dalpha/d. of the sub-pixel evaluation: (grad_params [4], grad_psi, grad_phi)
    with dense [T][H][W] image gradients (None unless images); None if Phi <= 0."""
    psi, phi, times = _f64(psi), _f64(phi), _f64(times)
    T, H, W = psi.shape
    keep = np.ascontiguousarray(keep, np.uint32)
    gp = np.zeros(4)
    gpsi = np.zeros((T, H, W)) if images else None
    gphi = np.zeros((T, H, W)) if images else None
    rc = lib().kbo_traj_vjp(_ptr(psi), _ptr(phi), _ptr(times), T, H, W, _ptr(keep), float(x0),
                            float(y0), float(vx), float(vy), float(gL), float(gA), _ptr(gp),
                            _ptr(gpsi), _ptr(gphi))
    if rc != 0:
        return None
    return gp, gpsi, gphi


def refine_adam(psi, phi, times, keep, params, n_steps, lr_pos, lr_vel, b1=0.9, b2=0.999,
                eps=1e-8):
    """Adam ascent of L from params (x0, y0, vx, vy); returns (params, L, alpha), L and alpha NaN
    if Phi <= 0 was met (params then as they were at that point)."""
    psi, phi, times = _f64(psi), _f64(phi), _f64(times)
    T, H, W = psi.shape
    keep = np.ascontiguousarray(keep, np.uint32)
    pr = np.array(params, dtype=np.float64)
    lh, fl = C.c_double(0), C.c_double(0)
    lib().kbo_refine_adam(_ptr(psi), _ptr(phi), _ptr(times), T, H, W, _ptr(keep), _ptr(pr),
                          int(n_steps), float(lr_pos), float(lr_vel), float(b1), float(b2),
                          float(eps), C.byref(lh), C.byref(fl))
    return pr, lh.value, fl.value


PAPER_MOMENT_LIMITS = (0.5, 0.5, 1.5, 36.5, 36.5)   # x, y, xy, xx, yy (Section 3.3)


def stamp_moments(stamps, limits=PAPER_MOMENT_LIMITS):
    """Moments (sum, x, y, xy, xx, yy) [n][6] of stamps [n][2r+1][2r+1] about their centres and
    the filter decision [n] (bool)."""
    st = _f64(stamps)
    n, side, _ = st.shape
    r = side // 2
    lim = np.ascontiguousarray(limits, dtype=np.float64)
    out = np.zeros((n, 6))
    ok = np.zeros(n, bool)
    for i in range(n):
        s_i = np.ascontiguousarray(st[i])
        ok[i] = bool(lib().kbo_stamp_moments(_ptr(s_i), r, _ptr(lim), _ptr(out[i])))
    return out, ok


def cluster(x0, y0, vx, vy, dt, radius, valid=None):
    """Greedy de-duplication in index order: (keep [n] bool, rep [n] int32)."""
    x0 = np.ascontiguousarray(x0, np.int32)
    y0 = np.ascontiguousarray(y0, np.int32)
    vx = np.ascontiguousarray(vx, np.float32)
    vy = np.ascontiguousarray(vy, np.float32)
    n = len(x0)
    va = None if valid is None else np.ascontiguousarray(valid, np.uint8)
    keep = np.zeros(n, np.uint8)
    rep = np.zeros(n, np.int32)
    lib().kbo_cluster(_ptr(x0), _ptr(y0), _ptr(vx), _ptr(vy), _ptr(va), n, float(dt),
                      float(radius), _ptr(keep), _ptr(rep))
    return keep.astype(bool), rep


def set_threads(n):
    """OpenMP threads of the oracle's parallel loops."""
    lib().kbo_set_threads(int(n))


def get_threads():
    return int(lib().kbo_get_threads())
