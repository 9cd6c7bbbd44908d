"""Pins of the FP64 oracle to things other than itself: the paper's printed numbers, closed forms,
library routines it does not use (scipy.special.erfinv, numpy percentiles/median), invariances,
and an independent numpy shift-and-stack brute force on tiny stacks."""
import json
import math
import os
import warnings

import numpy as np
import pytest
import scipy.special

import oracle
from synth import gaussian_psf, velocity_grid

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def paper():
    with open(os.path.join(GOLDEN, "paper_constants.json")) as f:
        return json.load(f)


# ------------------------------------------------------------------------------------------------
# sigma_G (Section 3.1, Eqs. 1-5)
# ------------------------------------------------------------------------------------------------

def test_sigma_g_coeff_matches_paper_and_closed_form():
    c = oracle.sigma_g_coeff(0.25, 0.75)
    printed = paper()["sigma_g_coeff_25_75"]["value"]
    assert abs(c - printed) < 5e-5                       # 0.7413 as printed in Section 3.1
    closed = 1.0 / (2.0 * math.sqrt(2.0) * scipy.special.erfinv(0.5))
    assert abs(c - closed) < 1e-13
    for lo, hi in [(0.1, 0.9), (0.16, 0.84), (0.3, 0.6), (0.05, 0.75)]:
        ref = 1.0 / (math.sqrt(2.0) * (scipy.special.erfinv(2 * hi - 1) -
                                       scipy.special.erfinv(2 * lo - 1)))
        assert abs(oracle.sigma_g_coeff(lo, hi) - ref) < 1e-12 * abs(ref)


def test_erfinv_against_scipy():
    for y in np.linspace(-0.999, 0.999, 101):
        assert abs(oracle.erfinv(y) - scipy.special.erfinv(y)) < 1e-12 * max(1.0, abs(y))


def test_sigma_g_estimates_gaussian_width():
    # Section 3.1: sigma_G estimates the standard deviation of the underlying Gaussian.
    rng = np.random.default_rng(11)
    x = rng.normal(3.0, 2.5, 400001)
    keep, med, sg = oracle.sigma_g_clip(x)
    assert abs(sg - 2.5) < 0.02
    assert abs(med - 3.0) < 0.02
    # +-2 sigma_G keeps ~95.45% of a Gaussian
    assert abs(keep.mean() - 0.9545) < 0.003


def test_percentile_matches_numpy_linear():
    rng = np.random.default_rng(5)
    for n in list(range(1, 41)) + [100, 128]:
        x = rng.normal(size=n) * rng.uniform(0.1, 10)
        for q in (0.0, 0.1, 0.25, 0.5, 0.75, 0.9, 1.0, 0.37):
            ref = np.percentile(x, 100 * q, method="linear")
            assert abs(oracle.percentile(x, q) - ref) <= 1e-12 * max(1.0, np.abs(x).max())


def test_sigma_g_clip_hand_worked_example():
    # values 1,2,3,4,100: h(q) = 4 q -> x25 = 2, median 3, x75 = 4; sigma_G = 2C;
    # bounds 3 -+ 4C = [0.0348, 5.9652]: 100 is rejected, the rest kept.
    keep, med, sg = oracle.sigma_g_clip([1.0, 2.0, 3.0, 4.0, 100.0])
    C = 1.0 / (2.0 * math.sqrt(2.0) * scipy.special.erfinv(0.5))
    assert med == 3.0
    assert abs(sg - 2.0 * C) < 1e-14
    assert keep.tolist() == [True, True, True, True, False]
    # order does not matter
    keep, _, _ = oracle.sigma_g_clip([100.0, 3.0, 1.0, 4.0, 2.0])
    assert keep.tolist() == [False, True, True, True, True]


def test_sigma_g_clip_constant_and_inclusive_bound():
    # a constant lightcurve has sigma_G = 0 and keeps every epoch (the bound is inclusive)
    keep, med, sg = oracle.sigma_g_clip([4.25] * 9)
    assert sg == 0.0 and keep.all()
    # five equal values and one other: x25 = x75 = median = 5, sigma_G = 0 -> only the 5s kept
    keep, med, sg = oracle.sigma_g_clip([5.0, 5.0, 6.0, 5.0, 5.0, 5.0])
    assert sg == 0.0 and med == 5.0
    assert keep.tolist() == [True, True, False, True, True, True]


def test_sigma_g_clip_rejects_spikes():
    rng = np.random.default_rng(3)
    x = rng.normal(0, 1, 200)
    spikes = np.full(20, 20.0)
    keep, med, sg = oracle.sigma_g_clip(np.concatenate([x, spikes]))
    assert not keep[200:].any()
    assert keep[:200].mean() > 0.9


# ------------------------------------------------------------------------------------------------
# Track rounding (R1): three IEEE single operations, round half up
# ------------------------------------------------------------------------------------------------

def np_offsets(times, v):
    dt = (np.asarray(times, np.float64) - times[0]).astype(np.float32)
    return np.floor(np.float32(v) * dt + np.float32(0.5)).astype(np.int64)


def _resting_track_case(a4):
    """T = 5 epochs of a 3 x 3 image with phi = 1 and psi = 0, 1, 2, 3, a4 at the centre: the
    flux lightcurve of the resting track (vx = vy = 0) started there."""
    T = 5
    psi = np.zeros((T, 3, 3))
    phi = np.ones((T, 3, 3))
    psi[:, 1, 1] = [0.0, 1.0, 2.0, 3.0, a4]
    times = np.array([0.0, 0.1, 0.2, 0.3, 0.4])
    return psi, phi, times


def test_clip_margin_closed_forms():
    """oracle.clip_margin (reading R6): quartiles 1 and 3, median 2, sigma_G = 2C and bounds
    2 -+ 4C at n = 2 (Section 3.1, Eqs. 3-5).  With a4 = 4 the nearest epochs (0 and 4) lie 4C - 2
    from a bound, i.e. 2C - 1 in units of max(sigma_G, |median|) = 2; with a4 on the upper bound
    the margin is 0; no clip decision (clip off, too few epochs) gives +inf."""
    c = 1.0 / (2.0 * math.sqrt(2.0) * scipy.special.erfinv(0.5))
    psi, phi, times = _resting_track_case(4.0)
    p = dict(min_obs=1, clip=1, q_lo=0.25, q_mid=0.5, q_hi=0.75, n_sigma=2.0)
    m = oracle.clip_margin(psi, phi, times, 1, 1, 0.0, 0.0, p)
    assert abs(m - (2.0 * c - 1.0)) < 1e-12
    upper = 2.0 + 2.0 * (oracle.sigma_g_coeff(0.25, 0.75) * 2.0)   # the oracle's own bound
    psi_b, phi_b, _ = _resting_track_case(upper)
    assert oracle.clip_margin(psi_b, phi_b, times, 1, 1, 0.0, 0.0, p) == 0.0
    # a first epoch on the lower bound (the quartiles and median are unchanged): margin 0
    psi_l, phi_l, _ = _resting_track_case(4.0)
    psi_l[0, 1, 1] = 2.0 - 2.0 * (oracle.sigma_g_coeff(0.25, 0.75) * 2.0)
    assert oracle.clip_margin(psi_l, phi_l, times, 1, 1, 0.0, 0.0, p) == 0.0
    # the margin is a property of one trajectory: the keep decision at the bound is inclusive
    r = oracle.eval_one(psi_b, phi_b, times, 1, 1, 0.0, 0.0, p)
    assert r["nkept"] == 5
    assert oracle.clip_margin(psi, phi, times, 1, 1, 0.0, 0.0, dict(p, clip=0)) == np.inf
    assert oracle.clip_margin(psi, phi, times, 1, 1, 0.0, 0.0, dict(p, min_obs=6)) == np.inf
    # a track that leaves the image after one epoch has one valid epoch: sigma_G = 0, bounds at
    # the value itself
    assert oracle.clip_margin(psi, phi, times, 1, 1, 30.0, 0.0, p) == 0.0


def test_track_offsets_match_float32_arithmetic():
    rng = np.random.default_rng(7)
    vx = rng.uniform(-600, 600, 200).astype(np.float32)
    vy = rng.uniform(-600, 600, 200).astype(np.float32)
    # epochs from 0 and as MJDs: the time difference is taken in float64, then rounded once
    for t0 in (0.0, 57000.37):
        times = t0 + np.sort(rng.uniform(0, 4, 30))
        ox, oy = oracle.track_offsets(times, vx, vy)
        for j in range(200):
            assert (ox[j] == np_offsets(times, vx[j])).all()
            assert (oy[j] == np_offsets(times, vy[j])).all()


def test_track_offsets_half_up():
    times = np.array([0.0, 1.0, 2.0])
    ox, oy = oracle.track_offsets(times, np.array([2.5, -2.5], np.float32),
                                  np.array([0.25, -0.75], np.float32))
    assert ox.tolist() == [[0, 3, 5], [0, -2, -5]]
    assert oy.tolist() == [[0, 0, 1], [0, -1, -1]]


# ------------------------------------------------------------------------------------------------
# psi / phi (Section 3; R0)
# ------------------------------------------------------------------------------------------------

def test_phi_constant_variance_closed_form():
    rng = np.random.default_rng(1)
    T, H, W, k = 2, 20, 23, 7
    psf = rng.uniform(0.0, 1.0, (T, k, k)).astype(np.float32)   # asymmetric on purpose
    v = np.float32(1.7)
    img = rng.normal(size=(T, H, W)).astype(np.float32)
    var = np.full((T, H, W), v, np.float32)
    psi, phi = oracle.psi_phi(img, var, None, psf)
    r = k // 2
    for t in range(T):
        ref = (psf[t].astype(np.float64) ** 2).sum() / float(v)
        inner = phi[t, r:H - r, r:W - r]
        assert np.allclose(inner, ref, rtol=1e-12, atol=0)
        # corner pixel (0, 0): only taps with u >= 0 fall inside
        corner = (psf[t, r:, r:].astype(np.float64) ** 2).sum() / float(v)
        assert abs(phi[t, 0, 0] - corner) < 1e-12 * corner


def test_psi_delta_image_is_correlation():
    rng = np.random.default_rng(2)
    T, H, W, k = 1, 17, 19, 5
    psf = rng.uniform(0.0, 1.0, (T, k, k)).astype(np.float32)   # asymmetric
    img = np.zeros((T, H, W), np.float32)
    A, v = 3.0, 0.5
    yd, xd = 8, 9
    img[0, yd, xd] = A
    var = np.full((T, H, W), v, np.float32)
    psi, _ = oracle.psi_phi(img, var, None, psf)
    r = k // 2
    ref = np.zeros((H, W))
    for y in range(H):
        for x in range(W):
            uy, ux = yd - y, xd - x
            if abs(uy) <= r and abs(ux) <= r:
                ref[y, x] = A / v * float(psf[0, uy + r, ux + r])
    assert np.allclose(psi[0], ref, rtol=1e-12, atol=1e-15)


def test_psi_phi_masking():
    rng = np.random.default_rng(4)
    T, H, W, k = 1, 15, 15, 5
    psf = rng.uniform(0.1, 1.0, (T, k, k)).astype(np.float32)
    img = rng.normal(size=(T, H, W)).astype(np.float32)
    var = np.full((T, H, W), 2.0, np.float32)
    mask = np.zeros((T, H, W), np.uint8)
    mask[0, 7, 7] = 1
    var[0, 3, 3] = np.inf            # non-finite variance is masked
    var[0, 10, 4] = -1.0             # non-positive variance is masked
    img[0, 11, 11] = np.nan          # non-finite image is masked
    psi, phi = oracle.psi_phi(img, var, mask, psf)
    for (y, x) in [(7, 7), (3, 3), (10, 4), (11, 11)]:
        assert psi[0, y, x] == 0.0 and phi[0, y, x] == 0.0
    # neighbour (7, 8) of the masked (7, 7): phi lacks exactly the tap u = (0, -1)
    r = k // 2
    full = (psf[0].astype(np.float64) ** 2).sum() / 2.0
    expect = full - float(psf[0, r + 0, r - 1]) ** 2 / 2.0
    assert abs(phi[0, 7, 8] - expect) < 1e-12


def test_psi_phi_at_matches_full():
    rng = np.random.default_rng(6)
    T, H, W, k = 3, 31, 29, 7
    psf = rng.uniform(0.0, 1.0, (T, k, k)).astype(np.float32)
    img = rng.normal(size=(T, H, W)).astype(np.float32)
    var = rng.uniform(0.5, 2, (T, H, W)).astype(np.float32)
    mask = (rng.random((T, H, W)) < 0.05).astype(np.uint8)
    psi, phi = oracle.psi_phi(img, var, mask, psf)
    tyx = np.stack([rng.integers(0, T, 50), rng.integers(0, H, 50), rng.integers(0, W, 50)], 1)
    ps, ph = oracle.psi_phi_at(img, var, mask, psf, tyx)
    assert np.array_equal(ps, psi[tyx[:, 0], tyx[:, 1], tyx[:, 2]])
    assert np.array_equal(ph, phi[tyx[:, 0], tyx[:, 1], tyx[:, 2]])
    # triples outside the stack read NaN
    bad = np.array([[T, 0, 0], [0, -1, 3], [1, 2, W]])
    ps, ph = oracle.psi_phi_at(img, var, mask, psf, bad)
    assert np.isnan(ps).all() and np.isnan(ph).all()


def test_psi_phi_match_scipy_correlate_with_varying_variance():
    # With masked pixels zeroed, psi_t and phi_t are the zero-padded correlations of I w and w
    # with P_t and P_t^2 (scipy.ndimage.correlate, a routine the oracle does not use), and 0 at
    # masked pixels.  The variance varies per pixel, so each tap must take its own pixel's weight.
    import scipy.ndimage
    rng = np.random.default_rng(8)
    T, H, W, k = 3, 26, 21, 7
    psf = rng.uniform(0.0, 1.0, (T, k, k)).astype(np.float32)   # asymmetric
    img = rng.normal(size=(T, H, W)).astype(np.float32)
    var = rng.uniform(0.3, 3.0, (T, H, W)).astype(np.float32)
    mask = (rng.random((T, H, W)) < 0.08).astype(np.uint8)
    psi, phi = oracle.psi_phi(img, var, mask, psf)
    good = mask == 0
    w = np.where(good, 1.0 / var.astype(np.float64), 0.0)
    for t in range(T):
        P = psf[t].astype(np.float64)
        ref_psi = scipy.ndimage.correlate(img[t] * w[t], P, mode="constant", cval=0.0)
        ref_phi = scipy.ndimage.correlate(w[t], P * P, mode="constant", cval=0.0)
        ref_psi[~good[t]] = 0.0
        ref_phi[~good[t]] = 0.0
        assert np.allclose(psi[t], ref_psi, rtol=1e-12, atol=1e-12)
        assert np.allclose(phi[t], ref_phi, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------------------------------------
# Search closed form: one noiseless mover, L = SNR sqrt(T), alpha = F  (Section 3: nu = Psi/sqrt Phi)
# ------------------------------------------------------------------------------------------------

def _noiseless_mover(T=8, H=64, W=64, snr=5.0, v=1.7, sigma=1.2, k=7, seed=0):
    rng = np.random.default_rng(seed)
    v = float(np.float32(v))            # the variance plane is float32
    times = np.sort(rng.uniform(0, 0.2, T))
    times[0] = 0.0
    vx, vy = velocity_grid(50.0, 120.0, 6, -0.3, 0.3, 5)
    j = 17
    psf = np.stack([gaussian_psf(sigma, k)] * T).astype(np.float32)
    sum_p2 = (psf[0].astype(np.float64) ** 2).sum()
    F = snr * math.sqrt(v) / math.sqrt(sum_p2)
    img = np.zeros((T, H, W), np.float32)
    x0, y0 = 20, 25
    ox, oy = np_offsets(times, vx[j]), np_offsets(times, vy[j])
    r = k // 2
    for t in range(T):
        x, y = x0 + ox[t], y0 + oy[t]
        assert r <= x < W - r and r <= y < H - r
        img[t, y - r:y + r + 1, x - r:x + r + 1] += (F * psf[t]).astype(np.float32)
    var = np.full((T, H, W), v, np.float32)
    return dict(img=img, var=var, psf=psf, times=times, vx=vx, vy=vy, j=j, x0=x0, y0=y0, F=F,
                T=T, snr=snr)


def test_search_noiseless_mover_closed_form():
    m = _noiseless_mover()
    # The image holds F * P exactly only up to float32 rounding of the injected values; build the
    # closed form from the stored image, which is F P rounded: the tolerance covers that rounding.
    psi, phi = oracle.psi_phi(m["img"], m["var"], None, m["psf"])
    res = oracle.search(psi, phi, m["times"], m["vx"], m["vy"],
                        dict(k=1, lh_min=1.0, min_obs=1), window=(m["x0"], m["x0"] + 1,
                                                                   m["y0"], m["y0"] + 1))
    L = res["lh"][0, 0, 0]
    a = res["flux"][0, 0, 0]
    assert abs(L - m["snr"] * math.sqrt(m["T"])) < 1e-6 * L
    assert abs(a - m["F"]) < 1e-6 * m["F"]
    assert res["nkept"][0, 0, 0] == m["T"] and res["nvalid"][0, 0, 0] == m["T"]
    idx = res["idx"][0, 0, 0]
    same_track = (np.array_equal(np_offsets(m["times"], m["vx"][idx]),
                                 np_offsets(m["times"], m["vx"][m["j"]])) and
                  np.array_equal(np_offsets(m["times"], m["vy"][idx]),
                                 np_offsets(m["times"], m["vy"][m["j"]])))
    assert idx == m["j"] or same_track


def test_search_noiseless_mover_exact_psi_phi():
    # With psi/phi written from the closed form directly (FP64), L and alpha match to 1e-9.
    m = _noiseless_mover(T=12, snr=6.5)
    T, H, W = m["img"].shape
    sum_p2 = (m["psf"][0].astype(np.float64) ** 2).sum()
    v = float(m["var"][0, 0, 0])
    phi = np.full((T, H, W), sum_p2 / v)
    psi = np.zeros((T, H, W))
    ox, oy = np_offsets(m["times"], m["vx"][m["j"]]), np_offsets(m["times"], m["vy"][m["j"]])
    for t in range(T):
        psi[t, m["y0"] + oy[t], m["x0"] + ox[t]] = m["F"] * sum_p2 / v
    res = oracle.search(psi, phi, m["times"], m["vx"], m["vy"], dict(k=2, lh_min=1.0, min_obs=1),
                        window=(m["x0"], m["x0"] + 1, m["y0"], m["y0"] + 1))
    assert abs(res["lh"][0, 0, 0] - m["snr"] * math.sqrt(T)) < 1e-9 * m["snr"] * math.sqrt(T)
    assert abs(res["flux"][0, 0, 0] - m["F"]) < 1e-9 * m["F"]
    assert res["mask"][0, 0, 0, 0] == (1 << T) - 1


# ------------------------------------------------------------------------------------------------
# Independent numpy shift-and-stack brute force (different formulation: whole shifted planes,
# numpy.nanpercentile for the quantiles, numpy sort for the selection)
# ------------------------------------------------------------------------------------------------

def numpy_search(psi, phi, times, vx, vy, K, lh_min, min_obs, clip=True, n_sigma=2.0,
                 clip_on=0, q=(25.0, 50.0, 75.0)):
    T, H, W = psi.shape
    C = 1.0 / (math.sqrt(2.0) * (scipy.special.erfinv(2 * q[2] / 100 - 1) -
                                 scipy.special.erfinv(2 * q[0] / 100 - 1)))
    cand = [[[] for _ in range(W)] for _ in range(H)]
    for j in range(len(vx)):
        ox, oy = np_offsets(times, vx[j]), np_offsets(times, vy[j])
        P = np.full((T, H, W), np.nan)
        F = np.full((T, H, W), np.nan)
        for t in range(T):
            ys = np.arange(H) + oy[t]
            xs = np.arange(W) + ox[t]
            yv = (ys >= 0) & (ys < H)
            xv = (xs >= 0) & (xs < W)
            P[t][np.ix_(yv, xv)] = psi[t][np.ix_(ys[yv], xs[xv])]
            F[t][np.ix_(yv, xv)] = phi[t][np.ix_(ys[yv], xs[xv])]
        valid = np.isfinite(P) & (np.nan_to_num(F) > 0)
        with np.errstate(divide="ignore", invalid="ignore"):
            a = np.where(valid, P / F if clip_on == 0 else P / np.sqrt(F), np.nan)
        nvalid = valid.sum(0)
        if clip:
            with warnings.catch_warnings():
                warnings.simplefilter("ignore")
                lo, mid, hi = np.nanpercentile(a, list(q), axis=0, method="linear")
            sg = C * (hi - lo)
            keep = valid & (a >= mid - n_sigma * sg) & (a <= mid + n_sigma * sg)
        else:
            keep = valid
        sp = np.where(keep, P, 0.0).sum(0)
        sf = np.where(keep, F, 0.0).sum(0)
        with np.errstate(divide="ignore", invalid="ignore"):
            L = sp / np.sqrt(sf)
        ok = (nvalid >= min_obs) & (keep.sum(0) > 0) & (sf > 0) & (L >= lh_min)
        for y, x in zip(*np.nonzero(ok)):
            bits = np.zeros((T + 31) // 32, np.uint64)
            for t in np.nonzero(keep[:, y, x])[0]:
                bits[t // 32] |= np.uint64(1) << np.uint64(t % 32)
            cand[y][x].append((-L[y, x], j, sp[y, x] / sf[y, x], nvalid[y, x],
                               keep[:, y, x].sum(), bits))
    out_idx = np.full((H, W, K), -1)
    out_lh = np.full((H, W, K), -np.inf)
    out_flux = np.zeros((H, W, K))
    out_nv = np.zeros((H, W, K), int)
    out_nk = np.zeros((H, W, K), int)
    out_mask = np.zeros((H, W, K, (T + 31) // 32), np.uint64)
    for y in range(H):
        for x in range(W):
            for s, c in enumerate(sorted(cand[y][x], key=lambda e: (e[0], e[1]))[:K]):
                out_lh[y, x, s], out_idx[y, x, s], out_flux[y, x, s] = -c[0], c[1], c[2]
                out_nv[y, x, s], out_nk[y, x, s], out_mask[y, x, s] = c[3], c[4], c[5]
    return dict(lh=out_lh, idx=out_idx, flux=out_flux, nvalid=out_nv, nkept=out_nk,
                mask=out_mask)


def _tiny_case(seed, T=6, H=12, W=14, n_traj=40, mask_frac=0.08):
    rng = np.random.default_rng(seed)
    times = np.sort(rng.uniform(0, 1.0, T))
    times[0] = 0.0
    phi = rng.uniform(0.2, 1.5, (T, H, W))
    psi = rng.normal(size=(T, H, W)) * np.sqrt(phi)
    psi += 3.0 * phi * (rng.random((T, H, W)) < 0.15)          # bright spots
    psi[:, 5, 6] += 8.0 * phi[:, 5, 6]                          # a static source
    m = rng.random((T, H, W)) < mask_frac
    psi[m] = 0.0
    phi[m] = 0.0
    vx = rng.uniform(-6, 6, n_traj).astype(np.float32)
    vy = rng.uniform(-6, 6, n_traj).astype(np.float32)
    vx[5], vy[5] = vx[3], vy[3]                                 # duplicate track -> index tie
    vx[9], vy[9] = np.nextafter(vx[8], np.float32(10)), vy[8]   # near-duplicate
    psi = psi.astype(np.float32).astype(np.float64)
    phi = phi.astype(np.float32).astype(np.float64)
    return psi, phi, times, vx, vy


@pytest.mark.parametrize("seed,clip,clip_on,K,T,q,n_sigma", [
    (0, True, 0, 3, 6, (0.25, 0.5, 0.75), 2.0),
    (1, True, 1, 2, 6, (0.25, 0.5, 0.75), 2.0),
    (2, False, 0, 4, 6, (0.25, 0.5, 0.75), 2.0),
    (3, True, 0, 1, 6, (0.25, 0.5, 0.75), 2.0),
    (4, True, 0, 5, 40, (0.1, 0.5, 0.9), 1.5),      # two mask words, other quantiles and width
    (5, True, 1, 8, 12, (0.2, 0.45, 0.8), 2.5),     # an off-centre "median"
])
def test_search_matches_numpy_brute_force(seed, clip, clip_on, K, T, q, n_sigma):
    psi, phi, times, vx, vy = _tiny_case(seed, T=T)
    lh_min, min_obs = 0.5, 3
    # the search takes its quantiles and width as float32 (both sides use the rounded values)
    q32 = [float(np.float32(v)) for v in q]
    ref = numpy_search(psi, phi, times, vx, vy, K, lh_min, min_obs, clip=clip, clip_on=clip_on,
                       n_sigma=n_sigma, q=tuple(100.0 * v for v in q32))
    got = oracle.search(psi, phi, times, vx, vy, dict(k=K, lh_min=lh_min, min_obs=min_obs,
                                                      clip=int(clip), clip_on=clip_on,
                                                      q_lo=q[0], q_mid=q[1], q_hi=q[2],
                                                      n_sigma=n_sigma))
    assert np.array_equal(got["idx"], ref["idx"])
    filled = ref["idx"] >= 0
    assert filled.sum() > 50
    assert np.allclose(got["lh"][filled], ref["lh"][filled], rtol=1e-12, atol=0)
    assert np.allclose(got["flux"][filled], ref["flux"][filled], rtol=1e-10, atol=1e-12)
    assert np.array_equal(got["nvalid"], ref["nvalid"])
    assert np.array_equal(got["nkept"], ref["nkept"])
    assert np.array_equal(got["mask"].astype(np.uint64), ref["mask"])


def test_search_duplicate_track_tie_break():
    psi, phi, times, vx, vy = _tiny_case(0)
    got = oracle.search(psi, phi, times, vx, vy, dict(k=40, lh_min=-1e9, min_obs=1))
    # trajectories 3 and 5 have identical tracks: wherever both appear, 3 ranks first and every
    # entry between them ties on L' with ascending indices (other tracks can reach the same
    # valid pixels when they leave the image)
    seen = 0
    for y in range(psi.shape[1]):
        for x in range(psi.shape[2]):
            row = got["idx"][y, x].tolist()
            if 3 in row and 5 in row:
                i3, i5 = row.index(3), row.index(5)
                assert i5 > i3
                assert (got["lh"][y, x, i3:i5 + 1] == got["lh"][y, x, i3]).all()
                assert row[i3:i5 + 1] == sorted(row[i3:i5 + 1])
                seen += 1
    assert seen > 20


def test_search_invariances():
    psi, phi, times, vx, vy = _tiny_case(4)
    p = dict(k=3, lh_min=0.5, min_obs=3)
    base = oracle.search(psi, phi, times, vx, vy, p)
    # (1) scaling psi and phi by c > 0 keeps the flux lightcurve, so masks and order are kept;
    #     L' scales by sqrt(c), alpha is unchanged (Section 3: nu = Psi / sqrt(Phi)).
    c = 4.0
    p2 = dict(p, lh_min=0.5 * 2.0)
    sc = oracle.search(psi * c, phi * c, times, vx, vy, p2)
    assert np.array_equal(sc["idx"], base["idx"])
    f = base["idx"] >= 0
    assert np.allclose(sc["lh"][f], 2.0 * base["lh"][f], rtol=1e-12)
    assert np.allclose(sc["flux"][f], base["flux"][f], rtol=1e-12)
    assert np.array_equal(sc["mask"], base["mask"])
    # (2) a common shift of all epoch times changes nothing (tracks use t - t_0).  The times are
    #     put on a 2^-30-day grid so that t + 57000.25 (an MJD-like origin) is exact in float64
    #     and every difference t - t_0 is unchanged: the results must be bit-identical, while a
    #     track measured from t = 0 instead of the first epoch would move by ~57000 days x v.
    tg = np.round(times * 2.0 ** 30) / 2.0 ** 30
    g0 = oracle.search(psi, phi, tg, vx, vy, p)
    sh = oracle.search(psi, phi, tg + 57000.25, vx, vy, p)
    assert not np.array_equal(tg + 57000.25, tg)
    for key in ("idx", "mask", "nvalid", "nkept"):
        assert np.array_equal(sh[key], g0[key]), key
    f0 = g0["idx"] >= 0
    assert f0.sum() > 10
    assert np.array_equal(sh["lh"][f0], g0["lh"][f0])
    assert np.array_equal(sh["flux"][f0], g0["flux"][f0])
    # (3) translating the content of every plane by (+2, +1) translates the results
    T, H, W = psi.shape
    psi2 = np.zeros_like(psi)
    phi2 = np.zeros_like(phi)
    psi2[:, 1:, 2:] = psi[:, :-1, :-2]
    phi2[:, 1:, 2:] = phi[:, :-1, :-2]
    big = dict(p, lh_min=-1e9)
    r1 = oracle.search(psi, phi, times, vx, vy, big, window=(3, 6, 3, 6))
    r2 = oracle.search(psi2, phi2, times, vx, vy, big, window=(5, 8, 4, 7))
    # only trajectories that stay clear of the borders are comparable: check the best one
    # whose track stays inside both frames at every epoch
    ox, oy = oracle.track_offsets(times, vx, vy)
    inside = [j for j in range(len(vx)) if
              (3 + ox[j].min() >= 0 and 5 + ox[j].max() < W - 2 and 3 + oy[j].min() >= 0 and
               5 + oy[j].max() < H - 1)]
    assert inside
    for j in inside[:5]:
        a = oracle.eval_one(psi, phi, times, 4, 4, vx[j], vy[j], p)
        b = oracle.eval_one(psi2, phi2, times, 6, 5, vx[j], vy[j], p)
        assert a["nvalid"] == b["nvalid"] and a["nkept"] == b["nkept"]
        if a["ok"]:
            assert abs(a["lh"] - b["lh"]) < 1e-12 * max(1, abs(a["lh"]))


def test_min_obs_and_off_image():
    psi, phi, times, vx, vy = _tiny_case(5, mask_frac=0.0)
    T = psi.shape[0]
    # min_obs above T: nothing can be selected
    r = oracle.search(psi, phi, times, vx, vy, dict(k=2, lh_min=-1e9, min_obs=T + 1))
    assert (r["idx"] < 0).all()
    # a trajectory that leaves the image has fewer valid epochs than T
    e = oracle.eval_one(psi, phi, times, 0, 0, -50.0, -50.0, dict(min_obs=1))
    assert e["nvalid"] == 1


def test_threshold_is_inclusive_at_an_exact_likelihood():
    # psi = phi = 1 on every pixel: a trajectory with all T = 16 epochs on the image has
    # Psi = Phi = 16 and L = 16 / sqrt(16) = 4 exactly (and a constant lightcurve keeps every
    # epoch), one with n < 16 epochs on the image has L = sqrt(n) < 4.  A threshold of exactly 4
    # keeps the former (ties to the lower trajectory index first); the next float32 above 4
    # keeps nothing anywhere.
    T, H, W = 16, 9, 12
    psi = np.ones((T, H, W))
    phi = np.ones((T, H, W))
    times = 0.05 * np.arange(T)
    vx = np.array([0.0, 10.0], np.float32)      # offsets 0 and round-half-up(0.5 t) <= 8
    vy = np.zeros(2, np.float32)
    r = oracle.search(psi, phi, times, vx, vy, dict(k=2, lh_min=4.0, min_obs=1))
    assert r["idx"][5, 1].tolist() == [0, 1] and r["lh"][5, 1].tolist() == [4.0, 4.0]
    assert r["idx"][5, 8].tolist() == [0, -1]   # trajectory 1 leaves the image from x0 = 8
    above = float(np.nextafter(np.float32(4.0), np.float32(5.0)))
    r = oracle.search(psi, phi, times, vx, vy, dict(k=2, lh_min=above, min_obs=1))
    assert (r["idx"] < 0).all()


# ------------------------------------------------------------------------------------------------
# Stamps (Section 3.3)
# ------------------------------------------------------------------------------------------------

def test_stamps_noiseless_mover_is_flux_times_psf():
    m = _noiseless_mover()
    j = m["j"]
    mean, med = oracle.stamps(m["img"], m["var"], None, m["times"], [m["x0"]], [m["y0"]],
                              [m["vx"][j]], [m["vy"][j]], radius=10)
    k = m["psf"].shape[-1]
    r = k // 2
    ref = np.zeros((21, 21))
    ref[10 - r:10 + r + 1, 10 - r:10 + r + 1] = (m["F"] * m["psf"][0]).astype(np.float32)
    assert np.allclose(mean[0], ref, rtol=1e-6, atol=1e-7)
    assert np.allclose(med[0], ref, rtol=1e-6, atol=1e-7)


def test_stamps_against_numpy_gather():
    rng = np.random.default_rng(9)
    T, H, W = 7, 30, 33
    img = rng.normal(size=(T, H, W)).astype(np.float32)
    var = np.ones((T, H, W), np.float32)
    mask = (rng.random((T, H, W)) < 0.1).astype(np.uint8)
    times = np.sort(rng.uniform(0, 0.5, T))
    x0 = rng.integers(0, W, 6)
    y0 = rng.integers(0, H, 6)
    vx = rng.uniform(-20, 20, 6).astype(np.float32)
    vy = rng.uniform(-20, 20, 6).astype(np.float32)
    keep = rng.integers(0, 2 ** T, 6).astype(np.uint32).reshape(6, 1)
    for km in (None, keep):
        R = 3
        mean, med = oracle.stamps(img, var, mask, times, x0, y0, vx, vy, radius=R, keep_mask=km)
        for c in range(6):
            ox, oy = np_offsets(times, vx[c]), np_offsets(times, vy[c])
            for sy in range(-R, R + 1):
                for sx in range(-R, R + 1):
                    vals = []
                    for t in range(T):
                        if km is not None and not (int(km[c, 0]) >> t) & 1:
                            continue
                        x, y = x0[c] + ox[t] + sx, y0[c] + oy[t] + sy
                        if 0 <= x < W and 0 <= y < H and not mask[t, y, x]:
                            vals.append(float(img[t, y, x]))
                    got_mean, got_med = mean[c, sy + R, sx + R], med[c, sy + R, sx + R]
                    if not vals:
                        assert np.isnan(got_mean) and np.isnan(got_med)
                    else:
                        assert abs(got_mean - np.mean(vals)) < 1e-12
                        assert got_med == np.median(vals)


# ------------------------------------------------------------------------------------------------
# Sub-pixel trajectory likelihood and gradient (refinement off the grid)
# ------------------------------------------------------------------------------------------------

def test_subpixel_eval_equals_integer_eval_on_integer_tracks():
    rng = np.random.default_rng(12)
    T, H, W = 6, 40, 40
    phi = rng.uniform(0.2, 1.0, (T, H, W))
    psi = rng.normal(size=(T, H, W)) * np.sqrt(phi)
    vx, vy = np.float32(8.0), np.float32(-4.0)        # integer positions at every epoch
    keep = np.array([(1 << T) - 1], np.uint32)
    # epochs counted from 0 and as MJDs: both paths measure time from the first epoch
    for t0 in (0.0, 57000.5):
        times = t0 + np.arange(T) * 0.25
        L, a, g = oracle.traj_eval_subpixel(psi, phi, times, keep, 10.0, 20.0, vx, vy)
        e = oracle.eval_one(psi, phi, times, 10, 20, vx, vy, dict(clip=0, min_obs=0))
        assert abs(L - e["lh"]) < 1e-12 * abs(e["lh"])
        assert abs(a - e["flux"]) < 1e-12 * abs(e["flux"])


def test_subpixel_gradient_against_finite_differences():
    rng = np.random.default_rng(13)
    T, H, W = 8, 48, 48
    times = np.sort(rng.uniform(0, 0.2, T))
    times[0] = 0.0
    phi = rng.uniform(0.2, 1.0, (T, H, W))
    psi = rng.normal(size=(T, H, W)) * np.sqrt(phi) + 2.0 * phi
    keep = np.array([0b10111011], np.uint32)
    checked = 0
    for trial in range(40):
        x0, y0 = rng.uniform(10, 30, 2)
        vx, vy = rng.uniform(-40, 40, 2)
        h = 1e-3
        dts = times - times[0]
        # skip points within 2h of a cell edge at any epoch (piecewise-bilinear kinks)
        xs = x0 + vx * dts
        ys = y0 + vy * dts
        edge = min(np.abs(xs - np.round(xs)).min(), np.abs(ys - np.round(ys)).min())
        if edge < 4 * h * (1 + dts.max()):
            continue
        L, a, g = oracle.traj_eval_subpixel(psi, phi, times, keep, x0, y0, vx, vy)
        p = np.array([x0, y0, vx, vy])
        fd = np.zeros(4)
        for i in range(4):
            pp, pm = p.copy(), p.copy()
            pp[i] += h
            pm[i] -= h
            Lp = oracle.traj_eval_subpixel(psi, phi, times, keep, *pp, grad=False)[0]
            Lm = oracle.traj_eval_subpixel(psi, phi, times, keep, *pm, grad=False)[0]
            fd[i] = (Lp - Lm) / (2 * h)
        assert np.all(np.abs(g - fd) <= 1e-3 * np.maximum(np.abs(fd), 1e-2)), (g, fd)
        checked += 1
    assert checked >= 10


def test_paper_grid_shape():
    pc = paper()
    vx, vy = velocity_grid(*pc["grid_speed_range_px_per_day"]["value"], pc["grid_speeds"]["value"],
                           -pc["grid_angle_half_width_rad"]["value"],
                           pc["grid_angle_half_width_rad"]["value"], pc["grid_angles"]["value"])
    assert len(vx) == 131072
    sp = np.hypot(vx.astype(np.float64), vy.astype(np.float64))
    assert abs(sp.min() - 92.0) < 1e-3 and abs(sp.max() - 550.0) < 1e-3


def _subpixel_case(seed, T=8, H=40, W=44):
    rng = np.random.default_rng(seed)
    times = np.sort(rng.uniform(0, 0.3, T))
    times[0] = 0.0
    phi = rng.uniform(0.2, 1.0, (T, H, W))
    psi = rng.normal(size=(T, H, W)) * np.sqrt(phi) + 2.0 * phi
    return rng, times, psi, phi


def _clear_of_kinks(times, p, h):
    dts = times - times[0]
    xs, ys = p[0] + p[2] * dts, p[1] + p[3] * dts
    edge = min(np.abs(xs - np.round(xs)).min(), np.abs(ys - np.round(ys)).min())
    return edge > 4 * h * (1 + dts.max())


def test_vjp_params_against_finite_differences_of_L_and_alpha():
    rng, times, psi, phi = _subpixel_case(21)
    keep = np.array([0b11011101], np.uint32)
    h = 1e-4
    checked = 0
    for trial in range(40):
        p = np.concatenate([rng.uniform(8, 30, 2), rng.uniform(-30, 30, 2)])
        if not _clear_of_kinks(times, p, h):
            continue
        gL, gA = rng.normal(size=2)
        g = oracle.traj_vjp(psi, phi, times, keep, *p, gL=gL, gA=gA, images=False)[0]
        fd = np.zeros(4)
        for i in range(4):
            pp, pm = p.copy(), p.copy()
            pp[i] += h
            pm[i] -= h
            Lp, Ap, _ = oracle.traj_eval_subpixel(psi, phi, times, keep, *pp, grad=False)
            Lm, Am, _ = oracle.traj_eval_subpixel(psi, phi, times, keep, *pm, grad=False)
            fd[i] = (gL * (Lp - Lm) + gA * (Ap - Am)) / (2 * h)
        assert np.all(np.abs(g - fd) <= 1e-6 * np.maximum(np.abs(fd), 1.0)), (g, fd)
        checked += 1
    assert checked >= 10


def test_vjp_images_against_finite_differences_and_support():
    rng, times, psi, phi = _subpixel_case(22)
    keep = np.array([0b10111111], np.uint32)
    T, H, W = psi.shape
    p = np.array([15.37, 20.71, 23.3, -17.9])
    gL, gA = 0.7, -1.3
    _, gpsi, gphi = oracle.traj_vjp(psi, phi, times, keep, *p, gL=gL, gA=gA)

    def obj(ps, ph):
        L, A, _ = oracle.traj_eval_subpixel(ps, ph, times, keep, *p, grad=False)
        return gL * L + gA * A

    # every pixel the track's taps touch, plus untouched pixels, which must read zero
    touched = np.argwhere((gpsi != 0) | (gphi != 0))
    assert 0 < len(touched) <= 4 * int(bin(int(keep[0])).count("1"))
    dts = times - times[0]
    for t in range(T):
        inside = (keep[0] >> t) & 1
        n_t = (touched[:, 0] == t).sum()
        assert n_t == (4 if inside else 0)
        if inside:   # the four taps of epoch t surround its position
            x, y = p[0] + p[2] * dts[t], p[1] + p[3] * dts[t]
            ys, xs = touched[touched[:, 0] == t, 1], touched[touched[:, 0] == t, 2]
            assert set(xs) == {math.floor(x), math.floor(x) + 1}
            assert set(ys) == {math.floor(y), math.floor(y) + 1}
    picks = [tuple(r) for r in touched[rng.choice(len(touched), 12, replace=False)]]
    picks += [(1, 2, 3), (5, 39, 43)]
    h = 1e-4
    for (t, y, x) in picks:
        for which, grad in (("psi", gpsi), ("phi", gphi)):
            a, b = psi.copy(), phi.copy()
            c, d = psi.copy(), phi.copy()
            if which == "psi":
                a[t, y, x] += h
                c[t, y, x] -= h
            else:
                b[t, y, x] += h
                d[t, y, x] -= h
            fd = (obj(a, b) - obj(c, d)) / (2 * h)
            assert abs(grad[t, y, x] - fd) <= 1e-6 * max(abs(fd), 1.0), (which, t, y, x)


def test_vjp_adds_to_its_outputs():
    # the VJP adds to the arrays it is given (what a caller summing over candidates relies on):
    # from arrays holding G0 it leaves G0 plus the values it writes into zeroed arrays
    import oracle.oracle as oo
    rng, times, psi, phi = _subpixel_case(23)
    T, H, W = psi.shape
    keep = np.array([0b11011111], np.uint32)
    p = (15.37, 20.71, 23.3, -17.9)
    gp0, gpsi0, gphi0 = oracle.traj_vjp(psi, phi, times, keep, *p, gL=0.7, gA=-1.3)
    g0 = np.array([1.0, -2.0, 3.0, 0.5])
    b_psi, b_phi = 1.0 + rng.random((T, H, W)), -1.0 - rng.random((T, H, W))
    gp, gpsi, gphi = g0.copy(), b_psi.copy(), b_phi.copy()
    psi64, phi64, t64 = (np.ascontiguousarray(a, np.float64) for a in (psi, phi, times))
    rc = oo.lib().kbo_traj_vjp(oo._ptr(psi64), oo._ptr(phi64), oo._ptr(t64), T, H, W,
                               oo._ptr(keep), *[float(v) for v in p], 0.7, -1.3, oo._ptr(gp),
                               oo._ptr(gpsi), oo._ptr(gphi))
    assert rc == 0
    assert np.allclose(gp - g0, gp0, rtol=1e-12, atol=1e-12)
    assert np.allclose(gpsi - b_psi, gpsi0, rtol=0, atol=1e-12)
    assert np.allclose(gphi - b_phi, gphi0, rtol=0, atol=1e-12)
    assert np.abs(gpsi0).max() > 1e-3 and np.abs(gphi0).max() > 1e-3


def test_vjp_euler_homogeneity():
    # L = Psi/sqrt(Phi) is homogeneous of degree 1 in the psi pixels and -1/2 in the phi pixels;
    # alpha = Psi/Phi of degree 1 and -1.  Euler's theorem fixes the pixel-weighted gradient sums.
    rng, times, psi, phi = _subpixel_case(23)
    keep = np.array([0b01111110], np.uint32)
    for trial in range(5):
        p = np.concatenate([rng.uniform(8, 30, 2), rng.uniform(-30, 30, 2)])
        L, A, _ = oracle.traj_eval_subpixel(psi, phi, times, keep, *p, grad=False)
        _, gpsi, gphi = oracle.traj_vjp(psi, phi, times, keep, *p, gL=1.0, gA=0.0)
        assert abs((gpsi * psi).sum() - L) <= 1e-12 * max(abs(L), 1)
        assert abs((gphi * phi).sum() + 0.5 * L) <= 1e-12 * max(abs(L), 1)
        _, gpsi, gphi = oracle.traj_vjp(psi, phi, times, keep, *p, gL=0.0, gA=1.0)
        assert abs((gpsi * psi).sum() - A) <= 1e-12 * max(abs(A), 1)
        assert abs((gphi * phi).sum() + A) <= 1e-12 * max(abs(A), 1)


def test_vjp_off_image_and_empty():
    _, times, psi, phi = _subpixel_case(24)
    keep = np.array([0xFF], np.uint32)
    assert oracle.traj_vjp(psi, phi, times, keep, -500.0, -500.0, 0.0, 0.0) is None
    assert oracle.traj_vjp(psi, phi, times, np.array([0], np.uint32), 10.0, 10.0, 1.0,
                           1.0) is None


def test_adam_first_step_closed_form():
    # After one step the bias-corrected moments are g and g^2, so the move is lr g/(|g| + eps).
    rng, times, psi, phi = _subpixel_case(25)
    keep = np.array([0xFF], np.uint32)
    p = np.array([17.3, 21.9, 11.0, -7.0])
    _, _, g = oracle.traj_eval_subpixel(psi, phi, times, keep, *p)
    lr = np.array([0.1, 0.1, 0.3, 0.3])
    pr, L, A = oracle.refine_adam(psi, phi, times, keep, p, 1, 0.1, 0.3)
    assert np.allclose(pr - p, lr * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    L1, A1, _ = oracle.traj_eval_subpixel(psi, phi, times, keep, *pr, grad=False)
    assert L == L1 and A == A1


def test_adam_refine_converges_on_a_noiseless_off_grid_mover():
    # A noiseless point source with a sub-pixel start and off-grid velocity: ascent from an offset
    # start must raise L to the maximum near the true track (bilinear sampling moves the maximum
    # by a fraction of a pixel) and bring position and velocity close to the truth.
    rng = np.random.default_rng(26)
    T, H, W, k, sig = 12, 64, 96, 9, 1.4
    times = np.sort(rng.uniform(0, 2.0, T))
    times[0] = 0.0
    tru = np.array([20.3, 30.6, 17.37, -4.81])
    img = np.zeros((T, H, W))
    psf = np.stack([gaussian_psf(sig, k, 0, 0)] * T)
    for t in range(T):
        x, y = tru[0] + tru[2] * times[t], tru[1] + tru[3] * times[t]
        ix, iy = math.floor(x + 0.5), math.floor(y + 0.5)
        img[t, iy - 7:iy + 8, ix - 7:ix + 8] += 10.0 * gaussian_psf(sig, 15, x - ix, y - iy)
    psi, phi = oracle.psi_phi(img, np.ones((T, H, W)), None, psf)
    keep = np.array([(1 << T) - 1], np.uint32)
    L_true = oracle.traj_eval_subpixel(psi, phi, times, keep, *tru, grad=False)[0]
    for off in ((0.8, -0.7, 1.0, -0.8), (-0.5, 0.5, -0.8, 0.6), (0.4, 0.9, 0.7, 0.9)):
        p0 = tru + np.array(off)
        L0 = oracle.traj_eval_subpixel(psi, phi, times, keep, *p0, grad=False)[0]
        pr, L, _ = oracle.refine_adam(psi, phi, times, keep, p0, 100, 0.1, 0.2)
        assert L0 < 0.8 * L_true
        assert L >= L_true * (1 - 1e-3)
        err = np.abs(pr - tru)
        assert err[:2].max() < 0.3 and err[2:].max() < 0.3, err


def test_adam_stops_where_phi_vanishes():
    _, times, psi, phi = _subpixel_case(27)
    keep = np.array([0xFF], np.uint32)
    pr, L, A = oracle.refine_adam(psi, phi, times, keep, [-300.0, -300.0, 0.0, 0.0], 5, 0.1, 0.1)
    assert np.isnan(L) and np.isnan(A)
    assert np.array_equal(pr, [-300.0, -300.0, 0.0, 0.0])


# ------------------------------------------------------------------------------------------------
# Central moments of coadded stamps (Section 3.3)
# ------------------------------------------------------------------------------------------------

def test_moments_of_single_pixels_and_their_mixtures():
    r = 10
    side = 2 * r + 1
    rng = np.random.default_rng(71)
    for _ in range(20):
        dx, dy = rng.integers(-r, r + 1, 2)
        s = np.zeros((side, side))
        s[dy + r, dx + r] = rng.uniform(0.5, 3.0)
        m, ok = oracle.stamp_moments(s[None])
        assert np.allclose(m[0, 1:], [dx, dy, dx * dy, dx * dx, dy * dy], atol=1e-12)
        assert ok[0] == (abs(dx) < 0.5 and abs(dy) < 0.5)
    # two lit pixels: moments are the weight-averaged ones
    s = np.zeros((side, side))
    s[r + 2, r - 3] = 1.0          # dx = -3, dy = +2
    s[r - 1, r + 4] = 3.0          # dx = +4, dy = -1
    m, _ = oracle.stamp_moments(s[None])
    w = np.array([0.25, 0.75])
    dxs, dys = np.array([-3, 4]), np.array([2, -1])
    assert np.allclose(m[0], [4.0, w @ dxs, w @ dys, w @ (dxs * dys), w @ dxs ** 2,
                              w @ dys ** 2], atol=1e-12)


def test_moments_of_a_flat_stamp_and_the_paper_limits():
    # a flat stamp with one dark pixel at its centre: every other pixel has weight 1, so
    # xx = sum dx^2 / (side^2 - 1) = side r(r+1)(2r+1)/3 / (side^2 - 1): 36.75 for the paper's
    # 21 x 21 stamps, just above the 36.5 limit (a flat, noise-like stamp is rejected)
    for r in (3, 7, 10):
        side = 2 * r + 1
        s = np.full((1, side, side), 0.37)
        s[0, r, r] = -0.2
        m, ok = oracle.stamp_moments(s)
        xx = side * r * (r + 1) * (2 * r + 1) / 3 / (side * side - 1)
        assert np.allclose(m[0], [(side * side - 1) * 0.57, 0, 0, 0, xx, xx], atol=1e-12)
    assert not ok[0] and abs(m[0, 4] - 16170.0 / 440) < 1e-12
    # a constant offset changes nothing (the weights are taken above the stamp's minimum)
    rng = np.random.default_rng(72)
    s = rng.normal(size=(1, 21, 21))
    m1, ok1 = oracle.stamp_moments(s)
    m2, ok2 = oracle.stamp_moments(s + 7.25)
    assert np.allclose(m1, m2, rtol=1e-9, atol=1e-9) and ok1[0] == ok2[0]
    # flat, empty and all-NaN stamps have no weight and are rejected
    assert not oracle.stamp_moments(np.zeros((1, 21, 21)))[1][0]
    assert not oracle.stamp_moments(np.full((1, 21, 21), -3.0))[1][0]
    assert not oracle.stamp_moments(np.full((1, 21, 21), np.nan))[1][0]
    # NaN pixels are left out of both the minimum and the sums
    s = np.full((1, 21, 21), np.nan)
    s[0, 10, 10] = 2.0
    s[0, 10, 12] = 1.0      # the minimum: weight 0
    m, ok = oracle.stamp_moments(s)
    assert ok[0] and m[0, 0] == 1.0 and np.allclose(m[0, 1:], 0)


def test_moments_of_a_sampled_gaussian():
    r = 10
    u = np.arange(-r, r + 1, dtype=np.float64)
    yy, xx = np.meshgrid(u, u, indexing="ij")
    for cx, cy, sig in ((0.2, -0.3, 1.5), (0.0, 0.0, 2.0), (0.7, 0.1, 1.2), (-2.0, 1.0, 1.4)):
        g = np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * sig ** 2))
        m, ok = oracle.stamp_moments(g[None])
        # a Gaussian well inside the stamp: centroid = centre, second moments = sig^2 + centre^2
        assert np.allclose(m[0, 1:3], [cx, cy], atol=1e-6)
        assert abs(m[0, 3] - cx * cy) < 1e-6
        assert abs(m[0, 4] - (sig ** 2 + cx ** 2)) < 1e-3
        assert abs(m[0, 5] - (sig ** 2 + cy ** 2)) < 1e-3
        assert ok[0] == (abs(cx) < 0.5 and abs(cy) < 0.5)
    # symmetric stamps have zero odd moments
    g = np.exp(-(xx ** 2 + 2 * yy ** 2) / 8.0) + 0.1 * (np.abs(xx) + np.abs(yy))
    m, _ = oracle.stamp_moments(g[None])
    assert np.allclose(m[0, 1:4], 0, atol=1e-12)
    # limits are strict
    s = np.zeros((1, 21, 21))
    s[0, 10, 10] = 1.0
    s[0, 10, 11] = 1.0      # x = 0.5 exactly
    assert not oracle.stamp_moments(s)[1][0]
    assert oracle.stamp_moments(s, limits=(0.5000001, 0.5, 1.5, 36.5, 36.5))[1][0]


def test_moment_filter_limits_apply_each_to_its_own_moment():
    # One lit pixel at (dx, dy) has x = dx, y = dy, xy = dx dy, xx = dx^2, yy = dy^2 exactly.
    # Limits just above those values pass it; a limit equal to its own moment's magnitude rejects
    # it (the bounds are strict and act on |x|, |y|, |xy|), and no other limit does.
    r = 10
    side = 2 * r + 1
    for dx, dy in ((2, -3), (-2, 3)):
        s = np.zeros((1, side, side))
        s[0, dy + r, dx + r] = 1.5
        vals = [abs(dx), abs(dy), abs(dx * dy), dx * dx, dy * dy]
        loose = [v + 1.0 for v in vals]
        assert oracle.stamp_moments(s, limits=tuple(loose))[1][0]
        for i in range(5):
            tight = list(loose)
            tight[i] = float(vals[i])
            assert not oracle.stamp_moments(s, limits=tuple(tight))[1][0], (dx, dy, i)


# ------------------------------------------------------------------------------------------------
# Clustering of candidates (greedy de-duplication, reading of the Fig. 3 step)
# ------------------------------------------------------------------------------------------------

def test_cluster_hand_cases():
    dt, r = 3.0, 4.0
    # identical tracks: the second duplicates the first
    keep, rep = oracle.cluster([10, 10], [20, 20], [100.0, 100.0], [5.0, 5.0], dt, r)
    assert keep.tolist() == [True, False] and rep.tolist() == [0, 0]
    # a chain a - b - c (a~b, b~c, a!~c): greedy keeps a, drops b, keeps c (b was not kept)
    keep, rep = oracle.cluster([0, 3, 6], [0, 0, 0], [10.0, 10.0, 10.0], [0.0, 0.0, 0.0], dt, r)
    assert keep.tolist() == [True, False, True] and rep.tolist() == [0, 0, 2]
    # the same start but velocities 2 px/day apart: 6 px apart at the last epoch -> distinct
    keep, rep = oracle.cluster([5, 5], [5, 5], [100.0, 102.0], [0.0, 0.0], dt, r)
    assert keep.tolist() == [True, True]
    # exactly r apart at both epochs counts as a duplicate (<= r)
    keep, _ = oracle.cluster([0, 4], [0, 0], [1.0, 1.0], [0.0, 0.0], dt, r)
    assert keep.tolist() == [True, False]
    # an invalid entry takes no part: c is compared with a only
    keep, rep = oracle.cluster([0, 3, 6], [0, 0, 0], [10.0] * 3, [0.0] * 3, dt, r,
                               valid=[1, 0, 1])
    assert keep.tolist() == [True, False, True] and rep.tolist() == [0, -1, 2]
    # a placeholder start far outside any image takes no part, even at a duplicate's position
    keep, rep = oracle.cluster([-(1 << 28), -(1 << 28), 5], [-(1 << 28), -(1 << 28), 5],
                               [1.0] * 3, [0.0] * 3, dt, r)
    assert keep.tolist() == [False, False, True] and rep.tolist() == [-1, -1, 2]
    # the representative is the first kept duplicate, not the nearest
    keep, rep = oracle.cluster([0, 6, 3], [0, 0, 0], [0.0] * 3, [0.0] * 3, dt, r)
    assert keep.tolist() == [True, True, False] and rep.tolist() == [0, 1, 0]


def test_cluster_properties_fix_the_greedy_result():
    rng = np.random.default_rng(91)
    dt, r = 3.0, 6.0
    n = 400
    # clusters of near-identical tracks plus scattered ones
    cx = rng.uniform(0, 300, 25)
    cy = rng.uniform(0, 300, 25)
    k = rng.integers(0, 25, n)
    x0 = np.round(cx[k] + rng.normal(0, 2.5, n)).astype(np.int32)
    y0 = np.round(cy[k] + rng.normal(0, 2.5, n)).astype(np.int32)
    vx = (100 + 3 * k + rng.normal(0, 0.8, n)).astype(np.float32)
    vy = (rng.normal(0, 0.8, n)).astype(np.float32)
    valid = rng.random(n) < 0.9
    keep, rep = oracle.cluster(x0, y0, vx, vy, dt, r, valid=valid)

    def dup(i, j):
        d0 = np.hypot(float(x0[i]) - x0[j], float(y0[i]) - y0[j])
        d1 = np.hypot(x0[i] + float(vx[i]) * dt - (x0[j] + float(vx[j]) * dt),
                      y0[i] + float(vy[i]) * dt - (y0[j] + float(vy[j]) * dt))
        return d0 <= r and d1 <= r

    kept = np.nonzero(keep)[0]
    for a in range(len(kept)):               # kept candidates are pairwise distinct
        for b in range(a):
            assert not dup(kept[a], kept[b])
    for i in range(n):
        if not valid[i]:
            assert not keep[i] and rep[i] == -1
        elif keep[i]:
            assert rep[i] == i
        else:                                 # the first kept lower-index duplicate
            firsts = [j for j in range(i) if keep[j] and dup(i, j)]
            assert firsts and rep[i] == firsts[0]
    assert 20 <= keep.sum() < valid.sum()


@pytest.mark.parametrize("name,H,W,window", [("tiny", None, None, (30, 40, 200, 210)),
                                             ("decam", 160, 520, (20, 28, 70, 78))])
def test_window_inputs_equal_whole_image_search(name, H, W, window):
    """oracle.window_inputs (psi/phi on the region a window's tracks reach) gives the results of
    the search of the whole image over that window, bit for bit."""
    from synth import make_stack
    s = make_stack(name, H=H, W=W)
    p = dict(k=3, lh_min=2.0, min_obs=5)
    if name == "decam":
        s.vx, s.vy = s.vx[::64].copy(), s.vy[::64].copy()     # a coarser grid keeps it fast
    psi, phi = oracle.psi_phi(s.img, s.var, s.mask, s.psf)
    whole = oracle.search(psi, phi, s.times, s.vx, s.vy, p, window=window)
    cp, cf, w2, (xa, ya) = oracle.window_inputs(s.img, s.var, s.mask, s.psf, s.times, s.vx, s.vy,
                                                window)
    assert cp.shape[1] < psi.shape[1] or cp.shape[2] < psi.shape[2]
    assert np.array_equal(cp, psi[:, ya:ya + cp.shape[1], xa:xa + cp.shape[2]])
    crop = oracle.search(cp, cf, s.times, s.vx, s.vy, p, window=w2)
    for k in whole:
        assert np.array_equal(whole[k], crop[k]), k
    assert (whole["idx"] >= 0).sum() > 0


def test_stage_counts_against_the_listing_and_a_numpy_count():
    """oracle.stage_counts: with lh_min far below every LH' and K = n_traj, the search lists every
    pair that passes, so the pass count and the n_kept / n_valid sums equal the listing's; the
    count of pairs with n_valid >= min_obs equals a numpy count of in-image epochs with phi > 0."""
    psi, phi, times, vx, vy = _tiny_case(9)
    T, H, W = psi.shape
    n = len(vx)
    for lh_min, min_obs in ((-1e9, 3), (0.8, 4)):
        p = dict(k=n, lh_min=lh_min, min_obs=min_obs)
        sc = oracle.stage_counts(psi, phi, times, vx, vy, p)
        r = oracle.search(psi, phi, times, vx, vy, p)
        f = r["idx"] >= 0
        assert sc[1] == int(f.sum()) > 0
        assert sc[2] == int(r["nkept"][f].sum()) and sc[3] == int(r["nvalid"][f].sum())
        assert sc[2] < sc[3]                    # the clip removes some epochs
        ox, oy = oracle.track_offsets(times, vx, vy)
        valid = 0
        for y in range(H):
            for x in range(W):
                xs, ys = x + ox, y + oy                               # [n][T]
                inside = (xs >= 0) & (xs < W) & (ys >= 0) & (ys < H)
                f_at = np.zeros(xs.shape)
                tt = np.broadcast_to(np.arange(T), xs.shape)
                f_at[inside] = phi[tt[inside], ys[inside], xs[inside]]
                nv = (inside & (f_at > 0)).sum(axis=1)
                valid += int(((nv >= min_obs) & (nv > 0)).sum())
        assert sc[0] == valid
