"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded inputs.

Sizes are chosen so the oracle finishes in seconds while spanning several tiles (the search tile
is 32 x 56 start pixels, psi/phi tiles 32 x 32) and ragged tails.  The decam-sized case runs the
search at full size in the bench's launch configuration and checks sampled windows.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2109_03296_b300 as kb
from helpers import compare_search, gpu_result_numpy, search_ctx
from synth import CONFIGS, make_likelihood_stack, make_stack, search_params_for

pytestmark = pytest.mark.gpu


def _cuda(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _oracle_params(sp):
    return dict(k=sp.k, lh_min=sp.lh_min, min_obs=sp.min_obs, clip=sp.clip, q_lo=sp.q_lo,
                q_mid=sp.q_mid, q_hi=sp.q_hi, n_sigma=sp.n_sigma, clip_on=sp.clip_on)


def _run_both(psi32, phi32, times, vx, vy, sp, window=None, oracle_window=None):
    T, H, W = psi32.shape
    if window is not None:
        sp.window = window
    res = kb.search(_cuda(psi32), _cuda(phi32), times, _cuda(vx), _cuda(vy), sp)
    torch.cuda.synchronize()
    stats = kb.search_stats(res["workspace"])
    assert stats[3] == 0, "device error flags %#x" % stats[3]
    g = gpu_result_numpy(res)
    ow = oracle_window if oracle_window is not None else (window or (0, W, 0, H))
    o = oracle.search(psi32, phi32, times, vx, vy, _oracle_params(sp), window=ow)
    if oracle_window is not None and window != oracle_window:
        x0 = ow[0] - (window or (0, W, 0, H))[0]
        y0 = ow[2] - (window or (0, W, 0, H))[2]
        g = {k: v[y0:y0 + (ow[3] - ow[2]), x0:x0 + (ow[1] - ow[0])] for k, v in g.items()}
    return g, o, stats, search_ctx(psi32, phi32, times, vx, vy, _oracle_params(sp), ow)


# ------------------------------------------------------------------------------------------------
# psi / phi
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("T,H,W,k,mask_frac", [(3, 70, 45, 15, 0.02), (2, 33, 97, 7, 0.0),
                                               (1, 5, 3, 3, 0.1), (2, 40, 40, 1, 0.05)])
def test_psi_phi_parity(cuda_device, T, H, W, k, mask_frac):
    rng = np.random.default_rng(100 + k)
    img = rng.normal(size=(T, H, W)).astype(np.float32)
    var = rng.uniform(0.5, 2.0, (T, H, W)).astype(np.float32)
    mask = (rng.random((T, H, W)) < mask_frac).astype(np.uint8)
    var[0, 0, 0] = np.inf
    img[-1, H // 2, W // 2] = np.nan
    psf = rng.uniform(0.0, 1.0, (T, k, k)).astype(np.float32)
    psf /= psf.sum(axis=(1, 2), keepdims=True)
    psi_g, phi_g = kb.make_psi_phi(_cuda(img), _cuda(var), _cuda(mask), _cuda(psf))
    psi_o, phi_o = oracle.psi_phi(img, var, mask, psf)
    psi_g, phi_g = psi_g.cpu().numpy(), phi_g.cpu().numpy()
    masked = (mask > 0) | ~np.isfinite(var) | ~np.isfinite(img) | (var <= 0)
    assert (psi_g[masked] == 0).all() and (phi_g[masked] == 0).all()
    scale_psi = np.sqrt(np.maximum(phi_o, 1e-30))   # psi ~ N(0, phi) for unit-variance noise
    assert np.all(np.abs(psi_g - psi_o) <= 1e-5 * (np.abs(psi_o) + scale_psi) + 1e-12)
    assert np.all(np.abs(phi_g - phi_o) <= 1e-5 * np.abs(phi_o) + 1e-12)
    assert ((phi_g > 0) == (phi_o > 0)).all()


def test_psi_phi_full_size_sampled(cuda_device):
    s = make_stack("decam")
    img, var, mask, psf = _cuda(s.img), _cuda(s.var), _cuda(s.mask), _cuda(s.psf)
    psi_g, phi_g = kb.make_psi_phi(img, var, mask, psf)
    rng = np.random.default_rng(7)
    T, H, W = s.img.shape
    n = 4000
    tyx = np.stack([rng.integers(0, T, n), rng.integers(0, H, n), rng.integers(0, W, n)], 1)
    tyx[:50, 1] = rng.integers(0, 8, 50)                 # borders
    tyx[50:100, 2] = W - 1 - rng.integers(0, 8, 50)
    ps_o, ph_o = oracle.psi_phi_at(s.img, s.var, s.mask, s.psf, tyx)
    t, y, x = (torch.from_numpy(tyx[:, i]).cuda().long() for i in range(3))
    ps_g = psi_g[t, y, x].cpu().numpy()
    ph_g = phi_g[t, y, x].cpu().numpy()
    assert np.all(np.abs(ps_g - ps_o) <= 1e-5 * (np.abs(ps_o) + np.sqrt(np.maximum(ph_o, 1e-30))))
    assert np.all(np.abs(ph_g - ph_o) <= 1e-5 * np.abs(ph_o) + 1e-12)


# ------------------------------------------------------------------------------------------------
# search
# ------------------------------------------------------------------------------------------------

def test_search_parity_tiny_pipeline(cuda_device):
    """The tiny workload end to end: oracle psi/phi (rounded to float32) feed both searches."""
    s = make_stack("tiny")
    psi, phi = oracle.psi_phi(s.img, s.var, s.mask, s.psf)
    psi32, phi32 = psi.astype(np.float32), phi.astype(np.float32)
    c = CONFIGS["tiny"]
    sp = kb.SearchParams(k=c["K"], lh_min=c["lh_min"], min_obs=c["min_obs"])
    g, o, stats, ctx = _run_both(psi32, phi32, s.times, s.vx, s.vy, sp)
    compare_search(g, o, sp.lh_min, ctx=ctx)
    assert stats[0] == 256 * 256 * 128 * 10
    # recovery: at each injected mover's start pixel the best trajectory follows the injected
    # track to within 2 px at every epoch (neighbouring grid velocities differ by < 3 px over the
    # 0.2-day span, so noise may pick either), with LH' near SNR sqrt(T)
    ox, oy = oracle.track_offsets(s.times, s.vx, s.vy)
    for i in range(len(s.movers["x0"])):
        x0, y0, j = int(s.movers["x0"][i]), int(s.movers["y0"][i]), int(s.movers["grid_idx"][i])
        got = g["idx"][y0, x0, 0]
        assert got >= 0
        assert np.abs(ox[got] - ox[j]).max() <= 2 and np.abs(oy[got] - oy[j]).max() <= 2
        assert 0.6 * 5.0 * math.sqrt(10) < g["lh"][y0, x0, 0] < 5.0 * math.sqrt(10) + 4.0


def _likelihood_case(seed, T, H, W, n_traj, mask_frac=0.05, spread=40.0, dup=True):
    rng = np.random.default_rng(seed)
    times = np.sort(rng.uniform(0, 1.0, T))
    times[0] = 0.0
    phi = rng.uniform(0.2, 1.5, (T, H, W))
    psi = rng.normal(size=(T, H, W)) * np.sqrt(phi)
    psi += 3.0 * phi * (rng.random((T, H, W)) < 0.05)
    m = rng.random((T, H, W)) < mask_frac
    psi[m] = 0.0
    phi[m] = 0.0
    vx = rng.uniform(-spread, spread, n_traj).astype(np.float32)
    vy = rng.uniform(-spread, spread, n_traj).astype(np.float32)
    if dup:
        vx[7], vy[7] = vx[2], vy[2]
        vx[n_traj - 1], vy[n_traj - 1] = vx[0], vy[0]
    return psi.astype(np.float32), phi.astype(np.float32), times, vx, vy


@pytest.mark.parametrize("seed,T,H,W,n_traj,K,lh,min_obs,clip,clip_on,window", [
    (1, 13, 101, 77, 70, 4, 1.5, 3, 1, 0, None),            # ragged tiles, many candidates
    (2, 6, 70, 130, 33, 32, -1e9, 1, 1, 0, None),          # every pair enters: K=32 lists
    (3, 40, 65, 40, 50, 3, 2.0, 10, 1, 1, None),           # two epochs per lane, likelihood clip
    (4, 100, 40, 36, 24, 2, 2.0, 30, 1, 0, None),          # four epochs per lane
    (5, 9, 90, 90, 40, 5, 1.0, 2, 0, 0, (3, 70, 5, 83)),   # clip off, window with x_lo % 4 != 0
    (6, 1, 20, 20, 5, 2, 0.5, 1, 1, 0, None),              # a single epoch
    (7, 17, 64, 32, 1, 1, 1.0, 5, 1, 0, None),             # a single trajectory, exact tile
    (8, 128, 24, 36, 16, 2, 2.0, 40, 1, 0, None),          # T = KB_MAX_T: four full mask words
])
def test_search_parity_cases(cuda_device, seed, T, H, W, n_traj, K, lh, min_obs, clip, clip_on,
                             window):
    psi, phi, times, vx, vy = _likelihood_case(seed, T, H, W, n_traj, dup=n_traj > 8)
    sp = kb.SearchParams(k=K, lh_min=lh, min_obs=min_obs, clip=clip, clip_on=clip_on)
    g, o, stats, ctx = _run_both(psi, phi, times, vx, vy, sp, window=window)
    compare_search(g, o, lh, ctx=ctx)


# The paper leaves the quantile pair and the width "user-determinable" (Section 3.1, after
# Eq. 5); the kernel forms the interpolation rank (n - 1) q in float64 like the oracle, so kept
# masks agree except where an epoch sits within rounding of a clip bound (reading R6, counted).
_QUANTILE_CASES = [
    # seed, T, (q_lo, q_mid, q_hi), n_sigma, clip_on
    (31, 26, (0.10, 0.50, 0.90), 1.5, 0),    # thread per pair, flux lightcurve
    (32, 26, (0.10, 0.50, 0.90), 1.5, 1),    # thread per pair, likelihood lightcurve
    (33, 13, (0.20, 0.45, 0.80), 2.5, 0),    # 16-wide sorting network
    (34, 29, (0.20, 0.45, 0.80), 2.5, 1),
    (35, 45, (0.10, 0.50, 0.90), 1.5, 0),    # warp per pair, two epochs per lane
    (36, 45, (0.10, 0.50, 0.90), 1.5, 1),
    (37, 45, (0.20, 0.45, 0.80), 2.5, 0),
    (38, 100, (0.20, 0.45, 0.80), 2.5, 1),   # four epochs per lane
]


@pytest.mark.parametrize("seed,T,q,n_sigma,clip_on", _QUANTILE_CASES)
def test_search_parity_quantiles(cuda_device, seed, T, q, n_sigma, clip_on):
    H, W = (70, 60) if T <= 45 else (40, 36)
    psi, phi, times, vx, vy = _likelihood_case(seed, T, H, W, 48)
    sp = kb.SearchParams(k=4, lh_min=1.0, min_obs=max(3, T // 4), q_lo=q[0], q_mid=q[1],
                         q_hi=q[2], n_sigma=n_sigma, clip_on=clip_on)
    g, o, stats, ctx = _run_both(psi, phi, times, vx, vy, sp)
    counts = {}
    compare_search(g, o, sp.lh_min, ctx=ctx, counts=counts)
    # the clip is doing work: some kept mask is not the full valid set
    f = o["idx"] >= 0
    assert int(f.sum()) > 100
    assert (o["nkept"][f] < o["nvalid"][f]).any()
    print("ambiguous pixels:", counts)


@pytest.mark.parametrize("seed,T,H,W,n_traj,K,lh,min_obs,clip_on", [
    (21, 13, 101, 77, 70, 4, 1.5, 3, 0),     # ragged tiles, many candidates
    (22, 26, 90, 64, 96, 8, 3.0, 10, 0),     # the decam epoch count, K = 8
    (23, 40, 65, 40, 50, 3, 2.0, 10, 1),     # warp-per-pair evaluation, likelihood clip
])
def test_search_bound_rows_equivalent(cuda_device, seed, T, H, W, n_traj, K, lh, min_obs,
                                      clip_on):
    """The pruning bound per start pixel (bound_rows=1) and per block of two rows
    (bound_rows=2) are both exact: the oracle's results, and bit-identical to each other."""
    psi, phi, times, vx, vy = _likelihood_case(seed, T, H, W, n_traj)
    sp = kb.SearchParams(k=K, lh_min=lh, min_obs=min_obs, clip_on=clip_on, bound_rows=1)
    g1, o, _, ctx = _run_both(psi, phi, times, vx, vy, sp)
    compare_search(g1, o, lh, ctx=ctx)
    sp2 = kb.SearchParams(k=K, lh_min=lh, min_obs=min_obs, clip_on=clip_on, bound_rows=2)
    res = kb.search(_cuda(psi), _cuda(phi), times, _cuda(vx), _cuda(vy), sp2)
    torch.cuda.synchronize()
    assert kb.search_stats(res["workspace"])[3] == 0
    g2 = gpu_result_numpy(res)
    for key in g1:
        assert np.array_equal(g1[key], g2[key], equal_nan=True), key
    assert int((g1["idx"] >= 0).sum()) > 0


@pytest.mark.parametrize("lh_min,K,n_traj", [(-1e9, 32, 30), (1.5, 32, 30), (1.5, 4, 40)])
def test_search_stage_counts(cuda_device, lh_min, K, n_traj):
    """kb_search_stage_counts against the oracle's counts over every pair (Fig. 3's stages).
    With fewer trajectories than K no list can fill, so the admission threshold stays at lh_min:
    with lh_min <= 0 every pair is evaluated and all four counts are exhaustive; with lh_min > 0
    every pair that reaches lh_min is evaluated, so the pass count and the kept / valid sums are
    exhaustive (the n_valid count covers the evaluated pairs only).  Once lists fill (K = 4) the
    threshold rises to the K-th LH', and the counts cover only the pairs evaluated."""
    psi, phi, times, vx, vy = _likelihood_case(41, 13, 70, 60, n_traj)
    sp = kb.SearchParams(k=K, lh_min=lh_min, min_obs=3)
    res = kb.search(_cuda(psi), _cuda(phi), times, _cuda(vx), _cuda(vy), sp)
    torch.cuda.synchronize()
    stats = kb.search_stats(res["workspace"])
    assert stats[3] == 0
    sc = kb.search_stage_counts(res["workspace"])
    o = oracle.stage_counts(psi, phi, times, vx, vy, _oracle_params(sp))
    assert o[1] > 0 and o[2] < o[3]
    if K < n_traj:
        assert all(a <= b for a, b in zip(sc, o)) and 0 < sc[1] <= o[1]
    elif lh_min <= 0:
        assert sc == o and stats[1] == 70 * 60 * n_traj
    else:
        assert sc[1:] == o[1:] and sc[0] <= o[0] and stats[1] < 70 * 60 * n_traj


@pytest.mark.parametrize("bound_rows", [1, 2])
def test_search_fast_movers_fallback(cuda_device, bound_rows):
    """Velocities spread so widely that the staged rectangle overflows: the direct-load path,
    with single-row sums and with two-row blocks."""
    psi, phi, times, vx, vy = _likelihood_case(11, 8, 80, 90, 48, spread=400.0)
    sp = kb.SearchParams(k=3, lh_min=1.0, min_obs=2, bound_rows=bound_rows)
    g, o, _, ctx = _run_both(psi, phi, times, vx, vy, sp)
    compare_search(g, o, 1.0, ctx=ctx)


def test_search_non_finite_and_negative_planes(cuda_device):
    """psi/phi planes given directly with NaN, +-inf and non-positive values: an epoch is valid
    only where phi > 0 and both are finite, on both sides (the bound counts nothing there)."""
    psi, phi, times, vx, vy = _likelihood_case(13, 12, 60, 75, 40)
    rng = np.random.default_rng(13)
    T, H, W = psi.shape
    for value, frac, plane in ((np.nan, 0.01, psi), (np.inf, 0.005, psi), (-np.inf, 0.005, psi),
                               (np.nan, 0.01, phi), (np.inf, 0.005, phi), (-1.0, 0.01, phi),
                               (0.0, 0.01, phi)):
        plane[rng.random((T, H, W)) < frac] = value
    sp = kb.SearchParams(k=4, lh_min=1.5, min_obs=3)
    g, o, stats, ctx = _run_both(psi, phi, times, vx, vy, sp)
    compare_search(g, o, 1.5, ctx=ctx)
    assert int((g["idx"] >= 0).sum()) > 0


def test_search_degenerate(cuda_device):
    psi, phi, times, vx, vy = _likelihood_case(12, 5, 40, 40, 16)
    # min_obs above T: nothing can be selected
    sp = kb.SearchParams(k=2, lh_min=-1e9, min_obs=6)
    r = kb.search(_cuda(psi), _cuda(phi), times, _cuda(vx), _cuda(vy), sp)
    assert (r["idx"] < 0).all() and torch.isneginf(r["lh"]).all()
    # every pixel masked: no valid epoch anywhere
    z = np.zeros_like(psi)
    r = kb.search(_cuda(z), _cuda(z), times, _cuda(vx), _cuda(vy), kb.SearchParams(k=1, lh_min=-1e9,
                                                                                min_obs=0))
    assert (r["idx"] < 0).all()
    # a one-pixel window
    sp = kb.SearchParams(k=3, lh_min=-1e9, min_obs=1, window=(17, 18, 30, 31))
    g, o, _, ctx = _run_both(psi, phi, times, vx, vy, sp, window=(17, 18, 30, 31))
    compare_search(g, o, -1e9, ctx=ctx)


def test_search_parity_decam_full_size(cuda_device):
    """Full 2046 x 4094, T=26, 32768-trajectory search (the bench's launch); oracle on windows
    around injected movers and at a corner."""
    name = "decam"
    psi, phi, times, vx, vy, movers = make_likelihood_stack(name)
    c = CONFIGS[name]
    sp = kb.SearchParams(k=c["K"], lh_min=c["lh_min"], min_obs=c["min_obs"])
    T, H, W = psi.shape
    res = kb.search(_cuda(psi), _cuda(phi), times, _cuda(vx), _cuda(vy), sp)
    torch.cuda.synchronize()
    stats = kb.search_stats(res["workspace"])
    assert stats[3] == 0
    g_all = gpu_result_numpy(res)
    del res
    torch.cuda.empty_cache()
    # windows: around three bright movers, plus the image corner
    order = np.argsort(-movers["snr"])
    wins = []
    for i in order[:3]:
        x0, y0 = int(movers["x0"][i]), int(movers["y0"][i])
        x0 = min(max(x0 - 6, 0), W - 12)
        y0 = min(max(y0 - 6, 0), H - 12)
        wins.append((x0, x0 + 12, y0, y0 + 12))
    wins.append((W - 10, W, H - 10, H))
    filled = 0
    for (xa, xb, ya, yb) in wins:
        o = oracle.search(psi, phi, times, vx, vy, _oracle_params(sp), window=(xa, xb, ya, yb))
        g = {k: v[ya:yb, xa:xb] for k, v in g_all.items()}
        compare_search(g, o, sp.lh_min,
                       ctx=search_ctx(psi, phi, times, vx, vy, _oracle_params(sp),
                                      (xa, xb, ya, yb)))
        filled += int((o["idx"] >= 0).sum())
    assert filled > 0


def test_search_parity_bench_stack(cuda_device):
    """The bench's own input: make_stack("decam") with the seed the bench times.  psi/phi are
    formed by the oracle at full size (the kernel's psi/phi of the same images are checked
    against them element by element), rounded to float32 and searched at full size in the
    bench's launch configuration; the oracle checks windows around the three brightest movers,
    a hot window at a mover's earliest +20 sigma spike (nearly every trajectory of a start pixel
    there passes the pruning bound and is evaluated in full), and a corner."""
    name = "decam"
    s = make_stack(name)
    c = CONFIGS[name]
    psi_o, phi_o = oracle.psi_phi(s.img, s.var, s.mask, s.psf)
    psi_g, phi_g = kb.make_psi_phi(_cuda(s.img), _cuda(s.var), _cuda(s.mask), _cuda(s.psf))
    for got, ref, is_psi in ((psi_g, psi_o, True), (phi_g, phi_o, False)):
        gt = got.cpu().numpy()
        tol = 1e-5 * (np.abs(ref) + np.sqrt(np.maximum(phi_o, 1e-30))) if is_psi else \
            1e-5 * np.abs(ref) + 1e-12
        assert np.all(np.abs(gt - ref) <= tol)
        del gt
    del psi_g, phi_g
    psi = psi_o.astype(np.float32)
    phi = phi_o.astype(np.float32)
    del psi_o, phi_o
    sp = kb.SearchParams(k=c["K"], lh_min=c["lh_min"], min_obs=c["min_obs"])
    T, H, W = psi.shape
    res = kb.search(_cuda(psi), _cuda(phi), s.times, _cuda(s.vx), _cuda(s.vy), sp)
    torch.cuda.synchronize()
    stats = kb.search_stats(res["workspace"])
    assert stats[3] == 0
    g_all = gpu_result_numpy(res)
    del res
    torch.cuda.empty_cache()
    psi64, phi64 = psi.astype(np.float64), phi.astype(np.float64)
    del psi, phi
    mv = s.movers
    wins = []
    for i in np.argsort(-mv["snr"])[:3]:
        x0 = min(max(int(mv["x0"][i]) - 6, 0), W - 12)
        y0 = min(max(int(mv["y0"][i]) - 6, 0), H - 12)
        wins.append((x0, x0 + 12, y0, y0 + 12))
    first = np.where(mv["spike"].any(axis=1), mv["spike"].argmax(axis=1), T)
    i = int(np.argmin(first))
    dt = s.times[first[i]] - s.times[0]
    xs, ys = int(mv["x0"][i] + mv["vx"][i] * dt), int(mv["y0"][i] + mv["vy"][i] * dt)
    x0, y0 = min(max(xs - 5, 0), W - 10), min(max(ys - 5, 0), H - 10)
    wins.append((x0, x0 + 10, y0, y0 + 10))
    wins.append((0, 10, H - 10, H))
    p = _oracle_params(sp)
    filled = 0
    for (xa, xb, ya, yb) in wins:
        o = oracle.search(psi64, phi64, s.times, s.vx, s.vy, p, window=(xa, xb, ya, yb))
        g = {k: v[ya:yb, xa:xb] for k, v in g_all.items()}
        compare_search(g, o, sp.lh_min,
                       ctx=search_ctx(psi64, phi64, s.times, s.vx, s.vy, p, (xa, xb, ya, yb)))
        filled += int((o["idx"] >= 0).sum())
    assert filled > 0


def test_search_parity_full_config_grid(cuda_device):
    """The full-scale configuration's shape -- T = 100 over five nights (warp-per-pair
    evaluation, four epochs per lane), the paper's 512 x 256 velocity grid (131072 trajectories,
    92-550 px/day, +-pi/10), 1% masked pixels, min_obs 50 -- on a 384 x 2560 image (wide
    enough that movers stay in it for most of the 4 days); the oracle on windows around the
    brightest movers that start in the left third, and at a corner."""
    name = "full"
    psi, phi, times, vx, vy, movers = make_likelihood_stack(name, H=384, W=2560, n_movers=60)
    c = CONFIGS[name]
    sp = kb.SearchParams(k=c["K"], lh_min=c["lh_min"], min_obs=c["min_obs"])
    T, H, W = psi.shape
    assert T == 100 and len(vx) == 131072
    res = kb.search(_cuda(psi), _cuda(phi), times, _cuda(vx), _cuda(vy), sp)
    torch.cuda.synchronize()
    assert kb.search_stats(res["workspace"])[3] == 0
    g_all = gpu_result_numpy(res)
    del res
    torch.cuda.empty_cache()
    inside = (movers["x0"] > 8) & (movers["x0"] < W // 3) & (movers["y0"] > 8) & \
        (movers["y0"] < H - 8)
    order = [i for i in np.argsort(-movers["snr"]) if inside[i]]
    wins = []
    for i in order[:2]:
        x0, y0 = int(movers["x0"][i]), int(movers["y0"][i])
        wins.append((x0 - 3, x0 + 3, y0 - 3, y0 + 3))
    wins.append((0, 5, H - 5, H))
    filled = 0
    for (xa, xb, ya, yb) in wins:
        o = oracle.search(psi, phi, times, vx, vy, _oracle_params(sp), window=(xa, xb, ya, yb))
        g = {k: v[ya:yb, xa:xb] for k, v in g_all.items()}
        compare_search(g, o, sp.lh_min,
                       ctx=search_ctx(psi, phi, times, vx, vy, _oracle_params(sp),
                                      (xa, xb, ya, yb)))
        filled += int((o["idx"] >= 0).sum())
    assert filled > 0


def test_search_parity_full_config_stated_size(cuda_device):
    """The full-scale configuration at its stated size: T = 100 over five nights, 4096 x 4096,
    the paper's 512 x 256 grid of 131072 trajectories (Section 4.1), drawn on the device as the
    bench draws it.  The kernel forms psi/phi; over the region each checked window's tracks can
    reach, those planes are replaced by the oracle's psi/phi of the same images (rounded to
    float32), so both sides search identical values there.  The whole image is searched in the
    bench's launch configuration and the oracle checks a window at the brightest mover's start
    and one at a corner."""
    from synth.gpu_stacks import make_config_stack_torch
    name = "full"
    c = CONFIGS[name]
    g = make_config_stack_torch(name, torch.device("cuda"))
    psi, phi = kb.make_psi_phi(g["img"], g["var"], g["mask"], g["psf"])
    T, H, W = psi.shape
    assert (T, H, W) == (100, 4096, 4096) and g["vx"].numel() == 131072
    img, var, mask = g["img"].cpu().numpy(), g["var"].cpu().numpy(), g["mask"].cpu().numpy()
    psf = g["psf"].cpu().numpy()
    vx, vy = g["vx"].cpu().numpy(), g["vy"].cpu().numpy()
    times = g["times"]
    mv = g["movers"]
    del g
    sp = kb.SearchParams(k=c["K"], lh_min=c["lh_min"], min_obs=c["min_obs"])
    p = _oracle_params(sp)
    span = times[-1] - times[0]
    xe, ye = mv["x0"] + mv["vx"] * span, mv["y0"] + mv["vy"] * span
    inside = (mv["x0"] > 4) & (mv["x0"] < W - 4) & (mv["y0"] > 4) & (mv["y0"] < H - 4) & \
        (xe > 4) & (xe < W - 4) & (ye > 4) & (ye < H - 4)     # on the image at every epoch
    i = int(np.argmax(np.where(inside, mv["snr"], -1.0)))
    x0, y0 = int(mv["x0"][i]), int(mv["y0"][i])
    wins = [(x0 - 1, x0 + 2, y0 - 1, y0 + 2), (0, 3, H - 3, H)]
    crops = []
    for w in wins:
        cp, cf, wc, (xa, ya) = oracle.window_inputs(img, var, mask, psf, times, vx, vy, w)
        cp32, cf32 = cp.astype(np.float32), cf.astype(np.float32)
        hh, ww = cp.shape[1], cp.shape[2]
        psi[:, ya:ya + hh, xa:xa + ww] = torch.from_numpy(cp32).cuda()
        phi[:, ya:ya + hh, xa:xa + ww] = torch.from_numpy(cf32).cuda()
        crops.append((cp32.astype(np.float64), cf32.astype(np.float64), wc, w))
    del img, var, mask
    res = kb.search(psi, phi, times, torch.from_numpy(vx).cuda(), torch.from_numpy(vy).cuda(), sp)
    torch.cuda.synchronize()
    assert kb.search_stats(res["workspace"])[3] == 0
    g_all = gpu_result_numpy(res)
    del res, psi, phi
    torch.cuda.empty_cache()
    filled = 0
    for cp, cf, wc, (xa, xb, ya, yb) in crops:
        o = oracle.search(cp, cf, times, vx, vy, p, window=wc)
        g_w = {k: v[ya:yb, xa:xb] for k, v in g_all.items()}
        compare_search(g_w, o, sp.lh_min, ctx=search_ctx(cp, cf, times, vx, vy, p, wc))
        filled += int((o["idx"] >= 0).sum())
    assert filled > 0     # the brightest mover is found at its start


# ------------------------------------------------------------------------------------------------
# stamps and the handoff
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("T,radius,with_keep", [(10, 10, False), (37, 4, True), (100, 2, False)])
def test_stamps_parity(cuda_device, T, radius, with_keep):
    rng = np.random.default_rng(T)
    H, W = 60, 70
    img = rng.normal(size=(T, H, W)).astype(np.float32)
    var = rng.uniform(0.5, 2, (T, H, W)).astype(np.float32)
    mask = (rng.random((T, H, W)) < 0.05).astype(np.uint8)
    times = np.sort(rng.uniform(0, 0.5, T))
    n = 40
    x0 = rng.integers(-5, W + 5, n).astype(np.int32)
    y0 = rng.integers(-5, H + 5, n).astype(np.int32)
    vx = rng.uniform(-60, 60, n).astype(np.float32)
    vy = rng.uniform(-60, 60, n).astype(np.float32)
    mw = (T + 31) // 32
    keep = rng.integers(0, 2 ** 32, (n, mw), dtype=np.uint64).astype(np.uint32) if with_keep else None
    mean_g, med_g = kb.stamps(_cuda(img), _cuda(var), _cuda(mask), times, _cuda(x0), _cuda(y0),
                              _cuda(vx), _cuda(vy), radius=radius,
                              keep_mask=None if keep is None else _cuda(keep.view(np.int32)))
    mean_o, med_o = oracle.stamps(img, var, mask, times, x0, y0, vx, vy, radius=radius,
                                  keep_mask=keep)
    mean_g, med_g = mean_g.cpu().numpy(), med_g.cpu().numpy()
    assert np.array_equal(np.isnan(mean_g), np.isnan(mean_o))
    ok = ~np.isnan(mean_o)
    assert np.all(np.abs(mean_g[ok] - mean_o[ok]) <= 1e-5 * (1 + np.abs(mean_o[ok])))
    assert np.all(np.abs(med_g[ok] - med_o[ok]) <= 1e-6 * (1 + np.abs(med_o[ok])))


def test_collect_orders_survivors(cuda_device):
    psi, phi, times, vx, vy = _likelihood_case(21, 8, 70, 66, 40)
    sp = kb.SearchParams(k=4, lh_min=1.0, min_obs=2)
    res = kb.search(_cuda(psi), _cuda(phi), times, _cuda(vx), _cuda(vy), sp)
    lh = res["lh"].cpu().numpy().reshape(-1, 4)
    idx = res["idx"].cpu().numpy().reshape(-1, 4)
    filled = np.nonzero(idx.ravel() >= 0)[0]
    keys = sorted(filled, key=lambda p: (-lh.ravel()[p], p))
    for n_max in (1, 7, 300, len(filled), len(filled) + 50):
        pix, slot, count = kb.collect(res, n_max)
        pix, slot = pix.cpu().numpy(), slot.cpu().numpy()
        assert int(count.item()) == len(filled)
        got = [p * 4 + s for p, s in zip(pix, slot) if p >= 0]
        assert got == [int(k) for k in keys[:n_max]]
        assert (pix[min(n_max, len(filled)):] == -1).all()
