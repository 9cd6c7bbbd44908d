"""Seeded synthetic difference-image stacks.

Workloads (sizes from the paper: 2K x 4K DECam CCDs, Section 2.1; 5-25 pointings over nearly
consecutive nights, ~5 per night; the 92-550 px/day x +-pi/10 velocity grid of 512 x 256,
Section 4.1).  The DECam NEO data are not available, so these stand in for them:

  tiny      T=10, 256x256, N(0,1), var 1, Gaussian PSF sigma 1.4 on 7x7, 3 movers at per-epoch
            SNR 5 on integer pixel tracks, grid 16 speeds 50-400 px/day x 8 angles +-0.2 rad.
  decam     T=26 over 4 nights (7,7,6,6 epochs, 20 min cadence), 2046x4094, var_t U[0.5,2],
            0.5% pixels masked, PSF sigma_t U[1,2] on 15x15, 200 movers SNR log-U[1.5,10] with
            10% of each mover's epochs replaced by +20 sigma spikes; grid 256 x 128
            (90-500 px/day, +-0.3 rad).
  full      T=100 over 5 nights, 4096x4096, var_t U[0.5,2], 1% masked, PSF sigma_t U[1,2.5] on
            15x15, 1000 movers SNR U[1,8]; grid 512 x 256 (92-550 px/day, +-pi/10).
  refine    the tiny stack with movers at off-grid sub-pixel starts and velocities.
  decam_refine  the decam recipe (own seed) with movers at sub-pixel starts and off-grid
            velocities, uniform between grid points: the workload of the off-grid refinement.
  decam_refine_half  the same at 2046x2048 with 100 movers (detailed refine profiles).
  decam_small  the decam recipe on 1024x1024 with 50 movers (psi+phi 218 MB, above the 126 MB
            L2).
  decam_half   the decam recipe on 2046x2048 with 100 movers (same mover density; psi+phi
            0.87 GB): the size used for detailed kernel profiles, with ~15 tiles per SM.

A mover of per-epoch matched-filter SNR s has flux F_t = s sqrt(var_t) / sqrt(sum P_t^2) and is
drawn as F_t times the PSF centred on its position (integer positions for 'tiny', exact
sub-pixel positions otherwise).  Masked pixels carry var = inf and mask = 1.
"""
import math
from dataclasses import dataclass, field

import numpy as np

__all__ = ["Stack", "velocity_grid", "gaussian_psf", "make_stack", "make_likelihood_stack",
           "CONFIGS", "search_params_for"]


@dataclass
class Stack:
    img: np.ndarray          # float32 [T][H][W]
    var: np.ndarray          # float32 [T][H][W]
    mask: np.ndarray         # uint8 [T][H][W] or None
    psf: np.ndarray          # float32 [T][k][k], sums to 1
    times: np.ndarray        # float64 [T] (days), ascending
    vx: np.ndarray           # float32 [n_traj]
    vy: np.ndarray           # float32 [n_traj]
    movers: dict = field(default_factory=dict)  # x0, y0, vx, vy, snr, flux [n][T], grid_idx
    name: str = ""


CONFIGS = {
    "tiny": dict(T=10, H=256, W=256, psf_k=7, psf_sigma=(1.4, 1.4), var=(1.0, 1.0),
                 mask_frac=0.0, n_movers=3, snr=("const", 5.0), spike_frac=0.0,
                 grid=(50.0, 400.0, 16, -0.2, 0.2, 8), times="uniform0.2",
                 integer_tracks=True, movers_on_grid=True, start_margin=28, seed=0,
                 K=1, lh_min=7.0, min_obs=5),
    "decam": dict(T=26, H=2046, W=4094, psf_k=15, psf_sigma=(1.0, 2.0), var=(0.5, 2.0),
                  mask_frac=0.005, n_movers=200, snr=("loguniform", 1.5, 10.0),
                  spike_frac=0.1, grid=(90.0, 500.0, 256, -0.3, 0.3, 128),
                  times=("nights", (7, 7, 6, 6)), integer_tracks=False, movers_on_grid=False,
                  start_margin=0, seed=1, K=8, lh_min=10.0, min_obs=15),
    "decam_small": dict(T=26, H=1024, W=1024, psf_k=15, psf_sigma=(1.0, 2.0), var=(0.5, 2.0),
                        mask_frac=0.005, n_movers=50, snr=("loguniform", 1.5, 10.0),
                        spike_frac=0.1, grid=(90.0, 500.0, 256, -0.3, 0.3, 128),
                        times=("nights", (7, 7, 6, 6)), integer_tracks=False,
                        movers_on_grid=False, start_margin=0, seed=5, K=8, lh_min=10.0,
                        min_obs=15),
    "decam_half": dict(T=26, H=2046, W=2048, psf_k=15, psf_sigma=(1.0, 2.0), var=(0.5, 2.0),
                       mask_frac=0.005, n_movers=100, snr=("loguniform", 1.5, 10.0),
                       spike_frac=0.1, grid=(90.0, 500.0, 256, -0.3, 0.3, 128),
                       times=("nights", (7, 7, 6, 6)), integer_tracks=False,
                       movers_on_grid=False, start_margin=0, seed=6, K=8, lh_min=10.0,
                       min_obs=15),
    "full": dict(T=100, H=4096, W=4096, psf_k=15, psf_sigma=(1.0, 2.5), var=(0.5, 2.0),
                 mask_frac=0.01, n_movers=1000, snr=("uniform", 1.0, 8.0), spike_frac=0.0,
                 grid=(92.0, 550.0, 512, -math.pi / 10, math.pi / 10, 256),
                 times=("nights", (20, 20, 20, 20, 20)), integer_tracks=False,
                 movers_on_grid=False, start_margin=0, seed=4, K=8, lh_min=10.0, min_obs=50),
    "refine": dict(T=10, H=256, W=256, psf_k=7, psf_sigma=(1.4, 1.4), var=(1.0, 1.0),
                   mask_frac=0.0, n_movers=3, snr=("const", 5.0), spike_frac=0.0,
                   grid=(50.0, 400.0, 16, -0.2, 0.2, 8), times="uniform0.2",
                   integer_tracks=False, movers_on_grid=False, start_margin=28, seed=3,
                   K=1, lh_min=7.0, min_obs=5, subpixel_starts=True),
    "decam_refine": dict(T=26, H=2046, W=4094, psf_k=15, psf_sigma=(1.0, 2.0), var=(0.5, 2.0),
                         mask_frac=0.005, n_movers=200, snr=("loguniform", 1.5, 10.0),
                         spike_frac=0.1, grid=(90.0, 500.0, 256, -0.3, 0.3, 128),
                         times=("nights", (7, 7, 6, 6)), integer_tracks=False,
                         movers_on_grid=False, start_margin=0, seed=7, K=8, lh_min=10.0,
                         min_obs=15, subpixel_starts=True),
    "decam_refine_half": dict(T=26, H=2046, W=2048, psf_k=15, psf_sigma=(1.0, 2.0),
                              var=(0.5, 2.0), mask_frac=0.005, n_movers=100,
                              snr=("loguniform", 1.5, 10.0), spike_frac=0.1,
                              grid=(90.0, 500.0, 256, -0.3, 0.3, 128),
                              times=("nights", (7, 7, 6, 6)), integer_tracks=False,
                              movers_on_grid=False, start_margin=0, seed=7, K=8, lh_min=10.0,
                              min_obs=15, subpixel_starts=True),
}


def search_params_for(name):
    c = CONFIGS[name]
    return dict(k=c["K"], lh_min=c["lh_min"], min_obs=c["min_obs"], clip=1, q_lo=0.25,
                q_mid=0.5, q_hi=0.75, n_sigma=2.0, clip_on=0)


def velocity_grid(v_min, v_max, n_speed, a_min, a_max, n_angle, ecliptic=0.0):
    """Linear grid: inclusive linspace of speeds and angles; index = i_speed * n_angle + i_angle."""
    v = np.linspace(v_min, v_max, n_speed)
    a = np.linspace(a_min, a_max, n_angle) + ecliptic
    vv, aa = np.meshgrid(v, a, indexing="ij")
    vx = (vv * np.cos(aa)).astype(np.float32).ravel()
    vy = (vv * np.sin(aa)).astype(np.float32).ravel()
    return vx, vy


def gaussian_psf(sigma, k, fx=0.0, fy=0.0):
    """k x k Gaussian of width sigma centred at (fx, fy) from the centre pixel, normalised so the
    centred profile sums to one."""
    r = k // 2
    u = np.arange(-r, r + 1, dtype=np.float64)
    yy, xx = np.meshgrid(u, u, indexing="ij")
    norm = np.exp(-(xx ** 2 + yy ** 2) / (2 * sigma ** 2)).sum()
    return np.exp(-((xx - fx) ** 2 + (yy - fy) ** 2) / (2 * sigma ** 2)) / norm


def _times(spec, T, rng):
    if spec == "uniform0.2":
        return np.sort(rng.uniform(0.0, 0.2, T))
    kind, per_night = spec
    assert kind == "nights" and sum(per_night) == T
    cadence = 20.0 / (60 * 24)
    ts = []
    for n, m in enumerate(per_night):
        start = n + rng.uniform(0.0, 0.05)
        ts.extend(start + cadence * np.arange(m))
    t = np.asarray(ts, np.float64)
    return t - t[0]


def _snr(spec, n, rng):
    if spec[0] == "const":
        return np.full(n, spec[1])
    if spec[0] == "uniform":
        return rng.uniform(spec[1], spec[2], n)
    lo, hi = math.log(spec[1]), math.log(spec[2])
    return np.exp(rng.uniform(lo, hi, n))


def _stamp_add(plane, x, y, stamp):
    """Adds stamp (k x k) centred on integer pixel (x, y), clipped to the plane."""
    H, W = plane.shape
    k = stamp.shape[0]
    r = k // 2
    y0, y1 = y - r, y + r + 1
    x0, x1 = x - r, x + r + 1
    sy0, sx0 = max(0, -y0), max(0, -x0)
    sy1, sx1 = k - max(0, y1 - H), k - max(0, x1 - W)
    if sy0 >= sy1 or sx0 >= sx1:
        return
    plane[max(0, y0):min(H, y1), max(0, x0):min(W, x1)] += stamp[sy0:sy1, sx0:sx1]


def make_stack(name="tiny", seed=None, H=None, W=None, T=None, n_movers=None, grid=None):
    """Draws a difference-image stack for the named workload (overrides for test sizes)."""
    c = dict(CONFIGS[name])
    if H is not None:
        c["H"] = H
    if W is not None:
        c["W"] = W
    if T is not None:
        c["T"] = T
        if isinstance(c["times"], tuple):
            c["times"] = "uniform0.2" if T < 4 else ("nights", _split(T, 4))
    if n_movers is not None:
        c["n_movers"] = n_movers
    if grid is not None:
        c["grid"] = grid
    seed = c["seed"] if seed is None else seed
    rng = np.random.default_rng(seed)
    T_, H_, W_, k = c["T"], c["H"], c["W"], c["psf_k"]

    times = _times(c["times"], T_, rng)
    sig = rng.uniform(c["psf_sigma"][0], c["psf_sigma"][1], T_)
    psf = np.stack([gaussian_psf(s, k) for s in sig]).astype(np.float32)
    var_t = rng.uniform(c["var"][0], c["var"][1], T_).astype(np.float32)

    img = rng.standard_normal((T_, H_, W_), dtype=np.float32)
    img *= np.sqrt(var_t)[:, None, None]
    var = np.broadcast_to(var_t[:, None, None], (T_, H_, W_)).copy()

    vx, vy = velocity_grid(*c["grid"])
    nm = c["n_movers"]
    m = c["start_margin"]
    mx0 = rng.integers(m, W_ - m, nm)
    my0 = rng.integers(m, H_ - m, nm)
    if c["movers_on_grid"]:
        gidx = rng.integers(0, len(vx), nm)
        mvx, mvy = vx[gidx].astype(np.float64), vy[gidx].astype(np.float64)
    else:
        v0, v1, ns, a0, a1, na = c["grid"]
        sp = rng.uniform(v0, v1, nm)
        an = rng.uniform(a0, a1, nm)
        mvx, mvy = sp * np.cos(an), sp * np.sin(an)
        gidx = np.full(nm, -1)
    mx0f, my0f = mx0.astype(np.float64), my0.astype(np.float64)
    if c.get("subpixel_starts"):
        mx0f = mx0f + rng.uniform(-0.5, 0.5, nm)
        my0f = my0f + rng.uniform(-0.5, 0.5, nm)
    snr = _snr(c["snr"], nm, rng)
    sum_p2 = (psf.astype(np.float64) ** 2).sum(axis=(1, 2))
    flux = snr[:, None] * np.sqrt(var_t.astype(np.float64))[None, :] / np.sqrt(sum_p2)[None, :]
    spike = np.zeros((nm, T_), bool)
    if c["spike_frac"] > 0:
        n_sp = max(1, int(round(c["spike_frac"] * T_)))
        for i in range(nm):
            spike[i, rng.choice(T_, n_sp, replace=False)] = True
        spike_flux = 20.0 * np.sqrt(var_t.astype(np.float64)) / np.sqrt(sum_p2)
        flux = np.where(spike, spike_flux[None, :], flux)
    for i in range(nm):
        for t in range(T_):
            dt = times[t] - times[0]
            px, py = mx0f[i] + mvx[i] * dt, my0f[i] + mvy[i] * dt
            if c["integer_tracks"]:
                ix, iy = int(math.floor(px + 0.5)), int(math.floor(py + 0.5))
                st = flux[i, t] * psf[t].astype(np.float64)
            else:
                ix, iy = int(math.floor(px + 0.5)), int(math.floor(py + 0.5))
                st = flux[i, t] * gaussian_psf(sig[t], k, px - ix, py - iy)
            _stamp_add(img[t], ix, iy, st.astype(np.float32))

    mask = None
    if c["mask_frac"] > 0:
        mask = (rng.random((T_, H_, W_), dtype=np.float32) < c["mask_frac"]).astype(np.uint8)
        var[mask.astype(bool)] = np.inf
    movers = dict(x0=mx0f, y0=my0f, vx=mvx, vy=mvy, snr=snr, flux=flux, grid_idx=gidx,
                  spike=spike)
    return Stack(img=img, var=var, mask=mask, psf=psf, times=times, vx=vx, vy=vy, movers=movers,
                 name=name)


def _split(T, n):
    base = [T // n] * n
    for i in range(T % n):
        base[i] += 1
    return tuple(base)


def make_likelihood_stack(name="decam", seed=None, H=None, W=None, T=None, n_movers=None,
                          grid=None):
    """Draws psi/phi-like planes directly (the search's own inputs), without image formation.

    phi_t is a positive per-epoch level with mild pixel texture (0 at masked pixels); psi_t is
    sqrt(phi_t) N(0,1) plus Gaussian blobs of per-epoch significance s along each mover's track
    (s = 20 on spike epochs).  Used where the search is checked on its own at full size.
    Returns (psi, phi, times, vx, vy, movers)."""
    c = dict(CONFIGS[name])
    for key, val in (("H", H), ("W", W), ("T", T), ("n_movers", n_movers), ("grid", grid)):
        if val is not None:
            c[key] = val
    if T is not None and isinstance(c["times"], tuple):
        c["times"] = "uniform0.2" if T < 4 else ("nights", _split(T, 4))
    seed = (c["seed"] + 1000) if seed is None else seed
    rng = np.random.default_rng(seed)
    T_, H_, W_ = c["T"], c["H"], c["W"]
    times = _times(c["times"], T_, rng)
    level = rng.uniform(0.05, 0.3, T_).astype(np.float32)
    phi = level[:, None, None] * (1.0 + 0.05 * rng.random((T_, H_, W_), dtype=np.float32))
    psi = rng.standard_normal((T_, H_, W_), dtype=np.float32) * np.sqrt(phi)
    vx, vy = velocity_grid(*c["grid"])
    nm = c["n_movers"]
    v0, v1, ns, a0, a1, na = c["grid"]
    gidx = rng.integers(0, len(vx), nm)
    on_grid = rng.random(nm) < 0.5
    sp = rng.uniform(v0, v1, nm)
    an = rng.uniform(a0, a1, nm)
    mvx = np.where(on_grid, vx[gidx], sp * np.cos(an))
    mvy = np.where(on_grid, vy[gidx], sp * np.sin(an))
    mx0 = rng.uniform(0, W_, nm)
    my0 = rng.uniform(0, H_, nm)
    snr = _snr(c["snr"], nm, rng)
    spike = rng.random((nm, T_)) < max(c["spike_frac"], 0.0)
    r = 4
    u = np.arange(-r, r + 1)
    for i in range(nm):
        for t in range(T_):
            dt = times[t] - times[0]
            px, py = mx0[i] + mvx[i] * dt, my0[i] + mvy[i] * dt
            ix, iy = int(math.floor(px + 0.5)), int(math.floor(py + 0.5))
            s = 20.0 if spike[i, t] else snr[i]
            yy, xx = np.meshgrid(u + iy - py, u + ix - px, indexing="ij")
            blob = s * np.sqrt(level[t]) * np.exp(-(xx ** 2 + yy ** 2) / (2 * 1.5 ** 2))
            _stamp_add(psi[t], ix, iy, blob.astype(np.float32))
    if c["mask_frac"] > 0:
        m = rng.random((T_, H_, W_), dtype=np.float32) < c["mask_frac"]
        psi[m] = 0.0
        phi[m] = 0.0
    movers = dict(x0=mx0, y0=my0, vx=mvx, vy=mvy, snr=snr, grid_idx=np.where(on_grid, gidx, -1),
                  spike=spike)
    return psi, phi, times, vx, vy, movers
