"""Seeded synthetic stacks drawn on the GPU with torch, for workloads too large to draw with numpy
in reasonable time (the 64-stack batch).  Same recipe as `make_stack` for the decam workload:
N(0, var_t) noise with var_t ~ U[0.5, 2], 0.5% masked pixels (var = inf), Gaussian PSFs with
sigma_t ~ U[1, 2] on 15 x 15, movers at real starts with velocities drawn uniformly in speed and
angle over the grid's range, per-epoch SNR log-U[1.5, 10] and 10% of each mover's epochs replaced
by +20 sigma spikes; times over 4 nights at 20-minute cadence.  No method arithmetic here; the
random draws differ from numpy's, so these stacks are not those of `make_stack`.
"""
import math

import numpy as np

from .stacks import CONFIGS, _snr, _split, _times, gaussian_psf, velocity_grid

__all__ = ["make_stack_torch", "make_config_stack_torch", "BATCH64"]

# 64 stacks: sizes uniform in {512x512, 1024x2048, 2046x4094}, epochs uniform in 10..40, velocity
# grids of 4096..32768 trajectories (speeds x angles over 90-500 px/day and +-0.3 rad); movers at
# the decam density (200 per 2046 x 4094).
BATCH64 = dict(n=64, sizes=((512, 512), (1024, 2048), (2046, 4094)), T=(10, 40),
               grids=((64, 64), (128, 64), (128, 128), (256, 128)), v=(90.0, 500.0),
               a=(-0.3, 0.3), density=200.0 / (2046 * 4094), seed=64)


def batch_specs(cfg=BATCH64):
    """Per-stack (H, W, T, n_speed, n_angle, n_movers, seed) of the batch, seeded."""
    rng = np.random.default_rng(cfg["seed"])
    out = []
    for i in range(cfg["n"]):
        H, W = cfg["sizes"][rng.integers(len(cfg["sizes"]))]
        T = int(rng.integers(cfg["T"][0], cfg["T"][1] + 1))
        ns, na = cfg["grids"][rng.integers(len(cfg["grids"]))]
        nm = max(1, int(round(cfg["density"] * H * W)))
        out.append((H, W, T, ns, na, nm, int(cfg["seed"] * 1000 + i)))
    return out


def _add_unique(img, idx, val, device):
    """img.view(-1)[idx] += val with repeated indices summed on the host first (float64), so that
    the device add sees each pixel once and the stack is the same bit for bit in every process
    (an index_add_ with repeated indices adds in an order that varies between runs)."""
    import torch
    uniq, inv = np.unique(np.asarray(idx, np.int64), return_inverse=True)
    sums = np.bincount(inv.ravel(), weights=np.asarray(val, np.float64).ravel()).astype(np.float32)
    img.view(-1).index_add_(0, torch.from_numpy(uniq).to(device), torch.from_numpy(sums).to(device))


def make_stack_torch(H, W, T, n_speed, n_angle, n_movers, seed, device, v=(90.0, 500.0),
                     a=(-0.3, 0.3)):
    """Returns dict(img, var, mask, psf (torch on device), times, vx, vy (torch), movers)."""
    import torch
    rng = np.random.default_rng(seed)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    times = _times(("nights", _split(T, 4)) if T >= 4 else "uniform0.2", T, rng)
    k = 15
    sig = rng.uniform(1.0, 2.0, T)
    psf = np.stack([gaussian_psf(s, k) for s in sig]).astype(np.float32)
    var_t = rng.uniform(0.5, 2.0, T).astype(np.float32)
    sd = torch.from_numpy(np.sqrt(var_t)).to(device)
    img = torch.randn((T, H, W), generator=g, device=device, dtype=torch.float32)
    img *= sd[:, None, None]
    var = torch.from_numpy(var_t).to(device)[:, None, None].expand(T, H, W).contiguous()
    vx, vy = velocity_grid(v[0], v[1], n_speed, a[0], a[1], n_angle)
    # movers: real starts, off-grid velocities
    x0 = rng.uniform(0, W, n_movers)
    y0 = rng.uniform(0, H, n_movers)
    sp = rng.uniform(v[0], v[1], n_movers)
    an = rng.uniform(a[0], a[1], n_movers)
    mvx, mvy = sp * np.cos(an), sp * np.sin(an)
    snr = np.exp(rng.uniform(math.log(1.5), math.log(10.0), n_movers))
    sum_p2 = (psf.astype(np.float64) ** 2).sum(axis=(1, 2))
    flux = snr[:, None] * np.sqrt(var_t.astype(np.float64))[None, :] / np.sqrt(sum_p2)[None, :]
    n_sp = max(1, int(round(0.1 * T)))
    spike = np.zeros((n_movers, T), bool)
    for i in range(n_movers):
        spike[i, rng.choice(T, n_sp, replace=False)] = True
    flux = np.where(spike, (20.0 * np.sqrt(var_t.astype(np.float64)) / np.sqrt(sum_p2))[None, :],
                    flux)
    r = k // 2
    idx, val = [], []
    u = np.arange(-r, r + 1)
    for i in range(n_movers):
        for t in range(T):
            dt = times[t] - times[0]
            px, py = x0[i] + mvx[i] * dt, y0[i] + mvy[i] * dt
            ix, iy = int(math.floor(px + 0.5)), int(math.floor(py + 0.5))
            if ix + r < 0 or ix - r >= W or iy + r < 0 or iy - r >= H:
                continue
            st = flux[i, t] * gaussian_psf(sig[t], k, px - ix, py - iy)
            yy, xx = np.meshgrid(iy + u, ix + u, indexing="ij")
            ok = (yy >= 0) & (yy < H) & (xx >= 0) & (xx < W)
            idx.append((t * H + yy[ok]) * W + xx[ok])
            val.append(st[ok])
    if idx:
        _add_unique(img, np.concatenate(idx), np.concatenate(val), device)
    mask = torch.rand((T, H, W), generator=g, device=device) < 0.005
    var[mask] = float("inf")
    movers = dict(x0=x0, y0=y0, vx=mvx, vy=mvy, snr=snr, spike=spike)
    return dict(img=img, var=var, mask=mask.to(torch.uint8), psf=torch.from_numpy(psf).to(device),
                times=times, vx=torch.from_numpy(vx).to(device),
                vy=torch.from_numpy(vy).to(device), movers=movers)


def make_config_stack_torch(name, device, seed=None, H=None, W=None, n_movers=None):
    """A named workload's stack (CONFIGS[name]: epochs and nights, image size, per-epoch variance
    and PSF width, masked fraction, movers with their SNR distribution and spikes, velocity grid)
    drawn on the device with torch, for sizes too large to draw with numpy in reasonable time
    (the full-scale 4096 x 4096 x 100 stack).  Movers start at real positions with velocities
    drawn uniformly in speed and angle over the grid's range.  The random draws differ from
    make_stack's.  H, W, n_movers override the config (test sizes).  Returns dict(img, var, mask,
    psf (torch, device), times, vx, vy (torch), movers, seed)."""
    import torch
    c = dict(CONFIGS[name])
    for key, v in (("H", H), ("W", W), ("n_movers", n_movers)):
        if v is not None:
            c[key] = v
    seed = c["seed"] if seed is None else seed
    rng = np.random.default_rng(seed)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    T, H, W, k = c["T"], c["H"], c["W"], c["psf_k"]
    times = _times(c["times"], T, rng)
    sig = rng.uniform(c["psf_sigma"][0], c["psf_sigma"][1], T)
    psf = np.stack([gaussian_psf(s_, k) for s_ in sig]).astype(np.float32)
    var_t = rng.uniform(c["var"][0], c["var"][1], T).astype(np.float32)
    sd = torch.from_numpy(np.sqrt(var_t)).to(device)
    img = torch.randn((T, H, W), generator=g, device=device, dtype=torch.float32)
    img *= sd[:, None, None]
    var = torch.from_numpy(var_t).to(device)[:, None, None].expand(T, H, W).contiguous()
    vx, vy = velocity_grid(*c["grid"])
    v0, v1, ns, a0, a1, na = c["grid"]
    nm = c["n_movers"]
    x0 = rng.uniform(0, W, nm)
    y0 = rng.uniform(0, H, nm)
    sp = rng.uniform(v0, v1, nm)
    an = rng.uniform(a0, a1, nm)
    mvx, mvy = sp * np.cos(an), sp * np.sin(an)
    snr = _snr(c["snr"], nm, rng)
    sum_p2 = (psf.astype(np.float64) ** 2).sum(axis=(1, 2))
    flux = snr[:, None] * np.sqrt(var_t.astype(np.float64))[None, :] / np.sqrt(sum_p2)[None, :]
    spike = np.zeros((nm, T), bool)
    if c["spike_frac"] > 0:
        n_sp = max(1, int(round(c["spike_frac"] * T)))
        for i in range(nm):
            spike[i, rng.choice(T, n_sp, replace=False)] = True
        flux = np.where(spike, (20.0 * np.sqrt(var_t.astype(np.float64)) /
                                np.sqrt(sum_p2))[None, :], flux)
    r = k // 2
    u = np.arange(-r, r + 1)
    idx, val = [], []
    for t in range(T):
        dt = times[t] - times[0]
        px, py = x0 + mvx * dt, y0 + mvy * dt
        ix, iy = np.floor(px + 0.5).astype(np.int64), np.floor(py + 0.5).astype(np.int64)
        fx, fy = px - ix, py - iy
        norm = np.exp(-(u[:, None] ** 2 + u[None, :] ** 2) / (2 * sig[t] ** 2)).sum()
        # [n][k][k] stamps of every mover at this epoch, centred on (fx, fy)
        sx = np.exp(-((u[None, :] - fx[:, None]) ** 2) / (2 * sig[t] ** 2))
        sy = np.exp(-((u[None, :] - fy[:, None]) ** 2) / (2 * sig[t] ** 2))
        st = flux[:, t][:, None, None] * sy[:, :, None] * sx[:, None, :] / norm
        yy = iy[:, None, None] + u[None, :, None]
        xx = ix[:, None, None] + u[None, None, :]
        yy, xx = np.broadcast_to(yy, st.shape), np.broadcast_to(xx, st.shape)
        ok = (yy >= 0) & (yy < H) & (xx >= 0) & (xx < W)
        idx.append((t * H + yy[ok]) * W + xx[ok])
        val.append(st[ok])
    _add_unique(img, np.concatenate(idx), np.concatenate(val), device)
    mask = torch.rand((T, H, W), generator=g, device=device) < c["mask_frac"]
    var[mask] = float("inf")
    movers = dict(x0=x0, y0=y0, vx=mvx, vy=mvy, snr=snr, spike=spike)
    return dict(img=img, var=var, mask=mask.to(torch.uint8), psf=torch.from_numpy(psf).to(device),
                times=times, vx=torch.from_numpy(vx).to(device),
                vy=torch.from_numpy(vy).to(device), movers=movers, seed=seed)
