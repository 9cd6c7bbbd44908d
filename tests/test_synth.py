"""The seeded input generators follow the stated recipes (checked on reduced image sizes; the
recipe's other parameters are those of the named workload)."""
import math

import numpy as np

from synth import CONFIGS, make_likelihood_stack, make_stack, velocity_grid


def test_decam_recipe():
    c = CONFIGS["decam"]
    s = make_stack("decam", H=192, W=256, n_movers=40)
    T = c["T"]
    assert s.img.shape == (T, 192, 256) and s.img.dtype == np.float32
    # 26 epochs over 4 nights (7, 7, 6, 6), 20-minute cadence within a night, from t = 0
    t = s.times
    assert len(t) == 26 and t[0] == 0.0 and np.all(np.diff(t) > 0)
    gaps = np.diff(t)
    night_breaks = np.nonzero(gaps > 0.5)[0]
    assert night_breaks.tolist() == [6, 13, 19]
    within = np.delete(gaps, night_breaks)
    assert np.allclose(within, 20.0 / (60 * 24), rtol=0, atol=1e-12)
    # nights start a day apart, each at a random offset of up to 0.05 d
    starts = t[[0, 7, 14, 20]] - np.arange(4)
    assert np.all(np.abs(starts) <= 0.05)
    # per-epoch variance U[0.5, 2] (inf at the ~0.5% masked pixels), PSFs normalised Gaussians
    good = ~s.mask.astype(bool)
    assert abs(s.mask.mean() - 0.005) < 0.001
    assert np.all(np.isinf(s.var[~good]))
    for e in range(T):
        v = np.unique(s.var[e][good[e]])
        assert len(v) == 1 and 0.5 <= v[0] <= 2.0
        p = s.psf[e].astype(np.float64)
        assert p.shape == (15, 15) and abs(p.sum() - 1.0) < 1e-5
        assert np.allclose(p, p[::-1, :]) and np.allclose(p, p.T)
        # the width from the second moment of the centred profile: sigma in [1, 2]
        u = np.arange(-7, 8)
        sig2 = (p.sum(0) * u ** 2).sum() / p.sum()
        assert 0.95 <= math.sqrt(sig2) <= 2.0
    # movers: SNR log-uniform in [1.5, 10], 10% of epochs (3 of 26) replaced by +20 sigma spikes
    mv = s.movers
    assert np.all((mv["snr"] >= 1.5) & (mv["snr"] <= 10.0))
    assert np.all(mv["spike"].sum(1) == 3)
    sum_p2 = (s.psf.astype(np.float64) ** 2).sum(axis=(1, 2))
    var_t = np.array([np.unique(s.var[e][good[e]])[0] for e in range(T)], np.float64)
    spike_flux = 20.0 * np.sqrt(var_t) / np.sqrt(sum_p2)
    assert np.allclose(mv["flux"][mv["spike"]], np.broadcast_to(spike_flux, mv["flux"].shape)[
        mv["spike"]])
    normal = mv["snr"][:, None] * np.sqrt(var_t)[None, :] / np.sqrt(sum_p2)[None, :]
    assert np.allclose(mv["flux"][~mv["spike"]], normal[~mv["spike"]])
    # movers' velocities between the grid's speed and angle limits (off the grid)
    sp = np.hypot(mv["vx"], mv["vy"])
    an = np.arctan2(mv["vy"], mv["vx"])
    assert np.all((sp >= 90.0) & (sp <= 500.0)) and np.all(np.abs(an) <= 0.3 + 1e-12)
    # background noise has the epoch's variance
    for e in (0, 13, 25):
        z = s.img[e][good[e]] / math.sqrt(var_t[e])
        assert abs(z.std() - 1.0) < 0.05


def test_velocity_grid_layout():
    vx, vy = velocity_grid(90.0, 500.0, 256, -0.3, 0.3, 128)
    assert vx.dtype == np.float32 and len(vx) == 256 * 128
    sp = np.hypot(vx.astype(np.float64), vy.astype(np.float64)).reshape(256, 128)
    an = np.arctan2(vy.astype(np.float64), vx.astype(np.float64)).reshape(256, 128)
    # index = i_speed * n_angle + i_angle, both inclusive linspaces
    assert np.allclose(sp[:, 0], np.linspace(90.0, 500.0, 256), rtol=1e-6)
    assert np.allclose(an[0], np.linspace(-0.3, 0.3, 128), atol=1e-6)


def test_tiny_recipe():
    s = make_stack("tiny")
    assert s.img.shape == (10, 256, 256) and s.mask is None
    assert np.all(s.var == 1.0) and np.all((s.times >= 0) & (s.times <= 0.2))
    mv = s.movers
    assert len(mv["x0"]) == 3 and np.all(mv["grid_idx"] >= 0) and np.all(mv["snr"] == 5.0)
    assert np.array_equal(mv["vx"], s.vx[mv["grid_idx"]].astype(np.float64))


def test_generators_are_seeded():
    a = make_stack("decam", H=64, W=96, n_movers=5)
    b = make_stack("decam", H=64, W=96, n_movers=5)
    c = make_stack("decam", H=64, W=96, n_movers=5, seed=99)
    assert np.array_equal(a.img, b.img) and np.array_equal(a.times, b.times)
    assert not np.array_equal(a.img, c.img)
    p1 = make_likelihood_stack("decam", H=64, W=96, n_movers=5)
    p2 = make_likelihood_stack("decam", H=64, W=96, n_movers=5)
    for x, y in zip(p1[:5], p2[:5]):
        assert np.array_equal(x, y)


def test_likelihood_stack_planes():
    psi, phi, times, vx, vy, mv = make_likelihood_stack("decam", H=128, W=160, n_movers=10)
    assert psi.shape == phi.shape == (26, 128, 160)
    assert psi.dtype == phi.dtype == np.float32
    assert np.all(phi >= 0.0) and np.all(np.isfinite(psi)) and np.all(np.isfinite(phi))
    # masked pixels carry psi = phi = 0, about 0.5% of them
    zero = phi == 0.0
    assert abs(zero.mean() - 0.005) < 0.0015 and np.all(psi[zero] == 0.0)
    assert len(vx) == 256 * 128 and times[0] == 0.0


def test_batch64_specs_and_torch_stacks():
    """The 64-stack batch: sizes, epoch counts and grids from the stated sets, movers at the decam
    density; one stack drawn by the torch generator (on the CPU here) follows the decam recipe."""
    import torch
    from synth.gpu_stacks import BATCH64, batch_specs, make_stack_torch
    specs = batch_specs()
    assert len(specs) == 64 and batch_specs() == specs
    sizes = {(H, W) for H, W, *_ in specs}
    assert sizes <= set(BATCH64["sizes"]) and len(sizes) == 3
    assert all(10 <= T <= 40 for _, _, T, *_ in specs)
    assert {(ns, na) for _, _, _, ns, na, _, _ in specs} <= set(BATCH64["grids"])
    for H, W, T, ns, na, nm, seed in specs:
        assert nm == max(1, int(round(200.0 / (2046 * 4094) * H * W)))
    assert len({s[-1] for s in specs}) == 64
    s = make_stack_torch(96, 128, 12, 16, 8, 6, 1234, "cpu")
    img, var, mask = s["img"], s["var"], s["mask"].bool()
    assert img.shape == var.shape == (12, 96, 128) and img.dtype == torch.float32
    assert torch.isinf(var[mask]).all() and torch.isfinite(var[~mask]).all()
    assert abs(mask.float().mean().item() - 0.005) < 0.003
    assert s["vx"].numel() == 16 * 8 and s["times"][0] == 0.0
    mv = s["movers"]
    assert np.all(mv["spike"].sum(1) == 1)               # round(0.1 * 12) spike epochs
    assert np.all((mv["snr"] >= 1.5) & (mv["snr"] <= 10.0))
    again = make_stack_torch(96, 128, 12, 16, 8, 6, 1234, "cpu")
    assert torch.equal(again["img"], img) and torch.equal(again["mask"], s["mask"])


def test_config_stack_torch_follows_the_full_recipe():
    """The device generator of the full-scale workload (drawn here on the CPU at a reduced image
    size): five nights of 20 epochs at a 20-minute cadence, per-epoch variance in [0.5, 2] with 1%
    of pixels masked (var = inf), PSF widths in [1, 2.5] on 15 x 15 normalised kernels, movers at
    SNR 1-8, the paper's 512 x 256 grid; seeded."""
    import torch
    from synth.gpu_stacks import make_config_stack_torch
    d = make_config_stack_torch("full", "cpu", H=256, W=320, n_movers=40)
    T, H, W = d["img"].shape
    assert (T, H, W) == (100, 256, 320)
    t = d["times"]
    gaps = np.diff(t)
    assert t[0] == 0.0 and (gaps > 0).all() and (gaps > 0.5).sum() == 4
    assert np.allclose(gaps[gaps < 0.5], 20.0 / 1440.0)
    m = d["mask"].bool()
    assert abs(m.float().mean().item() - 0.01) < 0.002
    assert torch.isinf(d["var"][m]).all()
    v = d["var"][~m]
    assert v.min().item() >= 0.5 and v.max().item() <= 2.0
    psf = d["psf"].numpy()
    assert psf.shape == (100, 15, 15) and np.allclose(psf.sum(axis=(1, 2)), 1.0, atol=1e-5)
    assert len(d["vx"]) == 512 * 256
    snr = d["movers"]["snr"]
    assert snr.min() >= 1.0 and snr.max() <= 8.0 and not d["movers"]["spike"].any()
    d2 = make_config_stack_torch("full", "cpu", H=256, W=320, n_movers=40)
    assert torch.equal(d["img"], d2["img"]) and torch.equal(d["mask"], d2["mask"])
