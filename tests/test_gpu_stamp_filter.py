"""Central-moment stamp filter (Section 3.3) against the FP64 oracle.

Stamps are drawn here (no input comes from the CUDA path): sampled Gaussians with random centres,
widths and amplitudes plus noise, flat stamps, single lit pixels, stamps with NaN pixels, all-zero
and negative stamps, at radius 10 (the paper's 21 x 21) and 5.  Moments are compared within
float32 output rounding (the weights are non-negative, so no sum cancels); decisions must be equal
except where an oracle moment lies within 1e-12 relative of its limit (none in these cases).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2109_03296_b300 as kb

pytestmark = pytest.mark.gpu


def _stamps(n, r, seed):
    rng = np.random.default_rng(seed)
    side = 2 * r + 1
    u = np.arange(-r, r + 1, dtype=np.float64)
    yy, xx = np.meshgrid(u, u, indexing="ij")
    out = np.zeros((n, side, side))
    for i in range(n):
        kind = i % 6
        if kind in (0, 1, 2):
            cx, cy = rng.uniform(-1.2, 1.2, 2)
            sig = rng.uniform(0.8, 3.5)
            g = np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * sig ** 2))
            out[i] = rng.uniform(0.5, 20) * g + rng.normal(0, 0.05 * kind, (side, side))
        elif kind == 3:
            out[i] = rng.uniform(-0.2, 1.0)
        elif kind == 4:
            dx, dy = rng.integers(-r, r + 1, 2)
            out[i, dy + r, dx + r] = 1.0
            out[i] += rng.normal(0, 0.01, (side, side))
        else:
            out[i] = rng.normal(0, 1, (side, side))
            out[i][rng.random((side, side)) < 0.3] = np.nan
    out[0] = 0.0
    out[1] = -np.abs(out[1])
    return out.astype(np.float32)


@pytest.mark.parametrize("r", [10, 5])
def test_stamp_filter_matches_oracle(cuda_device, r):
    st = _stamps(600, r, 81 + r)
    mom, ok = kb.stamp_filter(torch.from_numpy(st).cuda())
    mom, ok = mom.cpu().numpy(), ok.cpu().numpy()
    om, ook = oracle.stamp_moments(st.astype(np.float64))
    side = 2 * r + 1
    u = np.arange(-r, r + 1, dtype=np.float64)
    yy, xx = np.meshgrid(u, u, indexing="ij")
    s64 = st.astype(np.float64)
    a = np.nan_to_num(s64 - np.nanmin(s64, axis=(1, 2), keepdims=True))
    for k, w in enumerate([np.ones_like(xx), xx, yy, xx * yy, xx * xx, yy * yy]):
        scale = (a * np.abs(w)).sum(axis=(1, 2))
        if k > 0:
            scale = scale / np.maximum(np.abs(om[:, 0]), 1e-300)
        fin = np.isfinite(om[:, k])
        assert np.all(np.abs(mom[fin, k] - om[fin, k]) <= 2e-7 * np.abs(om[fin, k]) +
                      1e-12 * scale[fin]), k
    lim = np.array(oracle.PAPER_MOMENT_LIMITS)
    near = np.zeros(len(st), bool)
    for k, (j, absv) in enumerate(((1, True), (2, True), (3, True), (4, False), (5, False))):
        v = np.abs(om[:, j]) if absv else om[:, j]
        near |= np.abs(v - lim[k]) <= 1e-12 * lim[k]
    assert not near.any()
    assert np.array_equal(ok, ook)
    assert 0.1 < ook.mean() < 0.9


def test_stamp_filter_custom_limits_and_edges(cuda_device):
    st = _stamps(120, 10, 91)
    lim = (1.0, 0.8, 2.0, 30.0, 40.0)
    _, ok = kb.stamp_filter(torch.from_numpy(st).cuda(), limits=lim)
    _, ook = oracle.stamp_moments(st.astype(np.float64), limits=lim)
    assert np.array_equal(ok.cpu().numpy(), ook)
    e = torch.empty((0, 21, 21), dtype=torch.float32, device="cuda")
    m, ok = kb.stamp_filter(e)
    assert m.shape == (0, 6) and ok.numel() == 0
    with pytest.raises(kb.KbError):
        kb.stamp_filter(torch.zeros((2, 21, 21), device="cuda"), limits=(float("nan"),) * 5)


def test_stamp_filter_keeps_movers_and_rejects_noise(cuda_device):
    """Pipeline property on the tiny workload: the median coadds along the injected movers' own
    tracks pass the paper's limits; those along random tracks through noise mostly fail."""
    from synth import make_stack
    s = make_stack("tiny")
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    img, var = d(s.img), d(s.var)
    mv = s.movers
    x0 = d(np.round(mv["x0"]).astype(np.int32))
    y0 = d(np.round(mv["y0"]).astype(np.int32))
    _, med = kb.stamps(img, var, None, s.times, x0, y0, d(mv["vx"].astype(np.float32)),
                       d(mv["vy"].astype(np.float32)))
    _, ok = kb.stamp_filter(med)
    assert ok.all()
    rng = np.random.default_rng(5)
    n = 400
    rx = d(rng.integers(40, 216, n).astype(np.int32))
    ry = d(rng.integers(40, 216, n).astype(np.int32))
    k = rng.integers(0, len(s.vx), n)
    _, medr = kb.stamps(img, var, None, s.times, rx, ry, d(s.vx[k]), d(s.vy[k]))
    _, okr = kb.stamp_filter(medr)
    # a noise stamp has xx, yy = 36.67 +- 0.6 about the 36.5 limit: both below it ~15% of the time
    assert okr.float().mean() < 0.35
