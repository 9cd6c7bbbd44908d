"""Candidate clustering (greedy de-duplication in priority order) against the FP64 oracle: the
kept flags and representatives must be equal exactly (both sides decide with float64 distances
computed by the same separately rounded operations).  Candidates are drawn here: dense groups of
near-identical tracks (chains of duplicates), scattered tracks, invalid entries and the
out-of-range placeholders of empty survivor slots."""
import numpy as np
import pytest
import torch

import oracle
import paper_2109_03296_b300 as kb

pytestmark = pytest.mark.gpu


def _d(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _cands(seed, n, groups, spread_px, spread_v, W=4000, H=2000):
    rng = np.random.default_rng(seed)
    cx, cy = rng.uniform(0, W, groups), rng.uniform(0, H, groups)
    cvx, cvy = rng.uniform(90, 500, groups), rng.uniform(-150, 150, groups)
    k = rng.integers(0, groups, n)
    x0 = np.round(cx[k] + rng.normal(0, spread_px, n)).astype(np.int32)
    y0 = np.round(cy[k] + rng.normal(0, spread_px, n)).astype(np.int32)
    vx = (cvx[k] + rng.normal(0, spread_v, n)).astype(np.float32)
    vy = (cvy[k] + rng.normal(0, spread_v, n)).astype(np.float32)
    valid = (rng.random(n) < 0.92).astype(np.uint8)
    far = rng.random(n) < 0.02            # placeholders of empty slots
    x0[far] = -(1 << 28)
    y0[far] = -(1 << 28)
    return x0, y0, vx, vy, valid


@pytest.mark.parametrize("seed,n,groups,spx,sv,r", [(1, 5000, 60, 3.0, 1.0, 8.0),
                                                    (2, 20000, 400, 6.0, 3.0, 4.0),
                                                    (3, 3000, 3000, 500.0, 50.0, 8.0)])
def test_cluster_matches_oracle(cuda_device, seed, n, groups, spx, sv, r):
    x0, y0, vx, vy, valid = _cands(seed, n, groups, spx, sv)
    dt = 3.1
    keep, rep, rounds = kb.cluster(_d(x0), _d(y0), _d(vx), _d(vy), np.array([0.0, dt]),
                                   radius=r, valid=_d(valid), return_rounds=True)
    ok, orep = oracle.cluster(x0, y0, vx, vy, dt, r, valid=valid)
    assert np.array_equal(keep.cpu().numpy(), ok)
    assert np.array_equal(rep.cpu().numpy(), orep)
    assert 0 < ok.sum() < valid.sum()
    assert 1 <= rounds <= 64


def test_cluster_rounds_stay_few_on_dense_groups(cuda_device):
    # 3000 candidates in 3 groups of mutual duplicates, as a bright mover's survivors are: the
    # greedy result needs two rounds per group, not one per member
    rng = np.random.default_rng(9)
    n = 3000
    g = rng.integers(0, 3, n)
    x0 = (np.array([100, 900, 2000])[g] + rng.integers(-1, 2, n)).astype(np.int32)
    y0 = (np.array([50, 700, 1500])[g] + rng.integers(-1, 2, n)).astype(np.int32)
    vx = (np.array([120.0, 300.0, 450.0])[g] + rng.normal(0, 0.2, n)).astype(np.float32)
    vy = (np.array([10.0, -40.0, 90.0])[g] + rng.normal(0, 0.2, n)).astype(np.float32)
    keep, rep, rounds = kb.cluster(_d(x0), _d(y0), _d(vx), _d(vy), [0.0, 3.0], radius=8.0,
                                   return_rounds=True)
    ok, orep = oracle.cluster(x0, y0, vx, vy, 3.0, 8.0)
    assert np.array_equal(keep.cpu().numpy(), ok) and np.array_equal(rep.cpu().numpy(), orep)
    assert ok.sum() == 3
    assert rounds <= 4


def test_cluster_edges(cuda_device):
    e = torch.empty(0, dtype=torch.int32, device="cuda")
    ef = torch.empty(0, dtype=torch.float32, device="cuda")
    keep, rep = kb.cluster(e, e, ef, ef, [0.0, 1.0])
    assert keep.numel() == 0 and rep.numel() == 0
    one = torch.tensor([5], dtype=torch.int32, device="cuda")
    v1 = torch.tensor([100.0], device="cuda")
    keep, rep = kb.cluster(one, one, v1, v1, [0.0, 1.0])
    assert keep.tolist() == [True] and rep.tolist() == [0]
    keep, rep = kb.cluster(one, one, v1, v1, [0.0, 1.0],
                           valid=torch.zeros(1, dtype=torch.uint8, device="cuda"))
    assert keep.tolist() == [False] and rep.tolist() == [-1]
    with pytest.raises(kb.KbError):
        kb.cluster(one, one, v1, v1, [0.0, 1.0], radius=0.5)


def test_cluster_after_stamp_filter_keeps_one_track_per_mover(cuda_device):
    """Tiny workload end to end: search -> collect -> tracks -> stamps -> moment filter ->
    clustering.  Many survivors follow each injected mover; after clustering each mover is still
    represented and the number of candidates drops."""
    from synth import CONFIGS, make_stack
    s = make_stack("tiny")
    c = CONFIGS["tiny"]
    img, var = _d(s.img), _d(s.var)
    psi, phi = kb.make_psi_phi(img, var, None, _d(s.psf))
    vx, vy = _d(s.vx), _d(s.vy)
    res = kb.search(psi, phi, s.times, vx, vy, kb.SearchParams(k=4, lh_min=c["lh_min"],
                                                               min_obs=c["min_obs"]))
    pix, slot, count = kb.collect(res, 2000)
    x0, y0, cvx, cvy, traj = kb.candidate_tracks(pix, slot, res, vx, vy)
    _, med = kb.stamps(img, var, None, s.times, x0, y0, cvx, cvy)
    _, passed = kb.stamp_filter(med)
    valid = passed & (traj >= 0)
    keep, rep = kb.cluster(x0, y0, cvx, cvy, s.times, radius=8.0, valid=valid)
    k = keep.cpu().numpy()
    assert 0 < k.sum() < valid.sum().item()
    X0, Y0 = x0.cpu().numpy(), y0.cpu().numpy()
    for i in range(len(s.movers["x0"])):
        mx, my = s.movers["x0"][i], s.movers["y0"][i]
        near = (np.abs(X0 - mx) <= 2) & (np.abs(Y0 - my) <= 2) & k
        assert near.any(), "mover %d lost" % i
