"""Batched search (many stacks, one persistent launch): every stack's results must equal those of
kb_search on it, bit for bit (same kernels, same per-tile arithmetic; only the scheduling
differs), under every schedule, through the CUDA graph and on replay; three stacks are also
checked against the FP64 oracle.  Stacks mix T (thread-, half-warp- and warp-evaluated), sizes,
windows, K, clip settings and velocity counts.  Inputs are seeded likelihood planes (no input
comes from the CUDA path)."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import paper_2109_03296_b300 as kb
from helpers import compare_search, gpu_result_numpy

pytestmark = pytest.mark.gpu


def _stack(seed, T, H, W, n_traj, spread=30.0, params=None):
    rng = np.random.default_rng(seed)
    times = np.sort(rng.uniform(0, 1.0, T))
    times[0] = 0.0
    phi = rng.uniform(0.2, 1.5, (T, H, W))
    psi = rng.normal(size=(T, H, W)) * np.sqrt(phi)
    psi += 3.0 * phi * (rng.random((T, H, W)) < 0.05)
    m = rng.random((T, H, W)) < 0.04
    psi[m] = 0.0
    phi[m] = 0.0
    vx = rng.uniform(-spread, spread, n_traj).astype(np.float32)
    vy = rng.uniform(-spread, spread, n_traj).astype(np.float32)
    vx[3], vy[3] = vx[1], vy[1]
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return dict(psi=d(psi.astype(np.float32)), phi=d(phi.astype(np.float32)), times=times,
                vx=d(vx), vy=d(vy), params=params or kb.SearchParams(k=3, lh_min=2.0, min_obs=3),
                psi32=psi.astype(np.float32), phi32=phi.astype(np.float32), vxn=vx, vyn=vy)


def _stacks():
    return [
        _stack(1, 10, 70, 90, 100),
        _stack(2, 26, 130, 150, 220, params=kb.SearchParams(k=4, lh_min=2.5, min_obs=8,
                                                              clip_on=1)),
        _stack(3, 40, 60, 75, 90, params=kb.SearchParams(k=2, lh_min=2.0, min_obs=10)),
        _stack(4, 16, 57, 33, 64, params=kb.SearchParams(k=5, lh_min=1.5, min_obs=4, clip=0)),
        _stack(5, 20, 120, 200, 150, params=kb.SearchParams(k=3, lh_min=2.0, min_obs=5,
                                                              window=(17, 170, 9, 101))),
        _stack(6, 33, 40, 40, 33, spread=10.0, params=kb.SearchParams(k=1, lh_min=1.0,
                                                                      min_obs=2)),
        _stack(7, 80, 36, 44, 40, spread=12.0, params=kb.SearchParams(k=2, lh_min=2.0,
                                                                      min_obs=20)),
    ]


def _equal(a, b):
    for key in ("lh", "flux", "idx", "nvalid", "nkept", "mask"):
        x, y = a[key], b[key]
        if key in ("lh", "flux"):
            if not torch.equal(x.view(torch.int32), y.view(torch.int32)):
                return False
        elif not torch.equal(x, y):
            return False
    return True


@pytest.fixture(scope="module")
def batch_case():
    stacks = _stacks()
    ref = [kb.search(s["psi"], s["phi"], s["times"], s["vx"], s["vy"], s["params"])
           for s in stacks]
    torch.cuda.synchronize()
    return stacks, ref


def test_batch_equals_per_stack_search(cuda_device, batch_case):
    stacks, ref = batch_case
    b = kb.Batch(stacks)
    res = b.run()
    torch.cuda.synchronize()
    for i, (r, g) in enumerate(zip(ref, res)):
        assert _equal(r, g), "stack %d differs from kb_search" % i
    done, tot = b.stats()
    assert tot["err"] == 0
    assert tot["te"] == sum(b.te)
    assert np.all(done > 0)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("tile_cols", [0, 1, 2])
def test_batch_two_row_blocks(cuda_device, batch_case, mode, tile_cols):
    """Every stack summed over two-row blocks (bound_rows = 2; the automatic choice takes single
    rows for these small thresholds), so one persistent launch (mode 0) runs the block kernel, in
    tiles 32 or 64 pixels wide: results still bit-identical to kb_search with single rows."""
    stacks, ref = batch_case
    blocks = [dict(s, params=dataclasses.replace(s["params"], bound_rows=2)) for s in stacks]
    b = kb.Batch(blocks)
    b.schedule = kb.Schedule(mode=mode, tile_cols=tile_cols)
    res = b.run(graph=True)
    torch.cuda.synchronize()
    for i, (r, g) in enumerate(zip(ref, res)):
        assert _equal(r, g), "stack %d differs (mode %d, tile_cols %d)" % (i, mode, tile_cols)
    assert b.stats()[1]["err"] == 0
    words, offsets, staged, direct = b.pass_counts()
    assert words > 0 and offsets > 0 and staged > 0


def test_batch_graph_replay_and_schedules(cuda_device, batch_case):
    stacks, ref = batch_case
    b = kb.Batch(stacks)
    for sched in (kb.Schedule(), kb.Schedule(mode=0), kb.Schedule(tile_order=0, stack_order=0),
                  kb.Schedule(mode=0, hot_nu2=9.0, score_span=128, stack_order=0),
                  kb.Schedule(score_span=0), kb.Schedule(tile_cols=1), kb.Schedule(tile_cols=2),
                  kb.Schedule(mode=0, tile_cols=1, tile_order=0)):
        b.schedule = sched
        assert b.schedule == sched
        for _ in range(2):          # capture, then replay
            for r in b.results:     # stale outputs must be overwritten
                r["lh"].fill_(123.0)
                r["idx"].fill_(77)
            res = b.run(graph=True)
            torch.cuda.synchronize()
            for i, (r, g) in enumerate(zip(ref, res)):
                assert _equal(r, g), "stack %d differs under %s" % (i, sched)
    best = b.autotune(reps=1)
    assert b.schedule == best
    res = b.run(graph=True)
    torch.cuda.synchronize()
    for i, (r, g) in enumerate(zip(ref, res)):
        assert _equal(r, g), "stack %d differs after autotune" % i
    with pytest.raises(kb.KbError):
        b.schedule = kb.Schedule(tile_order=2)
    with pytest.raises(kb.KbError):
        b.schedule = kb.Schedule(hot_nu2=0.0)
    with pytest.raises(kb.KbError):
        b.schedule = kb.Schedule(mode=3)
    with pytest.raises(kb.KbError):
        b.schedule = kb.Schedule(tile_cols=3)


def test_batch_stacks_against_oracle(cuda_device, batch_case):
    stacks, _ = batch_case
    b = kb.Batch(stacks)
    res = b.run(graph=True)
    torch.cuda.synchronize()
    # T = 26 (thread path, clip on likelihood), T = 40 (half-warp pairs), T = 80 (warp per pair)
    for i in (1, 2, 6):
        s = stacks[i]
        sp = s["params"]
        o = oracle.search(s["psi32"], s["phi32"], s["times"], s["vxn"], s["vyn"],
                          dict(k=sp.k, lh_min=sp.lh_min, min_obs=sp.min_obs, clip=sp.clip,
                               clip_on=sp.clip_on))
        compare_search(gpu_result_numpy(res[i]), o, sp.lh_min)


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_completion_times(cuda_device, batch_case, mode):
    stacks, _ = batch_case
    b = kb.Batch(stacks)
    b.schedule = kb.Schedule(mode=mode)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    b.run()
    e1.record()
    torch.cuda.synchronize()
    done, tot = b.stats()
    # every stack finished within the run (the stamps are taken on the device)
    assert np.all(done > 0)
    assert done.max() <= e0.elapsed_time(e1) * 1e6 * 1.05 + 1e5
    assert tot["evals"] > 0 and tot["err"] == 0


def test_batch_refuses_bad_stacks(cuda_device):
    s = _stack(7, 10, 32, 32, 16)
    bad = dict(s, params=kb.SearchParams(k=0))
    with pytest.raises(kb.KbError, match="stack 1"):
        kb.Batch([s, bad])
    with pytest.raises(ValueError):
        kb.Batch([])
