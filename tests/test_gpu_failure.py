"""Failure detection without a GPU fault.

The search kernel bounds every device-side wait (mbarrier waits of producers and consumers, the
producers' tile hand-off) by time, and a block whose wait gave up raises an abort flag that ends
its other warps' waits.  kb_wait_check runs those wait routines on waits that nothing completes,
with a short limit: they must give up, the device must report it, the abort flag must end a wait
at once, and the context must stay usable for the next search.  Nothing here faults, traps or
hangs the GPU: every wait ends by its limit or by the flag.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
import paper_2109_03296_b300 as kb
from helpers import compare_search, gpu_result_numpy


def test_wait_check_validates_its_limit():
    from paper_2109_03296_b300 import _lib as K
    L = K.lib()
    out = (C.c_ulonglong * 4)()
    assert L.kb_wait_check(999, out, None) == K.KB_ERR_INVALID_ARG
    assert L.kb_wait_check(10 ** 10 + 1, out, None) == K.KB_ERR_INVALID_ARG
    assert "limit_ns" in L.kb_last_error().decode()


@pytest.mark.gpu
def test_bounded_waits_give_up_and_the_context_stays_usable(cuda_device):
    limit = 50_000_000                         # 50 ms
    status, (t_prod, t_cons, t_abort), msg = kb.wait_check(limit)
    assert status == 0x7, msg
    assert "gave up" in msg
    # each wait ran to its limit and stopped soon after (an attempt suspends for <= 20 us)
    assert limit <= t_prod < limit + 20_000_000
    assert limit <= t_cons < limit + 20_000_000
    # with the abort flag raised a consumer wait returns at the flag, not at the limit
    assert t_abort < 1_000_000

    # the same context then searches a small stack and matches the oracle
    rng = np.random.default_rng(31)
    T, H, W, n = 10, 70, 90, 300
    times = np.sort(rng.uniform(0, 1.0, T))
    times[0] = 0.0
    phi = rng.uniform(0.2, 1.5, (T, H, W))
    psi = rng.normal(size=(T, H, W)) * np.sqrt(phi) + 3.0 * phi * (rng.random((T, H, W)) < 0.05)
    psi32, phi32 = psi.astype(np.float32), phi.astype(np.float32)
    vx = rng.uniform(-30, 30, n).astype(np.float32)
    vy = rng.uniform(-30, 30, n).astype(np.float32)
    sp = kb.SearchParams(k=3, lh_min=3.0, min_obs=4)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    res = kb.search(d(psi32), d(phi32), times, d(vx), d(vy), sp)
    torch.cuda.synchronize()
    assert kb.search_stats(res["workspace"])[3] == 0
    o = oracle.search(psi32, phi32, times, vx, vy, dict(k=3, lh_min=3.0, min_obs=4))
    compare_search(gpu_result_numpy(res), o, sp.lh_min)


@pytest.mark.gpu
def test_injected_host_faults_are_reported_and_the_next_call_works(cuda_device, monkeypatch):
    """KB_FAULT_INJECT makes the named entry points fail on the host, before any device work; the
    binding raises, and the same search, batch and context then run normally."""
    rng = np.random.default_rng(32)
    T, H, W, n = 8, 50, 64, 120
    times = np.sort(rng.uniform(0, 1.0, T))
    times[0] = 0.0
    phi = rng.uniform(0.2, 1.5, (T, H, W)).astype(np.float32)
    psi = (rng.normal(size=(T, H, W)) * np.sqrt(phi) + 3.0 * phi * (rng.random((T, H, W)) < 0.05)
           ).astype(np.float32)
    vx = rng.uniform(-25, 25, n).astype(np.float32)
    vy = rng.uniform(-25, 25, n).astype(np.float32)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    gpsi, gphi, gvx, gvy = d(psi), d(phi), d(vx), d(vy)
    sp = kb.SearchParams(k=2, lh_min=2.0, min_obs=3)
    launches = kb.launch_count()
    monkeypatch.setenv("KB_FAULT_INJECT", "kb_search,kb_batch_create")
    with pytest.raises(kb.KbError, match="kb_search: injected fault"):
        kb.search(gpsi, gphi, times, gvx, gvy, sp)
    stack = dict(psi=gpsi, phi=gphi, times=times, vx=gvx, vy=gvy, params=sp)
    with pytest.raises(kb.KbError, match="kb_batch_create: injected fault"):
        kb.Batch([stack])
    assert kb.launch_count() == launches          # nothing reached the device
    monkeypatch.delenv("KB_FAULT_INJECT")
    b = kb.Batch([stack])
    monkeypatch.setenv("KB_FAULT_INJECT", "*")
    with pytest.raises(kb.KbError, match="kb_batch_run: injected fault"):
        b.run()
    with pytest.raises(kb.KbError, match="kb_batch_run_graph: injected fault"):
        b.run(graph=True)
    monkeypatch.delenv("KB_FAULT_INJECT")
    got = b.run(graph=True)[0]
    ref = kb.search(gpsi, gphi, times, gvx, gvy, sp)
    torch.cuda.synchronize()
    for key in ("idx", "nvalid", "nkept", "mask"):
        assert torch.equal(got[key], ref[key]), key
    assert torch.equal(got["lh"].view(torch.int32), ref["lh"].view(torch.int32))
    o = oracle.search(psi, phi, times, vx, vy, dict(k=2, lh_min=2.0, min_obs=3))
    compare_search(gpu_result_numpy(ref), o, sp.lh_min)
