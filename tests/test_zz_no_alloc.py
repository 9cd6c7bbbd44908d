"""kb_search_no_alloc, the search for callers that must not allocate device memory.

Callers such as a plug-in inside a host program whose device memory belongs to another allocator,
or code that must keep a fixed device footprint after start-up, cannot call cudaMalloc or pass a
workspace.  kb_search_no_alloc uses scratch memory built into the library instead.  This test calls
it through the C ABI twice in a row, on different inputs (the second call finds the first call's
data in the shared scratch), and checks each result against kb_search with a workspace, under the
same tolerance the parity tests use.  It also checks that a size beyond the built-in scratch is
refused.  It lives in its own file, collected last, and passes alone or after the other tests.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import paper_2109_03296_b300 as kb
from paper_2109_03296_b300 import _lib

pytestmark = pytest.mark.gpu


def _case(seed, T, H, W, n_traj):
    rng = np.random.default_rng(seed)
    times = np.sort(rng.uniform(0, 1.0, T))
    times[0] = 0.0
    phi = rng.uniform(0.2, 1.5, (T, H, W))
    psi = rng.normal(size=(T, H, W)) * np.sqrt(phi)
    psi += 3.0 * phi * (rng.random((T, H, W)) < 0.05)
    m = rng.random((T, H, W)) < 0.05
    psi[m] = 0.0
    phi[m] = 0.0
    vx = rng.uniform(-40, 40, n_traj).astype(np.float32)
    vy = rng.uniform(-40, 40, n_traj).astype(np.float32)
    vx[7], vy[7] = vx[2], vy[2]
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return d(psi.astype(np.float32)), d(phi.astype(np.float32)), times, d(vx), d(vy)


def _assert_same(a, b):
    for key in ("idx", "nvalid", "nkept", "mask"):
        assert torch.equal(a[key], b[key]), key
    la, lb = a["lh"].cpu().numpy(), b["lh"].cpu().numpy()
    f = a["idx"].cpu().numpy() >= 0
    assert np.array_equal(np.isneginf(la), np.isneginf(lb))
    assert np.all(np.abs(la[f] - lb[f]) <= 1e-4 * np.maximum(np.abs(lb[f]), 1.0))
    fa, fb = a["flux"].cpu().numpy()[f], b["flux"].cpu().numpy()[f]
    scale = np.abs(fb) * np.maximum(1.0, 1.0 / np.maximum(np.abs(lb[f]), 1e-30))
    assert np.all(np.abs(fa - fb) <= 1e-4 * np.maximum(scale, 1e-30))


def test_no_alloc_matches_workspace_search_twice(cuda_device):
    cases = [(31, 13, 101, 77, 70, kb.SearchParams(k=4, lh_min=1.5, min_obs=3)),
             (32, 40, 65, 40, 50, kb.SearchParams(k=3, lh_min=2.0, min_obs=10, clip_on=1))]
    filled = 0
    for seed, T, H, W, n, sp in cases:
        psi, phi, times, vx, vy = _case(seed, T, H, W, n)
        ref = kb.search(psi, phi, times, vx, vy, sp)
        got = kb.search_no_alloc(psi, phi, times, vx, vy, sp)
        torch.cuda.synchronize()
        _assert_same(got, ref)
        # the built-in scratch's counters: no device-side wait gave up, every pair was covered
        st = kb.search_no_alloc_stats()
        assert st[3] == 0 and st[0] == H * W * n * T == kb.search_stats(ref["workspace"])[0]
        filled += int((got["idx"] >= 0).sum())
    assert filled > 100


def test_no_alloc_refuses_sizes_beyond_its_scratch(cuda_device):
    # workspace need for 26 x 2046 x 4094 is ~2.6 GB, far above the built-in 32 MiB
    sp = _lib.SearchParamsC()
    _lib.lib().kb_search_params_default(C.byref(sp), 2046, 4094)
    need = C.c_size_t()
    assert _lib.lib().kb_search_workspace_size(26, 2046, 4094, 32768, C.byref(sp),
                                              C.byref(need)) == 0
    assert need.value > _lib.KB_STATIC_SCRATCH_BYTES
    times = np.linspace(0.0, 3.0, 26)
    dummy = torch.zeros(16, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    rc = _lib.lib().kb_search_no_alloc(p, p, times.ctypes.data_as(C.c_void_p), 26, 2046, 4094,
                                       p, p, 32768, C.byref(sp), p, p, p, p, p, p, None)
    assert rc == _lib.KB_ERR_UNSUPPORTED
    assert "built into the library" in _lib.lib().kb_last_error().decode()
