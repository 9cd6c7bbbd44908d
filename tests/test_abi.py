"""CPU-side checks of the C ABI: the library loads, exports every entry point include/kb.h
declares, and rejects bad arguments on the host (before any CUDA call)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2109_03296_b300 import build
    build.build()
    from paper_2109_03296_b300._lib import lib
    return lib()


def header_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"KB_API\s+[\w\s\*]+?\b(kb_\w+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(L):
    from paper_2109_03296_b300._lib import EXPORTS
    names = header_symbols()
    assert len(names) >= 13
    assert names == set(EXPORTS)
    for n in names:
        assert hasattr(L, n), n


def test_checked_build_exports_the_same_symbols():
    """libkb_b300_checked.so (the search kernel with KB_BOUNDS_CHECK=1) is the same C ABI."""
    from paper_2109_03296_b300 import _lib, build
    if not os.path.exists(build.LIB_CHECKED):
        build.build(checked=True)
    Lc = C.CDLL(build.LIB_CHECKED)
    for n in header_symbols():
        assert hasattr(Lc, n), n
    Lc.kb_version.restype = C.c_int
    assert Lc.kb_version() == _lib.lib().kb_version()


def test_version_and_defaults(L):
    from paper_2109_03296_b300._lib import SearchParamsC
    assert L.kb_version() >= 100
    p = SearchParamsC()
    L.kb_search_params_default(C.byref(p), 2046, 4094)
    assert (p.k_per_pixel, p.lh_min, p.min_obs, p.clip) == (8, 10.0, 15, 1)
    assert (p.q_lo, p.q_mid, p.q_hi, p.n_sigma, p.clip_on) == (0.25, 0.5, 0.75, 2.0, 0)
    assert (p.x_lo, p.x_hi, p.y_lo, p.y_hi) == (0, 4094, 0, 2046)
    assert p.bound_rows == 0


def _params(L, H=64, W=64, **kw):
    from paper_2109_03296_b300._lib import SearchParamsC
    p = SearchParamsC()
    L.kb_search_params_default(C.byref(p), H, W)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


FAKE = C.c_void_p(0x10000)   # never dereferenced: validation fails before any use


def _search(L, T=10, H=64, W=64, n=16, times=None, p=None, ws=FAKE, wsb=1 << 40, psi=FAKE):
    if times is None:
        times = np.linspace(0, 1, T)
    times = np.ascontiguousarray(times, np.float64)
    p = p or _params(L, H, W)
    return L.kb_search(psi, FAKE, times.ctypes.data_as(C.c_void_p), T, H, W, FAKE, FAKE, n,
                       C.byref(p), FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, ws, wsb, None)


def test_search_rejects_bad_arguments(L):
    from paper_2109_03296_b300 import _lib as K
    assert _search(L, psi=None) == K.KB_ERR_INVALID_ARG
    assert _search(L, T=0) == K.KB_ERR_INVALID_ARG
    assert _search(L, T=129) == K.KB_ERR_UNSUPPORTED
    assert _search(L, n=0) == K.KB_ERR_INVALID_ARG
    t = np.linspace(0, 1, 10)
    t[3] = np.nan
    assert _search(L, times=t) == K.KB_ERR_INVALID_ARG
    assert _search(L, p=_params(L, k_per_pixel=0)) == K.KB_ERR_INVALID_ARG
    assert _search(L, p=_params(L, k_per_pixel=33)) == K.KB_ERR_INVALID_ARG
    assert _search(L, p=_params(L, q_lo=0.8)) == K.KB_ERR_INVALID_ARG
    assert _search(L, p=_params(L, q_lo=0.0)) == K.KB_ERR_INVALID_ARG
    assert _search(L, p=_params(L, n_sigma=float("nan"))) == K.KB_ERR_INVALID_ARG
    assert _search(L, p=_params(L, x_hi=65)) == K.KB_ERR_INVALID_ARG
    assert _search(L, p=_params(L, bound_rows=3)) == K.KB_ERR_INVALID_ARG
    assert _search(L, p=_params(L, bound_rows=-1)) == K.KB_ERR_INVALID_ARG
    assert _search(L, p=_params(L, y_lo=10, y_hi=10)) == K.KB_ERR_INVALID_ARG
    assert _search(L, p=_params(L, clip_on=2)) == K.KB_ERR_INVALID_ARG
    assert _search(L, p=_params(L, min_obs=-1)) == K.KB_ERR_INVALID_ARG
    assert "window" in L.kb_last_error().decode() or "min_obs" in L.kb_last_error().decode()
    # too-small or misaligned workspace
    assert _search(L, ws=None) == K.KB_ERR_WORKSPACE
    assert _search(L, wsb=16) == K.KB_ERR_WORKSPACE
    assert _search(L, ws=C.c_void_p(0x10010)) == K.KB_ERR_WORKSPACE


def test_workspace_size_query(L):
    p = _params(L, 2046, 4094)
    n = C.c_size_t()
    assert L.kb_search_workspace_size(26, 2046, 4094, 32768, C.byref(p), C.byref(n)) == 0
    # dominated by the [T][H+3][Wp] bound planes (Wp = 4096), the interleaved (psi, phi) planes
    # [T][H][W] of 8-byte pairs and the evaluation records (256 blocks x 2048 x 32 bytes)
    planes = 26 * 2049 * 4096 * 4 + 26 * 2046 * 4094 * 8 + 256 * 2048 * 32
    assert planes < n.value < planes + 32 * 2 ** 20
    assert L.kb_search_workspace_size(200, 10, 10, 5, C.byref(p), C.byref(n)) == 2


def test_other_entry_points_validate(L):
    from paper_2109_03296_b300 import _lib as K
    times = np.linspace(0, 1, 5)
    tp = times.ctypes.data_as(C.c_void_p)
    arr = (C.c_ulonglong * 4)()
    assert L.kb_smem_probe(0, 10, FAKE, None) == K.KB_ERR_INVALID_ARG
    assert L.kb_smem_probe(4, 0, FAKE, None) == K.KB_ERR_INVALID_ARG
    assert L.kb_smem_probe(4, 10, None, None) == K.KB_ERR_INVALID_ARG
    assert L.kb_search_stage_counts(None, arr, None) == K.KB_ERR_INVALID_ARG
    assert L.kb_search_stage_counts(FAKE, None, None) == K.KB_ERR_INVALID_ARG
    assert L.kb_search_pass_counts(None, arr, None) == K.KB_ERR_INVALID_ARG
    assert L.kb_search_pass_counts(FAKE, None, None) == K.KB_ERR_INVALID_ARG
    assert L.kb_batch_pass_counts(None, arr, None) == K.KB_ERR_INVALID_ARG
    assert L.kb_search_no_alloc_stats(None, None) == K.KB_ERR_INVALID_ARG
    assert L.kb_make_psi_phi(FAKE, FAKE, None, FAKE, 5, 10, 10, 4, FAKE, FAKE, None) == \
        K.KB_ERR_INVALID_ARG
    assert L.kb_make_psi_phi(FAKE, FAKE, None, FAKE, 5, 10, 10, 33, FAKE, FAKE, None) == \
        K.KB_ERR_INVALID_ARG
    assert L.kb_make_psi_phi(None, FAKE, None, FAKE, 5, 10, 10, 3, FAKE, FAKE, None) == \
        K.KB_ERR_INVALID_ARG
    assert L.kb_stamps(FAKE, FAKE, None, tp, 5, 10, 10, FAKE, FAKE, FAKE, FAKE, None, 3, 16,
                       FAKE, FAKE, None) == K.KB_ERR_INVALID_ARG
    assert L.kb_stamps(FAKE, FAKE, None, tp, 200, 10, 10, FAKE, FAKE, FAKE, FAKE, None, 3, 10,
                       FAKE, FAKE, None) == K.KB_ERR_UNSUPPORTED
    # zero candidates: nothing to do, no CUDA call
    assert L.kb_stamps(FAKE, FAKE, None, tp, 5, 10, 10, None, None, None, None, None, 0, 10,
                       FAKE, FAKE, None) == K.KB_OK
    n = C.c_size_t()
    assert L.kb_collect_workspace_size(0, C.byref(n)) == K.KB_ERR_INVALID_ARG
    assert L.kb_collect_workspace_size(10000, C.byref(n)) == 0 and n.value >= 16384 * 8
    assert L.kb_collect(FAKE, FAKE, 100, 0, 10, FAKE, FAKE, FAKE, FAKE, 1 << 30, None) == \
        K.KB_ERR_INVALID_ARG
    assert L.kb_collect(FAKE, FAKE, 100, 8, 10, FAKE, FAKE, FAKE, FAKE, 8, None) == \
        K.KB_ERR_WORKSPACE
    assert L.kb_candidate_tracks(FAKE, FAKE, 0, FAKE, 8, FAKE, FAKE, 0, 0, 10, FAKE, FAKE, FAKE,
                                 FAKE, FAKE, None) == K.KB_OK


def test_binding_rejects_cpu_tensors():
    import torch
    import paper_2109_03296_b300 as kb
    x = torch.zeros((2, 4, 4))
    with pytest.raises(ValueError, match="CUDA"):
        kb.make_psi_phi(x, x, None, torch.zeros((2, 3, 3)))
    with pytest.raises(ValueError, match="CUDA"):
        kb.search(x, x, np.zeros(2), torch.zeros(3), torch.zeros(3))


def test_comparison_harness_catches_planted_mistakes():
    """Plants mistakes in oracle outputs (CPU) and checks the parity comparison rejects them."""
    import oracle
    from helpers import compare_search
    rng = np.random.default_rng(0)
    T, H, W = 6, 12, 14
    times = np.sort(rng.uniform(0, 1, T))
    phi = rng.uniform(0.2, 1.5, (T, H, W))
    psi = rng.normal(size=(T, H, W)) * np.sqrt(phi) + 2.0 * phi * (rng.random((T, H, W)) < 0.2)
    vx = rng.uniform(-6, 6, 30).astype(np.float32)
    vy = rng.uniform(-6, 6, 30).astype(np.float32)
    o = oracle.search(psi, phi, times, vx, vy, dict(k=3, lh_min=0.5, min_obs=2))
    g = {k: v.copy() for k, v in o.items()}
    assert compare_search(g, o, 0.5) == 0
    f = np.argwhere(o["idx"][..., 1] >= 0)[0]
    for plant in ("idx", "lh", "flux", "mask", "nkept"):
        g = {k: v.copy() for k, v in o.items()}
        y, x = f
        if plant == "idx":
            g["idx"][y, x, 0], g["idx"][y, x, 1] = o["idx"][y, x, 1], o["idx"][y, x, 0]
        elif plant == "lh":
            g["lh"][y, x, 0] *= 1.001
        elif plant == "flux":
            g["flux"][y, x, 0] *= -1.0
        elif plant == "mask":
            g["mask"][y, x, 0, 0] ^= 1
        else:
            g["nkept"][y, x, 0] += 1
        with pytest.raises(AssertionError):
            compare_search(g, o, 0.5)


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs have the C sizes and field offsets (gcc)."""
    import ctypes as C
    import subprocess
    from paper_2109_03296_b300 import _lib
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "layout.c"
    src.write_text(r"""
#include <stddef.h>
#include <stdio.h>
#include "kb.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(kb_search_params), sizeof(kb_refine_params),
         sizeof(kb_schedule), sizeof(kb_stack));
  printf("%zu %zu %zu %zu %zu\n", offsetof(kb_stack, vx), offsetof(kb_stack, n_traj),
         offsetof(kb_stack, params), offsetof(kb_stack, out_lh), offsetof(kb_stack, out_mask));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(root, "include"), str(src), "-o",
                           str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split()
    sizes = [int(v) for v in out[:4]]
    offs = [int(v) for v in out[4:]]
    assert sizes == [C.sizeof(_lib.SearchParamsC), C.sizeof(_lib.RefineParamsC),
                     C.sizeof(_lib.ScheduleC), C.sizeof(_lib.StackC)]
    S = _lib.StackC
    assert offs == [S.vx.offset, S.n_traj.offset, S.params.offset, S.out_lh.offset,
                    S.out_mask.offset]


def test_bench_traffic_line_matches_library_version(L):
    """The bench's roofline carries the DRAM traffic measured on this library version (a line in
    profiles/search_kernel_decam.md); a kernel change without a new capture would leave it null."""
    import bench
    v = L.kb_version()
    assert bench.search_traffic(v, "decam") is not None
    assert bench.search_traffic(v, "decam_half") is not None


MISALIGNED = C.c_void_p(0x10004)   # 4 bytes past a 16-byte boundary; never dereferenced


def _err(L):
    return L.kb_last_error().decode()


def test_refine_entry_points_validate(L):
    from paper_2109_03296_b300 import _lib as K
    T = 5
    times = np.linspace(0, 1, T)
    tp = times.ctypes.data_as(C.c_void_p)

    def fwd(n=3, params=FAKE, out=FAKE, grad=None, T=T, H=10, W=10, t=tp, psi=FAKE):
        return L.kb_traj_eval_fwd(psi, FAKE, t, T, H, W, params, None, n, out, out, grad, None)

    assert fwd(n=0, out=None) == K.KB_OK            # nothing to do, no CUDA call
    assert fwd(psi=None) == K.KB_ERR_INVALID_ARG
    assert fwd(T=0) == K.KB_ERR_INVALID_ARG
    assert fwd(n=-1) == K.KB_ERR_INVALID_ARG
    assert fwd(params=None) == K.KB_ERR_INVALID_ARG
    assert fwd(out=None) == K.KB_ERR_INVALID_ARG
    assert fwd(H=(1 << 20) + 1) == K.KB_ERR_UNSUPPORTED
    long_times = np.linspace(0, 1, K.KB_MAX_T + 1)
    assert fwd(T=K.KB_MAX_T + 1, t=long_times.ctypes.data_as(C.c_void_p)) == K.KB_ERR_UNSUPPORTED
    bad = times.copy()
    bad[2] = np.inf
    assert fwd(t=bad.ctypes.data_as(C.c_void_p)) == K.KB_ERR_INVALID_ARG
    # rows of params and of the gradient are float4: a pointer off a 16-byte boundary is refused
    assert fwd(params=MISALIGNED) == K.KB_ERR_INVALID_ARG and "aligned" in _err(L)
    assert fwd(grad=MISALIGNED) == K.KB_ERR_INVALID_ARG and "out_grad" in _err(L)

    def bwd(n=3, params=FAKE, gp=None):
        return L.kb_traj_eval_bwd(FAKE, FAKE, tp, T, 10, 10, params, None, n, None, None, gp,
                                  FAKE, None, None)

    assert bwd(n=0) == K.KB_OK
    assert bwd(params=MISALIGNED) == K.KB_ERR_INVALID_ARG
    assert bwd(gp=MISALIGNED) == K.KB_ERR_INVALID_ARG and "out_grad_params" in _err(L)

    rp0 = K.RefineParamsC()
    L.kb_refine_params_default(C.byref(rp0))
    assert (rp0.n_steps, rp0.beta1, rp0.eps) == (20, np.float32(0.9), np.float32(1e-8))

    def refine(rp, n=3, params=FAKE):
        return L.kb_refine(FAKE, FAKE, tp, T, 10, 10, params, None, n,
                           None if rp is None else C.byref(rp), FAKE, FAKE, None, None)

    assert refine(rp0, n=0) == K.KB_OK
    assert refine(None) == K.KB_ERR_INVALID_ARG
    assert refine(rp0, params=MISALIGNED) == K.KB_ERR_INVALID_ARG
    for field, value in (("n_steps", -1), ("n_steps", 100001), ("lr_pos", float("nan")),
                         ("lr_vel", -0.1), ("lr_pos", float("inf")), ("beta1", 1.0),
                         ("beta2", -0.5), ("eps", 0.0), ("eps", float("inf"))):
        rp = K.RefineParamsC.from_buffer_copy(rp0)
        setattr(rp, field, value)
        assert refine(rp) == K.KB_ERR_INVALID_ARG, (field, value)

    def cand(n=3, K_=8, T_=T, out=FAKE, keep=None, mask=FAKE):
        return L.kb_candidate_params(FAKE, FAKE, n, FAKE, mask, K_, T_, FAKE, FAKE, 0, 0, 10, out,
                                     keep, None)

    assert cand(n=0) == K.KB_OK
    assert cand(K_=0) == K.KB_ERR_INVALID_ARG
    assert cand(K_=K.KB_MAX_K + 1) == K.KB_ERR_INVALID_ARG
    assert cand(T_=K.KB_MAX_T + 1) == K.KB_ERR_UNSUPPORTED
    assert cand(keep=FAKE, mask=None) == K.KB_ERR_INVALID_ARG
    assert cand(out=MISALIGNED) == K.KB_ERR_INVALID_ARG and "out_params" in _err(L)


def test_filter_and_cluster_validate(L):
    from paper_2109_03296_b300 import _lib as K
    lim = np.array([0.5, 0.5, 1.5, 36.5, 36.5], np.float32)

    def filt(n=3, radius=10, limits=None, stamps=FAKE, out=FAKE):
        lp = None if limits is None else limits.ctypes.data_as(C.c_void_p)
        return L.kb_stamp_filter(stamps, n, radius, lp, None, out, None)

    assert filt(n=0) == K.KB_OK
    assert filt(n=-1) == K.KB_ERR_INVALID_ARG
    assert filt(radius=-1) == K.KB_ERR_INVALID_ARG and filt(radius=16) == K.KB_ERR_INVALID_ARG
    assert filt(stamps=None) == K.KB_ERR_INVALID_ARG and filt(out=None) == K.KB_ERR_INVALID_ARG
    bad = lim.copy()
    bad[3] = np.nan
    assert filt(limits=bad) == K.KB_ERR_INVALID_ARG and "NaN" in _err(L)

    n = C.c_size_t()
    assert L.kb_cluster_workspace_size(-1, C.byref(n)) == K.KB_ERR_INVALID_ARG
    assert L.kb_cluster_workspace_size((1 << 24) + 1, C.byref(n)) == K.KB_ERR_UNSUPPORTED
    assert L.kb_cluster_workspace_size(1000, C.byref(n)) == K.KB_OK and n.value > 0
    need = n.value

    def clus(n=1000, dt=3.0, radius=4.0, x0=FAKE, ws=C.c_void_p(1 << 20), wsb=need, rounds=None):
        return L.kb_cluster(x0, FAKE, FAKE, FAKE, None, n, dt, radius, FAKE, FAKE, ws, wsb, rounds,
                            None)

    r = C.c_int(7)
    assert clus(n=0, rounds=C.byref(r)) == K.KB_OK and r.value == 0
    assert clus(n=-1) == K.KB_ERR_INVALID_ARG
    assert clus(n=(1 << 24) + 1) == K.KB_ERR_UNSUPPORTED
    assert clus(radius=0.5) == K.KB_ERR_INVALID_ARG
    assert clus(radius=float("nan")) == K.KB_ERR_INVALID_ARG
    assert clus(dt=float("inf")) == K.KB_ERR_INVALID_ARG
    assert clus(x0=None) == K.KB_ERR_INVALID_ARG
    assert clus(wsb=need - 1) == K.KB_ERR_WORKSPACE
    assert clus(ws=None) == K.KB_ERR_WORKSPACE
    assert clus(ws=C.c_void_p((1 << 20) + 16)) == K.KB_ERR_WORKSPACE


def test_batch_validates_its_stacks(L):
    from paper_2109_03296_b300 import _lib as K
    T, H, W, n_traj = 10, 64, 64, 256
    times = np.linspace(0, 1, T)

    def stack(**kw):
        s = K.StackC()
        for name in ("psi", "phi", "vx", "vy", "out_lh", "out_flux", "out_idx", "out_nvalid",
                     "out_nkept", "out_mask"):
            setattr(s, name, 0x10000)
        s.times = times.ctypes.data
        s.T, s.H, s.W, s.n_traj = T, H, W, n_traj
        L.kb_search_params_default(C.byref(s.params), H, W)
        for k, v in kw.items():
            if hasattr(s.params, k) and k not in ("T", "H", "W"):
                setattr(s.params, k, v)
            else:
                setattr(s, k, v)
        return s

    def size(*stacks):
        arr = (K.StackC * len(stacks))(*stacks)
        n = C.c_size_t()
        return L.kb_batch_workspace_size(arr, len(stacks), C.byref(n)), n.value

    rc, one = size(stack())
    assert rc == K.KB_OK
    ws1 = C.c_size_t()
    assert L.kb_search_workspace_size(T, H, W, n_traj, C.byref(stack().params), C.byref(ws1)) == 0
    assert one >= ws1.value
    rc, two = size(stack(), stack())
    assert rc == K.KB_OK and two >= 2 * ws1.value
    assert L.kb_batch_workspace_size(None, 1, C.byref(C.c_size_t())) == K.KB_ERR_INVALID_ARG
    arr = (K.StackC * 1)(stack())
    assert L.kb_batch_workspace_size(arr, 0, C.byref(C.c_size_t())) == K.KB_ERR_INVALID_ARG
    assert size(stack(), stack(T=0))[0] == K.KB_ERR_INVALID_ARG and "stack 1" in _err(L)
    assert size(stack(T=K.KB_MAX_T + 1))[0] == K.KB_ERR_UNSUPPORTED
    assert size(stack(n_traj=(1 << 24) + 1))[0] == K.KB_ERR_UNSUPPORTED

    def create(stacks, ws=C.c_void_p(1 << 30), wsb=None):
        arr = (K.StackC * len(stacks))(*stacks)
        h = C.c_void_p(0x1234)
        wsb = size(*stacks)[1] if wsb is None else wsb
        rc = L.kb_batch_create(arr, len(stacks), ws, wsb, C.byref(h))
        return rc, h.value

    assert L.kb_batch_create(arr, 1, C.c_void_p(1 << 30), 1 << 40, None) == K.KB_ERR_INVALID_ARG
    assert create([stack()], wsb=one - 1) == (K.KB_ERR_WORKSPACE, None)
    assert create([stack()], ws=C.c_void_p((1 << 30) + 64)) == (K.KB_ERR_WORKSPACE, None)
    # the checks of kb_search run on every stack before any device work; the message names it
    for kw in (dict(q_lo=0.8), dict(k_per_pixel=0), dict(bound_rows=3), dict(x_hi=W + 1),
               dict(out_mask=None), dict(psi=None)):
        rc, h = create([stack(**kw)])
        assert rc == K.KB_ERR_INVALID_ARG and h is None, kw
        assert "stack 0" in _err(L), kw


def test_host_fault_injection(L, monkeypatch):
    """KB_FAULT_INJECT makes the named entry points fail with KB_ERR_CUDA after their argument
    checks and before any device work (valid arguments, device pointers never dereferenced)."""
    from paper_2109_03296_b300 import _lib as K
    T = 5
    times = np.linspace(0, 1, T)
    tp = times.ctypes.data_as(C.c_void_p)
    ws = C.c_void_p(1 << 20)
    nb = C.c_size_t()
    assert L.kb_collect_workspace_size(10, C.byref(nb)) == K.KB_OK
    collect_ws = nb.value
    assert L.kb_cluster_workspace_size(8, C.byref(nb)) == K.KB_OK
    cluster_ws = nb.value
    rp = K.RefineParamsC()
    L.kb_refine_params_default(C.byref(rp))
    sp_ = _params(L, 10, 10)
    calls = {
        "kb_search_no_alloc": lambda: L.kb_search_no_alloc(FAKE, FAKE, tp, T, 10, 10, FAKE, FAKE,
                                                           4, C.byref(sp_), FAKE, FAKE, FAKE,
                                                           FAKE, FAKE, FAKE, None),
        "kb_make_psi_phi": lambda: L.kb_make_psi_phi(FAKE, FAKE, None, FAKE, T, 10, 10, 3,
                                                     C.c_void_p(0x20000), C.c_void_p(0x30000),
                                                     None),
        "kb_stamps": lambda: L.kb_stamps(FAKE, FAKE, None, tp, T, 10, 10, FAKE, FAKE, FAKE, FAKE,
                                         None, 3, 10, FAKE, FAKE, None),
        "kb_stamp_filter": lambda: L.kb_stamp_filter(FAKE, 3, 10, None, None, FAKE, None),
        "kb_collect": lambda: L.kb_collect(FAKE, FAKE, 100, 8, 10, FAKE, FAKE, FAKE, ws,
                                           collect_ws, None),
        "kb_candidate_tracks": lambda: L.kb_candidate_tracks(FAKE, FAKE, 3, FAKE, 8, FAKE, FAKE,
                                                             0, 0, 10, FAKE, FAKE, FAKE, FAKE,
                                                             FAKE, None),
        "kb_cluster": lambda: L.kb_cluster(FAKE, FAKE, FAKE, FAKE, None, 8, 3.0, 4.0, FAKE, FAKE,
                                           ws, cluster_ws, None, None),
        "kb_traj_eval_fwd": lambda: L.kb_traj_eval_fwd(FAKE, FAKE, tp, T, 10, 10, FAKE, None, 3,
                                                       FAKE, FAKE, None, None),
        "kb_traj_eval_bwd": lambda: L.kb_traj_eval_bwd(FAKE, FAKE, tp, T, 10, 10, FAKE, None, 3,
                                                       None, None, FAKE, None, None, None),
        "kb_refine": lambda: L.kb_refine(FAKE, FAKE, tp, T, 10, 10, FAKE, None, 3, C.byref(rp),
                                         FAKE, FAKE, None, None),
        "kb_candidate_params": lambda: L.kb_candidate_params(FAKE, FAKE, 3, FAKE, FAKE, 8, T, FAKE,
                                                             FAKE, 0, 0, 10, FAKE, None, None),
    }
    monkeypatch.setenv("KB_FAULT_INJECT", "*")
    for name, call in calls.items():
        assert call() == K.KB_ERR_CUDA, name
        assert _err(L) == "%s: injected fault (KB_FAULT_INJECT)" % name
    # argument errors still come first
    assert L.kb_collect(FAKE, FAKE, 100, 0, 10, FAKE, FAKE, FAKE, ws, collect_ws, None) == \
        K.KB_ERR_INVALID_ARG
    # a list names entry points exactly; the others are unaffected (here: nothing to do, n = 0)
    monkeypatch.setenv("KB_FAULT_INJECT", "kb_refine_x,kb_collect")
    assert calls["kb_collect"]() == K.KB_ERR_CUDA and "injected" in _err(L)
    assert L.kb_refine(FAKE, FAKE, tp, T, 10, 10, FAKE, None, 0, C.byref(rp), FAKE, FAKE, None,
                       None) == K.KB_OK
    monkeypatch.setenv("KB_FAULT_INJECT", "kb_refine")
    assert calls["kb_refine"]() == K.KB_ERR_CUDA and "injected" in _err(L)


def test_plain_c_program_links_and_calls_the_library(L, tmp_path):
    """The ABI is usable from C alone: a C11 program includes kb.h, links libkb_b300.so and calls
    the host-only entry points (defaults, workspace query, argument checks, error text)."""
    import subprocess
    from paper_2109_03296_b300 import _lib as K
    libdir = os.path.dirname(K.LIB_PATH)
    src = tmp_path / "use_kb.c"
    src.write_text(r"""
#include <stdio.h>
#include <string.h>
#include "kb.h"
int main(void) {
  kb_search_params p;
  size_t bytes = 0;
  kb_search_params_default(&p, 2046, 4094);
  if (p.k_per_pixel != 8 || p.min_obs != 15 || p.x_hi != 4094 || p.y_hi != 2046) return 1;
  if (kb_search_workspace_size(26, 2046, 4094, 32768, &p, &bytes) != KB_OK || bytes == 0) return 2;
  if (kb_search_workspace_size(KB_MAX_T + 1, 10, 10, 5, &p, &bytes) != KB_ERR_UNSUPPORTED)
    return 3;
  if (kb_make_psi_phi(NULL, NULL, NULL, NULL, 1, 1, 1, 1, NULL, NULL, NULL) != KB_ERR_INVALID_ARG)
    return 4;
  if (strstr(kb_last_error(), "kb_make_psi_phi") == NULL) return 5;
  printf("%d %zu\n", kb_version(), bytes);
  return 0;
}
""")
    exe = tmp_path / "use_kb"
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror",
                           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                           "-L", libdir, "-lkb_b300", "-Wl,-rpath," + libdir])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out
    v, nbytes = out.stdout.split()
    assert int(v) == L.kb_version()
    n = C.c_size_t()
    p = _params(L, 2046, 4094)
    assert L.kb_search_workspace_size(26, 2046, 4094, 32768, C.byref(p), C.byref(n)) == 0
    assert int(nbytes) == n.value


def test_no_alloc_scratch_holds_the_documented_sizes(L):
    """The built-in scratch of kb_search_no_alloc (32 MiB, of which the evaluation records take
    a fixed 16 MiB) holds T = 26 searches up to 212 x 212 pixels with 4096 trajectories and
    120 x 120 with 32768, and no larger squares."""
    from paper_2109_03296_b300 import _lib as K
    n = C.c_size_t()
    for side, n_traj in ((212, 4096), (120, 32768)):
        for s, fits in ((side, True), (side + 4, False)):
            p = _params(L, s, s)
            assert L.kb_search_workspace_size(26, s, s, n_traj, C.byref(p), C.byref(n)) == 0
            assert (n.value <= K.KB_STATIC_SCRATCH_BYTES) == fits, (s, n_traj, n.value)
    p = _params(L, 64, 64)
    assert L.kb_search_workspace_size(26, 64, 64, 1, C.byref(p), C.byref(n)) == 0
    assert n.value > 16 * 2 ** 20          # the records alone


def test_missing_library_fails_loudly(monkeypatch):
    """No fallback: without libkb_b300.so every call into the binding raises."""
    import paper_2109_03296_b300 as kb
    from paper_2109_03296_b300 import _lib as K
    monkeypatch.setattr(K, "LIB_PATH", os.path.join(ROOT, "no_such_dir", "libkb_b300.so"))
    monkeypatch.setattr(K, "_LIB", None)
    with pytest.raises(ImportError, match="not built"):
        K.lib()
    with pytest.raises(ImportError):
        kb.version()
    with pytest.raises(ImportError):
        kb.launch_count()


def test_product_and_oracle_share_no_code():
    """The package never imports the oracle, the oracle never imports the package or includes its
    headers, and neither reads the other's sources."""
    pkg = os.path.join(ROOT, "paper_2109_03296_b300")
    orc = os.path.join(ROOT, "oracle")
    for folder, banned in ((pkg, ("import oracle", "from oracle", "kb_oracle", "libkb_oracle")),
                           (orc, ("import paper_2109_03296_b300", "from paper_2109_03296_b300",
                                  "kb.h\"", "csrc/", "libkb_b300"))):
        for dirpath, _, files in os.walk(folder):
            if "_build" in dirpath or "__pycache__" in dirpath:
                continue
            for f in files:
                if not f.endswith((".py", ".c", ".h", ".cu", ".cuh")):
                    continue
                text = open(os.path.join(dirpath, f)).read()
                for b in banned:
                    assert b not in text, (f, b)


def test_header_is_clean_c_and_cxx(tmp_path):
    """include/kb.h compiles warning-free as C11 and C++17 (-Wall -Wextra -Wpedantic)."""
    import subprocess
    inc = os.path.join(ROOT, "include")
    for lang, compiler, std, ext in (("c", "gcc", "-std=c11", ".c"),
                                     ("c++", "g++", "-std=c++17", ".cpp")):
        src = tmp_path / ("h" + ext)
        src.write_text('#include "kb.h"\nint main(void) { return KB_OK; }\n')
        subprocess.check_call([compiler, std, "-Wall", "-Wextra", "-Wpedantic", "-Werror",
                               "-I", inc, "-fsyntax-only", str(src)])


def test_comparison_harness_tolerance_edges():
    """The parity bar as the harness applies it: LH' and alpha within 1e-4 relative (LH' scale
    floored at 1) pass, just outside fail; counts, masks and empty slots are exact."""
    import oracle
    from helpers import compare_search
    rng = np.random.default_rng(1)
    T, H, W = 6, 12, 14
    times = np.sort(rng.uniform(0, 1, T))
    phi = rng.uniform(0.2, 1.5, (T, H, W))
    psi = rng.normal(size=(T, H, W)) * np.sqrt(phi) + 2.0 * phi * (rng.random((T, H, W)) < 0.2)
    vx = rng.uniform(-6, 6, 30).astype(np.float32)
    vy = rng.uniform(-6, 6, 30).astype(np.float32)
    o = oracle.search(psi, phi, times, vx, vy, dict(k=3, lh_min=0.5, min_obs=2))
    y, x = np.argwhere(o["idx"][..., 2] >= 0)[0]          # a pixel with three entries

    def planted(key, s, f):
        g = {k: v.copy() for k, v in o.items()}
        g[key][y, x, s] = f(g[key][y, x, s])
        return g

    L = o["lh"][y, x, 1]
    scale = max(abs(L), 1.0)
    assert compare_search(planted("lh", 1, lambda v: v + 0.9e-4 * scale), o, 0.5) == 0
    with pytest.raises(AssertionError):
        compare_search(planted("lh", 1, lambda v: v + 1.1e-4 * scale), o, 0.5)
    assert compare_search(planted("flux", 2, lambda v: v * (1 + 0.5e-4)), o, 0.5) == 0
    with pytest.raises(AssertionError):
        compare_search(planted("nvalid", 2, lambda v: v + 1), o, 0.5)
    with pytest.raises(AssertionError):
        compare_search(planted("mask", 2, lambda v: v ^ np.uint32(1 << (T - 1))), o, 0.5)
    e = np.argwhere(o["idx"] < 0)[0]
    g = {k: v.copy() for k, v in o.items()}
    g["lh"][tuple(e)] = 0.0                               # an empty slot must read -inf
    with pytest.raises(AssertionError):
        compare_search(g, o, 0.5)


def test_comparison_harness_clip_bound_rule():
    """Reading R6 for clip bounds: a kept-mask difference is accepted only for a trajectory whose
    lightcurve lies within 1e-5 max(sigma_G, |median|) of a clip bound (oracle.clip_margin), and
    then the GPU's LH' and alpha must be the sums over its own kept set.  Planted on the CPU in
    copies of oracle results."""
    import oracle
    from helpers import compare_search, search_ctx
    T = 5
    times = np.array([0.0, 0.1, 0.2, 0.3, 0.4])
    vx = np.zeros(1, np.float32)
    vy = np.zeros(1, np.float32)
    p = dict(k=1, lh_min=-1e9, min_obs=1, clip=1, q_lo=0.25, q_mid=0.5, q_hi=0.75, n_sigma=2.0)

    def planes(a4):
        psi = np.zeros((T, 3, 3))
        phi = np.ones((T, 3, 3))
        psi[:, 1, 1] = [0.0, 1.0, 2.0, 3.0, a4]
        return psi, phi

    upper = 2.0 + 2.0 * (oracle.sigma_g_coeff(0.25, 0.75) * 2.0)
    for a4, at_bound in ((upper, True), (4.0, False)):
        psi, phi = planes(a4)
        o = oracle.search(psi, phi, times, vx, vy, p)
        ctx = search_ctx(psi, phi, times, vx, vy, p)
        assert o["mask"][1, 1, 0, 0] == 0b11111
        g = {k: v.copy() for k, v in o.items()}
        g["mask"][1, 1, 0, 0] = 0b01111          # epoch 4 dropped
        g["nkept"][1, 1, 0] = 4
        g["lh"][1, 1, 0] = 6.0 / 2.0              # sum psi / sqrt(sum phi) over epochs 0..3
        g["flux"][1, 1, 0] = 6.0 / 4.0
        with pytest.raises(AssertionError):
            compare_search(g, o, p["lh_min"])     # no context: any mask difference fails
        if at_bound:
            counts = {}
            assert compare_search(g, o, p["lh_min"], ctx=ctx, counts=counts) == 1
            assert counts["clip_bound_mask"] == 1
            bad = {k: v.copy() for k, v in g.items()}
            bad["lh"][1, 1, 0] = o["lh"][1, 1, 0]   # values of the other kept set
            with pytest.raises(AssertionError):
                compare_search(bad, o, p["lh_min"], ctx=ctx)
        else:
            with pytest.raises(AssertionError, match="clip bound"):
                compare_search(g, o, p["lh_min"], ctx=ctx)
