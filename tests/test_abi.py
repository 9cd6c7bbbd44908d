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
    # dominated by the [T][H+1][Wp] bound planes (Wp = 4096) and the interleaved (psi, phi)
    # planes [T][H][W] of 8-byte pairs
    planes = 26 * 2047 * 4096 * 4 + 26 * 2046 * 4094 * 8
    assert planes < n.value < planes + 64 * 2 ** 20
    assert L.kb_search_workspace_size(200, 10, 10, 5, C.byref(p), C.byref(n)) == 2


def test_other_entry_points_validate(L):
    from paper_2109_03296_b300 import _lib as K
    times = np.linspace(0, 1, 5)
    tp = times.ctypes.data_as(C.c_void_p)
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
