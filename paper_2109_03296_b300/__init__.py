"""B300-native KBMOD shift-and-stack search with the in-line sigma-G clip (arXiv 2109.03296).

Thin Python binding over libkb_b300.so (C ABI in include/kb.h): it checks tensors, passes
device pointers and the current CUDA stream, and allocates outputs/workspaces with torch.
Every step of the computation runs in the library's sm_103a kernels; CPU tensors are rejected.

    psi, phi = make_psi_phi(img, var, mask, psf)                  # Section 3
    res = search(psi, phi, times, vx, vy, SearchParams(...))      # Sections 3, 3.1, 3.2
    pix, slot, count = collect(res, n_max)                        # GPU -> host handoff
    mean, median = stamps(img, var, mask, times, x0, y0, vx, vy)  # Section 3.3
"""
import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from ._lib import (KB_MAX_K, KB_MAX_T, KB_WORKSPACE_ALIGN, KbError, SearchParamsC, check, lib)

__all__ = ["SearchParams", "make_psi_phi", "search", "search_workspace_size", "search_stats",
           "stamps", "collect", "candidate_tracks", "launch_count", "profile_events", "KbError",
           "search_no_alloc",
           "KB_MAX_T", "KB_MAX_K", "lib", "version", "alloc_workspace"]


def version():
    return lib().kb_version()


@dataclass
class SearchParams:
    """kb_search_params (include/kb.h).  Defaults are the paper's settings (Sections 3.1-3.2)."""
    k: int = 8
    lh_min: float = 10.0
    min_obs: int = 15
    clip: int = 1
    q_lo: float = 0.25
    q_mid: float = 0.5
    q_hi: float = 0.75
    n_sigma: float = 2.0
    clip_on: int = 0
    window: tuple = None          # (x_lo, x_hi, y_lo, y_hi); None = whole image

    def to_c(self, H, W):
        x_lo, x_hi, y_lo, y_hi = self.window if self.window is not None else (0, W, 0, H)
        return SearchParamsC(int(self.k), float(self.lh_min), int(self.min_obs), int(self.clip),
                             float(self.q_lo), float(self.q_mid), float(self.q_hi),
                             float(self.n_sigma), int(self.clip_on), int(x_lo), int(x_hi),
                             int(y_lo), int(y_hi))


def _dev(t, dtype, name, ndim=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % name)
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor (no CPU path)" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if ndim is not None and t.dim() != ndim:
        raise ValueError("%s must have %d dims" % (name, ndim))
    return t


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _host_times(times):
    if isinstance(times, torch.Tensor):
        times = times.detach().cpu().numpy()
    return np.ascontiguousarray(times, dtype=np.float64)


def alloc_workspace(nbytes, device):
    """A device byte buffer whose data pointer is KB_WORKSPACE_ALIGN-aligned."""
    buf = torch.empty(int(nbytes) + KB_WORKSPACE_ALIGN, dtype=torch.uint8, device=device)
    off = (-buf.data_ptr()) % KB_WORKSPACE_ALIGN
    return buf[off:off + int(nbytes)]


def make_psi_phi(img, var, mask, psf, psi=None, phi=None, stream=None):
    """psi_t = (I_t/var_t) correlated with PSF_t, phi_t = (1/var_t) correlated with PSF_t^2."""
    _dev(img, torch.float32, "img", 3)
    _dev(var, torch.float32, "var", 3)
    _dev(psf, torch.float32, "psf", 3)
    if mask is not None:
        _dev(mask, torch.uint8, "mask", 3)
    T, H, W = img.shape
    if psi is None:
        psi = torch.empty_like(img)
    if phi is None:
        phi = torch.empty_like(img)
    check(lib().kb_make_psi_phi(_ptr(img), _ptr(var), _ptr(mask), _ptr(psf), T, H, W,
                                psf.shape[-1], _ptr(psi), _ptr(phi), _stream(stream)))
    return psi, phi


def search_workspace_size(T, H, W, n_traj, params):
    n = C.c_size_t(0)
    pc = params.to_c(H, W)
    check(lib().kb_search_workspace_size(T, H, W, n_traj, C.byref(pc), C.byref(n)))
    return n.value


def search(psi, phi, times, vx, vy, params=None, workspace=None, out=None, stream=None):
    """Exhaustive search with the in-line sigma-G clip and per-pixel top-K.

    Returns a dict of device tensors lh, flux [wy, wx, K], idx int32, nvalid/nkept int16
    (uint16 data), mask int32 [wy, wx, K, ceil(T/32)] (uint32 bits), plus 'workspace'."""
    params = params or SearchParams()
    _dev(psi, torch.float32, "psi", 3)
    _dev(phi, torch.float32, "phi", 3)
    _dev(vx, torch.float32, "vx", 1)
    _dev(vy, torch.float32, "vy", 1)
    T, H, W = psi.shape
    times = _host_times(times)
    pc = params.to_c(H, W)
    K = pc.k_per_pixel
    wy, wx = pc.y_hi - pc.y_lo, pc.x_hi - pc.x_lo
    mw = (T + 31) // 32
    dev = psi.device
    if out is None:
        out = dict(lh=torch.empty((wy, wx, K), dtype=torch.float32, device=dev),
                   flux=torch.empty((wy, wx, K), dtype=torch.float32, device=dev),
                   idx=torch.empty((wy, wx, K), dtype=torch.int32, device=dev),
                   nvalid=torch.empty((wy, wx, K), dtype=torch.int16, device=dev),
                   nkept=torch.empty((wy, wx, K), dtype=torch.int16, device=dev),
                   mask=torch.empty((wy, wx, K, mw), dtype=torch.int32, device=dev))
    if workspace is None:
        workspace = alloc_workspace(search_workspace_size(T, H, W, vx.numel(), params), dev)
    check(lib().kb_search(_ptr(psi), _ptr(phi), times.ctypes.data_as(C.c_void_p), T, H, W,
                          _ptr(vx), _ptr(vy), vx.numel(), C.byref(pc), _ptr(out["lh"]),
                          _ptr(out["flux"]), _ptr(out["idx"]), _ptr(out["nvalid"]),
                          _ptr(out["nkept"]), _ptr(out["mask"]), _ptr(workspace),
                          workspace.numel(), _stream(stream)))
    out["workspace"] = workspace
    return out


def search_stats(workspace, stream=None):
    """(trajectory-epochs, full evaluations, insertions, device error flags) of the last search
    that used this workspace.  Synchronises the stream."""
    arr = (C.c_ulonglong * 4)()
    check(lib().kb_search_stats(_ptr(workspace), arr, _stream(stream)))
    return tuple(int(v) for v in arr)


def stamps(img, var, mask, times, x0, y0, vx, vy, radius=10, keep_mask=None, stream=None):
    """Mean and median coadded stamps [n, 2r+1, 2r+1] along integer-pixel trajectories."""
    _dev(img, torch.float32, "img", 3)
    _dev(var, torch.float32, "var", 3)
    if mask is not None:
        _dev(mask, torch.uint8, "mask", 3)
    _dev(x0, torch.int32, "x0", 1)
    _dev(y0, torch.int32, "y0", 1)
    _dev(vx, torch.float32, "vx", 1)
    _dev(vy, torch.float32, "vy", 1)
    if keep_mask is not None:
        _dev(keep_mask, torch.int32, "keep_mask")
    T, H, W = img.shape
    n = x0.numel()
    side = 2 * radius + 1
    mean = torch.empty((n, side, side), dtype=torch.float32, device=img.device)
    med = torch.empty((n, side, side), dtype=torch.float32, device=img.device)
    times = _host_times(times)
    check(lib().kb_stamps(_ptr(img), _ptr(var), _ptr(mask), times.ctypes.data_as(C.c_void_p),
                          T, H, W, _ptr(x0), _ptr(y0), _ptr(vx), _ptr(vy), _ptr(keep_mask), n,
                          radius, _ptr(mean), _ptr(med), _stream(stream)))
    return mean, med


def collect(result, n_max, workspace=None, stream=None):
    """Best n_max filled slots of a search result, ordered by LH' desc, pixel, slot.

    Returns (cand_pix int32 [n_max] (window row-major index, -1 past the end), cand_slot,
    count int32 [1] = total filled slots), all on the device."""
    lh, idx = result["lh"], result["idx"]
    wy, wx, K = lh.shape
    npix = wy * wx
    dev = lh.device
    if workspace is None:
        n = C.c_size_t(0)
        check(lib().kb_collect_workspace_size(int(n_max), C.byref(n)))
        workspace = alloc_workspace(n.value, dev)
    pix = torch.empty(n_max, dtype=torch.int32, device=dev)
    slot = torch.empty(n_max, dtype=torch.int32, device=dev)
    count = torch.empty(1, dtype=torch.int32, device=dev)
    check(lib().kb_collect(_ptr(lh), _ptr(idx), npix, K, int(n_max), _ptr(pix), _ptr(slot),
                           _ptr(count), _ptr(workspace), workspace.numel(), _stream(stream)))
    return pix, slot, count


def candidate_tracks(pix, slot, result, vx, vy, window=None, stream=None):
    """(x0, y0, vx, vy, traj) device tensors of collected survivors, for stamps()."""
    idx = result["idx"]
    wy, wx, K = idx.shape
    x_lo, y_lo = (0, 0) if window is None else (window[0], window[2])
    n = pix.numel()
    dev = idx.device
    x0 = torch.empty(n, dtype=torch.int32, device=dev)
    y0 = torch.empty(n, dtype=torch.int32, device=dev)
    ovx = torch.empty(n, dtype=torch.float32, device=dev)
    ovy = torch.empty(n, dtype=torch.float32, device=dev)
    traj = torch.empty(n, dtype=torch.int32, device=dev)
    check(lib().kb_candidate_tracks(_ptr(pix), _ptr(slot), n, _ptr(idx), K, _ptr(vx), _ptr(vy),
                                    int(x_lo), int(y_lo), wx, _ptr(x0), _ptr(y0), _ptr(ovx),
                                    _ptr(ovy), _ptr(traj), _stream(stream)))
    return x0, y0, ovx, ovy, traj


def launch_count():
    """Kernels launched by the library in this process so far."""
    return int(lib().kb_launch_count())


def profile_events(start=None, stop=None):
    """Time the next searches' main kernel with these torch.cuda.Events (None, None: off)."""
    lib().kb_profile_events(None if start is None else C.c_void_p(start.cuda_event),
                            None if stop is None else C.c_void_p(stop.cuda_event))


def search_no_alloc(psi, phi, times, vx, vy, params=None, out=None, stream=None):
    """kb_search_no_alloc: the search with the library's built-in scratch instead of a workspace,
    for callers that must not allocate device memory.  Same results as search(); the outputs
    (`out`, same layout as search() returns) may be passed in so that the call allocates
    nothing.  Sizes beyond the built-in scratch raise KbError (KB_ERR_UNSUPPORTED)."""
    params = params or SearchParams()
    _dev(psi, torch.float32, "psi", 3)
    _dev(phi, torch.float32, "phi", 3)
    _dev(vx, torch.float32, "vx", 1)
    _dev(vy, torch.float32, "vy", 1)
    T, H, W = psi.shape
    times = _host_times(times)
    pc = params.to_c(H, W)
    K = pc.k_per_pixel
    wy, wx = pc.y_hi - pc.y_lo, pc.x_hi - pc.x_lo
    mw = (T + 31) // 32
    dev = psi.device
    if out is None:
        out = dict(lh=torch.empty((wy, wx, K), dtype=torch.float32, device=dev),
                   flux=torch.empty((wy, wx, K), dtype=torch.float32, device=dev),
                   idx=torch.empty((wy, wx, K), dtype=torch.int32, device=dev),
                   nvalid=torch.empty((wy, wx, K), dtype=torch.int16, device=dev),
                   nkept=torch.empty((wy, wx, K), dtype=torch.int16, device=dev),
                   mask=torch.empty((wy, wx, K, mw), dtype=torch.int32, device=dev))
    check(lib().kb_search_no_alloc(_ptr(psi), _ptr(phi), times.ctypes.data_as(C.c_void_p), T, H,
                                   W, _ptr(vx), _ptr(vy), vx.numel(), C.byref(pc),
                                   _ptr(out["lh"]), _ptr(out["flux"]), _ptr(out["idx"]),
                                   _ptr(out["nvalid"]), _ptr(out["nkept"]), _ptr(out["mask"]),
                                   _stream(stream)))
    return out
