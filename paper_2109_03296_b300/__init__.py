"""B300-native KBMOD shift-and-stack search with the in-line sigma-G clip (arXiv 2109.03296).

Thin Python binding over libkb_b300.so (C ABI in include/kb.h): it checks tensors, passes
device pointers and the current CUDA stream, and allocates outputs/workspaces with torch.
Every step of the computation runs in the library's sm_103a kernels; CPU tensors are rejected.

    psi, phi = make_psi_phi(img, var, mask, psf)                  # Section 3
    res = search(psi, phi, times, vx, vy, SearchParams(...))      # Sections 3, 3.1, 3.2
    batch = Batch([dict(psi=..., phi=..., times=..., vx=..., vy=..., params=...), ...])
    batch.run(graph=True); batch.results[i]                       # many stacks, one launch
    pix, slot, count = collect(res, n_max)                        # GPU -> host handoff
    mean, median = stamps(img, var, mask, times, x0, y0, vx, vy)  # Section 3.3
    moments, passed = stamp_filter(median)                        # Section 3.3 moment filter
    keep, rep = cluster(x0, y0, vx, vy, times, valid=passed)      # de-duplication (Fig. 3)
    params, keep = candidate_params(pix, slot, res, vx, vy)       # off-grid refinement:
    params, L, alpha, L0 = refine(psi, phi, times, params, keep)  #   Section 4.1, bilinear
    L, alpha = traj_likelihood(params, psi, phi, times, keep)     # differentiable (autograd)
"""
import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from ._lib import (KB_MAX_K, KB_MAX_T, KB_WORKSPACE_ALIGN, KbError, RefineParamsC, ScheduleC,
                   SearchParamsC, StackC, check, lib)

__all__ = ["SearchParams", "make_psi_phi", "search", "search_workspace_size", "search_stats",
           "stamps", "collect", "candidate_tracks", "launch_count", "profile_events", "KbError",
           "search_no_alloc", "RefineParams", "traj_eval", "traj_eval_backward", "TrajEval",
           "traj_likelihood", "refine", "candidate_params", "stamp_filter",
           "PAPER_MOMENT_LIMITS", "Schedule", "Batch", "cluster",
           "KB_MAX_T", "KB_MAX_K", "lib", "version", "alloc_workspace", "wait_check"]


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
    bound_rows: int = 0           # pruning bound per 1 or 2 start-pixel rows; 0 = automatic

    def to_c(self, H, W):
        x_lo, x_hi, y_lo, y_hi = self.window if self.window is not None else (0, W, 0, H)
        return SearchParamsC(int(self.k), float(self.lh_min), int(self.min_obs), int(self.clip),
                             float(self.q_lo), float(self.q_mid), float(self.q_hi),
                             float(self.n_sigma), int(self.clip_on), int(x_lo), int(x_hi),
                             int(y_lo), int(y_hi), int(self.bound_rows))


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
    _same_device([("psi", psi), ("phi", phi), ("vx", vx), ("vy", vy), ("workspace", workspace)]
                 + [("out[%s]" % k, v) for k, v in out.items() if k != "workspace"])
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


def search_stage_counts(workspace, stream=None):
    """Stage counts of the last search that used this workspace, over the pairs it evaluated in
    full: (n_valid >= min_obs, LH' >= lh_min after the clip, sum of n_kept and sum of n_valid over
    the latter).  Synchronises the stream."""
    arr = (C.c_ulonglong * 4)()
    check(lib().kb_search_stage_counts(_ptr(workspace), arr, _stream(stream)))
    return tuple(int(v) for v in arr)


def search_pass_counts(workspace, stream=None):
    """Shared-memory traffic of the last search that used this workspace: (bound words read,
    offsets read, bytes staged by TMA) in bytes, and iterations with direct global loads."""
    arr = (C.c_ulonglong * 4)()
    check(lib().kb_search_pass_counts(_ptr(workspace), arr, _stream(stream)))
    return tuple(int(v) for v in arr)


def search_no_alloc_stats(stream=None):
    """search_stats() of the last search_no_alloc() on the current device (stats[3] != 0: a
    device-side wait gave up and the lists may be partial)."""
    arr = (C.c_ulonglong * 4)()
    check(lib().kb_search_no_alloc_stats(arr, _stream(stream)))
    return tuple(int(v) for v in arr)


def _same_device(name_tensors):
    """Every tensor must live on the current CUDA device (the library launches there)."""
    cur = torch.cuda.current_device()
    for name, t in name_tensors:
        if t is not None and t.device.index != cur:
            raise ValueError("%s is on cuda:%s, the current device is cuda:%d"
                             % (name, t.device.index, cur))


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


PAPER_MOMENT_LIMITS = (0.5, 0.5, 1.5, 36.5, 36.5)   # x, y, xy, xx, yy (Section 3.3)


def stamp_filter(stamps_, limits=None, stream=None):
    """Central moments (M0, x, y, xy, xx, yy) [n, 6] of stamps [n, 2r+1, 2r+1] and the moment
    filter's decision [n] (bool tensor); limits default to the paper's."""
    _dev(stamps_, torch.float32, "stamps", 3)
    n, side, side2 = stamps_.shape
    if side != side2 or side % 2 != 1:
        raise ValueError("stamps must be [n, 2r+1, 2r+1]")
    mom = torch.empty((n, 6), dtype=torch.float32, device=stamps_.device)
    ok = torch.empty(n, dtype=torch.uint8, device=stamps_.device)
    lim = None
    if limits is not None:
        lim = (C.c_float * 5)(*[float(v) for v in limits])
    check(lib().kb_stamp_filter(_ptr(stamps_), n, side // 2, lim, _ptr(mom), _ptr(ok),
                                _stream(stream)))
    return mom, ok.view(torch.bool)


def cluster(x0, y0, vx, vy, times, radius=8.0, valid=None, workspace=None, stream=None,
            return_rounds=False):
    """De-duplicate candidates in index order (kb_cluster): (keep bool [n], rep int32 [n]).
    Two tracks are duplicates when they agree within `radius` pixels at the first and the last
    epoch of `times`.  Blocks the host until the result is final."""
    _dev(x0, torch.int32, "x0", 1)
    _dev(y0, torch.int32, "y0", 1)
    _dev(vx, torch.float32, "vx", 1)
    _dev(vy, torch.float32, "vy", 1)
    if valid is not None:
        if valid.dtype == torch.bool:
            valid = valid.view(torch.uint8)
        _dev(valid, torch.uint8, "valid", 1)
    n = x0.numel()
    t = _host_times(times)
    dt = float(t[-1] - t[0]) if len(t) else 0.0
    if workspace is None:
        nb = C.c_size_t(0)
        check(lib().kb_cluster_workspace_size(n, C.byref(nb)))
        workspace = alloc_workspace(nb.value, x0.device)
    keep = torch.empty(n, dtype=torch.uint8, device=x0.device)
    rep = torch.empty(n, dtype=torch.int32, device=x0.device)
    rounds = C.c_int(0)
    check(lib().kb_cluster(_ptr(x0), _ptr(y0), _ptr(vx), _ptr(vy), _ptr(valid), n, dt,
                           float(radius), _ptr(keep), _ptr(rep), _ptr(workspace),
                           workspace.numel(), C.byref(rounds), _stream(stream)))
    out = (keep.view(torch.bool), rep)
    return out + (rounds.value,) if return_rounds else out


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


def smem_read_bandwidth(iters=4000, device=None):
    """Shared-memory read bandwidth in GB/s from kb_smem_probe: conflict-free 32-bit loads, one
    128-byte wavefront each, from two 1024-thread blocks per SM (best of 3 timed calls after a
    warm-up)."""
    dev = torch.device("cuda") if device is None else device
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = sms * 2
    scratch = torch.zeros(blocks, dtype=torch.int32, device=dev)
    s = _stream(None)
    check(lib().kb_smem_probe(blocks, 200, _ptr(scratch), s))
    best = 0.0
    nbytes = blocks * 32 * iters * 32 * 128
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        check(lib().kb_smem_probe(blocks, iters, _ptr(scratch), s))
        e1.record()
        torch.cuda.synchronize()
        best = max(best, nbytes / (e0.elapsed_time(e1) / 1e3) / 1e9)
    return best


def l2_read_bandwidth(mbytes=64, reps=40, device=None):
    """L2 read bandwidth in GB/s from kb_l2_probe on a resident buffer of `mbytes` MB (best of 3
    timed calls after a warm-up)."""
    dev = torch.device("cuda") if device is None else device
    buf = torch.ones(mbytes * (1 << 20) // 4, dtype=torch.float32, device=dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = sms * 4
    scratch = torch.zeros(blocks, dtype=torch.float32, device=dev)
    s = _stream(None)
    check(lib().kb_l2_probe(_ptr(buf), buf.numel() * 4, 2, _ptr(scratch), blocks, s))
    best = 0.0
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        check(lib().kb_l2_probe(_ptr(buf), buf.numel() * 4, reps, _ptr(scratch), blocks, s))
        e1.record()
        torch.cuda.synchronize()
        best = max(best, buf.numel() * 4 * reps / (e0.elapsed_time(e1) / 1e3) / 1e9)
    return best


def launch_count():
    """Kernels launched by the library in this process so far."""
    return int(lib().kb_launch_count())


def wait_check(limit_ns=50_000_000, stream=None):
    """Runs the search kernel's bounded device-side waits on waits that cannot complete (see
    kb_wait_check) and returns (status bits, [duration of each wait in ns], message).  The
    expected outcome, every wait giving up and the device reporting it, is status 7 with the
    library's KB_ERR_TIMEOUT message; any other outcome raises KbError."""
    from ._lib import KB_ERR_TIMEOUT
    out = (C.c_ulonglong * 4)()
    rc = lib().kb_wait_check(int(limit_ns), out, _stream(stream))
    msg = lib().kb_last_error().decode(errors="replace")
    if rc != KB_ERR_TIMEOUT:
        check(rc)
        raise KbError(rc, "kb_wait_check returned without the expected timeouts")
    return int(out[0]), [int(v) for v in out[1:]], msg


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
    _same_device([("psi", psi), ("phi", phi), ("vx", vx), ("vy", vy)]
                 + [("out[%s]" % k, v) for k, v in out.items()])
    check(lib().kb_search_no_alloc(_ptr(psi), _ptr(phi), times.ctypes.data_as(C.c_void_p), T, H,
                                   W, _ptr(vx), _ptr(vy), vx.numel(), C.byref(pc),
                                   _ptr(out["lh"]), _ptr(out["flux"]), _ptr(out["idx"]),
                                   _ptr(out["nvalid"]), _ptr(out["nkept"]), _ptr(out["mask"]),
                                   _stream(stream)))
    return out


# ------------------------------------------------------------------------------------------------
# Sub-pixel evaluation, its backward pass and refinement off the velocity grid
# ------------------------------------------------------------------------------------------------

@dataclass
class RefineParams:
    """kb_refine_params (include/kb.h): Adam settings of refine()."""
    n_steps: int = 20
    lr_pos: float = 0.1
    lr_vel: float = 0.2
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8

    def to_c(self):
        return RefineParamsC(int(self.n_steps), float(self.lr_pos), float(self.lr_vel),
                             float(self.beta1), float(self.beta2), float(self.eps))


def _traj_args(psi, phi, params, keep):
    _dev(psi, torch.float32, "psi", 3)
    _dev(phi, torch.float32, "phi", 3)
    if psi.shape != phi.shape:
        raise ValueError("psi and phi shapes differ")
    _dev(params, torch.float32, "params", 2)
    if params.shape[1] != 4:
        raise ValueError("params must be [n, 4] (x0, y0, vx, vy)")
    T = psi.shape[0]
    if keep is not None:
        _dev(keep, torch.int32, "keep", 2)
        if keep.shape != (params.shape[0], (T + 31) // 32):
            raise ValueError("keep must be [n, ceil(T/32)]")
    return psi.shape


def traj_eval(psi, phi, times, params, keep=None, grad=False, stream=None):
    """L and alpha [n] of each trajectory by bilinear sampling over its kept epochs; with grad,
    also dL/dparams [n, 4]."""
    T, H, W = _traj_args(psi, phi, params, keep)
    n = params.shape[0]
    lh = torch.empty(n, dtype=torch.float32, device=psi.device)
    flux = torch.empty(n, dtype=torch.float32, device=psi.device)
    g = torch.empty((n, 4), dtype=torch.float32, device=psi.device) if grad else None
    times = _host_times(times)
    check(lib().kb_traj_eval_fwd(_ptr(psi), _ptr(phi), times.ctypes.data_as(C.c_void_p), T, H, W,
                                 _ptr(params), _ptr(keep), n, _ptr(lh), _ptr(flux), _ptr(g),
                                 _stream(stream)))
    return (lh, flux, g) if grad else (lh, flux)


def traj_eval_backward(psi, phi, times, params, keep, grad_lh=None, grad_flux=None,
                       want_params=True, want_psi=False, want_phi=False, grad_psi=None,
                       grad_phi=None, stream=None):
    """Vector-Jacobian product of traj_eval: (grad_params [n, 4], grad_psi, grad_phi [T, H, W]),
    each None unless asked for.  Image gradients go to new zeroed tensors, or are ACCUMULATED into
    the grad_psi / grad_phi tensors given."""
    T, H, W = _traj_args(psi, phi, params, keep)
    n = params.shape[0]
    dev = psi.device
    for name, g in (("grad_lh", grad_lh), ("grad_flux", grad_flux)):
        if g is not None:
            _dev(g, torch.float32, name, 1)
    for name, g in (("grad_psi", grad_psi), ("grad_phi", grad_phi)):
        if g is not None:
            _dev(g, torch.float32, name, 3)
            if g.shape != psi.shape:
                raise ValueError("%s must have the shape of psi" % name)
    gp = torch.empty((n, 4), dtype=torch.float32, device=dev) if want_params else None
    gpsi = grad_psi if grad_psi is not None else (
        torch.zeros((T, H, W), dtype=torch.float32, device=dev) if want_psi else None)
    gphi = grad_phi if grad_phi is not None else (
        torch.zeros((T, H, W), dtype=torch.float32, device=dev) if want_phi else None)
    times = _host_times(times)
    check(lib().kb_traj_eval_bwd(_ptr(psi), _ptr(phi), times.ctypes.data_as(C.c_void_p), T, H, W,
                                 _ptr(params), _ptr(keep), n, _ptr(grad_lh), _ptr(grad_flux),
                                 _ptr(gp), _ptr(gpsi), _ptr(gphi), _stream(stream)))
    return gp, gpsi, gphi


class TrajEval(torch.autograd.Function):
    """(L, alpha) = TrajEval.apply(params, psi, phi, times, keep) with the library's hand-written
    backward kernel; the kept set is fixed (no gradient flows through the clip)."""

    @staticmethod
    def forward(ctx, params, psi, phi, times, keep):
        lh, flux = traj_eval(psi, phi, times, params, keep)
        ctx.save_for_backward(params, psi, phi, keep)
        ctx.times = _host_times(times)
        return lh, flux

    @staticmethod
    def backward(ctx, grad_lh, grad_flux):
        params, psi, phi, keep = ctx.saved_tensors
        need_p, need_psi, need_phi = ctx.needs_input_grad[:3]
        if grad_lh is not None:
            grad_lh = grad_lh.contiguous()
        if grad_flux is not None:
            grad_flux = grad_flux.contiguous()
        gp, gpsi, gphi = traj_eval_backward(psi, phi, ctx.times, params, keep, grad_lh, grad_flux,
                                            need_p, need_psi, need_phi)
        return gp, gpsi, gphi, None, None


def traj_likelihood(params, psi, phi, times, keep=None):
    """Differentiable (L, alpha) of trajectories params [n, 4]; see TrajEval."""
    return TrajEval.apply(params, psi, phi, times, keep)


def refine(psi, phi, times, params, keep=None, rp=None, inplace=False, stream=None):
    """Adam ascent of L from params [n, 4] with the kept sets fixed.  Returns (params, L, alpha,
    L_start); params is updated in place when inplace, else a refined copy."""
    T, H, W = _traj_args(psi, phi, params, keep)
    rp = RefineParams() if rp is None else rp
    n = params.shape[0]
    if not inplace:
        params = params.clone()
    dev = psi.device
    lh = torch.empty(n, dtype=torch.float32, device=dev)
    flux = torch.empty(n, dtype=torch.float32, device=dev)
    lh0 = torch.empty(n, dtype=torch.float32, device=dev)
    c = rp.to_c()
    times = _host_times(times)
    check(lib().kb_refine(_ptr(psi), _ptr(phi), times.ctypes.data_as(C.c_void_p), T, H, W,
                          _ptr(params), _ptr(keep), n, C.byref(c), _ptr(lh), _ptr(flux), _ptr(lh0),
                          _stream(stream)))
    return params, lh, flux, lh0


def candidate_params(pix, slot, result, vx, vy, window=None, stream=None):
    """(params [n, 4], keep [n, ceil(T/32)]) of collected survivors, the inputs of refine()."""
    idx, mask = result["idx"], result["mask"]
    wy, wx, K = idx.shape
    MW = mask.shape[-1]
    T = 32 * MW     # any T with this word count gives the same gather
    x_lo, y_lo = (0, 0) if window is None else (window[0], window[2])
    n = pix.numel()
    dev = idx.device
    params = torch.empty((n, 4), dtype=torch.float32, device=dev)
    keep = torch.empty((n, MW), dtype=torch.int32, device=dev)
    check(lib().kb_candidate_params(_ptr(pix), _ptr(slot), n, _ptr(idx), _ptr(mask), K, T,
                                    _ptr(vx), _ptr(vy), int(x_lo), int(y_lo), wx, _ptr(params),
                                    _ptr(keep), _stream(stream)))
    return params, keep


# ------------------------------------------------------------------------------------------------
# Batched search: many stacks in one persistent launch (optionally replayed as a CUDA graph)
# ------------------------------------------------------------------------------------------------

@dataclass
class Schedule:
    """kb_schedule (include/kb.h): scheduling knobs of a batch; results never depend on them."""
    tile_order: int = 1
    hot_nu2: float = 64.0
    score_span: int = 64
    stack_order: int = 1
    mode: int = 1           # 0: one persistent launch; 1: concurrent per-stack launches
    tile_cols: int = 0      # tiles 32 * tile_cols pixels wide (two-row blocks); 0 = automatic

    def to_c(self):
        return ScheduleC(int(self.tile_order), float(self.hot_nu2), int(self.score_span),
                         int(self.stack_order), int(self.mode), int(self.tile_cols))

    @staticmethod
    def from_c(c):
        return Schedule(c.tile_order, c.hot_nu2, c.score_span, c.stack_order, c.mode, c.tile_cols)


class Batch:
    """A batch of stacks searched as one unit (kb_batch_*): one persistent launch or concurrent
    per-stack launches (Schedule.mode), optionally replayed as one CUDA graph.

    stacks: list of dicts with psi, phi ([T, H, W] float32 CUDA tensors), times (host array),
    vx, vy (float32 CUDA tensors) and params (SearchParams, optional).  Allocates each stack's
    outputs (``results[i]``, the dict kb.search returns) and the workspace."""

    def __init__(self, stacks, device=None):
        if not stacks:
            raise ValueError("empty batch")
        n = len(stacks)
        self._keep = []                    # host times and tensors referenced by the C structs
        arr = (StackC * n)()
        self.results = []
        self.te = []
        for i, st in enumerate(stacks):
            psi, phi, vx, vy = st["psi"], st["phi"], st["vx"], st["vy"]
            _dev(psi, torch.float32, "psi", 3)
            _dev(phi, torch.float32, "phi", 3)
            _dev(vx, torch.float32, "vx", 1)
            _dev(vy, torch.float32, "vy", 1)
            T, H, W = psi.shape
            sp = st.get("params") or SearchParams()
            pc = sp.to_c(H, W)
            x_lo, x_hi, y_lo, y_hi = pc.x_lo, pc.x_hi, pc.y_lo, pc.y_hi
            wy, wx, K = y_hi - y_lo, x_hi - x_lo, pc.k_per_pixel
            mw = (T + 31) // 32
            dev = psi.device
            out = dict(lh=torch.empty((wy, wx, K), dtype=torch.float32, device=dev),
                       flux=torch.empty((wy, wx, K), dtype=torch.float32, device=dev),
                       idx=torch.empty((wy, wx, K), dtype=torch.int32, device=dev),
                       nvalid=torch.empty((wy, wx, K), dtype=torch.int16, device=dev),
                       nkept=torch.empty((wy, wx, K), dtype=torch.int16, device=dev),
                       mask=torch.empty((wy, wx, K, mw), dtype=torch.int32, device=dev))
            times = _host_times(st["times"])
            self._keep += [times, psi, phi, vx, vy]
            arr[i] = StackC(psi.data_ptr(), phi.data_ptr(), times.ctypes.data, T, H, W,
                            vx.data_ptr(), vy.data_ptr(), vx.numel(), pc,
                            out["lh"].data_ptr(), out["flux"].data_ptr(), out["idx"].data_ptr(),
                            out["nvalid"].data_ptr(), out["nkept"].data_ptr(),
                            out["mask"].data_ptr())
            self.results.append(out)
            self.te.append(wy * wx * vx.numel() * T)
        self._arr = arr
        nbytes = C.c_size_t(0)
        check(lib().kb_batch_workspace_size(arr, n, C.byref(nbytes)))
        self.workspace = alloc_workspace(nbytes.value, stacks[0]["psi"].device)
        h = C.c_void_p()
        check(lib().kb_batch_create(arr, n, _ptr(self.workspace), self.workspace.numel(),
                                    C.byref(h)))
        self._h = h
        self.n = n

    def run(self, graph=False, stream=None):
        fn = lib().kb_batch_run_graph if graph else lib().kb_batch_run
        check(fn(self._h, _stream(stream)))
        return self.results

    @property
    def schedule(self):
        c = ScheduleC()
        check(lib().kb_batch_get_schedule(self._h, C.byref(c)))
        return Schedule.from_c(c)

    @schedule.setter
    def schedule(self, s):
        c = s.to_c()
        check(lib().kb_batch_set_schedule(self._h, C.byref(c)))

    def autotune(self, reps=1, stream=None):
        c = ScheduleC()
        check(lib().kb_batch_autotune(self._h, _stream(stream), int(reps), C.byref(c)))
        return Schedule.from_c(c)

    def stats(self, stream=None):
        """(done_ns [n] numpy uint64: completion of each stack from the start of the last run,
        totals {te, evals, inserts, err})."""
        done = np.zeros(self.n, np.uint64)
        tot = np.zeros(4, np.uint64)
        check(lib().kb_batch_stats(self._h, done.ctypes.data_as(C.c_void_p),
                                   tot.ctypes.data_as(C.c_void_p), _stream(stream)))
        return done, dict(te=int(tot[0]), evals=int(tot[1]), inserts=int(tot[2]),
                          err=int(tot[3]))

    def pass_counts(self, stream=None):
        """search_pass_counts() over the last run of the batch."""
        arr = (C.c_ulonglong * 4)()
        check(lib().kb_batch_pass_counts(self._h, arr, _stream(stream)))
        return tuple(int(v) for v in arr)

    def close(self):
        if getattr(self, "_h", None):
            lib().kb_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
