"""ctypes loader for libkb_b300.so (the C ABI declared in include/kb.h).

The library is built in-tree by ``paper_2109_03296_b300.build``.  There is no fallback: if the
library is missing or cannot be loaded, every call raises.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# KB_B300_LIBRARY=checked selects the build with device-side bounds checks (build.py --checked)
LIB_PATH = os.path.join(HERE, "libkb_b300_checked.so"
                        if os.environ.get("KB_B300_LIBRARY") == "checked" else "libkb_b300.so")

KB_OK = 0
KB_ERR_INVALID_ARG = 1
KB_ERR_UNSUPPORTED = 2
KB_ERR_CUDA = 3
KB_ERR_WORKSPACE = 4
KB_ERR_TIMEOUT = 5
KB_MAX_T = 128
KB_MAX_K = 32
KB_WORKSPACE_ALIGN = 256
KB_STATIC_SCRATCH_BYTES = 32 << 20

EXPORTS = ("kb_version", "kb_last_error", "kb_search_params_default", "kb_make_psi_phi",
           "kb_search_workspace_size", "kb_search", "kb_search_stats", "kb_stamps",
           "kb_collect_workspace_size", "kb_collect", "kb_candidate_tracks", "kb_launch_count",
           "kb_profile_events", "kb_search_no_alloc", "kb_traj_eval_fwd", "kb_traj_eval_bwd",
           "kb_refine_params_default", "kb_refine", "kb_candidate_params", "kb_stamp_filter",
           "kb_schedule_default", "kb_batch_workspace_size", "kb_batch_create", "kb_batch_run",
           "kb_batch_run_graph", "kb_batch_set_schedule", "kb_batch_get_schedule",
           "kb_batch_autotune", "kb_batch_stats", "kb_batch_destroy",
           "kb_cluster_workspace_size", "kb_cluster", "kb_l2_probe", "kb_wait_check",
           "kb_search_stage_counts", "kb_search_no_alloc_stats", "kb_smem_probe",
           "kb_search_pass_counts", "kb_batch_pass_counts")


class KbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("kb error %d: %s" % (code, msg))
        self.code = code


class SearchParamsC(C.Structure):
    _fields_ = [("k_per_pixel", C.c_int32), ("lh_min", C.c_float), ("min_obs", C.c_int32),
                ("clip", C.c_int32), ("q_lo", C.c_float), ("q_mid", C.c_float),
                ("q_hi", C.c_float), ("n_sigma", C.c_float), ("clip_on", C.c_int32),
                ("x_lo", C.c_int32), ("x_hi", C.c_int32), ("y_lo", C.c_int32),
                ("y_hi", C.c_int32), ("bound_rows", C.c_int32)]


class RefineParamsC(C.Structure):
    _fields_ = [("n_steps", C.c_int32), ("lr_pos", C.c_float), ("lr_vel", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float)]


class StackC(C.Structure):
    _fields_ = [("psi", C.c_void_p), ("phi", C.c_void_p), ("times", C.c_void_p),
                ("T", C.c_int32), ("H", C.c_int32), ("W", C.c_int32),
                ("vx", C.c_void_p), ("vy", C.c_void_p), ("n_traj", C.c_int32),
                ("params", SearchParamsC),
                ("out_lh", C.c_void_p), ("out_flux", C.c_void_p), ("out_idx", C.c_void_p),
                ("out_nvalid", C.c_void_p), ("out_nkept", C.c_void_p), ("out_mask", C.c_void_p)]


class ScheduleC(C.Structure):
    _fields_ = [("tile_order", C.c_int32), ("hot_nu2", C.c_float), ("score_span", C.c_int32),
                ("stack_order", C.c_int32), ("mode", C.c_int32), ("tile_cols", C.c_int32)]


_LIB = None


def lib():
    """Loads the library (building it first if the sources are newer and nvcc is present)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise ImportError("%s is not built: run paper_2109_03296_b300/build.py "
                          "(or __graft_entry__.build())" % os.path.basename(LIB_PATH))
    L = C.CDLL(LIB_PATH)
    p, i, f, sz = C.c_void_p, C.c_int, C.c_float, C.c_size_t
    L.kb_version.restype = i
    L.kb_version.argtypes = []
    L.kb_last_error.restype = C.c_char_p
    L.kb_last_error.argtypes = []
    L.kb_search_params_default.restype = None
    L.kb_search_params_default.argtypes = [C.POINTER(SearchParamsC), i, i]
    L.kb_make_psi_phi.restype = i
    L.kb_make_psi_phi.argtypes = [p, p, p, p, i, i, i, i, p, p, p]
    L.kb_search_workspace_size.restype = i
    L.kb_search_workspace_size.argtypes = [i, i, i, i, C.POINTER(SearchParamsC), C.POINTER(sz)]
    L.kb_search.restype = i
    L.kb_search.argtypes = [p, p, p, i, i, i, p, p, i, C.POINTER(SearchParamsC), p, p, p, p, p,
                            p, p, sz, p]
    L.kb_search_stats.restype = i
    L.kb_search_stats.argtypes = [p, p, p]
    L.kb_search_stage_counts.restype = i
    L.kb_search_stage_counts.argtypes = [p, p, p]
    L.kb_search_no_alloc_stats.restype = i
    L.kb_search_no_alloc_stats.argtypes = [p, p]
    L.kb_search_pass_counts.restype = i
    L.kb_search_pass_counts.argtypes = [p, p, p]
    L.kb_smem_probe.restype = i
    L.kb_smem_probe.argtypes = [i, i, p, p]
    L.kb_stamps.restype = i
    L.kb_stamps.argtypes = [p, p, p, p, i, i, i, p, p, p, p, p, i, i, p, p, p]
    L.kb_collect_workspace_size.restype = i
    L.kb_collect_workspace_size.argtypes = [i, C.POINTER(sz)]
    L.kb_collect.restype = i
    L.kb_collect.argtypes = [p, p, i, i, i, p, p, p, p, sz, p]
    L.kb_candidate_tracks.restype = i
    L.kb_candidate_tracks.argtypes = [p, p, i, p, i, p, p, i, i, i, p, p, p, p, p, p]
    L.kb_launch_count.restype = C.c_ulonglong
    L.kb_launch_count.argtypes = []
    L.kb_profile_events.restype = None
    L.kb_profile_events.argtypes = [p, p]
    L.kb_search_no_alloc.restype = i
    L.kb_search_no_alloc.argtypes = [p, p, p, i, i, i, p, p, i, C.POINTER(SearchParamsC), p, p, p,
                                     p, p, p, p]
    L.kb_traj_eval_fwd.restype = i
    L.kb_traj_eval_fwd.argtypes = [p, p, p, i, i, i, p, p, i, p, p, p, p]
    L.kb_traj_eval_bwd.restype = i
    L.kb_traj_eval_bwd.argtypes = [p, p, p, i, i, i, p, p, i, p, p, p, p, p, p]
    L.kb_refine_params_default.restype = None
    L.kb_refine_params_default.argtypes = [C.POINTER(RefineParamsC)]
    L.kb_refine.restype = i
    L.kb_refine.argtypes = [p, p, p, i, i, i, p, p, i, C.POINTER(RefineParamsC), p, p, p, p]
    SP, SCP = C.POINTER(StackC), C.POINTER(ScheduleC)
    L.kb_schedule_default.restype = None
    L.kb_schedule_default.argtypes = [SCP]
    L.kb_batch_workspace_size.restype = i
    L.kb_batch_workspace_size.argtypes = [SP, i, C.POINTER(sz)]
    L.kb_batch_create.restype = i
    L.kb_batch_create.argtypes = [SP, i, p, sz, C.POINTER(p)]
    L.kb_batch_run.restype = i
    L.kb_batch_run.argtypes = [p, p]
    L.kb_batch_run_graph.restype = i
    L.kb_batch_run_graph.argtypes = [p, p]
    L.kb_batch_set_schedule.restype = i
    L.kb_batch_set_schedule.argtypes = [p, SCP]
    L.kb_batch_get_schedule.restype = i
    L.kb_batch_get_schedule.argtypes = [p, SCP]
    L.kb_batch_autotune.restype = i
    L.kb_batch_autotune.argtypes = [p, p, i, SCP]
    L.kb_batch_stats.restype = i
    L.kb_batch_stats.argtypes = [p, p, p, p]
    L.kb_batch_pass_counts.restype = i
    L.kb_batch_pass_counts.argtypes = [p, p, p]
    L.kb_batch_destroy.restype = None
    L.kb_batch_destroy.argtypes = [p]
    L.kb_cluster_workspace_size.restype = i
    L.kb_cluster_workspace_size.argtypes = [i, C.POINTER(sz)]
    L.kb_cluster.restype = i
    L.kb_cluster.argtypes = [p, p, p, p, p, i, C.c_double, C.c_double, p, p, p, sz,
                             C.POINTER(C.c_int), p]
    L.kb_l2_probe.restype = i
    L.kb_l2_probe.argtypes = [p, sz, i, p, i, p]
    L.kb_wait_check.restype = i
    L.kb_wait_check.argtypes = [C.c_ulonglong, p, p]
    L.kb_stamp_filter.restype = i
    L.kb_stamp_filter.argtypes = [p, i, i, p, p, p, p]
    L.kb_candidate_params.restype = i
    L.kb_candidate_params.argtypes = [p, p, i, p, p, i, i, p, p, i, i, i, p, p, p]
    _LIB = L
    return L


def check(rc):
    if rc != KB_OK:
        raise KbError(rc, lib().kb_last_error().decode(errors="replace"))
    return rc
