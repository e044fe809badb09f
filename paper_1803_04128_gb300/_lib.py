"""ctypes declarations of the C ABI in include/bf.h (argument marshalling only).

The shared library is ``paper_1803_04128_gb300/_build/libbf.so``, built in tree
by ``build.py`` (``__graft_entry__.build()`` builds it).  There is no fallback:
if the library is missing, :func:`lib` raises.
"""
import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libbf.so")

BF_OK, BF_ERR_ARG, BF_ERR_NOMEM, BF_ERR_CUDA, BF_ERR_STATE, BF_ERR_TIMEOUT, BF_ERR_ACCURACY, \
    BF_ERR_IO, BF_ERR_UNSUPPORTED = range(9)
STATUS_NAMES = ["BF_OK", "BF_ERR_ARG", "BF_ERR_NOMEM", "BF_ERR_CUDA", "BF_ERR_STATE", "BF_ERR_TIMEOUT",
                "BF_ERR_ACCURACY", "BF_ERR_IO", "BF_ERR_UNSUPPORTED"]

PREC_F64, PREC_F32, PREC_BF16X3 = 0, 1, 2
PHASE_DFT, PHASE_FIO, PHASE_FIO_PW, PHASE_ONES, PHASE_SEP, PHASE_USER, PHASE_ENTRIES = 0, 1, 2, 3, 4, 100, 101
AMP_ONE, AMP_SMOOTH, AMP_USER = 0, 1, 100

PHASE_FN = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_void_p)
AMP_FN = ctypes.CFUNCTYPE(None, ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double))
ENTRIES_FN = ctypes.CFUNCTYPE(None, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), ctypes.c_int64,
                              ctypes.c_void_p, ctypes.POINTER(ctypes.c_double))
MATVEC_FN = ctypes.CFUNCTYPE(None, ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                             ctypes.POINTER(ctypes.c_double))


class KernelDesc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("phase_kind", ctypes.c_int), ("phase_param", ctypes.c_double),
                ("amp_kind", ctypes.c_int), ("phi", PHASE_FN), ("alpha", AMP_FN), ("user", ctypes.c_void_p),
                ("entry", AMP_FN), ("entries", ENTRIES_FN), ("matvec", MATVEC_FN)]


class Options(ctypes.Structure):
    _fields_ = [("r", ctypes.c_int), ("n0", ctypes.c_int), ("split", ctypes.c_int),
                ("amp_rank", ctypes.c_int), ("amp_oversample", ctypes.c_int), ("amp_tol", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("keep_host", ctypes.c_int), ("device", ctypes.c_int),
                ("indirect", ctypes.c_int), ("phase_rank", ctypes.c_int), ("phase_oversample", ctypes.c_int),
                ("phase_tol", ctypes.c_double), ("tau", ctypes.c_double), ("l1", ctypes.c_int)]


class BatchItem(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("F", ctypes.c_void_p), ("G", ctypes.c_void_p), ("m", ctypes.c_int64)]


class ApplyItem(ctypes.Structure):
    _fields_ = [("F", ctypes.c_void_p), ("G", ctypes.c_void_p), ("m", ctypes.c_int64)]


class ServerOptions(ctypes.Structure):
    _fields_ = [("n_slots", ctypes.c_int), ("hbm_budget", ctypes.c_int64), ("max_batch_rhs", ctypes.c_int64),
                ("precision", ctypes.c_int), ("per_request", ctypes.c_int), ("device", ctypes.c_int),
                ("n_priority_slots", ctypes.c_int), ("small_units", ctypes.c_int64), ("method", ctypes.c_int),
                ("nufft_eps", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("pending", ctypes.c_int64),
                ("in_flight", ctypes.c_int64), ("launches", ctypes.c_int64), ("mean_batch_rhs", ctypes.c_double),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("units_per_s", ctypes.c_double), ("wall_s", ctypes.c_double),
                ("device_busy_ms", ctypes.c_double), ("overlap_ms", ctypes.c_double),
                ("nufft_operators", ctypes.c_int64)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("r", ctypes.c_int), ("n0", ctypes.c_int), ("L", ctypes.c_int),
                ("h", ctypes.c_int), ("l1", ctypes.c_int), ("r_alpha", ctypes.c_int), ("split", ctypes.c_int),
                ("host_bytes", ctypes.c_int64), ("dev_bytes_f64", ctypes.c_int64),
                ("dev_bytes_f32", ctypes.c_int64), ("dev_bytes_bf16", ctypes.c_int64),
                ("uploaded", ctypes.c_int), ("amp_sigma_ratio", ctypes.c_double),
                ("phase_rank", ctypes.c_int), ("t_recover_s", ctypes.c_double), ("recover_err_k", ctypes.c_double),
                ("recover_err_amp", ctypes.c_double)]


_P = ctypes.c_void_p
_SIGS = {
    "bf_default_options": (ctypes.c_int, [ctypes.POINTER(Options)]),
    "bf_plan_create": (ctypes.c_int, [ctypes.POINTER(KernelDesc), ctypes.c_double, ctypes.POINTER(Options),
                                      ctypes.POINTER(_P)]),
    "bf_factor": (ctypes.c_int, [_P]),
    "bf_upload": (ctypes.c_int, [_P]),
    "bf_factor_device": (ctypes.c_int, [_P]),
    "bf_factor_otf": (ctypes.c_int, [_P]),
    "bf_reserve": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int64]),
    "bf_apply": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int64, _P, _P]),
    "bf_apply_host": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int64, _P, _P]),
    "bf_apply_f32_noalloc": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P]),
    "bf_sync_status": (ctypes.c_int, [_P, _P]),
    "bf_plan_get_info": (ctypes.c_int, [_P, ctypes.POINTER(PlanInfo)]),
    "bf_plan_view": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(ctypes.POINTER(ctypes.c_double)), ctypes.POINTER(ctypes.c_int64)]),
    "bf_plan_save": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "bf_plan_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(Options), ctypes.POINTER(_P)]),
    "bf_destroy": (None, [_P]),
    "bf_grid_indices": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_int)]),
    "bf_unwrap": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_double, _P, ctypes.c_int, _P, _P, ctypes.c_int64,
                                 ctypes.POINTER(ctypes.c_int64)]),
    "bf_nufft_decide": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int)]),
    "bf_nufft_prepare": (ctypes.c_int, [_P, ctypes.c_double, ctypes.POINTER(ctypes.c_int)]),
    "bf_nufft_apply": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P]),
    "bf_nufft_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int64)]),
    "bf_last_error": (ctypes.c_char_p, []),
    "bf_profile_begin": (ctypes.c_int, []),
    "bf_profile_end": (ctypes.c_int, []),
    "bf_profile_count": (ctypes.c_int, []),
    "bf_profile_get": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_double)]),
    "bf_version": (ctypes.c_char_p, []),
    "bf_fp32_peak": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "bf_fp64_peak": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "bf_batch_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(_P)]),
    "bf_batch_run": (ctypes.c_int, [_P, _P]),
    "bf_batch_capture_graph": (ctypes.c_int, [_P, _P]),
    "bf_batch_replay": (ctypes.c_int, [_P, _P]),
    "bf_batch_status": (ctypes.c_int, [_P, _P]),
    "bf_batch_get_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "bf_batch_set_spin_limit": (ctypes.c_int, [_P, ctypes.c_longlong]),
    "bf_batch_debug_hold": (ctypes.c_int, [_P, ctypes.c_int]),
    "bf_batch_destroy": (None, [_P]),
    "bf_batch_set_mode": (ctypes.c_int, [_P, ctypes.c_int]),
    "bf_batch_get_mode": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "bf_batch_tune": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "bf_batch_tune_times": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    "bf_apply_batched": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, _P]),
    "bf_apply_batched_release": (None, []),
    "bf_shard_info": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "bf_apply_shard_front": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int64, _P, _P]),
    "bf_apply_shard_back": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int64, _P, _P]),
    "bf_autotune": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int)]),
    "bf_autotune_get": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "bf_server_default_options": (ctypes.c_int, [ctypes.POINTER(ServerOptions)]),
    "bf_server_create": (ctypes.c_int, [ctypes.POINTER(ServerOptions), ctypes.POINTER(_P)]),
    "bf_server_add_operator": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int)]),
    "bf_server_start": (ctypes.c_int, [_P]),
    "bf_server_submit": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int64, _P, ctypes.POINTER(ctypes.c_uint64)]),
    "bf_server_wait": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
    "bf_server_drain": (ctypes.c_int, [_P, ctypes.c_double]),
    "bf_server_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(ServerStats)]),
    "bf_server_reset_stats": (ctypes.c_int, [_P]),
    "bf_server_destroy": (None, [_P]),
}

_lock = threading.Lock()
_lib = None


class BFError(RuntimeError):
    def __init__(self, status, where):
        msg = _lib.bf_last_error().decode() if _lib is not None else ""
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__("%s failed: %s: %s" % (where, name, msg))
        self.status = status


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libbf.so not built (%s); run __graft_entry__.build() or "
                                   "python -m paper_1803_04128_gb300.build" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(status, where):
    if status != BF_OK:
        raise BFError(status, where)


def declared_symbols():
    """The entry points include/*.h declares (parsed from the headers)."""
    import re
    inc = os.path.join(os.path.dirname(HERE), "include")
    names = []
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(bf_[a-z0-9_]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))
