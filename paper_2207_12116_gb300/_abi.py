"""ctypes declarations of the C ABI in include/pccp.h.

Argument marshalling only: every step of propagation and search runs in the
CUDA library.  Loading fails loudly if the library is missing; there is no
fallback of any kind."""
import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

PCCP_OK = 0
PCCP_ERR_INVALID = -1
PCCP_ERR_OVERFLOW = -2
PCCP_ERR_SMEM = -3
PCCP_ERR_TIMEOUT = -4
PCCP_ERR_CUDA = -5
PCCP_ERR_UNSUPPORTED = -6
PCCP_ERR_SCRATCH = -7

PCCP_FIXPOINT, PCCP_FAILED, PCCP_ERROR = 0, 1, 2
PCCP_INPUT_ORDER, PCCP_FIRST_FAIL, PCCP_LEARNED = 0, 1, 2
PCCP_OPTIMISE, PCCP_COUNT_ALL = 0, 1
PCCP_RES_OPTIMAL, PCCP_RES_INFEASIBLE, PCCP_RES_LIMIT = 0, 1, 2
PCCP_HOST_IN_PLACE = -1
PCCP_NOALLOC_SCRATCH_BYTES = 8 << 20
INT32_MAX = (1 << 31) - 1

P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64


class pccp_model_desc(ctypes.Structure):
    _fields_ = [
        ("n_vars", I32), ("lb0", P), ("ub0", P),
        ("n_temporal", I32), ("temporal", P),
        ("n_linear", I32), ("linear_c", P), ("linear_off", P), ("term_coef", P), ("term_var", P),
        ("n_reified", I32), ("reified", P),
        ("objective", I32), ("n_branch", I32), ("branch_vars", P),
        ("bool_store", I32),
    ]


class pccp_model_info(ctypes.Structure):
    _fields_ = [("n_vars", I32), ("n_temporal", I32), ("n_linear", I32), ("n_terms", I32),
                ("n_reified", I32), ("table_bytes", I32), ("bytes_per_sweep", I64),
                ("max_store_vars", I32), ("n_segments", I32), ("reordered", I32),
                ("bool_vars", I32), ("store_bytes", I32), ("temporal_levels", I32)]


class pccp_launch_config(ctypes.Structure):
    _fields_ = [("team_threads", I32), ("teams_per_cta", I32), ("ctas_per_sm", I32),
                ("max_iterations", I32), ("skip_stable", I32), ("stream_table", I32),
                ("temporal_levels", I32)]


class pccp_solve_opts(ctypes.Structure):
    _fields_ = [("strategy", I32), ("mode", I32), ("deterministic", I32), ("obj_ub", I32),
                ("node_limit", I64), ("time_limit_ms", I64), ("threads", I32), ("blocks", I32),
                ("skip_stable", I32), ("stream_table", I32), ("policy", P),
                ("teams_per_cta", I32), ("props_per_thread", I32), ("queue_granularity", I32),
                ("donate_nodes", I32), ("temporal_levels", I32)]


class pccp_policy_weights(ctypes.Structure):
    _fields_ = [("w1", P), ("b1", P), ("w2", P), ("b2", P), ("w3", P), ("b3", ctypes.c_float)]


class pccp_result(ctypes.Structure):
    _fields_ = [("status", I32), ("has_solution", I32), ("objective", I32),
                ("witness", ctypes.POINTER(I32)),
                ("nodes", I64), ("fails", I64), ("solutions", I64), ("iterations", I64),
                ("rows_evaluated", I64), ("max_depth", I32), ("elapsed_ms", ctypes.c_float),
                ("model_ms", ctypes.c_float)]


# name -> (restype, argtypes): every entry point declared in include/pccp.h
SIGNATURES = {
    "pccp_model_create": (ctypes.c_int, [ctypes.POINTER(pccp_model_desc), ctypes.POINTER(P)]),
    "pccp_model_destroy": (None, [P]),
    "pccp_model_get_info": (ctypes.c_int, [P, ctypes.POINTER(pccp_model_info)]),
    "pccp_propagate": (ctypes.c_int, [P, I32, P, P, P, P, P]),
    "pccp_propagate_ex": (ctypes.c_int, [P, I32, P, P, P, P, P, ctypes.POINTER(pccp_launch_config), P]),
    "pccp_propagate_host": (ctypes.c_int, [P, I32, P, P, P, P, I32, P]),
    "pccp_solve": (ctypes.c_int, [P, ctypes.POINTER(pccp_solve_opts), ctypes.POINTER(pccp_result), P]),
    "pccp_solve_batch": (ctypes.c_int, [ctypes.POINTER(P), I32, ctypes.POINTER(pccp_solve_opts),
                                        ctypes.POINTER(pccp_result), P]),
    "pccp_solve_batch_noalloc": (ctypes.c_int, [ctypes.POINTER(P), I32, ctypes.POINTER(pccp_solve_opts),
                                                ctypes.POINTER(pccp_result), P]),
    "pccp_batch_create": (ctypes.c_int, [ctypes.POINTER(P), I32, I32, I32, ctypes.POINTER(P)]),
    "pccp_batch_get_shape": (ctypes.c_int, [P, ctypes.POINTER(I32), ctypes.POINTER(I32),
                                            ctypes.POINTER(I32)]),
    "pccp_batch_solve_async": (ctypes.c_int, [P, ctypes.POINTER(pccp_solve_opts), P]),
    "pccp_batch_results": (ctypes.c_int, [P, ctypes.POINTER(pccp_result), P]),
    "pccp_batch_destroy": (None, [P]),
    "pccp_policy_create": (ctypes.c_int, [ctypes.POINTER(pccp_policy_weights), ctypes.POINTER(P)]),
    "pccp_policy_destroy": (None, [P]),
    "pccp_policy_get_weights": (ctypes.c_int, [P, P, P, P, P, P, P]),
    "pccp_policy_get_gradients": (ctypes.c_int, [P, P, P, P, P, P, P]),
    "pccp_policy_features": (ctypes.c_int, [P, I32, P, P, P, P, P]),
    "pccp_policy_score": (ctypes.c_int, [P, I32, P, P, P]),
    "pccp_policy_train_step": (ctypes.c_int, [P, I32, P, P, I32, P, ctypes.c_float,
                                              ctypes.POINTER(ctypes.c_float), P]),
    "pccp_error_string": (ctypes.c_char_p, [ctypes.c_int]),
}


class pccp_probe_result(ctypes.Structure):
    _fields_ = [("work", ctypes.c_double), ("ms", ctypes.c_double), ("sm_cycles", ctypes.c_double),
                ("n_sms", I32), ("ctas", I32)]


# every entry point declared in include/pccp_probe.h
PROBE_SIGNATURES = {
    "pccp_probe": (ctypes.c_int, [I32, I32, ctypes.POINTER(pccp_probe_result)]),
}
PCCP_PROBE_SMEM_LOAD, PCCP_PROBE_SMEM_ATOM, PCCP_PROBE_SMEM_DOM, PCCP_PROBE_L2_READ = 0, 1, 2, 3
_probe_lib = None


class PccpError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {error_string(code)} ({code})")


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libpccp.so (building it first if absent and allowed)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                if not build_if_missing:
                    raise ImportError(f"CUDA library not built: {path}")
                _build.build()
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def load_probe(build_if_missing: bool = True):
    """Load libpccp_probe.so, the roofline microbenchmarks."""
    global _probe_lib
    with _lock:
        if _probe_lib is None:
            path = _build.PROBE_LIB
            if not os.path.exists(path):
                if not build_if_missing:
                    raise ImportError(f"probe library not built: {path}")
                _build.build()
            lib = ctypes.CDLL(path)
            for name, (res, args) in PROBE_SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _probe_lib = lib
    return _probe_lib


def error_string(code: int) -> str:
    return load().pccp_error_string(code).decode()


def check(code: int, what: str):
    if code != PCCP_OK:
        raise PccpError(code, what)
