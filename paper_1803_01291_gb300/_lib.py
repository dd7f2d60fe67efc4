"""ctypes binding of libhbe.so (include/hbe.h).  Argument marshalling only:
every step of the solver runs in the CUDA library.  There is no CPU fallback:
if the library is missing the import of the binding fails loudly."""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhbe.so")

OK, EINVAL, ENOMEM, ECUDA, ESTATE, STOPPED, NONFINITE, ETIMEOUT = range(8)
DIRICHLET, PERIODIC = 0, 1
FP64, FP32, BF16, FP32_PLAIN = 0, 1, 2, 3
PREC_NAMES = {FP64: "fp64", FP32: "fp32", BF16: "bf16", FP32_PLAIN: "fp32_plain"}

# every entry point declared in include/hbe.h
EXPORTS = (
    "hbe_workspace_bytes", "hbe_create", "hbe_create_in", "hbe_destroy", "hbe_set_stream",
    "hbe_set_tuning", "hbe_set_schedule", "hbe_variant_info", "hbe_variant_count", "hbe_set_initial",
    "hbe_set_initial_device", "hbe_set_initial_bumps", "hbe_set_stop", "hbe_step", "hbe_step_async", "hbe_sync",
    "hbe_read", "hbe_read_device", "hbe_prefetch_initial", "hbe_set_initial_prefetched",
    "hbe_read_async", "hbe_read_wait", "hbe_profile_stages", "hbe_progress", "hbe_analysis", "hbe_set_monitor",
    "hbe_monitor_read", "hbe_diag", "hbe_save", "hbe_load",
    "hbe_last_error", "hbe_status_string", "hbe_launch_count", "hbe_batch_create",
    "hbe_batch_destroy", "hbe_batch_add", "hbe_batch_remove", "hbe_batch_run", "hbe_batch_launch",
    "hbe_batch_collect",
    "hbe_batch_size", "hbe_batch_last_error", "hbe_batch_launch_count", "hbe_step_fp64_noalloc",
    "hbe_radial_max_n", "hbe_radial_run", "hbe_slab_plan", "hbe_slabs_create",
    "hbe_slabs_destroy", "hbe_slabs_set_initial_device", "hbe_slabs_step",
    "hbe_slabs_read_device", "hbe_slabs_last_error",
)


class HbeDiag(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("step", ctypes.c_int64),
                ("max_abs_phi", ctypes.c_double), ("finite", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("n_pos", ctypes.c_int64),
                ("n_neg", ctypes.c_int64), ("bubble_count", ctypes.c_int64)]


class HbeAnalysis(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("integral_phi", ctypes.c_double),
                ("integral_phi3", ctypes.c_double), ("laplacian_monitor", ctypes.c_double),
                ("support_points", ctypes.c_int64), ("condition1_violations", ctypes.c_int64)]


class HbeVariant(ctypes.Structure):
    _fields_ = [("tile_x", ctypes.c_int32), ("tile_y", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("vec", ctypes.c_int32),
                ("rows_per_warp", ctypes.c_int32), ("consumer_warps", ctypes.c_int32),
                ("smem_bytes", ctypes.c_int32 * 4),
                ("ring", ctypes.c_int32 * 4),
                ("pair_tile_y", ctypes.c_int32 * 2), ("pair_threads", ctypes.c_int32 * 2),
                ("pair_smem_bytes", ctypes.c_int32 * 2), ("pair_ring", ctypes.c_int32 * 2)]


class HBEError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


STATUS_NAMES = {OK: "HBE_OK", EINVAL: "HBE_EINVAL", ENOMEM: "HBE_ENOMEM", ECUDA: "HBE_ECUDA",
                ESTATE: "HBE_ESTATE", STOPPED: "HBE_STOPPED", NONFINITE: "HBE_NONFINITE",
                ETIMEOUT: "HBE_ETIMEOUT"}

_lock = threading.Lock()
_lib = None


def load() -> ctypes.CDLL:
    """Load libhbe.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} not found: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'` "
                              "(the solver has no CPU fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        P, I, D, I64, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_size_t
        dp = ctypes.POINTER(ctypes.c_double)
        sig = {
            "hbe_workspace_bytes": (I, [I, I, I, ctypes.POINTER(SZ)]),
            "hbe_create": (I, [I, D, D, D, I, I, ctypes.POINTER(P)]),
            "hbe_create_in": (I, [I, D, D, D, I, I, P, SZ, ctypes.POINTER(P)]),
            "hbe_destroy": (None, [P]),
            "hbe_set_stream": (I, [P, P]),
            "hbe_set_tuning": (I, [P, I, I]),
            "hbe_set_schedule": (I, [P, I]),
            "hbe_variant_info": (I, [I, I, ctypes.POINTER(HbeVariant)]),
            "hbe_variant_count": (I, [I]),
            "hbe_set_initial": (I, [P, dp, dp, D]),
            "hbe_set_initial_device": (I, [P, P, P, D]),
            "hbe_set_initial_bumps": (I, [P, I, dp, dp, dp, I, dp, dp, dp, D]),
            "hbe_set_stop": (I, [P, D]),
            "hbe_step": (I, [P, I64, D]),
            "hbe_step_async": (I, [P, I64, D]),
            "hbe_sync": (I, [P]),
            "hbe_read": (I, [P, dp, dp, dp]),
            "hbe_read_device": (I, [P, P, P]),
            "hbe_prefetch_initial": (I, [P, dp, dp]),
            "hbe_set_initial_prefetched": (I, [P, D]),
            "hbe_read_async": (I, [P, dp, dp]),
            "hbe_read_wait": (I, [P]),
            "hbe_progress": (I, [P, ctypes.POINTER(I64), dp]),
            "hbe_profile_stages": (I, [P, I64, D, ctypes.POINTER(ctypes.c_float)]),
            "hbe_diag": (I, [P, D, ctypes.POINTER(HbeDiag), P, P]),
            "hbe_analysis": (I, [P, D, ctypes.POINTER(HbeAnalysis)]),
            "hbe_set_monitor": (I, [P, I]),
            "hbe_monitor_read": (I, [P, I64, I64, dp, dp]),
            "hbe_save": (I, [P, ctypes.c_char_p]),
            "hbe_load": (I, [P, ctypes.c_char_p]),
            "hbe_last_error": (ctypes.c_char_p, [P]),
            "hbe_status_string": (ctypes.c_char_p, [I]),
            "hbe_launch_count": (I64, [P]),
            "hbe_batch_create": (I, [I, I, P, ctypes.POINTER(P)]),
            "hbe_batch_destroy": (None, [P]),
            "hbe_batch_add": (I, [P, P, I64, D]),
            "hbe_batch_remove": (I, [P, P]),
            "hbe_batch_run": (I, [P, ctypes.POINTER(P), I, ctypes.POINTER(I)]),
            "hbe_batch_launch": (I, [P]),
            "hbe_batch_collect": (I, [P, ctypes.POINTER(P), I, ctypes.POINTER(I)]),
            "hbe_batch_size": (I, [P]),
            "hbe_batch_last_error": (ctypes.c_char_p, [P]),
            "hbe_batch_launch_count": (I64, [P]),
            "hbe_step_fp64_noalloc": (I, [I, D, D, D, I, P, P, D, D, I64, P, P, P]),
            "hbe_slab_plan": (I, [I, I, I, ctypes.POINTER(ctypes.c_int32),
                                  ctypes.POINTER(ctypes.c_int32), I]),
            "hbe_slabs_create": (I, [I, D, D, D, I, I, I, P, ctypes.POINTER(P)]),
            "hbe_slabs_destroy": (None, [P]),
            "hbe_slabs_set_initial_device": (I, [P, P, P, D]),
            "hbe_slabs_step": (I, [P, I64, D]),
            "hbe_slabs_read_device": (I, [P, P, P, dp]),
            "hbe_slabs_last_error": (ctypes.c_char_p, [P]),
            "hbe_radial_max_n": (I, [I]),
            "hbe_radial_run": (I, [I, I, D, P, P, P, P, D, D, I64, I, I, D, D, P, P, P, P, P,
                                   P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib
