"""ctypes binding of libhc.so (the C ABI in include/hc.h).

Argument marshalling only: every step of every call runs in the library's
CUDA kernels.  Loading fails loudly when the library has not been built;
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
# HC_LIBRARY selects another build of the same library (the debug bounds
# build, libhc_debug.so); it must exist like the default one.
LIB_PATH = os.environ.get("HC_LIBRARY") or os.path.join(HERE, "libhc.so")

# hc_kind
SET_U32, SET_U64, MAP_I64_I32, MAP_U64_U64 = 0, 1, 2, 3
# hc_rc
OK, ERR_ARG, ERR_OOM, ERR_OVERFLOW, ERR_CUDA, ERR_STATE, ERR_TIMEOUT = 0, 1, 2, 3, 4, 5, 6
RC_NAMES = {0: "HC_OK", 1: "HC_ERR_ARG", 2: "HC_ERR_OOM", 3: "HC_ERR_OVERFLOW", 4: "HC_ERR_CUDA", 5: "HC_ERR_STATE",
            6: "HC_ERR_TIMEOUT"}
# per-key status
INSERTED, EXISTS, OVERFLOW, ERASED, NOT_FOUND = 0, 1, 2, 3, 4
# selection predicates
PRED_ALL, PRED_KEY_RANGE, PRED_VALUE_RANGE, PRED_KEY_MASK, PRED_BLOCK_BOX, PRED_SHORT3_BOX = 0, 1, 2, 3, 4, 5
# ops, hash modes
OP_INSERT, OP_FIND, OP_ERASE = 0, 1, 2
HASH_MIX64, HASH_TESCHNER, HASH_TESCHNER_SHORT3 = 0, 1, 2

EXPORTS = [
    "hc_abi_version", "hc_last_error", "hc_table_bytes", "hc_create", "hc_destroy", "hc_set_launch",
    "hc_get_launch", "hc_insert", "hc_insert_if_absent", "hc_find", "hc_erase", "hc_insert_host", "hc_find_host", "hc_erase_host",
    "hc_size", "hc_stats", "hc_status", "hc_clear", "hc_rehash", "hc_dump", "hc_batch_create",
    "hc_batch_launch", "hc_batch_destroy", "hc_batch_run_noalloc", "hc_measure_random_reads",
    "hc_batch_scratch_bytes", "hc_batch_run", "hc_device_view_get", "hc_select",
    "hc_ordered_scratch_bytes", "hc_insert_ordered", "hc_erase_ordered", "hc_apply_mixed",
    "hc_pack_short3", "hc_unpack_short3", "hc_server_create", "hc_server_run", "hc_server_destroy",
    "hc_server_start", "hc_server_submit", "hc_server_wait", "hc_server_stop",
]


class HCError(RuntimeError):
    def __init__(self, rc: int, msg: str):
        super().__init__(f"{RC_NAMES.get(rc, rc)}: {msg}")
        self.rc = rc


class Config(ctypes.Structure):
    _fields_ = [("bucket_bytes", ctypes.c_int32), ("hash_mode", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class Launch(ctypes.Structure):
    _fields_ = [("lane_bytes", ctypes.c_int32), ("keys_per_group", ctypes.c_int32), ("block", ctypes.c_int32),
                ("fold_duplicates", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("live", ctypes.c_int64), ("used", ctypes.c_int64), ("capacity", ctypes.c_int64),
                ("slot_bytes", ctypes.c_int64), ("table_bytes", ctypes.c_int64), ("error_bits", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class BatchItem(ctypes.Structure):
    _fields_ = [("table", ctypes.c_void_p), ("op", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("d_keys", ctypes.c_void_p), ("d_vals", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("d_out", ctypes.c_void_p), ("d_vals_out", ctypes.c_void_p)]


class BatchConfig(ctypes.Structure):
    _fields_ = [("lane_bytes", ctypes.c_int32), ("keys_per_group", ctypes.c_int32), ("block", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("tile", ctypes.c_int32), ("use_graph", ctypes.c_int32)]


class Predicate(ctypes.Structure):
    """hc_predicate: which stored entries hc_select appends."""
    _fields_ = [("kind", ctypes.c_int32), ("negate", ctypes.c_int32), ("lo", ctypes.c_int64), ("hi", ctypes.c_int64),
                ("box", ctypes.c_int32 * 6)]


class DeviceView(ctypes.Structure):
    """hc_device_view: a table as the in-kernel functions see it."""
    _fields_ = [("buckets", ctypes.c_void_p), ("header", ctypes.c_void_p),
                ("nb", ctypes.c_uint64), ("seed", ctypes.c_uint64), ("kind", ctypes.c_int32),
                ("bucket_bytes", ctypes.c_int32), ("hash_mode", ctypes.c_int32), ("pad_from", ctypes.c_int32)]


class ServeConfig(ctypes.Structure):
    """hc_serve_config."""
    _fields_ = [("lanes", ctypes.c_int32), ("depth", ctypes.c_int32), ("slot_bytes", ctypes.c_int64),
                ("merge", ctypes.c_int32), ("max_items", ctypes.c_int32), ("batch", BatchConfig)]


class Request(ctypes.Structure):
    """hc_request: one served request."""
    _fields_ = [("table", ctypes.c_int32), ("op", ctypes.c_int32), ("h_keys", ctypes.c_void_p),
                ("h_vals", ctypes.c_void_p), ("n", ctypes.c_int64), ("h_status", ctypes.c_void_p),
                ("h_vals_out", ctypes.c_void_p), ("arrival", ctypes.c_double), ("deadline", ctypes.c_double),
                ("done", ctypes.c_double), ("rc", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ServeStats(ctypes.Structure):
    """hc_serve_stats."""
    _fields_ = [("requests", ctypes.c_int64), ("ops", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("queued_max", ctypes.c_int64), ("timed_out", ctypes.c_int64), ("wall_s", ctypes.c_double),
                ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("p999_ms", ctypes.c_double), ("max_ms", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def _declare(lib: ctypes.CDLL) -> ctypes.CDLL:
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    P = ctypes.POINTER
    sig = {
        "hc_abi_version": (i32, []),
        "hc_last_error": (ctypes.c_char_p, []),
        "hc_table_bytes": (i32, [i32, i64, P(Config), P(i64)]),
        "hc_create": (i32, [P(vp), i32, i64, P(Config), vp]),
        "hc_destroy": (i32, [vp]),
        "hc_set_launch": (i32, [vp, i32, P(Launch)]),
        "hc_get_launch": (i32, [vp, i32, P(Launch)]),
        "hc_insert": (i32, [vp, vp, vp, i64, vp, vp]),
        "hc_insert_if_absent": (i32, [vp, vp, vp, vp, i64, vp, vp]),
        "hc_find": (i32, [vp, vp, i64, vp, vp, vp]),
        "hc_erase": (i32, [vp, vp, i64, vp, vp]),
        "hc_insert_host": (i32, [vp, vp, vp, i64, vp, vp]),
        "hc_find_host": (i32, [vp, vp, i64, vp, vp, vp]),
        "hc_erase_host": (i32, [vp, vp, i64, vp, vp]),
        "hc_size": (i32, [vp, P(i64), vp]),
        "hc_stats": (i32, [vp, P(Stats), vp]),
        "hc_status": (i32, [vp, vp]),
        "hc_clear": (i32, [vp, vp]),
        "hc_rehash": (i32, [vp, i64, vp]),
        "hc_dump": (i32, [vp, vp, vp, i64, P(i64), vp]),
        "hc_batch_create": (i32, [P(vp), P(BatchItem), i64, P(BatchConfig), vp]),
        "hc_batch_launch": (i32, [vp, vp]),
        "hc_batch_destroy": (i32, [vp]),
        "hc_batch_run_noalloc": (i32, [P(BatchItem), i64, P(BatchConfig), vp]),
        "hc_measure_random_reads": (i32, [vp, i64, i64, i32, P(ctypes.c_float), vp]),
        "hc_batch_scratch_bytes": (i64, [i64]),
        "hc_batch_run": (i32, [P(BatchItem), i64, P(BatchConfig), vp, i64, vp]),
        "hc_device_view_get": (i32, [vp, P(DeviceView), vp]),
        "hc_select": (i32, [vp, P(Predicate), vp, vp, i64, vp, vp]),
        "hc_ordered_scratch_bytes": (i64, [i64]),
        "hc_insert_ordered": (i32, [vp, vp, vp, i64, vp, vp, i64, vp]),
        "hc_erase_ordered": (i32, [vp, vp, i64, vp, vp, i64, vp]),
        "hc_apply_mixed": (i32, [vp, vp, vp, vp, i64, vp, vp, vp]),
        "hc_pack_short3": (i32, [vp, i64, vp, vp]),
        "hc_unpack_short3": (i32, [vp, i64, vp, vp]),
        "hc_server_create": (i32, [P(vp), P(vp), i32, P(ServeConfig)]),
        "hc_server_run": (i32, [vp, P(Request), i64, i32, ctypes.c_double, P(ServeStats)]),
        "hc_server_start": (i32, [vp]),
        "hc_server_submit": (i32, [vp, P(Request)]),
        "hc_server_wait": (i32, [vp, P(Request), ctypes.c_double]),
        "hc_server_stop": (i32, [vp, P(ServeStats)]),
        "hc_server_destroy": (i32, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libhc.so.  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise ImportError(f"libhc.so is not built ({path}); run `python -m paper_1908_05936_gb300.build`")
            _lib = _declare(ctypes.CDLL(path))
    return _lib


def check(rc: int) -> None:
    if rc != OK:
        raise HCError(rc, load().hc_last_error().decode())
