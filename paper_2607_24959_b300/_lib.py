"""ctypes view of the C ABI in ``include/contact_solve.h``.

Argument marshalling only: every step of the solve runs in the CUDA kernels of
``libcs_b300.so``.  Loading fails loudly if the library is missing; there is
no CPU fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcs_b300.so")

c_int32 = ctypes.c_int32
c_int64 = ctypes.c_int64
c_float = ctypes.c_float
c_void_p = ctypes.c_void_p
c_size_t = ctypes.c_size_t

CS_OK = 0
CS_EINVAL = -1
CS_ECUDA = -2
CS_ENOMEM = -3
CS_EBUSY = -4
CS_ENOTFOUND = -5
CS_EUNSUPPORTED = -6
CS_PENDING = 1

ST_OK, ST_MAXITER, ST_CHOLFAIL, ST_NONFINITE, ST_BADSHAPE, ST_NOPROGRESS = range(6)
ST_FAILED, ST_TIMEOUT = 6, 7
STATUS_NAMES = {0: "OK", 1: "MAXITER", 2: "CHOLFAIL", 3: "NONFINITE",
                4: "BADSHAPE", 5: "NOPROGRESS", 6: "FAILED", 7: "TIMEOUT"}
SERVE_FAULT_H2D, SERVE_FAULT_LAUNCH, SERVE_FAULT_D2H, SERVE_FAULT_COMPLETE = range(4)
SERVE_FAULT_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p)


class CsBatch(ctypes.Structure):
    _fields_ = [("n", c_int32), ("nv_max", c_int32), ("m_max", c_int32),
                ("reserved", c_int32), ("inst", c_void_p), ("M", c_void_p),
                ("J", c_void_p), ("qfrc", c_void_p), ("aref", c_void_p),
                ("D", c_void_p), ("total_M", c_int64), ("total_J", c_int64),
                ("total_v", c_int64), ("total_r", c_int64)]


class CsOptions(ctypes.Structure):
    _fields_ = [("tol", c_float), ("max_iter", c_int32), ("keep_factor", c_int32),
                ("warps_per_block", c_int32)]


class CsState(ctypes.Structure):
    _fields_ = [("a_lo", c_void_p), ("act", c_void_p), ("L", c_void_p),
                ("status", c_void_p), ("iters", c_void_p)]


class CsPlanInfo(ctypes.Structure):
    _fields_ = [("n_kernels", c_int32), ("graph", c_int32),
                ("nv_bucket", c_int32 * 8), ("rows_per_lane", c_int32 * 8),
                ("instances", c_int32 * 8), ("warps_per_block", c_int32 * 8),
                ("tuned_ms", c_float * 8), ("cta", c_int32 * 8)]


CS_PLAN_AUTOTUNE = 1
CS_PLAN_GRAPH = 2
ST_FAILED = 6
CS_SERVE_CONTINUOUS = 0
CS_SERVE_FIXED = 1


class CsServeConfig(ctypes.Structure):
    _fields_ = [("arena_bytes", c_size_t), ("streams", c_int32), ("max_batch", c_int32),
                ("policy", c_int32), ("fixed_batch", c_int32), ("tol", c_float),
                ("max_iter", c_int32), ("max_queue", c_int32), ("queue_timeout_ms", c_int32)]


class CsRequest(ctypes.Structure):
    _fields_ = [("nv", c_int32), ("m", c_int32), ("M", c_void_p), ("J", c_void_p),
                ("qfrc", c_void_p), ("aref", c_void_p), ("D", c_void_p), ("g", c_void_p)]


class CsResult(ctypes.Structure):
    _fields_ = [("a", c_void_p), ("dqfrc", c_void_p), ("daref", c_void_p), ("dJ", c_void_p),
                ("status", c_int32), ("iters", c_int32), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]


class CsServeStats(ctypes.Structure):
    _fields_ = [("submitted", c_int64), ("completed", c_int64), ("batches", c_int64),
                ("batched_requests", c_int64), ("queued", c_int64),
                ("max_inflight", c_int32), ("failed_launches", c_int32),
                ("timed_out", c_int64)]

# name -> (restype, argtypes)
_SIGS = {
    "cs_version": (ctypes.c_int, []),
    "cs_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "cs_last_error": (ctypes.c_char_p, []),
    "cs_solve_fwd": (ctypes.c_int, [ctypes.POINTER(CsBatch), ctypes.POINTER(CsOptions),
                                    c_void_p, ctypes.POINTER(CsState), c_void_p]),
    "cs_solve_adjoint": (ctypes.c_int, [ctypes.POINTER(CsBatch), ctypes.POINTER(CsOptions),
                                        c_void_p, ctypes.POINTER(CsState), c_void_p,
                                        c_void_p, c_void_p, c_void_p, c_void_p]),
    "cs_solve_adjoint_theta": (ctypes.c_int, [ctypes.POINTER(CsBatch), ctypes.POINTER(CsOptions),
                                              c_void_p, ctypes.POINTER(CsState), c_void_p,
                                              c_void_p, c_void_p, c_void_p, c_void_p,
                                              c_void_p, c_void_p]),
    "cs_state_create": (ctypes.c_int, [ctypes.POINTER(CsBatch), c_int32,
                                       ctypes.POINTER(ctypes.POINTER(CsState))]),
    "cs_solve_fwd_alloc": (ctypes.c_int, [ctypes.POINTER(CsBatch), ctypes.POINTER(CsOptions),
                                          c_void_p, ctypes.POINTER(ctypes.POINTER(CsState)),
                                          c_void_p]),
    "cs_state_status": (ctypes.c_int, [ctypes.POINTER(CsState), c_void_p, c_void_p, c_void_p]),
    "cs_state_free": (None, [ctypes.POINTER(CsState)]),
    "cs_fused_workspace_bytes": (c_size_t, [c_int32]),
    "cs_solve_fused_ncg": (ctypes.c_int, [ctypes.POINTER(CsBatch), ctypes.POINTER(CsOptions),
                                          c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                          c_void_p, c_void_p, c_void_p, c_void_p, c_size_t,
                                          c_void_p]),
    "cs_solve_fused_elliptic": (ctypes.c_int, [ctypes.POINTER(CsBatch),
                                               ctypes.POINTER(CsOptions), c_void_p, c_void_p,
                                               c_void_p, c_void_p, c_void_p, c_void_p,
                                               c_void_p, c_void_p, c_void_p, c_void_p,
                                               c_void_p, c_void_p, c_void_p, c_size_t,
                                               c_void_p]),
    "cs_unrolled_trace_floats": (c_size_t, [ctypes.POINTER(CsBatch), c_int32]),
    "cs_unrolled_mask_bytes": (c_size_t, [ctypes.POINTER(CsBatch), c_int32]),
    "cs_unrolled_fwd": (ctypes.c_int, [ctypes.POINTER(CsBatch), ctypes.POINTER(CsOptions),
                                       c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                       c_void_p]),
    "cs_unrolled_bwd": (ctypes.c_int, [ctypes.POINTER(CsBatch), ctypes.POINTER(CsOptions),
                                       c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                       c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                       c_void_p, c_void_p]),
    "cs_solve_fused_theta": (ctypes.c_int, [ctypes.POINTER(CsBatch), ctypes.POINTER(CsOptions),
                                            c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                            c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                            c_void_p, c_size_t, c_void_p]),
    "cs_plan_create_fused_theta": (ctypes.c_int, [ctypes.POINTER(CsBatch),
                                                  ctypes.POINTER(CsOptions), c_void_p, c_void_p,
                                                  c_void_p, c_void_p, c_void_p, c_void_p,
                                                  c_void_p, c_void_p, c_void_p, c_void_p,
                                                  c_int32, c_void_p, ctypes.POINTER(c_void_p)]),
    "cs_solve_fused": (ctypes.c_int, [ctypes.POINTER(CsBatch), ctypes.POINTER(CsOptions),
                                      c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                      c_void_p, c_void_p, c_void_p, c_void_p, c_size_t,
                                      c_void_p]),
    "cs_plan_create_fused": (ctypes.c_int, [ctypes.POINTER(CsBatch), ctypes.POINTER(CsOptions),
                                            c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                            c_void_p, c_void_p, c_void_p, c_int32, c_void_p,
                                            ctypes.POINTER(c_void_p)]),
    "cs_plan_launch": (ctypes.c_int, [c_void_p, c_void_p]),
    "cs_plan_describe": (ctypes.c_int, [c_void_p, ctypes.POINTER(CsPlanInfo)]),
    "cs_plan_destroy": (None, [c_void_p]),
    "cs_autotune_cache_dump": (ctypes.c_int, [ctypes.c_char_p, c_size_t]),
    "cs_autotune_cache_load": (ctypes.c_int, [ctypes.c_char_p]),
    "cs_solve_fused_static": (ctypes.c_int, [ctypes.POINTER(CsBatch), ctypes.POINTER(CsOptions),
                                             c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                             c_void_p, c_void_p, c_void_p, c_void_p]),
    "cs_serve_create": (ctypes.c_int, [ctypes.POINTER(CsServeConfig), ctypes.POINTER(c_void_p)]),
    "cs_serve_submit": (ctypes.c_int, [c_void_p, ctypes.POINTER(CsRequest),
                                       ctypes.POINTER(ctypes.c_uint64)]),
    "cs_serve_poll": (ctypes.c_int, [c_void_p, ctypes.c_uint64, ctypes.POINTER(CsResult)]),
    "cs_serve_cancel": (ctypes.c_int, [c_void_p, ctypes.c_uint64]),
    "cs_serve_submit_batch": (ctypes.c_int, [c_void_p, c_int32, ctypes.POINTER(CsRequest),
                                             ctypes.POINTER(ctypes.c_uint64)]),
    "cs_serve_poll_batch": (ctypes.c_int, [c_void_p, c_int32, ctypes.POINTER(ctypes.c_uint64),
                                           ctypes.POINTER(CsResult), ctypes.POINTER(c_int32)]),
    "cs_serve_clock": (ctypes.c_double, []),
    "cs_serve_replay": (ctypes.c_int, [c_void_p, c_int32, ctypes.POINTER(CsRequest),
                                       ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                                       ctypes.POINTER(ctypes.c_uint64)]),
    "cs_serve_flush": (ctypes.c_int, [c_void_p]),
    "cs_serve_get_stats": (ctypes.c_int, [c_void_p, ctypes.POINTER(CsServeStats)]),
    "cs_serve_destroy": (None, [c_void_p]),
    "cs_serve_set_fault_hook": (ctypes.c_int, [c_void_p, SERVE_FAULT_FN, c_void_p]),
    "cs_serve_completed": (ctypes.c_int, [c_void_p, c_int32, c_void_p]),
}

STATIC_MAX_INSTANCES = 1 << 20

_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load libcs_b300.so (raises if it is missing or lacks a symbol)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(
                f"CUDA library {p} is missing: build it with "
                "`python -m paper_2607_24959_b300.build` (no CPU fallback exists)")
        lib = ctypes.CDLL(p)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def register(name, restype, argtypes):
    """Declare another entry point's signature (used by optional modules)."""
    _SIGS[name] = (restype, argtypes)
    if _lib is not None:
        fn = getattr(_lib, name)
        fn.restype = restype
        fn.argtypes = argtypes


def check(rc: int, what: str) -> int:
    if rc < 0:
        lib = load()
        msg = lib.cs_last_error().decode(errors="replace")
        raise RuntimeError(f"{what} failed: {lib.cs_strerror(rc).decode()} ({rc}): {msg}")
    return rc
