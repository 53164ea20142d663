"""ctypes declarations of the C ABI in ``include/bcfsort.h``.

Loads ``_build/libbcfsort.so`` from this package directory.  There is no
fallback: if the library is missing or does not load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libbcfsort.so")

BCF_U32, BCF_U64, BCF_F32, BCF_I32, BCF_I64, BCF_F64, BCF_U16, BCF_I16 = 0, 1, 2, 3, 4, 5, 6, 7
BCF_CPS_BANKED, BCF_CPS_ROWS = 0, 1
(BCF_OP_SORT, BCF_OP_MERGE, BCF_OP_SEGMENTED, BCF_OP_CPS, BCF_OP_SORT_PB, BCF_OP_SORT_HOST,
 BCF_OP_SORT_HOST_PB, BCF_OP_SORT_WIDE) = 0, 1, 2, 3, 4, 5, 6, 7
BCF_ALGO_MERGE, BCF_ALGO_PIVOT_BUCKETS, BCF_ALGO_AUTO = 0, 1, 2
STATUS = {0: "BCF_OK", 1: "BCF_EINVAL", 2: "BCF_ENOMEM", 3: "BCF_ECUDA", 4: "BCF_ETIMEOUT",
          5: "BCF_EUNSUPPORTED"}


class BcfOpts(ctypes.Structure):
    _fields_ = [("descending", ctypes.c_int), ("stable_required", ctypes.c_int),
                ("algorithm", ctypes.c_int)]


class BcfPlan(ctypes.Structure):
    _fields_ = [("block_tile", ctypes.c_uint32), ("merge_tile", ctypes.c_uint32),
                ("merge_passes", ctypes.c_uint32), ("launches", ctypes.c_uint32),
                ("bytes_per_pass", ctypes.c_uint64)]


class BcfTuningEntry(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("key_bytes", ctypes.c_int), ("has_vals", ctypes.c_int),
                ("n_min", ctypes.c_uint64), ("n_max", ctypes.c_uint64),
                ("block_cfg", ctypes.c_int), ("merge_cfg", ctypes.c_int), ("seg_cfg", ctypes.c_int)]


BCF_PROFILE_KINDS = 6


class BcfProfile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint32 * BCF_PROFILE_KINDS),
                ("total_ms", ctypes.c_double * BCF_PROFILE_KINDS)]


BCF_SERVE_BATCHED, BCF_SERVE_PLAIN = 0, 1


class BcfServerConfig(ctypes.Structure):
    _fields_ = [("arena", ctypes.c_void_p), ("arena_bytes", ctypes.c_uint64),
                ("streams", ctypes.c_int), ("mode", ctypes.c_int),
                ("small_max", ctypes.c_uint64), ("batch_max_keys", ctypes.c_uint64)]


class BcfRequest(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("kt", ctypes.c_int), ("descending", ctypes.c_int),
                ("n", ctypes.c_uint64), ("keys_in", ctypes.c_void_p), ("vals_in", ctypes.c_void_p),
                ("keys_out", ctypes.c_void_p), ("vals_out", ctypes.c_void_p),
                ("run_offsets", ctypes.c_void_p), ("k", ctypes.c_uint32), ("tag", ctypes.c_uint64)]


class BcfCompletion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int), ("submit_s", ctypes.c_double),
                ("admit_s", ctypes.c_double), ("done_s", ctypes.c_double)]


class BcfServerStats(ctypes.Structure):
    _fields_ = [("pending", ctypes.c_uint64), ("inflight", ctypes.c_uint64),
                ("arena_used", ctypes.c_uint64), ("arena_peak", ctypes.c_uint64),
                ("launched_units", ctypes.c_uint64), ("launched_batches", ctypes.c_uint64)]


# name -> (restype, argtypes); the exported symbol set of include/bcfsort.h
_vp, _u64, _u32, _i32, _sz = (ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                               ctypes.c_size_t)
SIGNATURES = {
    "bcf_workspace_bytes": (_sz, [_i32, _u64, _u64, _i32, _i32]),
    "bcf_sort_keys": (_i32, [_vp, _vp, _u64, _i32, ctypes.POINTER(BcfOpts), _vp, _sz, _vp]),
    "bcf_sort_pairs": (_i32, [_vp, _vp, _vp, _vp, _u64, _i32, ctypes.POINTER(BcfOpts), _vp, _sz,
                              _vp]),
    "bcf_merge_runs": (_i32, [_vp, _vp, _vp, _vp, _vp, _u32, _i32, ctypes.POINTER(BcfOpts), _vp,
                              _sz, _vp]),
    "bcf_segmented_sort": (_i32, [_vp, _vp, _vp, _vp, _vp, _u64, _u64, _i32,
                                  ctypes.POINTER(BcfOpts), _vp, _sz, _vp]),
    "bcf_status_string": (ctypes.c_char_p, [_i32]),
    "bcf_last_device_error": (_i32, [_vp]),
    "bcf_sort_plan": (_i32, [_u64, _i32, _i32, ctypes.POINTER(BcfPlan)]),
    "bcf_profile_enable": (_i32, [_i32]),
    "bcf_profile_collect": (_i32, [ctypes.POINTER(BcfProfile)]),
    "bcf_selftest_bounded_wait": (_i32, [_u32, _vp]),
    "bcf_set_wait_limit_us": (_i32, [_u32]),
    "bcf_wait_limit_us": (_u32, []),
    "bcf_selftest_segmented_wait": (_i32, [_vp, _sz, _vp]),
    "bcf_profile_set_smem_floor": (_i32, [_u32]),
    "bcf_profile_collect_launches": (_i32, [ctypes.POINTER(BcfProfile), ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_float), _u32,
                                            ctypes.POINTER(ctypes.c_uint32)]),
    "bcf_version": (ctypes.c_char_p, []),
    "bcf_sort_keys_static": (_i32, [_vp, _vp, _u64, _i32, ctypes.POINTER(BcfOpts), _vp]),
    "bcf_colored_prefix_sums": (_i32, [_vp, _vp, _vp, _u64, _u32, _i32, _i32, _vp, _sz, _vp]),
    "bcf_sort_pairs_wide": (_i32, [_vp, _vp, _vp, _vp, _u64, _u32, _i32, ctypes.POINTER(BcfOpts),
                                   _vp, _sz, _vp]),
    "bcf_sort_keys_host": (_i32, [_vp, _vp, _u64, _i32, ctypes.POINTER(BcfOpts), _vp, _sz, _vp]),
    "bcf_sort_pairs_host": (_i32, [_vp, _vp, _vp, _vp, _u64, _i32, ctypes.POINTER(BcfOpts), _vp,
                                   _sz, _vp]),
    "bcf_tuning_set": (_i32, [ctypes.POINTER(BcfTuningEntry), _i32]),
    "bcf_tuning_config": (_i32, [_i32, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "bcf_tuning_supported": (_i32, [_i32, _i32, _i32, _i32]),
    "bcf_server_create": (_i32, [ctypes.POINTER(BcfServerConfig), ctypes.POINTER(_vp)]),
    "bcf_server_now": (ctypes.c_double, [_vp]),
    "bcf_server_submit": (_i32, [_vp, ctypes.POINTER(BcfRequest)]),
    "bcf_server_step": (_i32, [_vp, ctypes.POINTER(_i32)]),
    "bcf_server_poll": (_i32, [_vp, ctypes.POINTER(BcfCompletion), _i32]),
    "bcf_server_stats": (_i32, [_vp, ctypes.POINTER(BcfServerStats)]),
    "bcf_server_drain": (_i32, [_vp]),
    "bcf_server_destroy": (_i32, [_vp]),
    "bcf_arena_create": (_i32, [_u64, ctypes.POINTER(_vp)]),
    "bcf_arena_alloc": (_i32, [_vp, _u64, ctypes.POINTER(_u64)]),
    "bcf_arena_free": (_i32, [_vp, _u64, _u64]),
    "bcf_arena_usage": (_i32, [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64)]),
    "bcf_arena_destroy": (_i32, [_vp]),
}

# keys per call accepted by bcf_sort_keys_static (BCF_STATIC_MAX_KEYS)
BCF_STATIC_MAX_KEYS = 1 << 20

_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load the library (once) and declare every exported signature."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(
                f"bcfsort CUDA library not found at {p}; build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _lib = lib
        return lib
