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

BCF_U32, BCF_U64, BCF_F32 = 0, 1, 2
BCF_OP_SORT, BCF_OP_MERGE, BCF_OP_SEGMENTED = 0, 1, 2
STATUS = {0: "BCF_OK", 1: "BCF_EINVAL", 2: "BCF_ENOMEM", 3: "BCF_ECUDA", 4: "BCF_ETIMEOUT",
          5: "BCF_EUNSUPPORTED"}


class BcfOpts(ctypes.Structure):
    _fields_ = [("descending", ctypes.c_int), ("stable_required", ctypes.c_int)]


class BcfPlan(ctypes.Structure):
    _fields_ = [("block_tile", ctypes.c_uint32), ("merge_tile", ctypes.c_uint32),
                ("merge_passes", ctypes.c_uint32), ("launches", ctypes.c_uint32),
                ("bytes_per_pass", ctypes.c_uint64)]


class BcfTuningEntry(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("key_bytes", ctypes.c_int), ("has_vals", ctypes.c_int),
                ("n_min", ctypes.c_uint64), ("n_max", ctypes.c_uint64),
                ("block_cfg", ctypes.c_int), ("merge_cfg", ctypes.c_int), ("seg_cfg", ctypes.c_int)]


class BcfProfile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint32 * 4), ("total_ms", ctypes.c_double * 4)]


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
    "bcf_version": (ctypes.c_char_p, []),
    "bcf_sort_keys_static": (_i32, [_vp, _vp, _u64, _i32, ctypes.POINTER(BcfOpts), _vp]),
    "bcf_tuning_set": (_i32, [ctypes.POINTER(BcfTuningEntry), _i32]),
    "bcf_tuning_config": (_i32, [_i32, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "bcf_tuning_supported": (_i32, [_i32, _i32, _i32, _i32]),
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
