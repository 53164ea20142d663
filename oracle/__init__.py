"""CPU oracle for the bank-conflict-free merge sort library.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product (``paper_1306_5076_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``bcf_oracle.c`` (plain C, built with gcc into
``oracle/_build/liboracle.so``); this module only marshals numpy arrays.
Each function states the definition it computes:

* :func:`sort` -- "sort N keys" (Sec. 3): stable ascending/descending order,
  f32/f64 keys under IEEE 754 totalOrder, i16/i32/i64 as signed integers,
  u16/u32/u64 as unsigned, payloads kept in input order on ties.
* :func:`merge_runs` -- "merge sorted sequences" (Sec. 3.2, Algorithm 6): the
  stable sort of the runs concatenated in run order.
* :func:`segmented_sort` -- :func:`sort` applied to every segment.
* :func:`colored_prefix_sums` -- d independent prefix sums, one per color
  (Appendix A), modulo 2^32, inclusive or exclusive.

Every function is pinned by ``tests/test_oracle_pins.py``; none is unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bcf_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

_DTYPE_CODE = {np.dtype(np.uint32): 0, np.dtype(np.uint64): 1, np.dtype(np.float32): 2,
               np.dtype(np.int32): 3, np.dtype(np.int64): 4, np.dtype(np.float64): 5,
               np.dtype(np.uint16): 6, np.dtype(np.int16): 7}

_lock = threading.Lock()
_lib = None


def build(force: bool = False, src: str = _SRC, out: str = _LIB_PATH) -> str:
    """Compile the oracle with gcc (plain C11, -O2) into a shared object."""
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                           src, "-o", tmp])
    os.replace(tmp, out)
    return out


def load(path: str | None = None):
    """Load (building first if needed) the oracle library and declare signatures."""
    global _lib
    if path is None and _lib is not None:
        return _lib
    with _lock:
        if path is None and _lib is not None:
            return _lib
        lib = ctypes.CDLL(path or build())
        vp, u64, i32, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32
        lib.oracle_sort.argtypes = [vp, vp, vp, vp, u64, i32, i32, i32]
        lib.oracle_sort.restype = i32
        lib.oracle_merge_runs.argtypes = [vp, vp, vp, vp, vp, u32, i32, i32]
        lib.oracle_merge_runs.restype = i32
        lib.oracle_segmented_sort.argtypes = [vp, vp, vp, vp, vp, u64, i32, i32]
        lib.oracle_segmented_sort.restype = i32
        lib.oracle_key_less.argtypes = [i32, u64, u64]
        lib.oracle_key_less.restype = i32
        lib.oracle_colored_prefix_sums.argtypes = [vp, vp, vp, u64, u32, i32]
        lib.oracle_colored_prefix_sums.restype = i32
        if path is None:
            _lib = lib
        return lib


def _code(keys: np.ndarray) -> int:
    try:
        return _DTYPE_CODE[keys.dtype]
    except KeyError:
        raise TypeError(f"oracle: unsupported key dtype {keys.dtype}") from None


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _prep(keys, vals):
    keys = np.ascontiguousarray(keys)
    if vals is not None:
        vals = np.ascontiguousarray(vals, dtype=np.uint32)
        if vals.shape != keys.shape:
            raise ValueError("oracle: keys and values differ in length")
    return keys, vals


def sort(keys, vals=None, descending: bool = False, nthreads: int = 1, lib=None):
    """Stable sort of ``keys`` (+ ``vals``).  Returns ``(keys_out, vals_out)``."""
    lib = lib or load()
    keys, vals = _prep(keys, vals)
    ko = np.empty_like(keys)
    vo = None if vals is None else np.empty_like(vals)
    rc = lib.oracle_sort(_ptr(ko), _ptr(vo), _ptr(keys), _ptr(vals), keys.size,
                         _code(keys), int(bool(descending)), int(nthreads))
    if rc != 0:
        raise RuntimeError("oracle_sort failed")
    return ko, vo


def merge_runs(keys, vals, run_offsets, descending: bool = False, lib=None):
    """Stable merge of the sorted runs ``[run_offsets[r], run_offsets[r+1])``."""
    lib = lib or load()
    keys, vals = _prep(keys, vals)
    offs = np.ascontiguousarray(run_offsets, dtype=np.uint64)
    ko = keys.copy()
    vo = None if vals is None else vals.copy()
    k = offs.size - 1
    rc = lib.oracle_merge_runs(_ptr(ko), _ptr(vo), _ptr(keys), _ptr(vals), _ptr(offs),
                               max(k, 0), _code(keys), int(bool(descending)))
    if rc != 0:
        raise RuntimeError("oracle_merge_runs failed")
    return ko, vo


def segmented_sort(keys, vals, seg_offsets, descending: bool = False, lib=None):
    """Stable sort of every segment ``[seg_offsets[s], seg_offsets[s+1])``."""
    lib = lib or load()
    keys, vals = _prep(keys, vals)
    offs = np.ascontiguousarray(seg_offsets, dtype=np.uint64)
    ko = keys.copy()
    vo = None if vals is None else vals.copy()
    rc = lib.oracle_segmented_sort(_ptr(ko), _ptr(vo), _ptr(keys), _ptr(vals), _ptr(offs),
                                   max(offs.size - 1, 0), _code(keys), int(bool(descending)))
    if rc != 0:
        raise RuntimeError("oracle_segmented_sort failed")
    return ko, vo


def key_less(dtype, a: int, b: int, lib=None) -> bool:
    """Strict ascending-order test on raw key bit patterns of ``dtype``."""
    lib = lib or load()
    return bool(lib.oracle_key_less(_DTYPE_CODE[np.dtype(dtype)], int(a), int(b)))


def colored_prefix_sums(values, colors, d: int, exclusive: bool = False, lib=None):
    """``out[i]`` = sum (mod 2^32) of ``values[j]`` over ``j <= i`` (``j < i`` if
    exclusive) with ``colors[j] == colors[i]``."""
    lib = lib or load()
    values = np.ascontiguousarray(values, dtype=np.uint32)
    colors = np.ascontiguousarray(colors, dtype=np.uint8)
    if values.shape != colors.shape:
        raise ValueError("oracle: values and colors differ in length")
    out = np.empty_like(values)
    rc = lib.oracle_colored_prefix_sums(_ptr(out), _ptr(values), _ptr(colors), values.size,
                                        int(d), int(bool(exclusive)))
    if rc != 0:
        raise RuntimeError("oracle_colored_prefix_sums failed (color >= d or bad d)")
    return out
