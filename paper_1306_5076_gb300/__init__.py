"""GB300-native bank-conflict-free comparison merge sort (arXiv 1306.5076).

Python binding of the C ABI in ``include/bcfsort.h``: the functions below have
the C names and only marshal arguments (tensor -> device pointer, stream,
options) and turn non-OK status codes into :class:`BcfError`.  Every step of
the sort runs in the CUDA kernels of ``libbcfsort.so``; there is no CPU or
library fallback.  PyTorch supplies device memory and streams only.

Keys (the code ``key_dtype_of`` picks from the tensor's dtype; pass ``kt`` to
read a tensor's bits as another type): torch.uint16 / uint32 / uint64 in
natural order, torch.int16 / int32 / int64 in two's-complement order,
torch.float32 / float64 under IEEE 754 totalOrder.
Values: 32-bit tensors (torch.int32 / torch.uint32).
"""
from __future__ import annotations

import ctypes

from . import _native
from ._native import (BCF_ALGO_MERGE, BCF_ALGO_PIVOT_BUCKETS, BCF_CPS_BANKED, BCF_CPS_ROWS,
                      BCF_F32, BCF_F64, BCF_I16, BCF_I32, BCF_I64, BCF_OP_CPS, BCF_OP_MERGE,
                      BCF_OP_SEGMENTED, BCF_OP_SORT, BCF_OP_SORT_PB, BCF_U16, BCF_U32, BCF_U64)

__all__ = [
    "BcfError", "bcf_workspace_bytes", "bcf_sort_keys", "bcf_sort_pairs", "bcf_merge_runs",
    "bcf_segmented_sort", "bcf_last_device_error", "bcf_sort_plan", "bcf_profile_enable",
    "bcf_profile_collect", "bcf_profile_collect_launches", "bcf_version",
    "bcf_sort_keys_static", "bcf_tuning_set",
    "bcf_tuning_config", "bcf_tuning_supported", "key_dtype_of", "BCF_U32",
    "BCF_U64", "BCF_F32", "BCF_I32", "BCF_I64", "BCF_F64", "BCF_U16", "BCF_I16",
    "BCF_OP_SORT", "BCF_OP_MERGE", "BCF_OP_SEGMENTED", "BCF_OP_CPS",
    "bcf_colored_prefix_sums", "BCF_CPS_BANKED", "BCF_CPS_ROWS", "BCF_OP_SORT_PB",
    "BCF_ALGO_MERGE", "BCF_ALGO_PIVOT_BUCKETS", "bcf_sort_keys_host", "bcf_sort_pairs_host",
    "bcf_sort_pairs_wide", "bcf_set_wait_limit_us", "bcf_wait_limit_us",
    "bcf_profile_set_smem_floor",
]


class BcfError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = _native.load().bcf_status_string(status).decode()
        super().__init__(f"{what}: {msg}" if what else msg)


def _check(status: int, what: str) -> None:
    if status != 0:
        raise BcfError(status, what)


def key_dtype_of(t) -> int:
    """C key-type code of a tensor's dtype: float32 / float64 sort under IEEE
    totalOrder, int16 / int32 / int64 as signed integers, uint16 / uint32 /
    uint64 as unsigned.
    (To sort the bits of a signed tensor as unsigned, pass ``kt`` explicitly.)"""
    import torch

    table = {torch.float32: BCF_F32, torch.float64: BCF_F64, torch.int32: BCF_I32,
             torch.int64: BCF_I64, torch.int16: BCF_I16}
    for name, code in (("uint32", BCF_U32), ("uint64", BCF_U64), ("uint16", BCF_U16)):
        if hasattr(torch, name):
            table[getattr(torch, name)] = code
    try:
        return table[t.dtype]
    except KeyError:
        raise TypeError(f"unsupported key dtype {t.dtype}") from None


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("bcfsort: tensors must be CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("bcfsort: tensors must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


_ALGORITHMS = {"merge": 0, "pivot_buckets": 1, "auto": 2}


def _opts(descending: bool, algorithm: str = "merge"):
    try:
        algo = _ALGORITHMS[algorithm]
    except KeyError:
        raise ValueError(f"unknown algorithm {algorithm!r} (merge, pivot_buckets, auto)") from None
    return ctypes.byref(_native.BcfOpts(int(bool(descending)), 1, algo))


def _workspace(op, n, k, kt, has_vals, ws, device):
    import torch

    need = bcf_workspace_bytes(op, n, k, kt, has_vals)
    if ws is None:
        ws = torch.empty(max(need, 1), dtype=torch.uint8, device=device)
    return ws, ws.numel() * ws.element_size()


def bcf_workspace_bytes(op: int, n: int, nseg_or_k: int, kt: int, has_vals: bool) -> int:
    return int(_native.load().bcf_workspace_bytes(op, n, nseg_or_k, kt, int(bool(has_vals))))


def _sort_op(algorithm: str) -> int:
    return BCF_OP_SORT_PB if algorithm in ("pivot_buckets", "auto") else BCF_OP_SORT


def bcf_sort_keys(keys_out, keys_in, *, descending=False, ws=None, stream=None, kt=None,
                  algorithm="merge"):
    """Sort ``keys_in`` into ``keys_out`` (may be the same tensor).  ``algorithm``:
    "merge" (block sort + merge passes) or "pivot_buckets" (BCFMergesortPB)."""
    kt = key_dtype_of(keys_in) if kt is None else kt
    n = keys_in.numel()
    opts = _opts(descending, algorithm)
    ws, wsb = _workspace(_sort_op(algorithm), n, 0, kt, False, ws, keys_in.device)
    _check(_native.load().bcf_sort_keys(_ptr(keys_out), _ptr(keys_in), n, kt, opts,
                                        _ptr(ws), wsb, _stream(stream)), "bcf_sort_keys")
    return keys_out


def bcf_sort_pairs_wide(keys_out, vals_out, keys_in, vals_in, *, descending=False, ws=None,
                        stream=None, kt=None, algorithm="merge"):
    """Stable sort by key with payload rows wider than 32 bits: ``vals_in`` is a
    CUDA tensor whose first dimension is n (any dtype; each row a multiple of 4
    bytes), e.g. int64 row ids or an [n, 3] float32 array.  ``vals_out`` must
    be a different tensor of the same shape."""
    kt = key_dtype_of(keys_in) if kt is None else kt
    n = keys_in.numel()
    if vals_in.shape != vals_out.shape or vals_in.shape[0] != n:
        raise ValueError("bcf_sort_pairs_wide: payloads must be n rows, in and out alike")
    row_bytes = vals_in.numel() * vals_in.element_size() // max(n, 1)
    ws, wsb = _workspace(_native.BCF_OP_SORT_WIDE, n, 0, kt, True, ws, keys_in.device)
    _check(_native.load().bcf_sort_pairs_wide(_ptr(keys_out), _ptr(vals_out), _ptr(keys_in),
                                              _ptr(vals_in), n, row_bytes, kt,
                                              _opts(descending, algorithm), _ptr(ws), wsb,
                                              _stream(stream)), "bcf_sort_pairs_wide")
    return keys_out, vals_out


def _host_ptr(t):
    if t is None:
        return None
    if t.is_cuda:
        raise ValueError("bcfsort: host-buffer calls take CPU tensors")
    if not t.is_contiguous():
        raise ValueError("bcfsort: tensors must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def bcf_sort_keys_host(keys_out, keys_in, *, descending=False, ws=None, stream=None, kt=None,
                       algorithm="merge", device=None):
    """Sort keys held in host memory (CPU tensors, ideally pinned): copy in, sort
    and copy out, asynchronously on ``stream``; the copy-in overlaps the block
    sort.  ``ws``: a device workspace of ``bcf_workspace_bytes(BCF_OP_SORT_HOST,
    ...)`` bytes (allocated if None)."""
    import torch

    kt = key_dtype_of(keys_in) if kt is None else kt
    n = keys_in.numel()
    op = (_native.BCF_OP_SORT_HOST_PB if algorithm in ("pivot_buckets", "auto")
          else _native.BCF_OP_SORT_HOST)
    device = device or torch.device("cuda", torch.cuda.current_device())
    ws, wsb = _workspace(op, n, 0, kt, False, ws, device)
    _check(_native.load().bcf_sort_keys_host(_host_ptr(keys_out), _host_ptr(keys_in), n, kt,
                                             _opts(descending, algorithm), _ptr(ws), wsb,
                                             _stream(stream)), "bcf_sort_keys_host")
    return keys_out


def bcf_sort_pairs_host(keys_out, vals_out, keys_in, vals_in, *, descending=False, ws=None,
                        stream=None, kt=None, algorithm="merge", device=None):
    """Stable sort of (key, value) pairs held in host memory (see
    :func:`bcf_sort_keys_host`)."""
    import torch

    kt = key_dtype_of(keys_in) if kt is None else kt
    n = keys_in.numel()
    op = (_native.BCF_OP_SORT_HOST_PB if algorithm in ("pivot_buckets", "auto")
          else _native.BCF_OP_SORT_HOST)
    device = device or torch.device("cuda", torch.cuda.current_device())
    ws, wsb = _workspace(op, n, 0, kt, True, ws, device)
    _check(_native.load().bcf_sort_pairs_host(_host_ptr(keys_out), _host_ptr(vals_out),
                                              _host_ptr(keys_in), _host_ptr(vals_in), n, kt,
                                              _opts(descending, algorithm), _ptr(ws), wsb,
                                              _stream(stream)), "bcf_sort_pairs_host")
    return keys_out, vals_out


def bcf_sort_pairs(keys_out, vals_out, keys_in, vals_in, *, descending=False, ws=None,
                   stream=None, kt=None, algorithm="merge"):
    """Stable sort of (key, value) pairs (``algorithm`` as for :func:`bcf_sort_keys`)."""
    kt = key_dtype_of(keys_in) if kt is None else kt
    n = keys_in.numel()
    if vals_in.numel() != n or vals_out.numel() != n or keys_out.numel() != n:
        raise ValueError("bcf_sort_pairs: length mismatch")
    opts = _opts(descending, algorithm)
    ws, wsb = _workspace(_sort_op(algorithm), n, 0, kt, True, ws, keys_in.device)
    _check(_native.load().bcf_sort_pairs(_ptr(keys_out), _ptr(vals_out), _ptr(keys_in),
                                         _ptr(vals_in), n, kt, opts, _ptr(ws), wsb,
                                         _stream(stream)), "bcf_sort_pairs")
    return keys_out, vals_out


def bcf_merge_runs(keys_out, vals_out, keys_in, vals_in, run_offsets, *, descending=False,
                   ws=None, stream=None, kt=None):
    """Stable merge of the sorted runs delimited by host ``run_offsets`` (k+1 ints)."""
    kt = key_dtype_of(keys_in) if kt is None else kt
    offs = [int(x) for x in run_offsets]
    k = len(offs) - 1
    arr = (ctypes.c_uint64 * max(len(offs), 1))(*offs)
    n = offs[-1] if offs else 0
    ws, wsb = _workspace(BCF_OP_MERGE, n, max(k, 0), kt, vals_in is not None, ws, keys_in.device)
    _check(_native.load().bcf_merge_runs(_ptr(keys_out), _ptr(vals_out), _ptr(keys_in),
                                         _ptr(vals_in), arr, k, kt, _opts(descending), _ptr(ws),
                                         wsb, _stream(stream)), "bcf_merge_runs")
    return keys_out, vals_out


def bcf_segmented_sort(keys_out, vals_out, keys_in, vals_in, seg_offsets, *, descending=False,
                       ws=None, stream=None, kt=None):
    """Sort every segment; ``seg_offsets`` is a CUDA uint64/int64 tensor of nseg+1 offsets."""
    kt = key_dtype_of(keys_in) if kt is None else kt
    nseg = seg_offsets.numel() - 1
    n = keys_in.numel()
    ws, wsb = _workspace(BCF_OP_SEGMENTED, n, nseg, kt, vals_in is not None, ws, keys_in.device)
    _check(_native.load().bcf_segmented_sort(_ptr(keys_out), _ptr(vals_out), _ptr(keys_in),
                                             _ptr(vals_in), _ptr(seg_offsets), nseg, n, kt,
                                             _opts(descending), _ptr(ws), wsb, _stream(stream)),
           "bcf_segmented_sort")
    return keys_out, vals_out


def bcf_colored_prefix_sums(out, values, colors, d: int, *, exclusive=False,
                            layout=BCF_CPS_BANKED, ws=None, stream=None):
    """Colored prefix sums (Appendix A): ``out[i]`` = sum mod 2^32 of ``values[j]``
    over ``j <= i`` (``j < i`` if exclusive) with ``colors[j] == colors[i]``.
    ``values`` / ``out`` are 4-byte integer CUDA tensors, ``colors`` a uint8 CUDA
    tensor with entries < d (1 <= d <= 64)."""
    n = values.numel()
    if colors.numel() != n or out.numel() != n:
        raise ValueError("bcf_colored_prefix_sums: out, values and colors differ in length")
    if values.element_size() != 4 or out.element_size() != 4 or colors.element_size() != 1:
        raise TypeError("bcf_colored_prefix_sums: 4-byte values/out and 1-byte colors expected")
    need = _native.load().bcf_workspace_bytes(BCF_OP_CPS, n, d, BCF_U32, 0)
    if need == 0 and n > 0:
        raise BcfError(1, "bcf_colored_prefix_sums: d must be in 1..64")
    ws, wsb = _workspace(BCF_OP_CPS, n, d, BCF_U32, False, ws, values.device)
    _check(_native.load().bcf_colored_prefix_sums(_ptr(out), _ptr(values), _ptr(colors), n, d,
                                                  int(bool(exclusive)), int(layout), _ptr(ws),
                                                  wsb, _stream(stream)),
           "bcf_colored_prefix_sums")
    return out


def bcf_last_device_error(stream=None) -> int:
    return int(_native.load().bcf_last_device_error(_stream(stream)))


def bcf_sort_plan(n: int, kt: int, has_vals: bool) -> dict:
    p = _native.BcfPlan()
    _check(_native.load().bcf_sort_plan(n, kt, int(bool(has_vals)), ctypes.byref(p)),
           "bcf_sort_plan")
    return {f: getattr(p, f) for f, _ in p._fields_}


def bcf_set_wait_limit_us(limit_us: int) -> None:
    """Limit of every device-side bounded wait, in microseconds (0: 2 s)."""
    _check(_native.load().bcf_set_wait_limit_us(int(limit_us)), "bcf_set_wait_limit_us")


def bcf_wait_limit_us() -> int:
    return int(_native.load().bcf_wait_limit_us())


def bcf_profile_set_smem_floor(nbytes: int) -> None:
    """Profiling control: minimum dynamic shared memory of the block sort and
    merge-pass launches (0: as built); limits the CTAs sharing an SM."""
    _check(_native.load().bcf_profile_set_smem_floor(int(nbytes)), "bcf_profile_set_smem_floor")


def bcf_profile_enable(on: bool = True) -> None:
    _check(_native.load().bcf_profile_enable(int(bool(on))), "bcf_profile_enable")


PROFILE_KINDS = ("block_sort", "partition", "merge", "segmented", "colored_prefix_sums",
                 "pivot_buckets")


def bcf_profile_collect() -> dict:
    p = _native.BcfProfile()
    _check(_native.load().bcf_profile_collect(ctypes.byref(p)), "bcf_profile_collect")
    return {k: {"launches": int(p.launches[i]), "total_ms": float(p.total_ms[i])}
            for i, k in enumerate(PROFILE_KINDS)}


def bcf_profile_collect_launches(max_launches: int = 4096):
    """Like bcf_profile_collect, plus every recorded launch in order as
    (kind name, ms) -- e.g. each merge pass of a sort on its own."""
    p = _native.BcfProfile()
    kinds = (ctypes.c_int * max_launches)()
    ms = (ctypes.c_float * max_launches)()
    count = ctypes.c_uint32(0)
    _check(_native.load().bcf_profile_collect_launches(ctypes.byref(p), kinds, ms, max_launches,
                                                       ctypes.byref(count)),
           "bcf_profile_collect_launches")
    totals = {k: {"launches": int(p.launches[i]), "total_ms": float(p.total_ms[i])}
              for i, k in enumerate(PROFILE_KINDS)}
    n = min(int(count.value), max_launches)
    return totals, [(PROFILE_KINDS[kinds[i]] if 0 <= kinds[i] < len(PROFILE_KINDS) else str(kinds[i]),
                     float(ms[i])) for i in range(n)]


def bcf_sort_keys_static(keys_out, keys_in, *, descending=False, stream=None, kt=None):
    """Sort without a caller workspace: the library's own device array serves as
    scratch, so neither this call nor the library allocates (at most
    ``_native.BCF_STATIC_MAX_KEYS`` keys; calls must not overlap on the GPU)."""
    kt = key_dtype_of(keys_in) if kt is None else kt
    _check(_native.load().bcf_sort_keys_static(_ptr(keys_out), _ptr(keys_in), keys_in.numel(),
                                               kt, _opts(descending), _stream(stream)),
           "bcf_sort_keys_static")
    return keys_out


def bcf_tuning_set(entries) -> None:
    """Install a tuning table: a list of dicts with the fields of bcf_tuning_entry
    ([] -> built-in defaults, None -> the package's table file again)."""
    lib = _native.load()
    if entries is None:
        _check(lib.bcf_tuning_set(None, -1), "bcf_tuning_set")
        return
    arr = (_native.BcfTuningEntry * max(len(entries), 1))()
    for i, e in enumerate(entries):
        for k, v in e.items():
            setattr(arr[i], k, v)
    _check(lib.bcf_tuning_set(arr, len(entries)), "bcf_tuning_set")


def bcf_tuning_config(kind: int, index: int):
    """(E, NT) of configuration `index` of kind 0 block / 1 merge / 2 segmented, or None."""
    e, t = ctypes.c_int(), ctypes.c_int()
    if not _native.load().bcf_tuning_config(kind, index, ctypes.byref(e), ctypes.byref(t)):
        return None
    return e.value, t.value


def bcf_tuning_supported(kind: int, index: int, key_bytes: int, has_vals: bool) -> bool:
    return bool(_native.load().bcf_tuning_supported(kind, index, key_bytes, int(bool(has_vals))))


def bcf_version() -> str:
    return _native.load().bcf_version().decode()
