"""Independent checks used to pin the oracle (and, later, the GPU path).

Nothing here is shared with ``oracle/`` or the CUDA library.  The key order is
re-derived from its definitions in a different formulation:

* integers: Python's integer ``<`` on the unsigned or two's-complement value;
* binary32 / binary64: IEEE 754-2008 Sec. 5.10 totalOrder written as the
  standard's case analysis on numeric value, sign of zero, and NaN sign / kind /
  payload (the oracle instead compares sign and magnitude bit fields).

The brute-force sorts (stable selection sort, stable insertion sort) are the
textbook algorithms written in plain Python.
"""
from __future__ import annotations

import struct

import numpy as np


def f32_value(bits: int) -> float:
    return struct.unpack("<f", struct.pack("<I", bits & 0xFFFFFFFF))[0]


def f64_value(bits: int) -> float:
    return struct.unpack("<d", struct.pack("<Q", bits & 0xFFFFFFFFFFFFFFFF))[0]


def ieee_total_order_lt(a_bits: int, b_bits: int, width: int = 32) -> bool:
    """totalOrder(a, b) and a != b, for binary32 (width 32) or binary64 (width
    64) bit patterns."""
    value = f32_value if width == 32 else f64_value
    frac_bits = 23 if width == 32 else 52  # the quiet bit is the top fraction bit
    a, b = value(a_bits), value(b_bits)
    a_nan, b_nan = a != a, b != b
    sa, sb = a_bits >> (width - 1) & 1, b_bits >> (width - 1) & 1
    if not a_nan and not b_nan:
        if a < b:
            return True
        if a > b:
            return False
        return sa == 1 and sb == 0  # only -0 vs +0 are numerically equal but distinct
    if a_nan and b_nan:
        if sa != sb:
            return sa == 1
        pmask = (1 << (frac_bits - 1)) - 1
        ka = (a_bits >> (frac_bits - 1) & 1, a_bits & pmask)  # (quiet bit, payload)
        kb = (b_bits >> (frac_bits - 1) & 1, b_bits & pmask)
        return ka < kb if sa == 0 else ka > kb
    if a_nan:
        return sa == 1  # -NaN is below every number, +NaN above
    return sb == 0


def lt_for(dtype, descending: bool = False):
    """Strict precedence on the keys :func:`as_bits` gives for ``dtype``: raw
    bit patterns for floats, integer values (signed for i32 / i64) otherwise."""
    dt = np.dtype(dtype)
    if dt == np.float32:
        base = ieee_total_order_lt
    elif dt == np.float64:
        base = lambda a, b: ieee_total_order_lt(a, b, 64)  # noqa: E731
    else:
        base = lambda a, b: a < b  # noqa: E731
    if descending:
        return lambda a, b: base(b, a)
    return base


def as_bits(keys: np.ndarray) -> list[int]:
    if keys.dtype == np.float32:
        return [int(x) for x in keys.view(np.uint32)]
    if keys.dtype == np.float64:
        return [int(x) for x in keys.view(np.uint64)]
    return [int(x) for x in keys]


def raw_bits(keys: np.ndarray) -> np.ndarray:
    """The keys' bit patterns as an unsigned array of the same width."""
    return keys.view({2: np.uint16, 4: np.uint32, 8: np.uint64}[keys.dtype.itemsize])


def stable_selection_sort(items, lt):
    """Repeatedly take the FIRST minimal remaining item (stable by construction)."""
    rest = list(items)
    out = []
    while rest:
        m = 0
        for i in range(1, len(rest)):
            if lt(rest[i][0], rest[m][0]):
                m = i
        out.append(rest.pop(m))
    return out


def stable_insertion_sort(items, lt):
    """Insertion sort that moves an item left only past strictly greater items."""
    a = list(items)
    for i in range(1, len(a)):
        x = a[i]
        j = i - 1
        while j >= 0 and lt(x[0], a[j][0]):
            a[j + 1] = a[j]
            j -= 1
        a[j + 1] = x
    return a


def check_sorted_stable(keys_in, vals_in, keys_out, vals_out, descending=False):
    """Invariants every correct stable sort output satisfies (vals_in = index).

    1. keys_out is non-decreasing under the (direction-adjusted) key order;
    2. (keys_out, vals_out) is a permutation of (keys_in, vals_in) -- checked
       exactly via vals_out being a permutation and keys_out[i] being the key
       that was at input position vals_out[i];
    3. stability: within a run of equal keys the row indices increase.
    Vectorised for integer dtypes; f32 is mapped through totalOrder ranks
    computed from the golden definition of the order (sign/magnitude by
    case analysis on numpy, not the oracle).
    """
    n = keys_in.size
    assert keys_out.size == n and vals_out.size == n
    perm = vals_out.astype(np.int64)
    assert np.array_equal(np.sort(perm), np.arange(n)), "payloads are not a permutation"
    kin, kout = raw_bits(keys_in), raw_bits(keys_out)
    assert np.array_equal(kin[perm], kout), "key/payload pairing broken"
    r = order_rank(keys_out)
    lo, hi = (r[1:], r[:-1]) if descending else (r[:-1], r[1:])  # no int64 overflow
    assert np.all(lo <= hi), "output not sorted"
    ties = lo == hi
    assert np.all(np.diff(perm)[ties] > 0), "equal keys out of input order (unstable)"


def order_rank(keys: np.ndarray) -> np.ndarray:
    """A vectorised int64 rank that is strictly monotone in the key order.

    u32 / i32 / i64: the value.  u64: the value with its top bit flipped,
    viewed as int64.  f32 / f64: negative-signed patterns rank by descending
    magnitude below every positive-signed pattern, which rank by ascending
    magnitude.  The float ranks are themselves checked against
    :func:`ieee_total_order_lt` in the pin tests.
    """
    if keys.dtype == np.float32:
        b = keys.view(np.uint32).astype(np.int64)
        sign = b >> 31
        mag = b & 0x7FFFFFFF
        return np.where(sign == 1, -1 - mag, mag)
    if keys.dtype == np.float64:
        b = keys.view(np.uint64)
        sign = (b >> np.uint64(63)).astype(np.int64)
        mag = (b & np.uint64(0x7FFFFFFFFFFFFFFF)).astype(np.int64)
        return np.where(sign == 1, -1 - mag, mag)
    if keys.dtype == np.int64:
        return keys.copy()
    if keys.dtype == np.uint64:
        # map to a signed int64 with the same order by flipping the top bit
        return (keys ^ np.uint64(1 << 63)).view(np.int64)
    return keys.astype(np.int64)
