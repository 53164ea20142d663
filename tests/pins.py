"""Independent checks used to pin the oracle (and, later, the GPU path).

Nothing here is shared with ``oracle/`` or the CUDA library.  The key order is
re-derived from its definitions in a different formulation:

* integers: Python's integer ``<``;
* binary32: IEEE 754-2008 Sec. 5.10 totalOrder written as the standard's case
  analysis on numeric value, sign of zero, and NaN sign / kind / payload (the
  oracle instead compares sign and magnitude bit fields).

The brute-force sorts (stable selection sort, stable insertion sort) are the
textbook algorithms written in plain Python.
"""
from __future__ import annotations

import struct

import numpy as np


def f32_value(bits: int) -> float:
    return struct.unpack("<f", struct.pack("<I", bits & 0xFFFFFFFF))[0]


def ieee_total_order_lt(a_bits: int, b_bits: int) -> bool:
    """totalOrder(a, b) and a != b, for binary32 bit patterns."""
    a, b = f32_value(a_bits), f32_value(b_bits)
    a_nan, b_nan = a != a, b != b
    sa, sb = a_bits >> 31 & 1, b_bits >> 31 & 1
    if not a_nan and not b_nan:
        if a < b:
            return True
        if a > b:
            return False
        return sa == 1 and sb == 0  # only -0 vs +0 are numerically equal but distinct
    if a_nan and b_nan:
        if sa != sb:
            return sa == 1
        ka = (a_bits >> 22 & 1, a_bits & 0x3FFFFF)  # (quiet bit, payload)
        kb = (b_bits >> 22 & 1, b_bits & 0x3FFFFF)
        return ka < kb if sa == 0 else ka > kb
    if a_nan:
        return sa == 1  # -NaN is below every number, +NaN above
    return sb == 0


def lt_for(dtype, descending: bool = False):
    """Strict precedence on raw key bits of ``dtype`` (numpy dtype or str)."""
    dt = np.dtype(dtype)
    base = ieee_total_order_lt if dt == np.float32 else (lambda a, b: a < b)
    if descending:
        return lambda a, b: base(b, a)
    return base


def as_bits(keys: np.ndarray) -> list[int]:
    if keys.dtype == np.float32:
        return [int(x) for x in keys.view(np.uint32)]
    return [int(x) for x in keys]


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
    kin = keys_in.view(np.uint32) if keys_in.dtype == np.float32 else keys_in
    kout = keys_out.view(np.uint32) if keys_out.dtype == np.float32 else keys_out
    assert np.array_equal(kin[perm], kout), "key/payload pairing broken"
    r = order_rank(keys_out)
    if descending:
        r = -r
    d = np.diff(r)
    assert np.all(d >= 0), "output not sorted"
    ties = d == 0
    assert np.all(np.diff(perm)[ties] > 0), "equal keys out of input order (unstable)"


def order_rank(keys: np.ndarray) -> np.ndarray:
    """A vectorised int64 rank that is strictly monotone in the key order.

    u32: the value.  u64: the value with its top bit flipped, viewed as int64.
    f32: negative-signed patterns rank by descending magnitude below every
    positive-signed pattern, which rank by ascending magnitude.  The f32 rank
    is itself checked against :func:`ieee_total_order_lt` in the pin tests.
    """
    if keys.dtype == np.float32:
        b = keys.view(np.uint32).astype(np.int64)
        sign = b >> 31
        mag = b & 0x7FFFFFFF
        return np.where(sign == 1, -1 - mag, mag)
    if keys.dtype == np.uint64:
        # map to a signed int64 with the same order by flipping the top bit
        return (keys ^ np.uint64(1 << 63)).view(np.int64)
    return keys.astype(np.int64)
