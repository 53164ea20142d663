"""The FMA-pipe forms of the compare-exchange (csrc/bcf_device.cuh, ce) are
exact in modular arithmetic (CPU only).

The kernels compute, with 32-bit integer multiply-adds (multiplier 1 or -1
read at run time):
  kFmaKeys:   max(x, y) = x * 1 + y - min(x, y)            (mod 2^32)
  kFmaPairs / kFmaKeys64, per 32-bit word, with s = 1 to swap and 0 to keep:
              x' = x + s * (y - x),  y' = (x + y) - x'     (mod 2^32)
This restates both with numpy's wrapping uint32 arithmetic and checks them
on the extremes and random words, and that a 64-bit key swapped half by half
is the swapped key.
"""
from __future__ import annotations

import numpy as np


def mad(a, b, c):
    """mad.lo.u32: the low 32 bits of a * b + c."""
    with np.errstate(over="ignore"):
        return (a.astype(np.uint64) * b.astype(np.uint64) + c.astype(np.uint64)).astype(np.uint32)


def words():
    r = np.random.default_rng(7)
    edge = np.array([0, 1, 2, 0x7FFFFFFF, 0x80000000, 0x80000001, 0xFFFFFFFE, 0xFFFFFFFF],
                    dtype=np.uint32)
    x = np.concatenate([np.repeat(edge, edge.size), r.integers(0, 1 << 32, 20000, dtype=np.uint64)
                        .astype(np.uint32)])
    y = np.concatenate([np.tile(edge, edge.size), r.integers(0, 1 << 32, 20000, dtype=np.uint64)
                        .astype(np.uint32)])
    return x, y


def test_fma_max_is_the_maximum():
    x, y = words()
    one, neg = np.uint32(1), np.uint32(0xFFFFFFFF)  # 1 and -1 mod 2^32
    lo = np.minimum(x, y)
    hi = mad(lo, np.full_like(x, neg), mad(x, np.full_like(x, one), y))
    assert np.array_equal(hi, np.maximum(x, y))


def swap_word(x, y, s):
    one, neg = np.full_like(x, 1), np.full_like(x, 0xFFFFFFFF)
    d = mad(x, neg, y)          # y - x
    nx = mad(s, d, x)           # x + s (y - x)
    t = mad(x, one, y)          # x + y
    ny = mad(nx, neg, t)        # x + y - x'
    return nx, ny


def test_fma_swap_swaps_or_keeps():
    x, y = words()
    for sval in (0, 1):
        s = np.full_like(x, sval)
        nx, ny = swap_word(x, y, s)
        assert np.array_equal(nx, y if sval else x)
        assert np.array_equal(ny, x if sval else y)


def test_64_bit_key_swapped_half_by_half():
    r = np.random.default_rng(11)
    a = r.integers(0, 1 << 63, 5000, dtype=np.uint64) * 2 + r.integers(0, 2, 5000, dtype=np.uint64)
    b = r.integers(0, 1 << 63, 5000, dtype=np.uint64) * 2 + r.integers(0, 2, 5000, dtype=np.uint64)
    s = (a > b).astype(np.uint32)  # ascending: swap when a > b
    lo_a, hi_a = (a & 0xFFFFFFFF).astype(np.uint32), (a >> 32).astype(np.uint32)
    lo_b, hi_b = (b & 0xFFFFFFFF).astype(np.uint32), (b >> 32).astype(np.uint32)
    nla, nlb = swap_word(lo_a, lo_b, s)
    nha, nhb = swap_word(hi_a, hi_b, s)
    na = nla.astype(np.uint64) | (nha.astype(np.uint64) << np.uint64(32))
    nb = nlb.astype(np.uint64) | (nhb.astype(np.uint64) << np.uint64(32))
    assert np.array_equal(na, np.minimum(a, b)) and np.array_equal(nb, np.maximum(a, b))
