"""Host model of the pivot-bucket sort (BCFMergesortPB; Sec. 3.2, paragraphs
"Distribution" and "Duplicate keys"), CPU only.

Restates, in numpy, what csrc/bcf_pb.cu and the host sequence in
csrc/bcf_api.cu compute: splitters from a sorted sample of every 256th key,
one open bucket between consecutive splitters and one bucket per splitter for
the keys equal to it, per-tile bucket counts of block-sorted tiles, an
exclusive scan in (bucket, tile) order, the scatter of every tile's pieces,
and a stable sort of the open buckets only.  Checks that the result is the
stable sort, that the equal buckets need no further work, and the bucket-size
bound of Lemma 1 on distinct keys.
"""
from __future__ import annotations

import numpy as np
import pytest

import workloads

STRIDE = 256       # sample stride
P = 256            # P - 1 splitters (the library default)
B = 2 * (P - 1) + 1  # open, equal, open, ..., open


def splitters(keys):
    samples = np.sort(keys[::STRIDE], kind="stable")
    ns = samples.size
    cand = [samples[((j + 1) * ns) // P] for j in range(P - 1) if ((j + 1) * ns) // P < ns]
    out = []
    for c in cand:
        if not out or c != out[-1]:
            out.append(c)
    return np.array(out, dtype=keys.dtype)


def pb_sort(keys, T):
    n = keys.size
    idx = np.arange(n)
    s = splitters(keys)
    m = s.size
    R = -(-n // T)
    counts = np.zeros((B, R), np.int64)
    tiles = []
    for t in range(R):
        kt, it = keys[t * T:(t + 1) * T], idx[t * T:(t + 1) * T]
        order = np.argsort(kt, kind="stable")
        kt, it = kt[order], it[order]
        tiles.append((kt, it))
        lo = np.searchsorted(kt, s, side="left")
        hi = np.searchsorted(kt, s, side="right")
        prev = 0
        for j in range(m):
            counts[2 * j, t] = lo[j] - prev
            counts[2 * j + 1, t] = hi[j] - lo[j]
            prev = hi[j]
        counts[2 * m, t] = kt.size - prev
    flat = counts.reshape(-1)
    offs = (np.cumsum(flat) - flat).reshape(B, R)
    out_k = np.empty_like(keys)
    out_i = np.empty_like(idx)
    for t, (kt, it) in enumerate(tiles):
        starts = np.cumsum(counts[:, t]) - counts[:, t]
        for b in range(B):
            c = counts[b, t]
            if c:
                out_k[offs[b, t]:offs[b, t] + c] = kt[starts[b]:starts[b] + c]
                out_i[offs[b, t]:offs[b, t] + c] = it[starts[b]:starts[b] + c]
    seg = np.append(offs[:, 0], n)
    for b in range(B):
        lo_, hi_ = seg[b], seg[b + 1]
        if b > 2 * m:  # buckets past the last splitter's are empty
            assert hi_ == lo_
            continue
        if b % 2 == 1:  # equal bucket: already in its final, stable order
            assert np.all(out_k[lo_:hi_] == s[b // 2])
            assert np.all(np.diff(out_i[lo_:hi_]) > 0)
            continue
        o = np.argsort(out_k[lo_:hi_], kind="stable")
        out_k[lo_:hi_] = out_k[lo_:hi_][o]
        out_i[lo_:hi_] = out_i[lo_:hi_][o]
    return out_k, out_i, counts, seg, m


@pytest.mark.parametrize("dist", ["uniform", "distinct16", "zipf", "gaussian", "sorted"])
@pytest.mark.parametrize("n,T", [(70_000, 4096), (3 * 16384 + 5, 16384)])
def test_pb_equals_stable_sort(dist, n, T):
    keys = workloads.keys(dist, "u32", n, seed=n + T)
    out_k, out_i, counts, seg, m = pb_sort(keys, T)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(out_k, keys[order])
    assert np.array_equal(out_i, order)
    assert np.all(np.diff(seg) >= 0) and seg[-1] == n


def test_pb_all_equal_and_zero_one():
    n, T = 50_000, 4096
    for keys in (np.full(n, 9, np.uint32), workloads.paper_keys("zero_one", n)):
        out_k, out_i, counts, seg, m = pb_sort(keys, T)
        assert np.array_equal(out_i, np.argsort(keys, kind="stable"))
        open_keys = sum(seg[b + 1] - seg[b] for b in range(0, B, 2))
        assert open_keys == 0  # every key sits in an equal bucket: nothing left to sort


def test_duplicates_land_in_equal_buckets():
    """16 distinct values: every value is a splitter, so no key is left in an
    open bucket (the paper's point for BCFMergesortPB)."""
    keys = workloads.keys("distinct16", "u32", 1 << 18, seed=3)
    out_k, out_i, counts, seg, m = pb_sort(keys, 16384)
    assert m == 16
    assert sum(seg[b + 1] - seg[b] for b in range(0, B, 2)) == 0


def test_lemma_1_bucket_bound_on_distinct_keys():
    """Lemma 1 (distinct keys): every bucket holds O(N/t (1 + t/P)) keys; with
    regular samples every 256 keys the open buckets stay within a small
    constant of N / P."""
    n = 1 << 20
    keys = workloads.paper_keys("distinct", n)
    out_k, out_i, counts, seg, m = pb_sort(keys, 16384)
    sizes = np.diff(seg)[0::2]
    assert sizes.max() <= 2 * n / P
