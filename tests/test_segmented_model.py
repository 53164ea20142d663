"""Host model of the segmented sort's plan and work-item geometry (CPU only).

Restates, as plain index arithmetic, what csrc/bcf_segmented.cuh computes for
every work item -- the segment classes, the T-aligned tiles clipped to a
segment, the merge pieces of every pass (pair index, A/B windows, output range,
diagonals), the splits the publishing CTA finds for every piece of a pass and
the buffer each pass reads and writes -- and executes the schedule on numpy
data, each piece merging only the windows its published splits give.  Checks that every read
and write stays inside its segment, that each pass's pieces tile the segment
exactly once, that the simulated result is the sorted segment, and that the
work count the plan publishes equals the items executed.
"""
from __future__ import annotations

import numpy as np
import pytest

TINY_MAX = 512


def ceil_log2(x):
    p = 0
    while (1 << p) < x:
        p += 1
    return p


def seg_geo(lo, hi, T):
    size = hi - lo
    tiny = 0 < size <= TINY_MAX
    tiles = 0 if (size == 0 or tiny) else (hi - 1) // T - lo // T + 1
    passes = ceil_log2(tiles) if tiles > 1 else 0
    return tiny, tiles, passes, tiles


def tile_item(lo, hi, T, q):
    base = (lo // T + q) * T
    s0, s1 = max(lo, base), min(hi, base + T)
    assert lo <= s0 < s1 <= hi
    return base, s0, s1


def piece_item(lo, hi, T, p, rel):
    G0 = lo // T
    gt = G0 + rel
    q = rel >> p
    half = 1 << (p - 1)
    A0 = max((G0 + (q << p)) * T, lo)
    A1 = min((G0 + (q << p) + half) * T, hi)
    B1 = min((G0 + ((q + 1) << p)) * T, hi)
    na, nb = A1 - A0, max(B1 - A1, 0)
    ps = max(gt * T, A0)
    pe = min((gt + 1) * T, A0 + na + nb)
    assert lo <= A0 < A1 <= hi and A1 <= max(B1, A1) <= hi
    assert A0 <= ps < pe <= A0 + na + nb
    return A0, A1, na, nb, ps, pe, ps - A0, pe - A0, gt


def merge_path(src, A0, A1, na, nb, d):
    """Smallest i with A[i] > B[d-1-i] (the number of A-keys among the first d
    outputs of the stable merge, A first on ties), or min(d, na)."""
    A, B = src[A0:A1], src[A1:A1 + nb]
    lo, hi = max(0, d - nb), min(d, na)
    while lo < hi:
        mid = (lo + hi) // 2
        if A[mid] > B[d - 1 - mid]:
            hi = mid
        else:
            lo = mid + 1
    return lo


def simulate(offs, keys, T, per_group=8):
    out = keys.copy()
    buf = np.zeros_like(keys)
    total_items = 0
    ntiny = 0
    executed = 0
    for s in range(len(offs) - 1):
        lo, hi = int(offs[s]), int(offs[s + 1])
        tiny, tiles, passes, pieces = seg_geo(lo, hi, T)
        if tiny:
            ntiny += 1
            out[lo:hi] = np.sort(keys[lo:hi], kind="stable")
            continue
        total_items += tiles + passes * pieces
        dst = out if passes % 2 == 0 else buf
        covered = np.zeros(hi - lo, np.int32)
        for q in range(tiles):
            base, s0, s1 = tile_item(lo, hi, T, q)
            assert base <= s0 and s1 <= base + T
            dst[s0:s1] = np.sort(keys[s0:s1], kind="stable")
            covered[s0 - lo:s1 - lo] += 1
            executed += 1
        assert np.all(covered == 1)
        for p in range(1, passes + 1):
            src = out if (passes - (p - 1)) % 2 == 0 else buf
            dst = out if (passes - p) % 2 == 0 else buf
            assert src is not dst
            # publication: the CTA that completed pass p-1 finds every piece's
            # start split (A-keys before the piece's first output)
            split = []
            for rel in range(pieces):
                A0, A1, na, nb, _ps, _pe, d0, _d1, _gt = piece_item(lo, hi, T, p, rel)
                split.append(merge_path(src, A0, A1, na, nb, d0))
            covered = np.zeros(hi - lo, np.int32)
            for rel in range(pieces):
                A0, A1, na, nb, ps, pe, d0, d1, gt = piece_item(lo, hi, T, p, rel)
                A, B = src[A0:A1], src[A1:A1 + nb]
                assert np.all(np.diff(A) >= 0) and np.all(np.diff(B) >= 0), "runs not sorted"
                # the piece's windows from the published splits: its own start
                # split and the next piece's, or |A| at the end of its pair
                i0 = split[rel]
                i1 = na if d1 == na + nb else split[rel + 1]
                if d1 < na + nb:
                    assert (rel + 1) >> p == rel >> p, "next piece is in another pair"
                wa, wb = A[i0:i1], B[d0 - i0:d1 - i1]
                assert wa.size + wb.size == pe - ps
                window = np.sort(np.concatenate([wa, wb]), kind="stable")
                merged = np.sort(np.concatenate([A, B]), kind="stable")
                assert np.array_equal(window, merged[d0:d1])
                dst[ps:pe] = window
                assert gt * T <= ps and pe <= (gt + 1) * T
                covered[ps - lo:pe - lo] += 1
                executed += 1
            assert np.all(covered == 1), "pieces do not tile the segment exactly once"
        assert np.array_equal(out[lo:hi], np.sort(keys[lo:hi]))
    groups = -(-ntiny // per_group)  # one tiny segment per warp of the worker CTA
    return out, total_items + groups, executed + groups


@pytest.mark.parametrize("T,per_group", [(2048, 4), (4096, 8), (4096, 4)])
def test_schedule_sorts_every_segment(T, per_group):
    r = np.random.default_rng(T)
    for trial in range(4):
        sizes = np.concatenate([np.zeros(5, np.int64), np.ones(5, np.int64),
                                r.integers(2, 513, size=20), r.integers(513, 2 * T, size=20),
                                r.integers(2 * T, 40 * T, size=6)])
        sizes = sizes[r.permutation(sizes.size)]
        offs = np.concatenate([[0], np.cumsum(sizes)])
        keys = r.integers(0, 1000, size=int(offs[-1]))
        out, planned, executed = simulate(offs, keys, T, per_group)
        assert planned == executed


def test_queue_capacity_bound_holds():
    """The host's queue bound (tiles <= n/2048 + 2*nseg + 2, times 1 + passes,
    plus tiny groups of at least 4) covers the plan's item count, including a
    batch of nothing but tiny segments."""
    r = np.random.default_rng(5)
    for T in (2048, 4096):
        for _ in range(20):
            nseg = int(r.integers(1, 300))
            hi = 600 if _ % 4 == 0 else 200000  # every fourth mix: (almost) all tiny
            sizes = r.integers(0, hi, size=nseg)
            offs = np.concatenate([[0], np.cumsum(sizes)])
            n = int(offs[-1])
            items = 0
            ntiny = 0
            for s in range(nseg):
                tiny, tiles, passes, pieces = seg_geo(int(offs[s]), int(offs[s + 1]), T)
                ntiny += tiny
                items += tiles + passes * pieces
            items += -(-ntiny // 4)
            tiles_bound = n // 2048 + 2 * nseg + 2
            passes_bound = max(1, ceil_log2(tiles_bound))
            capacity = tiles_bound * (1 + passes_bound) + nseg // 4 + 2
            assert items <= capacity
