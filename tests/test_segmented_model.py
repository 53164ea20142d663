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

The second model covers the other way the merge passes can run: segments of
two or more tiles are only block-sorted by the worker and listed by the plan
(most passes first, with prefix sums of their Tm-aligned merge tiles); the
host then launches one partition and one merge per number q of passes to go,
from the pass count of a segment of all n keys down to 1, and each launch
merges, for every listed segment with q or more passes left, the runs of its
pass P_s - q + 1.  The model restates the plan's list, the work-item
geometry of csrc/bcf_seg_merge.cu (seg_pass_geo, seg_item_at, piece_of_item) and the buffer
parity of each launch, checks every item's pair against run boundaries
derived independently from the segment and the pass, and executes the
launches on numpy data.
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


# ---------------------------------------------------------------- merge passes as launches


def plan_list(offs, T, Tm):
    """The plan's list: multi-tile segments, most passes first (ties in index
    order here; the device's order within a pass count is arbitrary), with the
    inclusive prefix sums of their Tm-tiles, and count_ge[q]."""
    listed = []
    for s in range(len(offs) - 1):
        lo, hi = int(offs[s]), int(offs[s + 1])
        _tiny, _tiles, passes, _ = seg_geo(lo, hi, T)
        if passes > 0:
            listed.append((passes, s, (hi - 1) // Tm - lo // Tm + 1))
    listed.sort(key=lambda t: -t[0])
    order = [s for _p, s, _m in listed]
    piece_end = np.cumsum([m for _p, _s, m in listed]).tolist()
    count_ge = [sum(1 for p, _s, _m in listed if p >= q) for q in range(64)]
    return order, piece_end, count_ge


def seg_pass_geo(offs, order, piece_end, idx, T, q):
    """Restates seg_pass_geo in csrc/bcf_seg_merge.cu: the listed segment at list
    position idx, this launch's pass j of it, its first item and item count.
    (seg_partition_kernel finds idx for an item from the chunk table that
    seg_chunk_kernel writes: the list position of every 32nd item.)"""
    s = order[idx]
    lo, hi = int(offs[s]), int(offs[s + 1])
    first = piece_end[idx - 1] if idx else 0
    G0 = lo // T
    tiles = (hi - 1) // T - G0 + 1
    j = ceil_log2(tiles) - q + 1
    return s, lo, hi, G0, j, first, piece_end[idx] - first


def seg_item_at(lo, hi, G0, j, t, T, Tm):
    """Restates seg_item_at: (src, na, nb, out0) of the segment's merge tile t."""
    out0 = (lo // Tm + t) * Tm
    pos = max(out0, lo)
    r = pos // T - G0
    t0 = G0 + ((r >> j) << j)
    a0, a1, b1 = t0 * T, (t0 + (1 << (j - 1))) * T, (t0 + (1 << j)) * T
    src = max(a0, lo)
    A1, B1 = min(a1, hi), min(b1, hi)
    return src, A1 - src, max(B1 - A1, 0), out0


def piece_of_item(src, na, nb, out0, Tm):
    end = src + na + nb
    start, stop = max(src, out0), min(end, out0 + Tm)
    return start - out0, start - src, stop - src, stop == end


def runs_of(lo, hi, T, j):
    """Independent definition: the sorted runs a segment holds before its pass
    j are its T-aligned tiles joined 2^(j-1) at a time (clipped to the
    segment); pass j merges runs 2k and 2k+1."""
    G0 = lo // T
    cuts = sorted({lo, hi} | {(G0 + k) * T for k in range(1, (hi - 1) // T - G0 + 1)
                              if k % (1 << (j - 1)) == 0 and lo < (G0 + k) * T < hi})
    runs = list(zip(cuts[:-1], cuts[1:]))
    return [(runs[i], runs[i + 1] if i + 1 < len(runs) else (runs[i][1], runs[i][1]))
            for i in range(0, len(runs), 2)]


def simulate_listed(offs, keys, T, Tm):
    n = int(offs[-1])
    out = np.zeros_like(keys)
    buf = np.zeros_like(keys)
    # the worker: tiny segments and one-tile segments to the output, the
    # tiles of listed segments to the buffer their first pass reads
    for s in range(len(offs) - 1):
        lo, hi = int(offs[s]), int(offs[s + 1])
        tiny, tiles, passes, _ = seg_geo(lo, hi, T)
        if tiny:
            out[lo:hi] = np.sort(keys[lo:hi], kind="stable")
            continue
        dst = out if passes % 2 == 0 else buf
        for qq in range(tiles):
            _base, s0, s1 = tile_item(lo, hi, T, qq)
            dst[s0:s1] = np.sort(keys[s0:s1], kind="stable")
    order, piece_end, count_ge = plan_list(offs, T, Tm)
    total = piece_end[-1] if piece_end else 0
    chunk_seg = [int(np.searchsorted(piece_end, 32 * c, side="right"))
                 for c in range(-(-total // 32))]
    qmax = ceil_log2((n - 1) // T + 2)
    launches = 0
    for q in range(qmax, 0, -1):
        to_out = q & 1
        src_buf, dst_buf = (buf, out) if to_out else (out, buf)
        count = count_ge[q]
        nitems = piece_end[count - 1] if count else 0
        if nitems:
            launches += 1
        covered = np.zeros(n, np.int32)
        # one thread per item: its list position from the chunk table (the
        # position of every 32nd item) and a search among the next 32
        recs = []
        for it in range(nitems):
            lo_i = chunk_seg[it // 32]
            hi_i = min(lo_i + 31, count - 1)
            while lo_i < hi_i:
                mid = (lo_i + hi_i) // 2
                if piece_end[mid] > it:
                    hi_i = mid
                else:
                    lo_i = mid + 1
            assert piece_end[lo_i] > it and (lo_i == 0 or piece_end[lo_i - 1] <= it)
            s, lo, hi, G0, j, first, _items = seg_pass_geo(offs, order, piece_end, lo_i, T, q)
            recs.append((s,) + seg_item_at(lo, hi, G0, j, it - first, T, Tm) + (j,))
        splits = []
        for s, src, na, nb, out0, _j in recs:
            _front, d0, _d1, _last = piece_of_item(src, na, nb, out0, Tm)
            splits.append(merge_path(src_buf, src, src + na, na, nb, d0))
        for it, (s, src, na, nb, out0, j) in enumerate(recs):
            lo, hi = int(offs[s]), int(offs[s + 1])
            assert seg_geo(lo, hi, T)[2] >= q
            front, d0, d1, last = piece_of_item(src, na, nb, out0, Tm)
            # the item's pair is the pair of runs that holds its first output
            ((a0, a1), (b0, b1)), = [pr for pr in runs_of(lo, hi, T, j)
                                     if pr[0][0] <= out0 + front < max(pr[0][1], pr[1][1])]
            assert (src, na, nb) == (a0, a1 - a0, b1 - b0)
            assert lo <= src and src + na + nb <= hi and out0 % Tm == 0
            A, B = src_buf[src:src + na], src_buf[src + na:src + na + nb]
            assert np.all(np.diff(A) >= 0) and np.all(np.diff(B) >= 0), "runs not sorted"
            i0 = splits[it]
            i1 = na if last else splits[it + 1]
            if not last:
                assert recs[it + 1][1] == src, "next item is in another pair"
            window = np.sort(np.concatenate([A[i0:i1], B[d0 - i0:d1 - i1]]), kind="stable")
            merged = np.sort(np.concatenate([A, B]), kind="stable")
            assert np.array_equal(window, merged[d0:d1])
            p0, p1 = out0 + front, out0 + front + (d1 - d0)
            assert out0 <= p0 < p1 <= out0 + Tm
            dst_buf[p0:p1] = window
            covered[p0:p1] += 1
        # every listed segment with q or more passes left is written once
        for s in range(len(offs) - 1):
            lo, hi = int(offs[s]), int(offs[s + 1])
            want = 1 if seg_geo(lo, hi, T)[2] >= q else 0
            assert np.all(covered[lo:hi] == want), (q, s)
    return out, launches, max(count_ge[1:2] + [0]), qmax


@pytest.mark.parametrize("T,Tm", [(4096, 2048), (4096, 4096), (2048, 2048), (8192, 2048)])
def test_listed_merge_passes_sort_every_segment(T, Tm):
    r = np.random.default_rng(T + Tm)
    for trial in range(3):
        sizes = np.concatenate([np.zeros(4, np.int64), np.ones(4, np.int64),
                                r.integers(2, 513, size=12), r.integers(513, 2 * T, size=12),
                                r.integers(2 * T, 40 * T, size=5), [T, T + 1, 2 * T - 1]])
        sizes = sizes[r.permutation(sizes.size)]
        offs = np.concatenate([[0], np.cumsum(sizes)])
        keys = r.integers(0, 1000, size=int(offs[-1]))
        out, launches, _listed, qmax = simulate_listed(offs, keys, T, Tm)
        for s in range(len(offs) - 1):
            lo, hi = int(offs[s]), int(offs[s + 1])
            assert np.array_equal(out[lo:hi], np.sort(keys[lo:hi])), s
        longest = max(seg_geo(int(a), int(b), T)[2] for a, b in zip(offs[:-1], offs[1:]))
        assert launches == longest <= qmax


def test_listed_one_segment_of_everything():
    """One segment of all n keys: the host's first q is its pass count."""
    T, Tm = 2048, 2048
    for n in (2 * T, 2 * T + 1, 5 * T + 7, 16 * T):
        keys = np.random.default_rng(n).integers(0, 50, size=n)
        offs = np.array([0, n])
        out, launches, _l, qmax = simulate_listed(offs, keys, T, Tm)
        assert np.array_equal(out, np.sort(keys))
        assert launches == seg_geo(0, n, T)[2]
        assert qmax in (launches, launches + 1)
