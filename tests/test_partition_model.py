"""Host model of the sampled merge-path searches of the partition kernel
(csrc/bcf_merge.cu, partition_kernel), CPU only.

The splitter of diagonal d of the stable merge of sorted runs A and B (A first
on equal keys) is the number of A-keys among the first d outputs.  The kernel
keeps a sample of every array position that is a multiple of S and first runs
merge path on the runs' samples, then searches exactly only in a window
around the result.  Two cases:
  - the sort's passes: runs start at multiples of S and d is one, the samples
    are A[kS] and B[kS]; merge path at D = d / S gives sa and the split lies
    in [sa*S - S, sa*S + S];
  - merges of given runs at any offsets: the samples are A[cA + kS] and
    B[cB + kS] (cA, cB < S, where the array's multiples of S fall); merge path
    at D = floor((d - cA - cB) / S) + 1 gives sa and the split lies in
    [cA + sa*S - S, cA + sa*S + S].
A split outside its window would fail the kernel's check and fall back to a
full search; this model shows the windows always hold it, for every diagonal
of small runs with many ties, empty runs and every pair of offsets.
"""
from __future__ import annotations

import numpy as np
import pytest


def merge_path(A, B, d):
    lo, hi = max(0, d - len(B)), min(d, len(A))
    while lo < hi:
        mid = (lo + hi) // 2
        if A[mid] > B[d - 1 - mid]:
            hi = mid
        else:
            lo = mid + 1
    return lo


def splitter_by_definition(A, B, d):
    tagged = sorted([(int(k), 0, i) for i, k in enumerate(A)] + [(int(k), 1, i) for i, k in enumerate(B)])
    return sum(1 for t in tagged[:d] if t[1] == 0)


def runs(r, S, trial):
    na, nb = int(r.integers(0, 10 * S)), int(r.integers(0, 10 * S))
    if trial % 10 == 0:
        na = 0
    if trial % 10 == 1:
        nb = 0
    hi_key = int(r.choice([1, 2, 5, 40, 1 << 30]))
    return np.sort(r.integers(0, hi_key, size=na)), np.sort(r.integers(0, hi_key, size=nb))


@pytest.mark.parametrize("S", [4, 8, 16])
def test_aligned_runs_window(S):
    r = np.random.default_rng(S)
    for trial in range(200):
        A, B = runs(r, S, trial)
        for d in range(0, len(A) + len(B) + 1, S):
            i = merge_path(A, B, d)
            sa = merge_path(A[::S], B[::S], d // S)
            assert sa * S - S <= i <= sa * S + S, (trial, d)


@pytest.mark.parametrize("S", [4, 8, 16, 32])
def test_runs_at_any_offsets_window(S):
    r = np.random.default_rng(100 + S)
    for trial in range(400):
        A, B = runs(r, S, trial)
        cA = S - 1 if trial % 7 == 0 else int(r.integers(0, S))
        cB = S - 1 if trial % 5 == 0 else int(r.integers(0, S))
        As, Bs = A[cA::S], B[cB::S]
        for d in range(len(A) + len(B) + 1):
            i = merge_path(A, B, d)
            if d < 24 and trial % 20 == 0:
                assert i == splitter_by_definition(A, B, d)
            D = max(0, (d - cA - cB) // S + 1) if d >= cA + cB else 0
            sa = merge_path(As, Bs, min(D, len(As) + len(Bs)))
            c = cA + sa * S
            assert c - S <= i <= c + S, (trial, d, i, c)


def test_irregular_merge_writes_every_sample_once():
    """The merge kernel's sample writes for a pass of given runs
    (csrc/bcf_merge.cu, merge_kernel with IRREG): pieces are the Tm-aligned
    output tiles clipped to each pair's range; thread tid of a piece writes the
    sample of array position out0 + tid*E when that position is a multiple of
    S and lies in the piece's slots [front, front + count).  Every multiple
    of S in the merged span must be written exactly once."""
    S, E, NT = 256, 16, 128
    Tm = E * NT
    r = np.random.default_rng(3)
    for trial in range(60):
        k = int(r.integers(1, 9))
        lens = r.integers(0, 3 * Tm, size=k)
        lo = int(r.integers(0, 5000))
        offs = np.concatenate([[lo], lo + np.cumsum(lens)])
        runs = [(int(offs[i]), int(lens[i])) for i in range(k)]
        # one pass: pair adjacent runs (an odd last run pairs with an empty one)
        written = []
        for q in range(0, len(runs), 2):
            off = runs[q][0]
            length = runs[q][1] + (runs[q + 1][1] if q + 1 < len(runs) else 0)
            if length == 0:
                continue
            end = off + length
            for g in range(off // Tm, (end - 1) // Tm + 1):
                out0 = g * Tm
                start, stop = max(off, out0), min(end, out0 + Tm)
                front, count = start - out0, stop - start
                for tid in range(NT):
                    s0 = tid * E
                    if (out0 + s0) % S == 0 and front <= s0 < front + count:
                        written.append(out0 + s0)
        hi = int(offs[-1])
        expect = list(range((lo + S - 1) // S * S, hi, S))
        assert sorted(written) == expect, trial

