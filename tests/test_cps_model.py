"""Host model of the colored prefix sums kernel (csrc/bcf_cps.cu), CPU only.

Restates the kernel's decomposition in numpy -- tiles of 16384 elements, 64
consecutive elements per thread, a d x 256 counter matrix, row scans over the
threads, a sequential look-back across tiles, and the final running sums --
and checks that it reproduces the oracle, that every counter index stays
inside the matrix, and that the conflict-free layout gives the 32 lanes of a
warp 32 different banks whatever colors they hold, while the row-per-thread
layout collides as the paper describes (Appendix A).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads

NT, E = 256, 64  # threads, consecutive elements per thread (4 steps of 16)
T = NT * E


def word(c, t, d, banked):
    return c * NT + t if banked else t * d + c


def model(values, colors, d, exclusive, banked):
    n = values.size
    out = np.zeros(n, np.uint64)
    ntiles = -(-n // T)
    inclusive_prefix = np.zeros((ntiles, d), np.uint64)  # published status words
    for tile in range(ntiles):
        base = tile * T
        cnt = min(T, n - base)
        mat = np.zeros(d * NT, np.uint64)
        for t in range(NT):  # phase 1
            for e in range(E):
                p = t * E + e
                if p < cnt:
                    w = word(int(colors[base + p]), t, d, banked)
                    assert 0 <= w < d * NT
                    mat[w] += values[base + p]
        agg = np.zeros(d, np.uint64)
        for c in range(d):  # phase 2: exclusive scan of row c over the threads
            carry = 0
            for t in range(NT):
                w = word(c, t, d, banked)
                x = mat[w]
                mat[w] = carry
                carry += x
            agg[c] = carry
        excl = inclusive_prefix[tile - 1] if tile > 0 else np.zeros(d, np.uint64)
        inclusive_prefix[tile] = excl + agg  # look-back result
        for t in range(NT):  # phase 3
            for e in range(E):
                p = t * E + e
                if p < cnt:
                    c = int(colors[base + p])
                    w = word(c, t, d, banked)
                    r = mat[w] + values[base + p]
                    mat[w] = r
                    out[base + p] = (r - values[base + p] if exclusive else r) + excl[c]
    return (out & 0xFFFFFFFF).astype(np.uint32)


@pytest.mark.parametrize("n,d", [(1, 1), (4097, 3), (2 * T + 100, 16), (T, 64)])
@pytest.mark.parametrize("banked", [True, False])
def test_model_matches_oracle(n, d, banked):
    values, colors = workloads.colored_elements(n, d, seed=n * 7 + d)
    for excl in (False, True):
        exp = oracle.colored_prefix_sums(values, colors, d, exclusive=excl)
        got = model(values.astype(np.uint64), colors, d, excl, banked)
        assert np.array_equal(got, exp)


def max_bank_load(d, banked, colors_of_lanes, warp=0):
    banks = [word(int(c), warp * 32 + lane, d, banked) % 32
             for lane, c in enumerate(colors_of_lanes)]
    return max(np.bincount(banks, minlength=32))


def test_banked_layout_is_conflict_free_for_any_colors():
    r = workloads.rng(5)
    for d in (1, 2, 3, 16, 32, 33, 64):
        for _ in range(200):
            cols = r.integers(0, d, size=32)
            for warp in range(NT // 32):
                assert max_bank_load(d, True, cols, warp) == 1
        # the row scan reads row c at threads j*32 + lane: 32 consecutive words
        for c in range(d):
            for j in range(NT // 32):
                banks = {word(c, j * 32 + lane, d, True) % 32 for lane in range(32)}
                assert len(banks) == 32


def test_row_layout_conflicts_grow_with_d():
    """The paper's baseline: with all lanes on one color, lanes t and t' share a
    bank when (t - t') * d is a multiple of 32, i.e. gcd(d, 32)-way."""
    for d in (1, 2, 4, 8, 16, 32):
        assert max_bank_load(d, False, [0] * 32) == np.gcd(d, 32)


def windowed_lookback(status, tile, d, warp, kwarps=8, loads=4, publish=None):
    """Lane-level restatement of the kernel's look-back for one warp: returns
    {color: exclusive prefix}.  `status[p][c]` = (flag, value) with flag 0
    (nothing published yet), 1 (tile total only) or 2 (inclusive prefix).
    `publish(round)` may update `status` between rounds (predecessors making
    progress while this tile waits)."""
    ncol = (d - warp + kwarps - 1) // kwarps if d > warp else 0
    if ncol == 0:
        return {}
    K = 1
    while K < ncol:
        K <<= 1
    J = 32 // K
    lanes = range(32)
    slot = [l & (K - 1) for l in lanes]
    jj = [l // K for l in lanes]
    color = [warp + kwarps * slot[l] for l in lanes]
    slot_lanes = [sum(1 << m for m in range(slot[l], 32, K)) for l in lanes]
    done = [slot[l] >= ncol or tile == 0 for l in lanes]
    excl = [0] * 32
    top = [tile - 1] * 32
    rounds = 0
    while not all(done):
        rounds += 1
        assert rounds < 10_000
        if publish is not None:
            publish(rounds)
        st = [[(0, 0)] * 32 for _ in range(loads)]
        for q in range(loads):
            for l in lanes:
                if not done[l]:
                    p = top[l] - (jj[l] + q * J)
                    st[q][l] = status[p][color[l]] if p >= 0 else (2, 0)
        found = [False] * 32
        wait = [False] * 32
        x = [0] * 32
        for q in range(loads):
            incl = sum(1 << l for l in lanes if not done[l] and st[q][l][0] == 2)
            none = sum(1 << l for l in lanes if not done[l] and st[q][l][0] == 0)
            y = [0] * 32
            mine = [0] * 32
            live = [False] * 32
            for l in lanes:
                mine[l] = incl & slot_lanes[l]
                last = (mine[l] & -mine[l]).bit_length() - 1 if mine[l] else 31
                upto = (1 << (last + 1)) - 1
                live[l] = not done[l] and not found[l] and not wait[l]
                if live[l] and (none & slot_lanes[l] & upto):
                    wait[l] = True
                if live[l] and not wait[l] and l <= last:
                    y[l] = st[q][l][1]
            o = K
            while o < 32:  # butterfly over the lanes of a slot
                y = [y[l] + y[l ^ o] for l in lanes]
                o <<= 1
            for l in lanes:
                if live[l] and not wait[l]:
                    x[l] += y[l]
                    if mine[l]:
                        found[l] = True
        for l in lanes:
            if done[l] or wait[l]:
                continue
            excl[l] += x[l]
            if found[l]:
                done[l] = True
            else:
                top[l] -= J * loads
    return {color[l]: excl[l] for l in lanes if jj[l] == 0 and slot[l] < ncol}


@pytest.mark.parametrize("d", [1, 2, 3, 8, 16, 33, 64])
@pytest.mark.parametrize("loads", [1, 4])
def test_windowed_lookback_matches_prefix(d, loads):
    r = workloads.rng(d + 100 * loads)
    ntiles = 600
    agg = r.integers(0, 1000, size=(ntiles, d))
    prefix = np.cumsum(agg, axis=0) - agg  # exclusive prefix per tile and color
    for trial in range(12):
        # a random mix of predecessors that have published nothing yet (0),
        # only their total (1), or also their inclusive prefix (2); the
        # unpublished ones publish their total after a few rounds
        incl_p = [0.0, 0.05, 0.5, 1.0][trial % 4]
        none_p = [0.0, 0.2][trial % 2]
        status = []
        pending = []
        for p in range(ntiles):
            row = []
            for c in range(d):
                u = r.random()
                if u < none_p:
                    row.append((0, 0))
                    pending.append((p, c, int(r.integers(1, 4))))
                elif r.random() < incl_p:
                    row.append((2, int(prefix[p, c] + agg[p, c])))
                else:
                    row.append((1, int(agg[p, c])))
            status.append(row)

        def publish(rnd):
            for p, c, when in pending:
                if rnd >= when and status[p][c][0] == 0:
                    status[p][c] = (1, int(agg[p, c]))

        tile = int(r.integers(0, ntiles))
        got = {}
        for warp in range(8):
            got.update(windowed_lookback(status, tile, d, warp, loads=loads, publish=publish))
        assert sorted(got) == list(range(d))
        for c in range(d):
            assert got[c] == prefix[tile, c], (d, tile, c)
