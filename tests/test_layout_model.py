"""Host model of the CTA layouts and sorting schedule of csrc/bcf_device.cuh.

The three register layouts (BLK / MID / STR), the padded shared-memory
addresses of every layout change, the bitonic "flip" folded into a layout
change, and the level schedule of the block sort and of the merge are restated
here as plain index arithmetic and checked on the CPU:

* every layout is a bijection (thread, register) <-> tile index k;
* every warp-wide shared access of every layout change touches 32 distinct
  banks (the paper's bank-conflict-free principle, Sec. 2.1) -- and the
  paper's Fig. 1 mapping (element A_k of a contiguous load in bank k mod w) is
  reproduced for w = 8;
* the simulated block sort sorts random inputs, and the simulated merge
  network sorts the 0-1 bitonic inputs (0-1 principle, Knuth vol. 3; the
  paper invokes it in Sec. 3.1 / 3.2) -- all of them for 1024-element tiles,
  an evenly spaced grid for larger ones -- and random merges.
"""
from __future__ import annotations

import numpy as np
import pytest

BLK, MID, STR = 0, 1, 2


class Geo:
    def __init__(self, E, NT):
        self.E, self.NT = E, NT
        self.r = E.bit_length() - 1
        self.t = (E * NT).bit_length() - 1
        assert self.r in (4, 5) and 10 <= self.t <= 3 * self.r

    def win(self, L):
        return 0 if L == BLK else (self.r if L == MID else self.t - self.r)

    def k(self, L, tid, e):
        E, NT = self.E, self.NT
        if L == BLK:
            return tid * E + e
        if L == STR:
            return e * NT + tid
        w, l = tid >> 5, tid & 31
        if self.r == 5:
            return (w << 10) | (e << 5) | l
        return (l & 15) | (e << 4) | ((w & 1) << 8) | ((l >> 4) << 9) | ((w >> 1) << 10)

    def base(self, L, tid, mirror=False):
        E, NT = self.E, self.NT
        if L == BLK:
            assert not mirror
            k0 = tid * E
            return k0 + (k0 >> 5)
        if L == STR:
            tt = tid ^ (NT - 1) if mirror else tid
            return tt + (tt >> 5)
        w, l = tid >> 5, tid & 31
        if self.r == 5:
            return w * 1056 + ((l ^ 31) if mirror else l)
        lo = ((l & 15) ^ 15) if mirror else (l & 15)
        return lo + 264 * (w & 1) + 528 * (l >> 4) + 1056 * (w >> 1)

    def off(self, L, e):
        NT = self.NT
        if L == BLK:
            return e
        if L == STR:
            return e * (NT + NT // 32)
        return 33 * e if self.r == 5 else 16 * e + (e >> 1)

    def addr(self, L, tid, e):
        return self.base(L, tid) + self.off(L, e)


def phys(k):
    return k + (k >> 5)


GEOS = [(16, 64), (16, 256), (16, 128), (32, 32), (32, 128), (32, 256), (32, 512), (32, 1024)]


@pytest.mark.parametrize("E,NT", GEOS)
def test_layouts_are_bijections_and_addresses_match_padding(E, NT):
    g = Geo(E, NT)
    for L in (BLK, MID, STR):
        ks = set()
        for tid in range(NT):
            for e in range(E):
                k = g.k(L, tid, e)
                ks.add(k)
                assert g.addr(L, tid, e) == phys(k)
        assert ks == set(range(E * NT))


@pytest.mark.parametrize("E,NT", GEOS)
def test_every_warp_access_is_bank_conflict_free(E, NT):
    g = Geo(E, NT)
    for L in (BLK, MID, STR):
        for w in range(NT // 32):
            for e in range(E):
                banks = {g.addr(L, 32 * w + l, e) % 32 for l in range(32)}
                assert len(banks) == 32, (L, w, e)
                if L != BLK:
                    # mirrored reads (the folded bitonic flip) as well
                    for q in range(g.r):
                        ee = e ^ ((1 << q) - 1)
                        mb = {(g.base(L, 32 * w + l, True) + g.off(L, ee)) % 32
                              for l in range(32)}
                        assert len(mb) == 32


@pytest.mark.parametrize("w", [8, 32])
def test_paper_fig1_mapping_and_padded_skew(w):
    """Fig. 1: a contiguous load puts element A_k in bank k mod w, so a thread
    per row (bank) is conflict-free but reading a column of the w x w matrix
    hits one bank w times.  One pad word per w words stores element k at
    k + k // w: column c then starts at bank c (the shifted diagonal of Sec.
    3.3), and both a row and a column read touch w distinct banks."""
    for c in range(w):
        col = [c * w + i for i in range(w)]  # k of column c, rows 0..w-1
        assert [k % w for k in col] == list(range(w))  # Fig. 1: A_k in bank k mod w
    row_unpadded = {(c * w + 0) % w for c in range(w)}
    assert len(row_unpadded) == 1  # same bank for every column: w-way conflict
    pad = lambda k: k + k // w  # noqa: E731
    for i in range(w):
        assert len({pad(c * w + i) % w for c in range(w)}) == w
    for c in range(w):
        assert len({pad(c * w + i) % w for i in range(w)}) == w
        assert pad(c * w) % w == c


def read_addrs(g, L, flipj=0):
    """[NT, E] shared-memory word each register of layout L is read from."""
    a = np.empty((g.NT, g.E), dtype=np.int64)
    q = flipj - 1 - g.win(L) if flipj else -1
    if flipj:
        assert 0 <= q < g.r
    for tid in range(g.NT):
        for e in range(g.E):
            if flipj and e & (1 << q):
                a[tid, e] = g.base(L, tid, True) + g.off(L, e ^ ((1 << q) - 1))
            else:
                a[tid, e] = g.addr(L, tid, e)
    return a


def simulate_relayout(g, X, FROM, TO, flipj=0, cache={}):
    """X: [B, NT, E] registers in layout FROM -> registers in layout TO."""
    key = (g.E, g.NT, FROM, TO, flipj)
    if key not in cache:
        cache[key] = (read_addrs(g, FROM).ravel(), read_addrs(g, TO, flipj).ravel())
    wa, ra = cache[key]
    sm = np.empty((X.shape[0], int(max(wa.max(), ra.max())) + 1), dtype=X.dtype)
    sm[:, wa] = X.reshape(X.shape[0], -1)
    return sm[:, ra].reshape(X.shape)


def simulate_stages(g, X, L, hi, lo):
    for b in range(hi, lo - 1, -1):
        q = b - g.win(L)
        assert 0 <= q < g.r
        for e in range(g.E):
            if not e & (1 << q):
                f = e | (1 << q)
                lo_, hi_ = np.minimum(X[..., e], X[..., f]), np.maximum(X[..., e], X[..., f])
                X[..., e], X[..., f] = lo_, hi_


def oem_pairs(n):
    out = []
    p = 1
    while p < n:
        kk = p
        while kk >= 1:
            j = kk % p
            while j + kk < n:
                for i in range(kk):
                    if i + j + kk < n and (i + j) // (2 * p) == (i + j + kk) // (2 * p):
                        out.append((i + j, i + j + kk))
                j += 2 * kk
            kk >>= 1
        p <<= 1
    return out


def layout_index(g, L):
    return np.array([[g.k(L, tid, e) for e in range(g.E)] for tid in range(g.NT)])


def simulate_block_sort(g, vals):
    """vals: [B, T] -> [B, T] after the simulated CTA sort."""
    B = vals.shape[0]
    X = vals.reshape(B, g.NT, g.E).copy()  # BLK: thread tid holds tid*E .. tid*E+E-1
    for a, b in oem_pairs(g.E):
        lo_, hi_ = np.minimum(X[..., a], X[..., b]), np.maximum(X[..., a], X[..., b])
        X[..., a], X[..., b] = lo_, hi_
    r, t = g.r, g.t
    for J in range(r + 1, t + 1):
        top = J - 1
        if top >= 2 * r:  # the level's top bit lies above the MID window
            X = simulate_relayout(g, X, BLK, STR, J)
            simulate_stages(g, X, STR, top, t - r)
            if t - r - 1 >= r:
                X = simulate_relayout(g, X, STR, MID)
                simulate_stages(g, X, MID, t - r - 1, r)
                X = simulate_relayout(g, X, MID, BLK)
            else:
                X = simulate_relayout(g, X, STR, BLK)
        else:
            X = simulate_relayout(g, X, BLK, MID, J)
            simulate_stages(g, X, MID, top, r)
            X = simulate_relayout(g, X, MID, BLK)
        simulate_stages(g, X, BLK, r - 1, 0)
    out = np.empty_like(vals)
    out[:, layout_index(g, BLK).ravel()] = X.reshape(B, -1)
    return out


def simulate_merge(g, seqs):
    """Bitonic merge of bitonic sequences [B, Tm] read into STR layout."""
    B = seqs.shape[0]
    X = seqs[:, layout_index(g, STR)].copy()
    r, t = g.r, g.t
    simulate_stages(g, X, STR, t - 1, t - r)
    if t - r - 1 >= r:
        X = simulate_relayout(g, X, STR, MID)
        simulate_stages(g, X, MID, t - r - 1, r)
        X = simulate_relayout(g, X, MID, BLK)
    else:
        X = simulate_relayout(g, X, STR, BLK)
    simulate_stages(g, X, BLK, r - 1, 0)
    out = np.empty_like(seqs)
    out[:, layout_index(g, BLK).ravel()] = X.reshape(B, -1)
    return out


@pytest.mark.parametrize("E,NT", [(16, 64), (16, 256), (32, 32), (32, 256)])
def test_simulated_block_sort_sorts(E, NT):
    g = Geo(E, NT)
    rng = np.random.default_rng(E * NT)
    n = E * NT
    vals = np.concatenate([rng.integers(0, 2**31, size=(6, n)), rng.integers(0, 3, size=(6, n)),
                           rng.integers(0, 2, size=(4, n))])
    got = simulate_block_sort(g, vals)
    assert np.array_equal(got, np.sort(vals, axis=1))


@pytest.mark.parametrize("E,NT", [(16, 64), (32, 32), (16, 256), (32, 128)])
def test_simulated_merge_on_01_bitonic_inputs(E, NT):
    """0-1 principle: a network sorts every bitonic sequence iff it sorts the
    0-1 bitonic ones, 0^a 1^b 0^c (ascending A, then reversed ascending B).
    All (a, b) for the 1024-element tiles, an evenly spaced grid otherwise."""
    g = Geo(E, NT)
    Tm = E * NT
    step = 1 if Tm <= 1024 else 37
    rows = []
    for a in range(0, Tm + 1, step):
        for b in range(0, Tm - a + 1, step):
            rows.append((a, b))
    rows = np.array(rows)
    idx = np.arange(Tm)
    for chunk in np.array_split(rows, max(1, len(rows) // 4096)):
        seqs = ((idx[None, :] >= chunk[:, :1]) & (idx[None, :] < chunk[:, :1] + chunk[:, 1:2]))
        seqs = seqs.astype(np.int8)
        got = simulate_merge(g, seqs)
        assert np.array_equal(got, np.sort(seqs, axis=1))


@pytest.mark.parametrize("E,NT", [(16, 256), (32, 128)])
def test_simulated_merge_of_random_runs(E, NT):
    g = Geo(E, NT)
    Tm = E * NT
    rng = np.random.default_rng(3)
    seqs = []
    for na in rng.integers(0, Tm + 1, size=64):
        A = np.sort(rng.integers(0, 50, size=na))
        B = np.sort(rng.integers(0, 50, size=Tm - na))
        seqs.append(np.concatenate([A, B[::-1]]))
    seqs = np.array(seqs)
    assert np.array_equal(simulate_merge(g, seqs), np.sort(seqs, axis=1))


@pytest.mark.parametrize("E", [16, 32])
def test_lane_shuffle_levels_pair_the_bitonic_partners(E):
    """The block sort's low levels exchange elements between lanes (BLK
    layout, k = tid*E + e): the flip stage of level J pairs register e of
    lane l with register E-1-e of lane l ^ (2^(J-r) - 1), a half-cleaner on
    lane bit b-r pairs lanes l and l ^ 2^(b-r) at the same register, and the
    lane with k bit J-1 (resp. b) set keeps the maximum.  These must be the
    bitonic network's partners k ^ (2^J - 1) and k ^ 2^b."""
    r = E.bit_length() - 1
    for J in range(r + 1, r + 6):
        m = (1 << (J - r)) - 1
        for tid in range(64):
            lane, warp = tid & 31, tid >> 5
            for e in range(E):
                k = tid * E + e
                pk = ((warp << 5) | (lane ^ m)) * E + (E - 1 - e)
                assert pk == k ^ ((1 << J) - 1)
                assert (((lane >> (J - 1 - r)) & 1) == 1) == bool(k >> (J - 1) & 1)
                for b in range(J - 2, r - 1, -1):
                    mb = 1 << (b - r)
                    pk = ((warp << 5) | (lane ^ mb)) * E + e
                    assert pk == k ^ (1 << b)
                    assert ((lane & mb) != 0) == bool(k >> b & 1)
