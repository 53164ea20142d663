"""Parity of bcf_segmented_sort (persistent launch, through the C ABI) with the
oracle -- bit-exact.

Segment sizes cover every class of the plan: empty, 1, tiny (<= 512 keys, one
warp), one tile, a few tiles (one or two merge passes) and many tiles (several
passes), at arbitrary (unaligned) offsets; keys and stable pairs, every key
type, both directions, in place, repeated, and replayed from a CUDA graph.

Every test runs with each of the two ways the merge passes can run (chosen by
the tuning table's merge_cfg for the segmented sort): in the persistent worker
("worker"), and as launches of the merge kernel over the list of multi-tile
segments with 2048-key merge tiles in 4096-key sort tiles ("passes") or with
merge tiles as large as the sort tiles ("passes_eq").
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import bits, from_dev, kt_of, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


# (seg_cfg, merge_cfg) of the segmented rows: 16 x 256 sort tiles (4096 keys);
# merge_cfg -1: the worker merges; 3: 16 x 128 merge tiles (2048 keys); 0:
# 16 x 256 (4096 keys)
MODES = {"worker": (0, -1), "passes": (0, 3), "passes_eq": (0, 0)}


@pytest.fixture(scope="module", params=list(MODES))
def bcf(request):
    import paper_1306_5076_gb300 as m
    from paper_1306_5076_gb300 import build

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    m._native.load()
    seg_cfg, merge_cfg = MODES[request.param]
    m.bcf_tuning_set([dict(op=m.BCF_OP_SEGMENTED, key_bytes=kb, has_vals=hv, n_min=0,
                           n_max=1 << 48, block_cfg=0, merge_cfg=merge_cfg, seg_cfg=seg_cfg)
                      for kb in (4, 8) for hv in (0, 1)])
    yield m
    m.bcf_tuning_set(None)


def mixed_sizes(r, count):
    """A mix of every size class, shuffled."""
    parts = [np.zeros(count // 10, np.int64), np.ones(count // 10, np.int64),
             r.integers(2, 513, size=count // 4), r.integers(513, 4097, size=count // 6),
             r.integers(4097, 40000, size=count // 8), r.integers(40000, 140000, size=3)]
    sizes = np.concatenate(parts)
    return sizes[r.permutation(sizes.size)]


def run(bcf, keys, offs, vals=None, descending=False, inplace=False):
    kd = to_dev(keys)
    vd = None if vals is None else to_dev(vals)
    ko = kd if inplace else torch.empty_like(kd)
    vo = None if vals is None else (vd if inplace else torch.empty_like(vd))
    od = torch.from_numpy(offs.astype(np.int64)).to("cuda")
    bcf.bcf_segmented_sort(ko, vo, kd, vd, od, descending=descending, kt=kt_of(keys))
    torch.cuda.synchronize()
    assert bcf.bcf_last_device_error() == 0
    return from_dev(ko, keys.dtype), (None if vals is None else from_dev(vo, np.uint32))


def check(bcf, keys, offs, vals, descending=False, inplace=False):
    ek, ev = oracle.segmented_sort(keys, vals, offs, descending=descending)
    gk, gv = run(bcf, keys, offs, vals, descending, inplace)
    bad = np.flatnonzero(bits(gk) != bits(ek))
    assert bad.size == 0, f"keys differ at {bad.size} positions, first {bad[:6]}"
    if vals is not None:
        assert np.array_equal(gv, ev)


@pytest.mark.parametrize("dtype", list(workloads.DTYPES))
@pytest.mark.parametrize("descending", [False, True])
def test_mixed_size_classes(bcf, dtype, descending):
    r = workloads.rng(31)
    sizes = mixed_sizes(r, 400)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    keys = workloads.keys("uniform" if dtype != "u32" else "gaussian", dtype, int(offs[-1]),
                          seed=7)
    vals = workloads.row_index(keys.size)
    check(bcf, keys, offs, None, descending)
    check(bcf, keys, offs, vals, descending)


def test_ties_and_extreme_keys(bcf):
    r = workloads.rng(32)
    sizes = mixed_sizes(r, 300)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    n = int(offs[-1])
    keys = np.where(r.random(n) < 0.5, np.uint32(0), np.uint32(0xFFFFFFFF)).astype(np.uint32)
    vals = workloads.row_index(n)
    for desc in (False, True):
        check(bcf, keys, offs, vals, desc)


@pytest.mark.parametrize("dtype", ["u32", "f32", "u64", "f64"])
def test_presorted_and_reversed_segments(bcf, dtype):
    """Keys already in order, in reverse order, and in few values: most merge
    tiles then draw every output from one of their two runs (the tiles that
    copy one window instead of merging), in both directions and with the key
    maps of the float types."""
    r = workloads.rng(34)
    sizes = mixed_sizes(r, 120)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    n = int(offs[-1])
    vals = workloads.row_index(n)
    for dist in ("sorted", "reverse", "distinct16"):
        keys = workloads.keys(dist, dtype, n, seed=10)
        for desc in (False, True):
            check(bcf, keys, offs, vals, desc)
        check(bcf, keys, offs, None, False)


def test_one_big_segment_and_empty_edges(bcf):
    n = (1 << 20) + 333
    keys = workloads.keys("uniform", "u32", n, seed=8)
    vals = workloads.row_index(n)
    for offs in ([0, n], [0, 0, n, n], [0, 1, n - 1, n]):
        check(bcf, keys, np.array(offs, np.uint64), vals)


def test_log_uniform_family_scaled(bcf):
    """The batched workload's size law (log-uniform in [1, 2^18]) on fewer segments."""
    keys, offs = workloads.segments(1500, 1 << 18, "u32", seed=4000)
    vals = workloads.row_index(keys.size)
    check(bcf, keys, offs, vals)
    check(bcf, keys, offs, None)


def test_in_place_and_repeat(bcf):
    r = workloads.rng(33)
    sizes = mixed_sizes(r, 200)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    keys = workloads.keys("distinct16", "u32", int(offs[-1]), seed=9)
    vals = workloads.row_index(keys.size)
    check(bcf, keys, offs, vals, inplace=True)
    first = run(bcf, keys, offs, vals)
    for _ in range(3):
        again = run(bcf, keys, offs, vals)
        assert np.array_equal(first[0], again[0]) and np.array_equal(first[1], again[1])


def test_cuda_graph_replay(bcf):
    """Captured once (after a warm-up call), replayed; every replay is exact."""
    keys, offs = workloads.segments(800, 1 << 16, "u32", seed=4001)
    vals = workloads.row_index(keys.size)
    ek, ev = oracle.segmented_sort(keys, vals, offs)
    kd, vd = to_dev(keys), to_dev(vals)
    ko, vo = torch.empty_like(kd), torch.empty_like(vd)
    od = torch.from_numpy(offs.astype(np.int64)).to("cuda")
    ws = torch.empty(bcf.bcf_workspace_bytes(bcf.BCF_OP_SEGMENTED, keys.size, offs.size - 1,
                                             bcf.BCF_U32, True), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        bcf.bcf_segmented_sort(ko, vo, kd, vd, od, kt=0, ws=ws, stream=s)  # warm-up
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        bcf.bcf_segmented_sort(ko, vo, kd, vd, od, kt=0, ws=ws, stream=s)
    for _ in range(3):
        ko.zero_()
        vo.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(from_dev(ko, np.uint32), ek)
        assert np.array_equal(from_dev(vo, np.uint32), ev)
    assert bcf.bcf_last_device_error() == 0


@pytest.mark.parametrize("pairs", [False, True])
def test_segments_past_2p32_keys(bcf, pairs):
    """Maximum sizes: 2^32 + 2^20 + 37 keys in segments of every class, one of
    them 2^31 keys long and one crossing position 2^32, so tile indices,
    merge-piece offsets and the queue go past 32 bits.  Key i is
    (i * C) mod 2^32 (odd C) and payload i mod 2^32, so every output element
    must satisfy key == payload * C mod 2^32; each segment must come out
    sorted with the multiset of its input (sum and sum of squares mod a prime,
    per segment)."""
    need = (100 if pairs else 60) << 30
    if torch.cuda.get_device_properties(0).total_memory < need + (8 << 30):
        pytest.skip("needs a large device memory")
    C = 0x9E3779B1
    n = (1 << 32) + (1 << 20) + 37
    offs = np.array([0, 0, 1, 300, 5000, 70000, (1 << 31) + 70000, (1 << 32) - 999,
                     (1 << 32) + 4096 + 17, n], dtype=np.int64)
    chunk = 1 << 27

    def u32_as_i32(x):
        return torch.where(x >= (1 << 31), x - (1 << 32), x).to(torch.int32)

    kd = torch.empty(n, dtype=torch.int32, device="cuda")
    vd = torch.empty(n, dtype=torch.int32, device="cuda") if pairs else None
    for c0 in range(0, n, chunk):
        i = torch.arange(c0, min(n, c0 + chunk), dtype=torch.int64, device="cuda")
        kd[c0:c0 + i.numel()] = u32_as_i32((i * C) & 0xFFFFFFFF)
        if pairs:
            vd[c0:c0 + i.numel()] = u32_as_i32(i & 0xFFFFFFFF)
    P = 1000000007

    def fingerprint(x):
        s1 = s2 = 0
        for c0 in range(0, x.numel(), chunk):
            v = x[c0:c0 + chunk].to(torch.int64) & 0xFFFFFFFF
            s1 += int(v.sum())
            s2 += int(((v * v) % P).sum())
        return s1, s2 % P

    before = [fingerprint(kd[a:b]) for a, b in zip(offs[:-1], offs[1:])]
    ko = torch.empty_like(kd)
    vo = torch.empty_like(vd) if pairs else None
    od = torch.from_numpy(offs).to("cuda")
    bcf.bcf_segmented_sort(ko, vo, kd, vd, od, kt=0)
    torch.cuda.synchronize()
    assert bcf.bcf_last_device_error() == 0
    del kd, vd
    for s, (a, b) in enumerate(zip(offs[:-1], offs[1:])):
        a, b = int(a), int(b)
        for c0 in range(a, b, chunk):
            c1 = min(b, c0 + chunk + 1)  # one element of overlap joins the chunks
            v = ko[c0:c1].to(torch.int64) & 0xFFFFFFFF
            assert bool((v[1:] >= v[:-1]).all()), (s, c0)
            if pairs:
                p = vo[c0:c1].to(torch.int64) & 0xFFFFFFFF
                assert torch.equal(v, (p * C) & 0xFFFFFFFF), (s, c0)
        assert fingerprint(ko[a:b]) == before[s], s
