"""Parity of bcf_merge_runs (through the C ABI) with the oracle -- bit-exact.

Runs of uneven, unaligned lengths (zero-length runs included), k = 1 .. 300,
keys and stable pairs, every key type, both directions, aliasing, and the
benchmark family of k in {2, 16, 256} runs with log-uniform lengths.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import bits, from_dev, kt_of, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bcf():
    import paper_1306_5076_gb300 as m
    from paper_1306_5076_gb300 import build

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    m._native.load()
    return m


def make_runs(r, dtype, lens, descending=False, alphabet=None):
    """Runs sorted under the requested order: each run is put in order with
    numpy's stable argsort of its totalOrder rank (input construction only)."""
    from tests.pins import order_rank

    parts = []
    for m in lens:
        if alphabet:
            pool = workloads.keys("uniform", dtype, alphabet, seed=int(r.integers(1 << 30)))
            k = pool[r.integers(0, alphabet, size=int(m))]
        else:
            k = workloads.keys("uniform", dtype, int(m), seed=int(r.integers(1 << 30)))
        rank = order_rank(k)
        order = np.argsort(~rank if descending else rank, kind="stable")  # ~: no overflow
        parts.append(k[order])
    offs = np.zeros(len(lens) + 1, np.uint64)
    offs[1:] = np.cumsum(lens)
    keys = np.concatenate(parts) if parts else np.zeros(0, workloads.DTYPES[dtype])
    return keys, offs


def gpu_merge(bcf, keys, offs, vals=None, descending=False, inplace=False):
    kd = to_dev(keys)
    vd = None if vals is None else to_dev(vals)
    ko = kd if inplace else torch.empty_like(kd)
    vo = None if vals is None else (vd if inplace else torch.empty_like(vd))
    bcf.bcf_merge_runs(ko, vo, kd, vd, [int(x) for x in offs], descending=descending,
                       kt=kt_of(keys))
    torch.cuda.synchronize()
    return from_dev(ko, keys.dtype), (None if vals is None else from_dev(vo, np.uint32))


def check(bcf, keys, offs, vals, descending, inplace=False):
    ek, ev = oracle.merge_runs(keys, vals, offs, descending=descending)
    gk, gv = gpu_merge(bcf, keys, offs, vals, descending, inplace)
    assert np.array_equal(bits(gk), bits(ek))
    if vals is not None:
        assert np.array_equal(gv, ev)


@pytest.mark.parametrize("dtype", list(workloads.DTYPES))
@pytest.mark.parametrize("descending", [False, True])
def test_random_uneven_runs(bcf, dtype, descending):
    r = workloads.rng(21)
    for case in range(8):
        k = int(r.choice([1, 2, 3, 5, 16, 33, 300]))
        lens = r.integers(0, 20000, size=k)
        lens[r.random(k) < 0.15] = 0
        alphabet = [None, 3, 50][case % 3]
        keys, offs = make_runs(r, dtype, lens, descending, alphabet)
        vals = workloads.row_index(keys.size)
        check(bcf, keys, offs, None, descending)
        check(bcf, keys, offs, vals, descending)


@pytest.mark.parametrize("k", [2, 16, 256])
def test_benchmark_family_scaled(bcf, k):
    total = 1 << 22
    keys, offs = workloads.sorted_runs(k, total)
    vals = workloads.row_index(total)
    check(bcf, keys, offs, None, False)
    check(bcf, keys, offs, vals, False)


@pytest.mark.parametrize("dtype", ["u32", "f32", "u64"])
@pytest.mark.parametrize("descending", [False, True])
def test_runs_of_disjoint_ranges(bcf, dtype, descending):
    """Runs that are consecutive stretches of one sorted array, in order and in
    reverse order of the stretches: every merge then takes all of one run
    before the other, so nearly every merge tile copies one window."""
    from tests.pins import order_rank

    r = workloads.rng(24)
    lens = r.integers(1, 40000, size=9)
    lens[3] = 0
    n = int(lens.sum())
    keys = workloads.keys("uniform", dtype, n, seed=12)
    rank = order_rank(keys)
    keys = keys[np.argsort(~rank if descending else rank, kind="stable")]
    bounds = np.concatenate([[0], np.cumsum(lens)])
    for flip in (False, True):
        idx = range(len(lens) - 1, -1, -1) if flip else range(len(lens))
        parts = [keys[bounds[i]:bounds[i + 1]] for i in idx]
        ks = np.concatenate(parts)
        offs = np.concatenate([[0], np.cumsum([p.size for p in parts])]).astype(np.uint64)
        vals = workloads.row_index(n)
        check(bcf, ks, offs, None, descending)
        check(bcf, ks, offs, vals, descending)
        check(bcf, ks, offs, vals, descending, inplace=True)


def test_in_place_odd_and_even_pass_counts(bcf):
    r = workloads.rng(22)
    for k in (2, 3, 4, 7, 8):
        lens = r.integers(1, 30000, size=k)
        keys, offs = make_runs(r, "u32", lens)
        vals = workloads.row_index(keys.size)
        check(bcf, keys, offs, vals, False, inplace=True)


def test_runs_not_starting_at_zero(bcf):
    r = workloads.rng(23)
    lens = np.array([5000, 12345, 1, 0, 9999])
    keys, offs = make_runs(r, "u32", lens)
    offs_shift = offs.copy()
    offs_shift[0] = 3  # runs cover [3, n); a suffix of a sorted run is sorted
    vals = workloads.row_index(keys.size)
    ek, ev = oracle.merge_runs(keys, vals, offs_shift)
    kd, vd = to_dev(keys), to_dev(vals)
    ko, vo = torch.zeros_like(kd), torch.zeros_like(vd)
    bcf.bcf_merge_runs(ko, vo, kd, vd, [int(x) for x in offs_shift], kt=0)
    torch.cuda.synchronize()
    gk, gv = from_dev(ko, np.uint32), from_dev(vo, np.uint32)
    assert np.array_equal(gk[3:], ek[3:]) and np.array_equal(gv[3:], ev[3:])
    assert np.all(gk[:3] == 0) and np.all(gv[:3] == 0)  # outside the runs: untouched


def test_unsorted_runs_stay_in_bounds(bcf):
    """Runs that are not sorted break bcf_merge_runs' precondition: the order
    of the output is then undefined, but every access stays inside the runs
    and the tiles' shared memory (the merge kernel clamps each tile's end
    split into what its start split allows).  The call completes, reports no
    device error, and the context sorts exactly afterwards."""
    r = np.random.default_rng(99)
    for k, total in ((2, 50_000), (5, 300_001), (64, (1 << 20) + 3)):
        keys = workloads.keys("uniform", "u32", total, seed=int(r.integers(1 << 30)))
        cuts = np.sort(r.choice(np.arange(1, total), size=k - 1, replace=False))
        offs = np.concatenate([[0], cuts, [total]]).astype(np.uint64)
        vals = workloads.row_index(total)
        kd, vd = to_dev(keys), to_dev(vals)
        ko, vo = torch.empty_like(kd), torch.empty_like(vd)
        bcf.bcf_merge_runs(ko, vo, kd, vd, [int(x) for x in offs], kt=0)
        bcf.bcf_merge_runs(ko, None, kd, None, [int(x) for x in offs], kt=0)
        torch.cuda.synchronize()
        assert bcf.bcf_last_device_error() == 0
    keys = workloads.keys("uniform", "u32", 100_000, seed=3)
    kd = to_dev(keys)
    ko = torch.empty_like(kd)
    bcf.bcf_sort_keys(ko, kd, kt=0)
    torch.cuda.synchronize()
    exp, _ = oracle.sort(keys)
    assert np.array_equal(from_dev(ko, np.uint32), exp)
