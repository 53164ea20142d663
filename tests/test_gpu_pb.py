"""Parity of the pivot-bucket sort (BCFMergesortPB, Sec. 3.2 "Duplicate
keys") with the CPU oracle -- bit-exact, and bit-identical to the merge-pass
sort.  Covers every workload distribution, the paper's duplicate data sets,
key types, payloads, both directions, in place, the fall-back below two tiles,
and workspace errors.
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


def pb_sort(bcf, keys, vals=None, descending=False, inplace=False, algorithm="pivot_buckets"):
    kd = to_dev(keys)
    ko = kd if inplace else torch.empty_like(kd)
    kt = kt_of(keys)
    if vals is None:
        bcf.bcf_sort_keys(ko, kd, descending=descending, kt=kt, algorithm=algorithm)
        torch.cuda.synchronize()
        return from_dev(ko, keys.dtype), None
    vd = to_dev(vals)
    vo = vd if inplace else torch.empty_like(vd)
    bcf.bcf_sort_pairs(ko, vo, kd, vd, descending=descending, kt=kt, algorithm=algorithm)
    torch.cuda.synchronize()
    return from_dev(ko, keys.dtype), from_dev(vo, np.uint32)


def check(bcf, keys, pairs=True, descending=False, inplace=False):
    vals = workloads.row_index(keys.size) if pairs else None
    ek, ev = oracle.sort(keys, vals, descending=descending, nthreads=8)
    gk, gv = pb_sort(bcf, keys, vals, descending, inplace)
    bad = np.flatnonzero(bits(gk) != bits(ek))
    assert bad.size == 0, f"keys differ at {bad.size} positions, first {bad[:6]}"
    if pairs:
        assert np.array_equal(gv, ev)
    assert bcf.bcf_last_device_error() == 0


N = 3 * 16384 + 4321  # several block tiles, a ragged last tile


@pytest.mark.parametrize("dtype", ["u32", "f32", "i64", "f64"])
@pytest.mark.parametrize("dist", workloads.DISTRIBUTIONS)
def test_distributions(bcf, dtype, dist):
    keys = workloads.keys(dist, dtype, N)
    for desc in (False, True):
        check(bcf, keys, pairs=True, descending=desc)
        check(bcf, keys, pairs=False, descending=desc)


@pytest.mark.parametrize("name", workloads.PAPER_SETS)
def test_paper_data_sets(bcf, name):
    keys = workloads.paper_keys(name, (1 << 19) + 17)
    check(bcf, keys, pairs=True)


@pytest.mark.parametrize("n", [16384 * 2 + 1, 200_001, (1 << 21) + 3])
def test_sizes_and_all_equal(bcf, n):
    for keys in (workloads.keys("zipf", "u32", n, seed=n), np.full(n, 0xFFFFFFFF, np.uint32),
                 np.full(n, 0, np.uint32)):
        check(bcf, keys, pairs=True)


def test_small_inputs_take_the_merge_path(bcf):
    for n in (0, 1, 1000, 16384, 2 * 16384):
        keys = workloads.keys("distinct16", "u32", n, seed=n)
        check(bcf, keys, pairs=True)


def test_in_place(bcf):
    keys = workloads.keys("distinct16", "u64", N, seed=5)
    check(bcf, keys, pairs=True, inplace=True)
    check(bcf, keys, pairs=False, descending=True, inplace=True)


def test_identical_to_merge_path(bcf):
    for dist in ("uniform", "zipf", "distinct16"):
        keys = workloads.keys(dist, "u32", (1 << 20) + 5, seed=11)
        vals = workloads.row_index(keys.size)
        a = pb_sort(bcf, keys, vals, algorithm="pivot_buckets")
        b = pb_sort(bcf, keys, vals, algorithm="merge")
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_workspace_sized_for_the_merge_path_is_too_small(bcf):
    n = 1 << 20
    kd = torch.zeros(n, dtype=torch.int32, device="cuda")
    ko = torch.empty_like(kd)
    ws = torch.empty(bcf.bcf_workspace_bytes(bcf.BCF_OP_SORT, n, 0, bcf.BCF_U32, False),
                     dtype=torch.uint8, device="cuda")
    with pytest.raises(bcf.BcfError) as ei:
        bcf.bcf_sort_keys(ko, kd, kt=bcf.BCF_U32, ws=ws, algorithm="pivot_buckets")
    assert ei.value.status == 2
    with pytest.raises(ValueError):
        bcf.bcf_sort_keys(ko, kd, kt=bcf.BCF_U32, algorithm="radix")


def test_large_duplicate_heavy_against_oracle(bcf):
    import os

    n = 1 << 26
    keys = workloads.keys("distinct16", "u32", n)
    vals = workloads.row_index(n)
    gk, gv = pb_sort(bcf, keys, vals)
    ek, ev = oracle.sort(keys, vals, nthreads=os.cpu_count() or 8)
    assert np.array_equal(gk, ek) and np.array_equal(gv, ev)


@pytest.mark.parametrize("dist,expect_pb", [("distinct16", True), ("zipf", True),
                                            ("uniform", False), ("sorted", False)])
@pytest.mark.parametrize("pairs", [False, True])
def test_auto_chooses_by_duplication_and_matches_the_oracle(bcf, dist, expect_pb, pairs):
    """algorithm="auto": pivot buckets when at least a third of the sampled keys
    (the splitters' own occurrences aside) equal a splitter (16 distinct values;
    Zipf(1.1) keys, about half), the merge path otherwise; the result is the oracle's
    either way.  The choice shows in the library's launch records: the
    decision itself launches three distribution-kind kernels (sample,
    splitters, count), the pivot-bucket sort five more."""
    n = (1 << 21) + 777
    keys = workloads.keys(dist, "u32", n)
    vals = workloads.row_index(n) if pairs else None
    bcf.bcf_profile_collect()
    bcf.bcf_profile_enable(True)
    try:
        got_k, got_v = pb_sort(bcf, keys, vals, algorithm="auto")
    finally:
        bcf.bcf_profile_enable(False)
    prof = bcf.bcf_profile_collect()
    ek, ev = oracle.sort(keys, vals)
    assert np.array_equal(bits(got_k), bits(ek))
    if pairs:
        assert np.array_equal(got_v, ev)
    distribution_launches = prof["pivot_buckets"]["launches"]
    assert distribution_launches == (8 if expect_pb else 3), prof


def test_auto_with_16_bit_and_descending_keys(bcf):
    n = (1 << 20) + 3
    for dtype, dist in (("i16", "distinct16"), ("u16", "uniform"), ("f32", "distinct16")):
        keys = workloads.keys(dist, dtype, n)
        for desc in (False, True):
            got, _ = pb_sort(bcf, keys, descending=desc, algorithm="auto")
            exp, _ = oracle.sort(keys, descending=desc)
            assert np.array_equal(bits(got), bits(exp)), (dtype, dist, desc)
