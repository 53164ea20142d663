"""Parity of the GPU sort (through the C ABI) with the CPU oracle -- bit-exact.

Sizes span several block tiles and merge passes with ragged tails; every key
type, both directions, keys-only and stable pairs, every workload
distribution and the paper's data sets; edge cases (empty, single, all-equal,
extreme key values that coincide with the network's pads, NaN / signed-zero
floats, aliasing, misalignment, short workspace).
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


def gpu_sort(bcf, keys, vals=None, descending=False, inplace=False):
    kd = to_dev(keys)
    kt = kt_of(keys)
    if vals is None:
        ko = kd if inplace else torch.empty_like(kd)
        bcf.bcf_sort_keys(ko, kd, descending=descending, kt=kt)
        torch.cuda.synchronize()
        return from_dev(ko, keys.dtype), None
    vd = to_dev(vals)
    ko = kd if inplace else torch.empty_like(kd)
    vo = vd if inplace else torch.empty_like(vd)
    bcf.bcf_sort_pairs(ko, vo, kd, vd, descending=descending, kt=kt)
    torch.cuda.synchronize()
    return from_dev(ko, keys.dtype), from_dev(vo, np.uint32)


def assert_same(got_k, got_v, exp_k, exp_v):
    gk, ek = bits(got_k), bits(exp_k)
    if not np.array_equal(gk, ek):
        bad = np.flatnonzero(gk != ek)
        raise AssertionError(f"keys differ at {bad.size} positions, first {bad[:8]}: "
                             f"got {gk[bad[:4]]} expected {ek[bad[:4]]}")
    if exp_v is not None:
        if not np.array_equal(got_v, exp_v):
            bad = np.flatnonzero(got_v != exp_v)
            raise AssertionError(f"values differ at {bad.size} positions, first {bad[:8]}")


SIZES = [0, 1, 2, 31, 1000, 4095, 4096, 4097, 8191, 8192, 8193, 3 * 8192 + 17, 65536,
         (1 << 17) + 123, (1 << 20) + 5]


@pytest.mark.parametrize("dtype", list(workloads.DTYPES))
@pytest.mark.parametrize("n", SIZES)
def test_uniform_keys_and_pairs_all_sizes(bcf, dtype, n):
    keys = workloads.keys("uniform", dtype, n, seed=100 + n)
    vals = workloads.row_index(n)
    for desc in (False, True):
        ek, _ = oracle.sort(keys, descending=desc)
        gk, _ = gpu_sort(bcf, keys, descending=desc)
        assert_same(gk, None, ek, None)
        ek, ev = oracle.sort(keys, vals, descending=desc)
        gk, gv = gpu_sort(bcf, keys, vals, descending=desc)
        assert_same(gk, gv, ek, ev)


@pytest.mark.parametrize("dtype", list(workloads.DTYPES))
@pytest.mark.parametrize("dist", workloads.DISTRIBUTIONS)
def test_workload_distributions(bcf, dtype, dist):
    n = (1 << 18) + 4321
    keys = workloads.keys(dist, dtype, n)
    vals = workloads.row_index(n)
    for desc in (False, True):
        ek, ev = oracle.sort(keys, vals, descending=desc, nthreads=8)
        gk, gv = gpu_sort(bcf, keys, vals, descending=desc)
        assert_same(gk, gv, ek, ev)
        gk, _ = gpu_sort(bcf, keys, descending=desc)
        assert_same(gk, None, ek, None)


@pytest.mark.parametrize("name", workloads.PAPER_SETS)
def test_paper_data_sets(bcf, name):
    n = (1 << 19) + 99
    keys = workloads.paper_keys(name, n)
    vals = workloads.row_index(n)
    ek, ev = oracle.sort(keys, vals, nthreads=8)
    gk, gv = gpu_sort(bcf, keys, vals)
    assert_same(gk, gv, ek, ev)


def test_extreme_keys_tie_with_pads(bcf):
    """Real keys equal to the network's +inf/-inf pads must sort by position."""
    n = 3 * 8192 + 77
    r = workloads.rng(5)
    i32, i64 = np.iinfo(np.int32), np.iinfo(np.int64)
    for dtype, lo, hi in (("u32", 0, 0xFFFFFFFF), ("u64", 0, 2**64 - 1),
                          ("i32", i32.min, i32.max), ("i64", i64.min, i64.max)):
        dt = workloads.DTYPES[dtype]
        keys = np.where(r.random(n) < 0.5, dt(lo), dt(hi)).astype(dt)
        vals = workloads.row_index(n)
        for desc in (False, True):
            ek, ev = oracle.sort(keys, vals, descending=desc)
            gk, gv = gpu_sort(bcf, keys, vals, descending=desc)
            assert_same(gk, gv, ek, ev)
    # float patterns that map to the extremes of the order: -NaN max and +NaN max
    for ut, ft, lo, hi in ((np.uint32, np.float32, 0xFFFFFFFF, 0x7FFFFFFF),
                           (np.uint64, np.float64, 2**64 - 1, 2**63 - 1)):
        keys = np.where(r.random(n) < 0.5, ut(lo), ut(hi)).astype(ut).view(ft)
        vals = workloads.row_index(n)
        for desc in (False, True):
            ek, ev = oracle.sort(keys, vals, descending=desc)
            gk, gv = gpu_sort(bcf, keys, vals, descending=desc)
            assert_same(gk, gv, ek, ev)


@pytest.mark.parametrize("width", [32, 64])
def test_float_golden_total_order(bcf, width):
    from tests.test_oracle_pins import FLOAT, read_golden

    g = read_golden(width)
    r = workloads.rng(9)
    keys = g[r.integers(0, g.size, size=50_000)].view(FLOAT[width][0])
    vals = workloads.row_index(keys.size)
    for desc in (False, True):
        ek, ev = oracle.sort(keys, vals, descending=desc)
        gk, gv = gpu_sort(bcf, keys, vals, descending=desc)
        assert_same(gk, gv, ek, ev)
        # every golden pattern appears, in golden order (reversed if descending)
        seen = np.unique(bits(gk), return_index=True)
        order = np.argsort(seen[1])
        assert np.array_equal(seen[0][order], g[::-1] if desc else g)


@pytest.mark.parametrize("dtype", ["i32", "i64"])
def test_signed_keys_around_zero(bcf, dtype):
    """Small signed values on both sides of zero: an unsigned compare would
    put every negative key after every positive one."""
    n = 3 * 8192 + 5
    r = workloads.rng(10)
    keys = r.integers(-50, 50, size=n).astype(workloads.DTYPES[dtype])
    vals = workloads.row_index(n)
    for desc in (False, True):
        ek, ev = oracle.sort(keys, vals, descending=desc)
        gk, gv = gpu_sort(bcf, keys, vals, descending=desc)
        assert_same(gk, gv, ek, ev)


def test_all_equal_and_sorted_inputs(bcf):
    n = 100_003
    for keys in (np.full(n, 7, np.uint32), np.arange(n, dtype=np.uint32),
                 np.arange(n, 0, -1, dtype=np.uint32)):
        vals = workloads.row_index(n)
        ek, ev = oracle.sort(keys, vals)
        gk, gv = gpu_sort(bcf, keys, vals)
        assert_same(gk, gv, ek, ev)


@pytest.mark.parametrize("n", [5000, 8192 * 5 + 3])
def test_in_place(bcf, n):
    keys = workloads.keys("gaussian", "u32", n, seed=3)
    vals = workloads.row_index(n)
    ek, ev = oracle.sort(keys, vals)
    gk, gv = gpu_sort(bcf, keys, vals, inplace=True)
    assert_same(gk, gv, ek, ev)
    ek, _ = oracle.sort(keys, descending=True)
    gk, _ = gpu_sort(bcf, keys, descending=True, inplace=True)
    assert_same(gk, None, ek, None)


def test_deterministic_repeat(bcf):
    keys = workloads.keys("distinct16", "u32", 300_001, seed=4)
    vals = workloads.row_index(keys.size)
    first = gpu_sort(bcf, keys, vals)
    for _ in range(5):
        again = gpu_sort(bcf, keys, vals)
        assert np.array_equal(first[0], again[0]) and np.array_equal(first[1], again[1])


def test_errors_on_device_buffers(bcf):
    n = 1 << 16
    kd = torch.zeros(n + 4, dtype=torch.int32, device="cuda")
    ko = torch.zeros(n + 4, dtype=torch.int32, device="cuda")
    with pytest.raises(bcf.BcfError) as ei:  # misaligned input
        bcf.bcf_sort_keys(ko[:n], kd[1:n + 1], kt=0)
    assert ei.value.status == 1
    small = torch.zeros(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(bcf.BcfError) as ei:
        bcf.bcf_sort_keys(ko[:n], kd[:n], kt=0, ws=small)
    assert ei.value.status == 2
    assert bcf.bcf_last_device_error() == 0


def test_full_size_bench_config_against_oracle(bcf):
    """The benchmark's workload (2^28 uniform u32 keys) in its launch
    configuration, compared with the oracle on every element."""
    n = 1 << 28
    keys = workloads.keys("uniform", "u32", n)
    kd = to_dev(keys)
    ko = torch.empty_like(kd)
    bcf.bcf_sort_keys(ko, kd, kt=0)
    torch.cuda.synchronize()
    got = from_dev(ko, np.uint32)
    del kd, ko
    import os

    exp, _ = oracle.sort(keys, nthreads=os.cpu_count() or 8)
    assert np.array_equal(got, exp)


@pytest.mark.parametrize("dtype", ["u32", "u64", "f64"])
@pytest.mark.parametrize("n", [8192, 3 * 16384 + 40, (1 << 20) + 8])
def test_outputs_16_but_not_32_byte_aligned(bcf, dtype, n):
    """The ABI asks for 16-byte alignment only: outputs (and inputs) that start
    16 bytes past a 32-byte boundary take the 16-byte store path."""
    keys = workloads.keys("uniform", dtype, n, seed=77)
    vals = workloads.row_index(n)
    per16 = 16 // keys.dtype.itemsize  # elements in 16 bytes
    kin = torch.zeros(n + 2 * per16, dtype=to_dev(keys[:1]).dtype, device="cuda")
    vin = torch.zeros(n + 8, dtype=torch.int32, device="cuda")
    kin[per16:per16 + n] = to_dev(keys)
    vin[4:4 + n] = to_dev(vals)
    kout = torch.zeros_like(kin)
    vout = torch.zeros_like(vin)
    ki, ko = kin[per16:per16 + n], kout[per16:per16 + n]
    vi, vo = vin[4:4 + n], vout[4:4 + n]
    assert ko.data_ptr() % 32 == 16 and vo.data_ptr() % 32 == 16
    kt = kt_of(keys)
    for desc in (False, True):
        bcf.bcf_sort_pairs(ko, vo, ki, vi, kt=kt, descending=desc)
        torch.cuda.synchronize()
        ek, ev = oracle.sort(keys, vals, descending=desc)
        assert_same(from_dev(ko, keys.dtype), from_dev(vo, np.uint32), ek, ev)
        bcf.bcf_sort_keys(ko, ki, kt=kt, descending=desc)
        torch.cuda.synchronize()
        assert_same(from_dev(ko, keys.dtype), None, ek, None)
    # nothing written outside the output slices
    assert not kout[:per16].any() and not kout[per16 + n:].any()
    assert not vout[:4].any() and not vout[4 + n:].any()


def test_more_than_2p32_keys_closed_form(bcf):
    """Maximum sizes: n = 2^32 + 2^20 + 37 keys, past every 32-bit index
    (tiles, merge items, samples, run offsets).  Key i is (i * C) mod 2^32 for
    an odd C, a bijection on the first 2^32 positions, so the multiset is every
    u32 value once plus the values D of positions 2^32 .. n-1 (those of
    i - 2^32) once more.  The sorted output is then known in closed form: value
    v fills positions [v + #(D < v), v + #(D <= v)], checked at every position.
    Payload i mod 2^32 must come out as (key * C^-1) mod 2^32 (both copies of a
    value carry the same payload)."""
    need = 100 << 30
    if torch.cuda.get_device_properties(0).total_memory < need + (8 << 30):
        pytest.skip("needs about 100 GB of device memory")
    C = 0x9E3779B1
    Cinv = pow(C, -1, 1 << 32)
    n = (1 << 32) + (1 << 20) + 37
    r = n - (1 << 32)
    chunk = 1 << 27

    def u32_as_i32(x):
        return torch.where(x >= (1 << 31), x - (1 << 32), x).to(torch.int32)

    kd = torch.empty(n, dtype=torch.int32, device="cuda")
    for c0 in range(0, n, chunk):
        i = torch.arange(c0, min(n, c0 + chunk), dtype=torch.int64, device="cuda")
        kd[c0:c0 + i.numel()] = u32_as_i32((i * C) & 0xFFFFFFFF)
    D = torch.sort((torch.arange(r, dtype=torch.int64, device="cuda") * C) & 0xFFFFFFFF).values

    def check_keys(ko):
        for c0 in range(0, n, chunk):
            c1 = min(n, c0 + chunk)
            v = ko[c0:c1].to(torch.int64) & 0xFFFFFFFF
            p = torch.arange(c0, c1, dtype=torch.int64, device="cuda")
            lt = torch.searchsorted(D, v, right=False)
            le = torch.searchsorted(D, v, right=True)
            bad = ~((v + lt <= p) & (p <= v + le))
            if bool(bad.any()):
                j = int(torch.nonzero(bad)[0, 0]) + c0
                raise AssertionError(f"position {j} holds {int(ko[j]) & 0xFFFFFFFF}")

    ko = torch.empty_like(kd)
    bcf.bcf_sort_keys(ko, kd, kt=0)
    torch.cuda.synchronize()
    check_keys(ko)

    vd = torch.empty_like(kd)
    for c0 in range(0, n, chunk):
        i = torch.arange(c0, min(n, c0 + chunk), dtype=torch.int64, device="cuda")
        vd[c0:c0 + i.numel()] = u32_as_i32(i & 0xFFFFFFFF)
    vo = torch.empty_like(vd)
    ko.zero_()
    bcf.bcf_sort_pairs(ko, vo, kd, vd, kt=0)
    torch.cuda.synchronize()
    check_keys(ko)
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        k = ko[c0:c1].to(torch.int64) & 0xFFFFFFFF
        v = vo[c0:c1].to(torch.int64) & 0xFFFFFFFF
        assert torch.equal(v, (k * Cinv) & 0xFFFFFFFF), c0
    assert bcf.bcf_last_device_error() == 0
