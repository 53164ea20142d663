"""Pins of the CPU oracle against things other than itself (CPU only).

What fixes the expected results here:
* brute force on tiny inputs: every permutation for n <= 8 (the inverse
  permutation is the closed-form answer) and every sequence over a 3-letter
  alphabet for n <= 7 against a stable selection sort;
* a stable insertion sort (textbook) for random n <= 1000;
* a library routine for the special cases it covers: numpy's stable argsort
  (integers, and floats without NaN or -0) and heapq.merge for merging;
* IEEE 754 totalOrder: the hand-listed golden vectors
  tests/golden/f32_total_order.txt and f64_total_order.txt, and the standard's
  case analysis in tests/pins.py;
* two's-complement order (i32 / i64): Python's integers and numpy's signed sort;
* closed forms of the paper's data sets (Sec. 4): sorted -> identity,
  reversed distinct keys -> reversal, 0-1 -> zero count, k copies -> k-blocks;
* invariants: sorted, permutation of the input, stable.
Mutation checks at the end compile broken copies of the oracle and show that
each plausible mistake fails at least one of these pins.
"""
from __future__ import annotations

import heapq
import itertools
import os
import re
import shutil

import numpy as np
import pytest

import oracle
import workloads
from tests import pins

GOLDEN_DIR = os.path.join(os.path.dirname(__file__), "golden")
FLOAT = {32: (np.float32, np.uint32), 64: (np.float64, np.uint64)}


def read_golden(width=32):
    out = []
    with open(os.path.join(GOLDEN_DIR, f"f{width}_total_order.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(int(line.split()[0], 16))
    return np.array(out, dtype=FLOAT[width][1])


def _keys(values, dtype):
    if dtype == "f32":
        return np.array(values, dtype=np.uint32).view(np.float32)
    if dtype == "f64":
        return np.array(values, dtype=np.uint64).view(np.float64)
    return np.array(values, dtype=workloads.DTYPES[dtype])


# ---------------------------------------------------------------- key order

@pytest.mark.parametrize("width", [32, 64])
def test_golden_list_is_in_ieee_total_order(width):
    g = [int(x) for x in read_golden(width)]
    assert len(g) == 28
    for i in range(len(g)):
        for j in range(len(g)):
            assert pins.ieee_total_order_lt(g[i], g[j], width) == (i < j), (hex(g[i]), hex(g[j]))


def check_golden_order(lib, width=32):
    g = read_golden(width)
    ft = FLOAT[width][0]
    for i in range(len(g)):
        for j in range(len(g)):
            assert oracle.key_less(ft, int(g[i]), int(g[j]), lib=lib) == (i < j)
    r = workloads.rng(11)
    for _ in range(20):
        shuffled = g[r.permutation(g.size)]
        ko, _ = oracle.sort(shuffled.view(ft), lib=lib)
        assert np.array_equal(ko.view(g.dtype), g)
        kd, _ = oracle.sort(shuffled.view(ft), descending=True, lib=lib)
        assert np.array_equal(kd.view(g.dtype), g[::-1])


@pytest.mark.parametrize("width", [32, 64])
def test_oracle_float_golden_order(oracle_lib, width):
    check_golden_order(oracle_lib, width)


@pytest.mark.parametrize("width", [32, 64])
def test_oracle_float_order_matches_ieee_case_analysis(oracle_lib, width):
    ft, ut = FLOAT[width]
    r = workloads.rng(12)
    bits = r.integers(0, 2**width, size=3000, dtype=np.uint64).astype(ut)
    bits[:28] = read_golden(width)
    # also pairs that differ only in sign, or only in the lowest bit
    bits[100:200:2] = bits[101:201:2] ^ ut(1 << (width - 1))
    bits[200:300:2] = bits[201:301:2] ^ ut(1)
    for a, b in zip(bits[:-1], bits[1:]):
        a, b = int(a), int(b)
        assert oracle.key_less(ft, a, b) == pins.ieee_total_order_lt(a, b, width)
        assert oracle.key_less(ft, b, a) == pins.ieee_total_order_lt(b, a, width)


@pytest.mark.parametrize("width", [32, 64])
def test_order_rank_helper_matches_ieee(width):
    g = read_golden(width)
    r = pins.order_rank(g.view(FLOAT[width][0]))
    assert np.all(r[1:] > r[:-1])


@pytest.mark.parametrize("dtype,width", [(np.int16, 16), (np.int32, 32), (np.int64, 64)])
def test_oracle_signed_order_matches_python_integers(oracle_lib, dtype, width):
    """Two's-complement order: the oracle's comparison of raw bit patterns
    agrees with Python's ``<`` on the values the patterns encode."""
    lo, hi = -(1 << (width - 1)), (1 << (width - 1)) - 1
    special = [lo, lo + 1, -2, -1, 0, 1, 2, hi - 1, hi]
    r = workloads.rng(18)
    vals = special + [int(x) for x in r.integers(lo, hi, size=2000, dtype=np.int64,
                                                  endpoint=True)]
    mask = (1 << width) - 1
    for a, b in itertools.chain(itertools.product(special, special), zip(vals[:-1], vals[1:])):
        assert oracle.key_less(dtype, a & mask, b & mask, lib=oracle_lib) == (a < b), (a, b)


# ---------------------------------------------------------------- brute force

def check_all_permutations(lib, max_n=8):
    for n in range(0, max_n + 1):
        for perm in itertools.permutations(range(n)):
            keys = np.array(perm, dtype=np.uint32)
            ko, vo = oracle.sort(keys, np.arange(n, dtype=np.uint32), lib=lib)
            inv = np.empty(n, dtype=np.uint32)
            inv[keys] = np.arange(n, dtype=np.uint32)
            assert np.array_equal(ko, np.arange(n, dtype=np.uint32))
            assert np.array_equal(vo, inv)


def test_all_permutations_up_to_8(oracle_lib):
    check_all_permutations(oracle_lib)


ALPHABETS = {
    "u32": [7, 3, 0xFFFFFFFF],
    "u64": [2**63 + 5, 3, 2**64 - 1],
    # -0.0, +0.0 and a quiet NaN: ties, signed zeros and NaN placement
    "f32": [0x80000000, 0x00000000, 0x7FC00000],
    # a positive value, -1 and the most negative value: unsigned order differs
    "i32": [5, -1, -(2**31)],
    "i64": [5, -1, -(2**63)],
    "u16": [7, 3, 0xFFFF],
    "i16": [5, -1, -(2**15)],
    "f64": [0x8000000000000000, 0x0000000000000000, 0x7FF8000000000000],
}


def check_ternary_sequences(lib, dtype, descending, max_n=7):
    alpha = ALPHABETS[dtype]
    lt = pins.lt_for(workloads.DTYPES[dtype], descending)
    for n in range(0, max_n + 1):
        for seq in itertools.product(range(3), repeat=n):
            kb = [alpha[s] for s in seq]
            keys = _keys(kb, dtype)
            ko, vo = oracle.sort(keys, np.arange(n, dtype=np.uint32), descending=descending,
                                 lib=lib)
            exp = pins.stable_selection_sort(list(zip(kb, range(n))), lt)
            assert pins.as_bits(ko) == [k for k, _ in exp]
            assert [int(v) for v in vo] == [v for _, v in exp]


@pytest.mark.parametrize("dtype", list(workloads.DTYPES))
@pytest.mark.parametrize("descending", [False, True])
def test_all_ternary_sequences_stable(oracle_lib, dtype, descending):
    check_ternary_sequences(oracle_lib, dtype, descending, max_n=7 if dtype == "u32" else 6)


def random_bits(r, dtype, n, alphabet):
    if alphabet is not None:
        pool = workloads.keys("uniform", dtype, alphabet, seed=int(r.integers(1 << 30)))
        return pool[r.integers(0, alphabet, size=n)]
    return workloads.keys("uniform", dtype, n, seed=int(r.integers(1 << 30)))


@pytest.mark.parametrize("dtype", list(workloads.DTYPES))
def test_insertion_sort_random(oracle_lib, dtype):
    r = workloads.rng(13)
    for case in range(6):
        n = int(r.integers(0, 1001)) if case else 1000
        alphabet = [None, 2, 5, 40][case % 4]
        keys = random_bits(r, dtype, n, alphabet)
        for desc in (False, True):
            ko, vo = oracle.sort(keys, np.arange(n, dtype=np.uint32), descending=desc)
            exp = pins.stable_insertion_sort(list(zip(pins.as_bits(keys), range(n))),
                                             pins.lt_for(keys.dtype, desc))
            assert pins.as_bits(ko) == [k for k, _ in exp]
            assert [int(v) for v in vo] == [v for _, v in exp]


# ---------------------------------------------------------------- library special cases

@pytest.mark.parametrize("dtype", ["u32", "u64", "i32", "i64", "u16", "i16"])
def test_matches_numpy_stable_argsort_integers(oracle_lib, dtype):
    r = workloads.rng(14)
    for n, alpha in [(100_000, None), (50_000, 97)]:
        keys = random_bits(r, dtype, n, alpha)
        idx = np.arange(n, dtype=np.uint32)
        ko, vo = oracle.sort(keys, idx)
        order = np.argsort(keys, kind="stable")
        assert np.array_equal(ko, keys[order]) and np.array_equal(vo, order.astype(np.uint32))
        # descending: stable argsort of the order-reversing bijection ~key
        # (max - key for unsigned, -1 - key for two's complement)
        rev = ~keys
        order_d = np.argsort(rev, kind="stable")
        kd, vd = oracle.sort(keys, idx, descending=True)
        assert np.array_equal(kd, keys[order_d]) and np.array_equal(vd, order_d.astype(np.uint32))


@pytest.mark.parametrize("ft", [np.float32, np.float64])
def test_matches_numpy_stable_argsort_finite_floats(oracle_lib, ft):
    r = workloads.rng(15)
    vals = r.normal(0, 1e3, size=60_000).astype(ft)
    vals = np.round(vals)  # many ties
    vals[vals == 0] = 1.0  # numpy treats -0 == +0; totalOrder does not
    ko, vo = oracle.sort(vals, np.arange(vals.size, dtype=np.uint32))
    order = np.argsort(vals, kind="stable")
    assert np.array_equal(pins.raw_bits(ko), pins.raw_bits(vals[order]))
    assert np.array_equal(vo, order.astype(np.uint32))


# ---------------------------------------------------------------- closed forms

def test_closed_forms_paper_data_sets(oracle_lib):
    n = 1 << 15
    idx = np.arange(n, dtype=np.uint32)
    srt = workloads.keys("sorted", "u32", n, seed=1)
    ko, vo = oracle.sort(srt, idx)
    assert np.array_equal(ko, srt) and np.array_equal(vo, idx)
    distinct = workloads.paper_keys("distinct", n)
    rev = np.ascontiguousarray(np.arange(n, 0, -1, dtype=np.uint32))
    ko, vo = oracle.sort(rev, idx)
    assert np.array_equal(ko, np.arange(1, n + 1, dtype=np.uint32))
    assert np.array_equal(vo, idx[::-1])
    ko, _ = oracle.sort(distinct)
    assert np.array_equal(ko, np.arange(1, n + 1, dtype=np.uint32))
    z = workloads.paper_keys("zero_one", n)
    ko, vo = oracle.sort(z, idx)
    zeros = int(np.count_nonzero(z == 0))
    assert np.all(ko[:zeros] == 0) and np.all(ko[zeros:] == 1)
    assert np.array_equal(vo[:zeros], np.flatnonzero(z == 0).astype(np.uint32))
    for k in (2, 16, 2250):
        d = workloads.paper_keys(f"dup{k}", n)
        ko, vo = oracle.sort(d, idx)
        pins.check_sorted_stable(d, idx, ko, vo)
        _, counts = np.unique(ko, return_counts=True)
        short = counts[counts != k]
        assert counts.size == -(-n // k) and short.size <= 1
        assert short.size == 0 or short[0] == n - k * (counts.size - 1)


@pytest.mark.parametrize("dtype", list(workloads.DTYPES))
@pytest.mark.parametrize("dist", workloads.DISTRIBUTIONS)
def test_invariants_on_workload_distributions(oracle_lib, dtype, dist):
    n = (1 << 14) + 77
    keys = workloads.keys(dist, dtype, n)
    idx = np.arange(n, dtype=np.uint32)
    for desc in (False, True):
        ko, vo = oracle.sort(keys, idx, descending=desc)
        pins.check_sorted_stable(keys, idx, ko, vo, descending=desc)
    if dist == "distinct16":
        ko, vo = oracle.sort(keys, idx)
        assert np.unique(pins.order_rank(ko)).size <= 16


def test_multithreaded_equals_single_thread(oracle_lib):
    for dtype in workloads.DTYPES:
        keys = workloads.keys("distinct16", dtype, (1 << 17) + 3, seed=5)
        idx = np.arange(keys.size, dtype=np.uint32)
        k1, v1 = oracle.sort(keys, idx, nthreads=1)
        k4, v4 = oracle.sort(keys, idx, nthreads=4)
        assert np.array_equal(k1.view(np.uint8), k4.view(np.uint8))
        assert np.array_equal(v1, v4)


# ---------------------------------------------------------------- merge and segments

def check_merge_runs(lib, dtype="u32", descending=False):
    r = workloads.rng(16)
    lt = pins.lt_for(workloads.DTYPES[dtype], descending)
    for case in range(25):
        k = int(r.integers(1, 9))
        lens = r.integers(0, 40, size=k)
        lens[r.random(k) < 0.2] = 0
        runs = []
        for m in lens:
            rb = random_bits(r, dtype, int(m), int(r.integers(1, 6)))
            items = pins.stable_insertion_sort(list(zip(pins.as_bits(rb), range(int(m)))), lt)
            runs.append([b for b, _ in items])
        flat = [b for run in runs for b in run]
        keys = _keys(flat, dtype) if flat else np.zeros(0, workloads.DTYPES[dtype])
        offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
        n = len(flat)
        ko, vo = oracle.merge_runs(keys, np.arange(n, dtype=np.uint32), offs,
                                   descending=descending, lib=lib)
        # heapq.merge is stable across iterables: ties come from earlier runs first
        tagged = []
        pos = 0
        for run in runs:
            tagged.append([(b, pos + i) for i, b in enumerate(run)])
            pos += len(run)
        rank = ((lambda b: pins.order_rank(_keys([b], dtype))[0]) if dtype in ("f32", "f64")
                else int)
        sign = -1 if descending else 1
        exp = list(heapq.merge(*tagged, key=lambda t: sign * int(rank(t[0]))))
        assert pins.as_bits(ko) == [b for b, _ in exp]
        assert [int(v) for v in vo] == [p for _, p in exp]


@pytest.mark.parametrize("dtype", list(workloads.DTYPES))
@pytest.mark.parametrize("descending", [False, True])
def test_merge_runs_matches_heapq_merge(oracle_lib, dtype, descending):
    check_merge_runs(oracle_lib, dtype, descending)


def test_segmented_sort_brute_force(oracle_lib):
    r = workloads.rng(17)
    for dtype in workloads.DTYPES:
        sizes = r.integers(0, 30, size=40)
        sizes[::7] = 0
        sizes[::11] = 1
        offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
        n = int(offs[-1])
        keys = random_bits(r, dtype, n, 4)
        idx = np.arange(n, dtype=np.uint32)
        for desc in (False, True):
            ko, vo = oracle.segmented_sort(keys, idx, offs, descending=desc)
            lt = pins.lt_for(keys.dtype, desc)
            bits = pins.as_bits(keys)
            for s in range(sizes.size):
                lo, hi = int(offs[s]), int(offs[s + 1])
                exp = pins.stable_selection_sort(list(zip(bits[lo:hi], range(lo, hi))), lt)
                assert pins.as_bits(ko[lo:hi]) == [b for b, _ in exp]
                assert [int(v) for v in vo[lo:hi]] == [v for _, v in exp]


def test_empty_and_single(oracle_lib):
    for dtype in workloads.DTYPES:
        e = np.zeros(0, workloads.DTYPES[dtype])
        ko, vo = oracle.sort(e, np.zeros(0, np.uint32))
        assert ko.size == 0 and vo.size == 0
        one = workloads.keys("uniform", dtype, 1, seed=3)
        ko, vo = oracle.sort(one, np.zeros(1, np.uint32))
        assert pins.as_bits(ko) == pins.as_bits(one) and vo[0] == 0


# ---------------------------------------------------------------- mutation checks

MUTANTS = {
    # ties taken from the right run: breaks stability
    "unstable_merge": (r"if \(precedes\(c, right\[j\], left\[i\]\)\)",
                       "if (!precedes(c, left[i], right[j]))"),
    # negative floats ordered by ascending magnitude
    "f32_negative_magnitude": (r"return mag_a > mag_b;", "return mag_a < mag_b;"),
    # sign rule inverted
    "f32_sign": (r"return sign_a == 1; /\*", "return sign_a == 0; /*"),
    # descending implemented as a reversed ascending output (ties reversed too)
    "desc_reverses_ties": (r"return c->descending \? bits_less\(c->dtype, b, a\) : "
                           r"bits_less\(c->dtype, a, b\);",
                           "return bits_less(c->dtype, a, b);"),
    # f64 negatives ordered by ascending magnitude, and the f64 sign rule inverted
    "f64_negative_magnitude": (r"return abs_a > abs_b;", "return abs_a < abs_b;"),
    "f64_sign": (r"return neg_a == 1;", "return neg_a == 0;"),
    # signed keys compared as unsigned bit patterns
    "i32_unsigned": (r"return \(int32_t\)\(uint32_t\)a < \(int32_t\)\(uint32_t\)b;",
                     "return (uint32_t)a < (uint32_t)b;"),
    "i64_unsigned": (r"return \(int64_t\)a < \(int64_t\)b;", "return a < b;"),
    "i16_unsigned": (r"return \(int16_t\)\(uint16_t\)a < \(int16_t\)\(uint16_t\)b;",
                     "return (uint16_t)a < (uint16_t)b;"),
    # 16-bit keys read as 32-bit ones
    "u16_as_32bit": (r"    case 2:  return \(\(const uint16_t\*\)c->keys\)\[i\];\n", ""),
    # 64-bit floats read through the 32-bit key path
    "f64_as_32bit": (r"dtype == ORACLE_I64 \|\| dtype == ORACLE_F64\) \? 8 : 4",
                     "dtype == ORACLE_I64) ? 8 : 4"),
    # right-run tail dropped
    "drop_tail": (r"while \(j < nr\) out\[o\+\+\] = right\[j\+\+\];",
                  "while (j + 1 < nr) out[o++] = right[j++]; if (j < nr) out[o++] = left[0];"),
}


def _pins_fail(lib, mutant):
    checks = [
        lambda: check_golden_order(lib),
        lambda: check_golden_order(lib, 64),
        lambda: check_all_permutations(lib, 6),
        lambda: check_ternary_sequences(lib, "i32", False, 3),
        lambda: check_ternary_sequences(lib, "i64", False, 3),
        lambda: check_ternary_sequences(lib, "i16", False, 3),
        lambda: check_ternary_sequences(lib, "u16", False, 3),
        lambda: check_ternary_sequences(lib, "u32", False, 5),
        lambda: check_ternary_sequences(lib, "f32", True, 4),
        lambda: check_merge_runs(lib, "u32", False),
    ]
    for chk in checks:
        try:
            chk()
        except AssertionError:
            return True
    return False


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_catch_planted_mistakes(tmp_path, mutant):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = open(os.path.join(os.path.dirname(oracle.__file__), "bcf_oracle.c")).read()
    pat, rep = MUTANTS[mutant]
    mutated, count = re.subn(pat, rep, src)
    assert count == 1, f"mutation {mutant} did not apply"
    if mutant == "desc_reverses_ties":
        # ascending-only comparator; reverse the whole output when descending
        mutated = mutated.replace(
            "    gather(keys_out, vals_out, keys_in, vals_in, perm, n, dtype);\n    free(perm);",
            "    if (descending) for (uint64_t i = 0; i < n / 2; ++i) { uint64_t t = perm[i];"
            " perm[i] = perm[n - 1 - i]; perm[n - 1 - i] = t; }\n"
            "    gather(keys_out, vals_out, keys_in, vals_in, perm, n, dtype);\n    free(perm);")
    path = tmp_path / "mutant.c"
    path.write_text(mutated)
    so = oracle.build(force=True, src=str(path), out=str(tmp_path / "libmutant.so"))
    lib = oracle.load(so)
    assert _pins_fail(lib, mutant), f"planted mistake {mutant} passed every pin"
