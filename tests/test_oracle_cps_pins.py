"""Pins of the oracle's colored prefix sums (Appendix A) against things other
than itself (CPU only).

What fixes the expected results here:
* brute force on small inputs: the definition summed term by term in Python
  integers (quadratic, no running state);
* a library routine for the special cases it covers: numpy's cumsum for one
  color, and for each color's subsequence taken on its own;
* closed forms: all values 1 gives each element's 1-based rank within its
  color; the last element of each color holds that color's total (bincount);
* the exclusive result is the inclusive one minus the element's own value;
* invalid colors are rejected.
Mutation checks compile broken copies of the oracle and show that each
plausible mistake fails at least one of these pins.
"""
from __future__ import annotations

import os
import re
import shutil

import numpy as np
import pytest

import oracle
import workloads

M32 = (1 << 32) - 1


def brute_force(values, colors, exclusive):
    out = []
    for i in range(len(values)):
        s = 0
        for j in range(i + (0 if exclusive else 1)):
            if colors[j] == colors[i]:
                s += int(values[j])
        out.append(s & M32)
    return np.array(out, dtype=np.uint32)


def check_brute_force(lib):
    r = workloads.rng(61)
    for case in range(30):
        n = int(r.integers(0, 120))
        d = int(r.choice([1, 2, 3, 7, 16, 64, 256]))
        values = r.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
        colors = r.integers(0, d, size=n).astype(np.uint8)
        for excl in (False, True):
            got = oracle.colored_prefix_sums(values, colors, d, exclusive=excl, lib=lib)
            assert np.array_equal(got, brute_force(values, colors, excl)), (case, excl)


def check_per_color_cumsum(lib):
    for law in ("uniform", "skewed", "runs"):
        values, colors = workloads.colored_elements(50_000, 16, seed=62, law=law)
        got = oracle.colored_prefix_sums(values, colors, 16, lib=lib)
        for c in range(16):
            m = colors == c
            exp = (np.cumsum(values[m].astype(np.uint64)) & M32).astype(np.uint32)
            assert np.array_equal(got[m], exp), (law, c)


def check_closed_forms(lib):
    r = workloads.rng(63)
    n = 10_000
    colors = r.integers(0, 5, size=n).astype(np.uint8)
    ones = np.ones(n, np.uint32)
    got = oracle.colored_prefix_sums(ones, colors, 5, lib=lib)
    # rank within color: stable argsort by color groups positions; ranks 1, 2, ...
    order = np.argsort(colors, kind="stable")
    starts = np.searchsorted(colors[order], np.arange(5))
    rank = np.empty(n, np.int64)
    rank[order] = np.arange(n) - starts[colors[order]] + 1
    assert np.array_equal(got, rank.astype(np.uint32))
    values = r.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
    got = oracle.colored_prefix_sums(values, colors, 5, lib=lib)
    totals = np.zeros(5, np.uint64)
    np.add.at(totals, colors, values.astype(np.uint64))
    for c in range(5):
        last = np.flatnonzero(colors == c)[-1]
        assert int(got[last]) == int(totals[c]) & M32


def check_exclusive_relation(lib):
    values, colors = workloads.colored_elements(20_000, 7, seed=64)
    inc = oracle.colored_prefix_sums(values, colors, 7, lib=lib)
    exc = oracle.colored_prefix_sums(values, colors, 7, exclusive=True, lib=lib)
    assert np.array_equal(exc, (inc.astype(np.uint64) - values + (1 << 32)).astype(np.uint64)
                          .astype(np.uint32) & np.uint32(M32))


def test_brute_force(oracle_lib):
    check_brute_force(oracle_lib)


def test_one_color_is_numpy_cumsum(oracle_lib):
    values, colors = workloads.colored_elements(100_000, 1, seed=65)
    assert not colors.any()
    for excl in (False, True):
        got = oracle.colored_prefix_sums(values, colors, 1, exclusive=excl)
        cs = np.cumsum(values.astype(np.uint64)) & M32
        exp = np.concatenate([[0], cs[:-1]]) if excl else cs
        assert np.array_equal(got, exp.astype(np.uint32))


def test_each_color_is_numpy_cumsum(oracle_lib):
    check_per_color_cumsum(oracle_lib)


def test_closed_forms(oracle_lib):
    check_closed_forms(oracle_lib)


def test_exclusive_is_inclusive_minus_value(oracle_lib):
    check_exclusive_relation(oracle_lib)


def test_rejects_bad_colors_and_d(oracle_lib):
    v = np.ones(4, np.uint32)
    with pytest.raises(RuntimeError):
        oracle.colored_prefix_sums(v, np.array([0, 1, 2, 3], np.uint8), 3)
    with pytest.raises(RuntimeError):
        oracle.colored_prefix_sums(v, np.zeros(4, np.uint8), 0)
    assert oracle.colored_prefix_sums(v[:0], np.zeros(0, np.uint8), 4).size == 0


MUTANTS = {
    # one running sum shared by all colors
    "shared_accumulator": (r"uint32_t c = colors\[i\];", "uint32_t c = 0; (void)colors;"),
    # inclusive and exclusive swapped
    "swapped_inclusive": (r"if \(exclusive\) \{", "if (!exclusive) {"),
    # running sums not reset at the start
    "no_reset": (r"        acc\[c\] = 0;\n", "        acc[c] = c;\n"),
    # the element's own value dropped from the inclusive sum
    "drop_own_value": (r"            acc\[c\] \+= values\[i\];\n            out\[i\] = acc\[c\];",
                       "            out[i] = acc[c];\n            acc[c] += values[i];"),
}


def _pins_fail(lib):
    for chk in (check_brute_force, check_per_color_cumsum, check_closed_forms,
                check_exclusive_relation):
        try:
            chk(lib)
        except (AssertionError, RuntimeError):
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
    path = tmp_path / "mutant.c"
    path.write_text(mutated)
    so = oracle.build(force=True, src=str(path), out=str(tmp_path / "libmutant.so"))
    lib = oracle.load(so)
    assert _pins_fail(lib), f"planted mistake {mutant} passed every pin"
