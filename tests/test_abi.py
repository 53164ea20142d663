"""The C-ABI library loads and exports what include/bcfsort.h declares (CPU only).

No call here launches GPU work: only host-side entry points (sizes, plans,
status strings) and argument checks that return before any CUDA call.
"""
from __future__ import annotations

import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bcfsort.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1306_5076_gb300 import _native, build

    build.build()
    return _native.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(bcf_[a-z_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("bcf_sort_keys", "bcf_sort_pairs", "bcf_merge_runs", "bcf_segmented_sort",
                     "bcf_workspace_bytes", "bcf_status_string", "bcf_last_device_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1306_5076_gb300 import _native

    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in bcfsort.h but not exported"
        assert name in _native.SIGNATURES, f"{name} has no Python binding"


def test_status_strings_and_version(lib):
    for code in range(6):
        s = lib.bcf_status_string(code).decode()
        assert s.startswith("BCF_")
    assert b"sm_103a" in lib.bcf_version()


def test_workspace_bytes_scale_with_input(lib):
    from paper_1306_5076_gb300 import (BCF_F32, BCF_F64, BCF_I32, BCF_I64, BCF_OP_MERGE,
                                       BCF_OP_SORT, BCF_U32, BCF_U64)

    n = 1 << 20
    keys = lib.bcf_workspace_bytes(BCF_OP_SORT, n, 0, BCF_U32, 0)
    pairs = lib.bcf_workspace_bytes(BCF_OP_SORT, n, 0, BCF_U32, 1)
    wide = lib.bcf_workspace_bytes(BCF_OP_SORT, n, 0, BCF_U64, 0)
    assert keys >= 4 * n and pairs >= 8 * n and wide >= 8 * n
    assert keys % 256 == 0 and pairs % 256 == 0
    assert lib.bcf_workspace_bytes(BCF_OP_SORT, n, 0, BCF_F32, 0) == keys
    # the signed and double key types take the space of their width
    for kt, same in ((BCF_I32, keys), (BCF_I64, wide), (BCF_F64, wide)):
        assert lib.bcf_workspace_bytes(BCF_OP_SORT, n, 0, kt, 0) == same
    assert lib.bcf_workspace_bytes(BCF_OP_SORT, n, 0, 8, 0) == 0
    # 16-bit keys: widened copies in and out (4 bytes each) on top of the 32-bit sort's
    for kt16 in (6, 7):
        w16 = lib.bcf_workspace_bytes(BCF_OP_SORT, n, 0, kt16, 0)
        assert w16 >= keys + 8 * n
        assert lib.bcf_workspace_bytes(BCF_OP_SORT, n, 0, kt16, 1) >= pairs + 8 * n
    # colored prefix sums: one look-back word per (tile, color); u32 values only
    from paper_1306_5076_gb300 import BCF_OP_CPS
    cps = lib.bcf_workspace_bytes(BCF_OP_CPS, n, 16, BCF_U32, 0)
    assert cps >= (n // 16384) * 16 * 8 and cps % 256 == 0
    assert lib.bcf_workspace_bytes(BCF_OP_CPS, n, 0, BCF_U32, 0) == 0
    assert lib.bcf_workspace_bytes(BCF_OP_CPS, n, 65, BCF_U32, 0) == 0
    assert lib.bcf_workspace_bytes(BCF_OP_CPS, n, 16, BCF_U64, 0) == 0
    # pivot buckets: the block-sorted copy, the segmented-sort scratch and small
    # tables; always at least the merge path's (its fall-back) workspace
    from paper_1306_5076_gb300 import BCF_OP_SORT_PB
    for kt, hv in ((BCF_U32, 0), (BCF_U32, 1), (BCF_U64, 0)):
        pb = lib.bcf_workspace_bytes(BCF_OP_SORT_PB, n, 0, kt, hv)
        assert pb >= 2 * lib.bcf_workspace_bytes(BCF_OP_SORT, n, 0, kt, hv) - (1 << 20)
        assert pb >= lib.bcf_workspace_bytes(BCF_OP_SORT, 10, 0, kt, hv)
    assert lib.bcf_workspace_bytes(BCF_OP_MERGE, n, 256, BCF_U32, 0) >= keys
    assert lib.bcf_workspace_bytes(9, n, 0, BCF_U32, 0) == 0
    assert lib.bcf_workspace_bytes(BCF_OP_SORT, n, 0, 9, 0) == 0


@pytest.mark.parametrize("n", [0, 1, 4095, 4096, 8192, 8193, 1 << 20, (1 << 28) + 1])
def test_plan_pass_count_is_lemma_2(lib, n):
    """Lemma 2: one base-case pass plus ceil(log2(n / T)) merge passes."""
    from paper_1306_5076_gb300 import _native

    for kt in range(8):
        for has_vals in (0, 1):
            p = _native.BcfPlan()
            assert lib.bcf_sort_plan(n, kt, has_vals, ctypes.byref(p)) == 0
            runs = -(-n // p.block_tile)
            expect = 0 if runs <= 1 else math.ceil(math.log2(runs))
            assert p.merge_passes == expect
            assert p.launches == (0 if n == 0 else 1 + 2 * expect)
            kb = 8 if kt in (1, 4, 5) else 4
            assert p.bytes_per_pass == 2 * n * (kb + 4 * has_vals)
            assert p.merge_tile <= 2 * p.block_tile


def test_host_side_argument_errors_return_before_launch(lib):
    from paper_1306_5076_gb300 import _native

    opts = ctypes.byref(_native.BcfOpts(0, 1, 0))
    EINVAL = 1
    # bad dtype (one past the last key type, and a negative code)
    assert lib.bcf_sort_keys(None, None, 0, 9, opts, None, 0, None) == EINVAL
    assert lib.bcf_sort_keys(None, None, 0, 8, opts, None, 0, None) == EINVAL
    assert lib.bcf_sort_keys(None, None, 0, -1, opts, None, 0, None) == EINVAL
    # n == 0 is a no-op
    assert lib.bcf_sort_keys(None, None, 0, 0, opts, None, 0, None) == 0
    # null pointers with n > 0
    assert lib.bcf_sort_keys(None, None, 10, 0, opts, None, 0, None) == EINVAL
    # misaligned pointers (never dereferenced: rejected on the host)
    assert lib.bcf_sort_keys(ctypes.c_void_p(0x1004), ctypes.c_void_p(0x2000), 10, 0, opts, None,
                             0, None) == EINVAL
    # partial overlap of output and input
    assert lib.bcf_sort_keys(ctypes.c_void_p(0x10000), ctypes.c_void_p(0x10010), 100, 0, opts,
                             None, 0, None) == EINVAL
    # wide payloads: rows must be a positive multiple of 4 bytes; null pointers
    assert lib.bcf_sort_pairs_wide(None, None, None, None, 10, 6, 0, opts, None, 0, None) == EINVAL
    assert lib.bcf_sort_pairs_wide(None, None, None, None, 10, 8, 0, opts, None, 0, None) == EINVAL
    assert lib.bcf_sort_pairs_wide(None, None, None, None, 0, 8, 0, opts, None, 0, None) == 0
    assert lib.bcf_workspace_bytes(7, 1 << 20, 0, 0, 1) >= 8 * (1 << 20)
    # host-buffer sorts: null host pointers, short workspace
    assert lib.bcf_sort_keys_host(None, None, 10, 0, opts, None, 0, None) == EINVAL
    assert lib.bcf_sort_keys_host(None, None, 0, 0, opts, None, 0, None) == 0
    assert lib.bcf_sort_keys_host(ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000), 1 << 20, 0,
                                  opts, ctypes.c_void_p(0x300000000), 4096, None) == 2
    assert lib.bcf_sort_pairs_host(ctypes.c_void_p(0x1000), None, ctypes.c_void_p(0x2000), None,
                                   10, 0, opts, None, 0, None) == EINVAL
    # unknown algorithm
    bad_algo = ctypes.byref(_native.BcfOpts(0, 1, 7))
    assert lib.bcf_sort_keys(ctypes.c_void_p(0x10000), ctypes.c_void_p(0x20000), 10, 0, bad_algo,
                             None, 0, None) == EINVAL
    # pairs need both value pointers
    assert lib.bcf_sort_pairs(ctypes.c_void_p(0x10000), None, ctypes.c_void_p(0x20000), None, 10,
                              0, opts, None, 0, None) == EINVAL
    # merge: k == 0, and decreasing offsets
    offs = (ctypes.c_uint64 * 3)(0, 5, 3)
    assert lib.bcf_merge_runs(None, None, None, None, offs, 0, 0, opts, None, 0, None) == EINVAL
    assert lib.bcf_merge_runs(ctypes.c_void_p(0x10000), None, ctypes.c_void_p(0x20000), None,
                              offs, 2, 0, opts, None, 0, None) == EINVAL
    # colored prefix sums: d outside 1..64, layout unknown, null pointers
    assert lib.bcf_colored_prefix_sums(None, None, None, 10, 0, 0, 0, None, 0, None) == EINVAL
    assert lib.bcf_colored_prefix_sums(None, None, None, 10, 65, 0, 0, None, 0, None) == EINVAL
    assert lib.bcf_colored_prefix_sums(None, None, None, 10, 4, 0, 2, None, 0, None) == EINVAL
    assert lib.bcf_colored_prefix_sums(None, None, None, 10, 4, 0, 0, None, 0, None) == EINVAL
    assert lib.bcf_colored_prefix_sums(None, None, None, 0, 4, 0, 0, None, 0, None) == 0
    # merge: values on one side only
    good = (ctypes.c_uint64 * 2)(0, 4)
    assert lib.bcf_merge_runs(ctypes.c_void_p(0x10000), ctypes.c_void_p(0x30000),
                              ctypes.c_void_p(0x20000), None, good, 1, 0, opts, None, 0,
                              None) == EINVAL


def test_workspace_too_small_is_enomem(lib):
    from paper_1306_5076_gb300 import _native

    opts = ctypes.byref(_native.BcfOpts(0, 1, 0))
    n = 1 << 20  # needs merge passes, hence a workspace
    assert lib.bcf_sort_keys(ctypes.c_void_p(0x100000000), ctypes.c_void_p(0x200000000), n, 0,
                             opts, ctypes.c_void_p(0x300000000), 1024, None) == 2


def test_committed_tuning_table_rows_are_valid(lib):
    """Every row of the package's tuning table names a built configuration."""
    import paper_1306_5076_gb300 as bcf

    path = os.path.join(ROOT, "paper_1306_5076_gb300", "tuning", "gb300.tsv")
    rows = []
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            op, kb, hv, lo, hi, b, m, s = (int(x) for x in line.split())
            rows.append(dict(op=op, key_bytes=kb, has_vals=hv, n_min=lo, n_max=hi, block_cfg=b,
                             merge_cfg=m, seg_cfg=s))
    assert rows
    for r in rows:
        bcf.bcf_tuning_set([r])  # raises BcfError(EINVAL) for an unbuilt configuration
    bcf.bcf_tuning_set(None)
    with pytest.raises(bcf.BcfError):
        bcf.bcf_tuning_set([dict(op=0, key_bytes=8, has_vals=1, n_min=0, n_max=10, block_cfg=1,
                                 merge_cfg=0, seg_cfg=0)])  # no E = 32 for 64-bit pairs


def test_segmented_tuning_rows_name_who_merges(lib):
    """Segmented rows: merge_cfg -1 (the worker merges) or a built merge
    configuration whose tile is at most the sort tile (it must divide it)."""
    import paper_1306_5076_gb300 as bcf

    def row(merge_cfg, seg_cfg, kb=4, hv=0):
        return dict(op=2, key_bytes=kb, has_vals=hv, n_min=0, n_max=1 << 40, block_cfg=0,
                    merge_cfg=merge_cfg, seg_cfg=seg_cfg)

    tile = lambda kind, i: bcf.bcf_tuning_config(kind, i)[0] * bcf.bcf_tuning_config(kind, i)[1]
    for si in range(5):
        bcf.bcf_tuning_set([row(-1, si)])
        for mi in range(4):
            if tile(1, mi) <= tile(2, si):
                bcf.bcf_tuning_set([row(mi, si)])
            else:
                with pytest.raises(bcf.BcfError):
                    bcf.bcf_tuning_set([row(mi, si)])
    for bad in (-2, 4):
        with pytest.raises(bcf.BcfError):
            bcf.bcf_tuning_set([row(bad, 0)])
    with pytest.raises(bcf.BcfError):
        bcf.bcf_tuning_set([row(1, 0, kb=8)])  # no E = 32 merge for 64-bit keys
    bcf.bcf_tuning_set(None)


def test_profile_collect_launches_without_records(lib):
    """Host-side only: nothing recorded gives zero launches; missing output
    pointers are BCF_EINVAL."""
    from paper_1306_5076_gb300 import _native

    p = _native.BcfProfile()
    count = ctypes.c_uint32(7)
    kinds = (ctypes.c_int * 4)()
    ms = (ctypes.c_float * 4)()
    assert lib.bcf_profile_collect_launches(ctypes.byref(p), kinds, ms, 4, ctypes.byref(count)) == 0
    assert count.value == 0 and sum(p.launches) == 0
    assert lib.bcf_profile_collect_launches(ctypes.byref(p), None, None, 0, ctypes.byref(count)) == 0
    assert lib.bcf_profile_collect_launches(None, kinds, ms, 4, ctypes.byref(count)) == 1
    assert lib.bcf_profile_collect_launches(ctypes.byref(p), kinds, ms, 4, None) == 1
    assert lib.bcf_profile_collect_launches(ctypes.byref(p), None, ms, 4, ctypes.byref(count)) == 1


def test_selftest_wait_rejects_bad_limits_before_any_launch(lib):
    assert lib.bcf_selftest_bounded_wait(0, None) == 1
    assert lib.bcf_selftest_bounded_wait(2000001, None) == 1


def test_wait_limit_setting_range(lib):
    assert lib.bcf_wait_limit_us() == 2_000_000  # default: 2 s
    assert lib.bcf_set_wait_limit_us(60_000_001) == 1
    assert lib.bcf_wait_limit_us() == 2_000_000  # a rejected value changes nothing
    assert lib.bcf_set_wait_limit_us(1500) == 0
    assert lib.bcf_wait_limit_us() == 1500
    assert lib.bcf_set_wait_limit_us(0) == 0  # back to the default
    assert lib.bcf_wait_limit_us() == 2_000_000


def test_segmented_wait_selftest_checks_its_scratch_before_any_launch(lib):
    assert lib.bcf_selftest_segmented_wait(None, 4096, None) == 2  # BCF_ENOMEM
    assert lib.bcf_selftest_segmented_wait(ctypes.c_void_p(1 << 20), 511, None) == 2
    assert lib.bcf_selftest_segmented_wait(ctypes.c_void_p((1 << 20) + 16), 4096, None) == 1


def test_smem_floor_range(lib):
    assert lib.bcf_profile_set_smem_floor(227 * 1024 + 1) == 1
    assert lib.bcf_profile_set_smem_floor(200 * 1024) == 0
    assert lib.bcf_profile_set_smem_floor(0) == 0
