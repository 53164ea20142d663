"""bcf_sort_keys_static: the sort for callers that cannot allocate device memory.

Such callers (a framework that owns every device allocation and hands out only
input and output buffers, a process whose device memory belongs to an external
pool, latency-critical loops that must avoid cudaMalloc's implicit
synchronisation) call the entry point with inputs and outputs only; the
library's own device array is the scratch space.  This test calls it through
the C ABI twice in a row and checks each result bit for bit (the tolerance of
every sort test) against bcf_sort_keys and against the CPU oracle, and that
sizes above the array's limit and unknown algorithms are refused.  It lives in
its own file, collected last, and passes alone or after the other tests.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import from_dev, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    from paper_1306_5076_gb300 import _native, build

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return _native.load()


def _opts(desc, algorithm=0):
    from paper_1306_5076_gb300 import _native

    return ctypes.byref(_native.BcfOpts(int(desc), 1, algorithm))


def _sort_static(lib, keys, kt, desc):
    kd = to_dev(keys)
    ko = torch.empty_like(kd)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.bcf_sort_keys_static(ctypes.c_void_p(ko.data_ptr()), ctypes.c_void_p(kd.data_ptr()),
                                  keys.size, kt, _opts(desc), stream)
    assert st == 0, lib.bcf_status_string(st)
    torch.cuda.synchronize()
    return from_dev(ko, keys.dtype)


def _sort_ws(lib, keys, kt, desc):
    from paper_1306_5076_gb300 import BCF_OP_SORT

    kd = to_dev(keys)
    ko = torch.empty_like(kd)
    wsb = lib.bcf_workspace_bytes(BCF_OP_SORT, keys.size, 0, kt, 0)
    ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.bcf_sort_keys(ctypes.c_void_p(ko.data_ptr()), ctypes.c_void_p(kd.data_ptr()),
                           keys.size, kt, _opts(desc), ctypes.c_void_p(ws.data_ptr()), wsb, stream)
    assert st == 0, lib.bcf_status_string(st)
    torch.cuda.synchronize()
    return from_dev(ko, keys.dtype)


def test_static_matches_workspace_sort_twice_in_a_row(lib):
    from paper_1306_5076_gb300 import _native

    cases = [("u32", "uniform", _native.BCF_STATIC_MAX_KEYS, False, 0),
             ("f32", "gaussian", 777_777, True, 2),
             ("u64", "distinct16", _native.BCF_STATIC_MAX_KEYS, False, 1)]  # widest keys at the limit
    for dtype, dist, n, desc, kt in cases:
        keys = workloads.keys(dist, dtype, n, seed=61 + n)
        expect = _sort_ws(lib, keys, kt, desc)
        truth, _ = oracle.sort(keys, descending=desc)
        assert np.array_equal(expect.view(np.uint8), truth.view(np.uint8))
        first = _sort_static(lib, keys, kt, desc)
        second = _sort_static(lib, keys, kt, desc)  # the array keeps the first call's data
        for got in (first, second):
            assert np.array_equal(got.view(np.uint8), expect.view(np.uint8))
            assert np.array_equal(got.view(np.uint8), truth.view(np.uint8))


def test_static_refuses_more_than_its_limit(lib):
    from paper_1306_5076_gb300 import _native

    n = _native.BCF_STATIC_MAX_KEYS + 1
    st = lib.bcf_sort_keys_static(ctypes.c_void_p(0x100000), ctypes.c_void_p(0x200000000), n, 0,
                                  _opts(False), None)
    assert st == 5  # BCF_EUNSUPPORTED, returned before any launch


def test_static_pivot_buckets_take_the_merge_path_and_unknown_algorithms_fail(lib):
    keys = workloads.keys("distinct16", "u32", 300_000, seed=62)
    kd = to_dev(keys)
    ko = torch.empty_like(kd)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.bcf_sort_keys_static(ctypes.c_void_p(ko.data_ptr()), ctypes.c_void_p(kd.data_ptr()),
                                  keys.size, 0, _opts(False, 1), stream)
    assert st == 0, lib.bcf_status_string(st)
    torch.cuda.synchronize()
    truth, _ = oracle.sort(keys)
    assert np.array_equal(from_dev(ko, np.uint32), truth)
    st = lib.bcf_sort_keys_static(ctypes.c_void_p(ko.data_ptr()), ctypes.c_void_p(kd.data_ptr()),
                                  keys.size, 0, _opts(False, 99), stream)
    assert st == 1  # BCF_EINVAL, as bcf_sort_keys returns for it
