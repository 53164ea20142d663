"""Sorting host buffers (bcf_sort_keys_host / bcf_sort_pairs_host): the copy
in, the sort and the copy out through the C ABI give the oracle's result,
bit-exact, for both algorithms, keys and pairs, sizes from empty to many
chunks with a ragged tail, and for calls overlapping on several streams."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import bits, kt_of

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


def pinned(a: np.ndarray):
    ibits = np.int32 if a.dtype.itemsize == 4 else np.int64
    return torch.from_numpy(np.ascontiguousarray(a).view(ibits)).pin_memory()


def host_sort(bcf, keys, vals=None, descending=False, algorithm="merge", stream=None, ws=None):
    hk = pinned(keys)
    ko = torch.empty_like(hk).pin_memory()
    kt = kt_of(keys)
    if vals is None:
        bcf.bcf_sort_keys_host(ko, hk, descending=descending, kt=kt, algorithm=algorithm,
                               stream=stream, ws=ws)
        return ko, None
    hv = pinned(vals)
    vo = torch.empty_like(hv).pin_memory()
    bcf.bcf_sort_pairs_host(ko, vo, hk, hv, descending=descending, kt=kt, algorithm=algorithm,
                            stream=stream, ws=ws)
    return ko, vo


def as_np(t, dtype):
    return t.numpy().view(dtype)


@pytest.mark.parametrize("algorithm", ["merge", "pivot_buckets"])
@pytest.mark.parametrize("n", [0, 1, 1000, 16384 * 9 + 77, (1 << 22) + 5])
@pytest.mark.parametrize("dtype", ["u32", "f64"])
def test_host_sort_matches_oracle(bcf, algorithm, n, dtype):
    keys = workloads.keys("zipf" if n % 2 else "uniform", dtype, n, seed=n + 1)
    vals = workloads.row_index(n)
    for desc in (False, True):
        ko, _ = host_sort(bcf, keys, descending=desc, algorithm=algorithm)
        torch.cuda.synchronize()
        ek, _ = oracle.sort(keys, descending=desc)
        assert np.array_equal(bits(as_np(ko, keys.dtype)), bits(ek))
        ko, vo = host_sort(bcf, keys, vals, descending=desc, algorithm=algorithm)
        torch.cuda.synchronize()
        ek, ev = oracle.sort(keys, vals, descending=desc)
        assert np.array_equal(bits(as_np(ko, keys.dtype)), bits(ek))
        assert np.array_equal(as_np(vo, np.uint32), ev)
    assert bcf.bcf_last_device_error() == 0


def test_overlapping_calls_on_several_streams(bcf):
    """Calls on three streams, each with its own workspace, issued back to back
    so that one call's copies overlap another's sort: every result is exact."""
    n = (1 << 21) + 3
    streams = [torch.cuda.Stream() for _ in range(3)]
    wss = [torch.empty(bcf.bcf_workspace_bytes(bcf._native.BCF_OP_SORT_HOST, n, 0, 0, False),
                       dtype=torch.uint8, device="cuda") for _ in streams]
    inputs = [workloads.keys("uniform", "u32", n, seed=900 + i) for i in range(6)]
    outs = []
    for i, keys in enumerate(inputs):
        outs.append(host_sort(bcf, keys, stream=streams[i % 3], ws=wss[i % 3])[0])
    torch.cuda.synchronize()
    for keys, ko in zip(inputs, outs):
        assert np.array_equal(as_np(ko, np.uint32), np.sort(keys))
