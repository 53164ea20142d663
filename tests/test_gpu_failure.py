"""Failure detection on the GPU without a fault: a bounded wait that runs out
is reported through the device error word, and the context stays usable.

bcf_selftest_bounded_wait makes one thread wait, bounded by the GPU's global
timer, for a device flag that nothing sets -- the same form of wait the
library's kernels use for bulk copies, work-queue slots and look-back words.
"""
from __future__ import annotations

import time

import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import from_dev, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BCF_OK, BCF_EINVAL, BCF_ETIMEOUT = 0, 1, 4


@pytest.fixture(scope="module")
def bcf():
    import paper_1306_5076_gb300 as m
    from paper_1306_5076_gb300 import build

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    m._native.load()
    return m


def test_wait_that_runs_out_is_reported_and_the_context_survives(bcf):
    lib = bcf._native.load()
    assert bcf.bcf_last_device_error() == BCF_OK  # start clean
    t0 = time.perf_counter()
    assert lib.bcf_selftest_bounded_wait(20000, None) == BCF_OK  # 20 ms
    assert lib.bcf_last_device_error(None) == BCF_ETIMEOUT
    assert time.perf_counter() - t0 >= 0.019
    assert lib.bcf_last_device_error(None) == BCF_OK  # read and cleared
    # the context is still usable: a sort afterwards is exact and reports nothing
    keys = workloads.keys("uniform", "u32", 100_000, seed=5)
    kd = to_dev(keys)
    ko = torch.empty_like(kd)
    bcf.bcf_sort_keys(ko, kd, kt=0)
    torch.cuda.synchronize()
    assert bcf.bcf_last_device_error() == BCF_OK
    exp, _ = oracle.sort(keys)
    assert np.array_equal(from_dev(ko, np.uint32), exp)


def test_segmented_worker_wait_on_an_unpublished_slot_runs_out(bcf):
    """The segmented sort's own worker kernel waits for a queue slot that the
    host set-up announces but never publishes; with the library's wait limit
    set short, the wait runs out, BCF_ETIMEOUT is reported, and sorts
    afterwards (segmented and plain) are exact."""
    lib = bcf._native.load()
    assert bcf.bcf_last_device_error() == BCF_OK
    scratch = torch.empty(4096, dtype=torch.uint8, device="cuda")
    bcf.bcf_set_wait_limit_us(50_000)  # 50 ms
    try:
        t0 = time.perf_counter()
        assert lib.bcf_selftest_segmented_wait(scratch.data_ptr(), 4096, None) == BCF_OK
        assert lib.bcf_last_device_error(None) == BCF_ETIMEOUT
        assert time.perf_counter() - t0 >= 0.049
        assert lib.bcf_last_device_error(None) == BCF_OK
        # with the short limit still in force, a real segmented sort never
        # comes near it
        keys, offs = workloads.segments(300, 1 << 14, "u32", seed=77)
        kd = to_dev(keys)
        ko = torch.empty_like(kd)
        od = torch.from_numpy(offs.astype(np.int64)).to("cuda")
        bcf.bcf_segmented_sort(ko, None, kd, None, od, kt=0)
        torch.cuda.synchronize()
        assert bcf.bcf_last_device_error() == BCF_OK
        got = from_dev(ko, np.uint32)
        for i in range(len(offs) - 1):
            a, b = int(offs[i]), int(offs[i + 1])
            exp, _ = oracle.sort(keys[a:b])
            assert np.array_equal(got[a:b], exp), f"segment {i}"
    finally:
        bcf.bcf_set_wait_limit_us(0)
    assert bcf.bcf_wait_limit_us() == 2_000_000
    keys = workloads.keys("uniform", "u32", 200_000, seed=6)
    kd = to_dev(keys)
    ko = torch.empty_like(kd)
    bcf.bcf_sort_keys(ko, kd, kt=0)
    torch.cuda.synchronize()
    assert bcf.bcf_last_device_error() == BCF_OK
    exp, _ = oracle.sort(keys)
    assert np.array_equal(from_dev(ko, np.uint32), exp)
