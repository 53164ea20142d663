"""Payloads wider than 32 bits (bcf_sort_pairs_wide): every payload row ends
up beside its key in the stable order, i.e. vals_out = vals_in[p] with p the
oracle's stable permutation; both algorithms, several key types and row
widths, and the argument errors."""
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


def payloads(kind, n, seed):
    r = workloads.rng(seed)
    if kind == "u64":
        return r.integers(0, 2**63, size=n, dtype=np.int64)
    if kind == "f32x3":
        return r.standard_normal((n, 3)).astype(np.float32)
    return r.integers(0, 256, size=(n, 16)).astype(np.uint8)  # 16-byte rows


@pytest.mark.parametrize("algorithm", ["merge", "pivot_buckets"])
@pytest.mark.parametrize("dtype,dist", [("u32", "uniform"), ("f64", "gaussian"),
                                        ("u16", "distinct16"), ("i64", "zipf")])
@pytest.mark.parametrize("kind", ["u64", "f32x3", "u8x16"])
def test_rows_follow_their_keys(bcf, algorithm, dtype, dist, kind):
    n = 3 * 16384 + 999
    keys = workloads.keys(dist, dtype, n, seed=5)
    vals = payloads(kind, n, 6)
    idx = workloads.row_index(n)
    for desc in (False, True):
        ek, perm = oracle.sort(keys, idx, descending=desc)
        kd = to_dev(keys)
        ko = torch.empty_like(kd)
        vd = torch.from_numpy(vals).to("cuda")
        vo = torch.empty_like(vd)
        bcf.bcf_sort_pairs_wide(ko, vo, kd, vd, kt=kt_of(keys), descending=desc,
                                algorithm=algorithm)
        torch.cuda.synchronize()
        assert np.array_equal(bits(from_dev(ko, keys.dtype)), bits(ek))
        assert np.array_equal(vo.cpu().numpy(), vals[perm])
    assert bcf.bcf_last_device_error() == 0


def test_wide_argument_errors(bcf):
    n = 1000
    kd = torch.zeros(n, dtype=torch.int32, device="cuda")
    ko = torch.empty_like(kd)
    v = torch.zeros((n, 2), dtype=torch.int64, device="cuda")
    with pytest.raises(bcf.BcfError) as ei:  # payloads in place
        bcf.bcf_sort_pairs_wide(ko, v, kd, v, kt=bcf.BCF_U32)
    assert ei.value.status == 1
    w = torch.zeros((n, 3), dtype=torch.int16, device="cuda")  # 6-byte rows
    with pytest.raises(bcf.BcfError) as ei:
        bcf.bcf_sort_pairs_wide(ko, torch.empty_like(w), kd, w, kt=bcf.BCF_U32)
    assert ei.value.status == 1
