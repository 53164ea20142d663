"""The sort's output does not depend on the tuning (GPU): every compiled
(E, NT) configuration of the block sort, the merge pass and the segmented sort
gives the oracle's result, bit-exact, for keys and stable pairs."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import bits, from_dev, to_dev

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
    yield m
    m.bcf_tuning_set(None)


def configs(bcf, kind, kb, pairs):
    out, i = [], 0
    while bcf.bcf_tuning_config(kind, i) is not None:
        if bcf.bcf_tuning_supported(kind, i, kb, pairs):
            out.append(i)
        i += 1
    return out


@pytest.mark.parametrize("dtype,pairs", [("u32", False), ("u32", True), ("u64", False),
                                         ("f32", True)])
def test_sort_invariant_to_tuning(bcf, dtype, pairs):
    kb = 8 if dtype == "u64" else 4
    kt = {"u32": 0, "u64": 1, "f32": 2}[dtype]
    n = (1 << 19) + 1234
    keys = workloads.keys("gaussian", dtype, n, seed=71)
    vals = workloads.row_index(n) if pairs else None
    ek, ev = oracle.sort(keys, vals, descending=True)
    for bi in configs(bcf, 0, kb, pairs):
        for mi in configs(bcf, 1, kb, pairs):
            be, bnt = bcf.bcf_tuning_config(0, bi)
            me, mnt = bcf.bcf_tuning_config(1, mi)
            if me * mnt > 2 * be * bnt:
                continue
            bcf.bcf_tuning_set([dict(op=0, key_bytes=kb, has_vals=int(pairs), n_min=0,
                                     n_max=1 << 40, block_cfg=bi, merge_cfg=mi, seg_cfg=0)])
            kd = to_dev(keys)
            ko = torch.empty_like(kd)
            if pairs:
                vd = to_dev(vals)
                vo = torch.empty_like(vd)
                bcf.bcf_sort_pairs(ko, vo, kd, vd, kt=kt, descending=True)
            else:
                bcf.bcf_sort_keys(ko, kd, kt=kt, descending=True)
            torch.cuda.synchronize()
            assert np.array_equal(bits(from_dev(ko, keys.dtype)), bits(ek)), (bi, mi)
            if pairs:
                assert np.array_equal(from_dev(vo, np.uint32), ev), (bi, mi)
    bcf.bcf_tuning_set(None)


@pytest.mark.parametrize("pairs", [False, True])
def test_segmented_invariant_to_tuning(bcf, pairs):
    keys, offs = workloads.segments(600, 1 << 15, "u32", seed=4100)
    vals = workloads.row_index(keys.size) if pairs else None
    ek, ev = oracle.segmented_sort(keys, vals, offs)
    od = torch.from_numpy(offs.astype(np.int64)).to("cuda")
    choices = []
    for si in configs(bcf, 2, 4, pairs):
        tile = np.prod(bcf.bcf_tuning_config(2, si))
        choices.append((si, -1))  # the worker merges
        choices += [(si, mi) for mi in configs(bcf, 1, 4, pairs)
                    if np.prod(bcf.bcf_tuning_config(1, mi)) <= tile]
    for si, mi in choices:
        bcf.bcf_tuning_set([dict(op=2, key_bytes=4, has_vals=int(pairs), n_min=0, n_max=1 << 40,
                                 block_cfg=0, merge_cfg=mi, seg_cfg=si)])
        kd = to_dev(keys)
        ko = torch.empty_like(kd)
        vd = to_dev(vals) if pairs else None
        vo = torch.empty_like(vd) if pairs else None
        bcf.bcf_segmented_sort(ko, vo, kd, vd, od, kt=0)
        torch.cuda.synchronize()
        assert np.array_equal(from_dev(ko, np.uint32), ek), (si, mi)
        if pairs:
            assert np.array_equal(from_dev(vo, np.uint32), ev), (si, mi)
    bcf.bcf_tuning_set(None)
