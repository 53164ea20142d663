"""The compiled merge and block-sort networks on 0-1 inputs (the 0-1 principle
the paper invokes for its merging networks, Sec. 3.2), through the C ABI and
compared bit for bit with the oracle.

The host model of the network schedule is checked exhaustively on 0-1 inputs
elsewhere; these tests run the kernels themselves, so a divergence between the
model and the compiled code cannot hide.

Merge: bcf_merge_runs with k = 2 on A = 0^a 1^(|A|-a) and B = 0^c 1^(|B|-c).
Run lengths sit around the 2048-key merge tile and its multiples, and a and c
cover every boundary class: 0, 1, the middle, the tile - 1, the tile, the tile
+ 1, the run length - 1 and the run length.  So the output tile that holds the
0/1 transition is cut at every position class, and the A and B windows of the
merge-path split are empty, full or ragged.  Keys only and with payloads (the
payload is the input position, so stability is checked exactly).

Block sort: bcf_sort_keys on 0-1 vectors one tile long and a tile +- 1, with
zero counts from every boundary class and random placements.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests.gpu_util import from_dev, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TM = 2048  # merge tile of the tuned 32-bit configurations


@pytest.fixture(scope="module")
def bcf():
    import paper_1306_5076_gb300 as m
    from paper_1306_5076_gb300 import build

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    m._native.load()
    return m


def zero_counts(length):
    cand = {0, 1, length // 2, TM - 1, TM, TM + 1, length - 1, length}
    return sorted(c for c in cand if 0 <= c <= length)


def zero_one_run(length, zeros):
    r = np.ones(length, dtype=np.uint32)
    r[:zeros] = 0
    return r


def test_merge_tile_plan_is_the_one_swept(bcf):
    plan = bcf.bcf_sort_plan(1 << 20, bcf.BCF_U32, False)
    assert plan["merge_tile"] == TM
    plan = bcf.bcf_sort_plan(1 << 20, bcf.BCF_U32, True)
    assert plan["merge_tile"] == TM


@pytest.mark.parametrize("pairs", [False, True])
@pytest.mark.parametrize("la,lb", [(TM, TM), (TM - 1, TM + 1), (TM + 1, 1), (1, TM - 1),
                                   (2 * TM + 1, TM), (3 * TM, 2 * TM - 1), (5, 3 * TM + 7)])
def test_two_way_merge_of_zero_one_runs(bcf, la, lb, pairs):
    bad = []
    for a in zero_counts(la):
        for c in zero_counts(lb):
            keys = np.concatenate([zero_one_run(la, a), zero_one_run(lb, c)])
            offs = [0, la, la + lb]
            vals = np.arange(keys.size, dtype=np.uint32) if pairs else None
            kd = to_dev(keys)
            ko = torch.empty_like(kd)
            vd = to_dev(vals) if pairs else None
            vo = torch.empty_like(vd) if pairs else None
            bcf.bcf_merge_runs(ko, vo, kd, vd, offs, kt=bcf.BCF_U32)
            torch.cuda.synchronize()
            ek, ev = oracle.merge_runs(keys, vals, np.array(offs, dtype=np.uint64))
            ok = np.array_equal(from_dev(ko, np.uint32), ek)
            if pairs:
                ok = ok and np.array_equal(from_dev(vo, np.uint32), ev)
            if not ok:
                bad.append((a, c))
    assert bcf.bcf_last_device_error() == 0
    assert not bad, f"0-1 merges that differ from the oracle (zeros in A, zeros in B): {bad}"


@pytest.mark.parametrize("pairs", [False, True])
def test_block_sort_of_zero_one_tiles(bcf, pairs):
    plan = bcf.bcf_sort_plan(1 << 20, bcf.BCF_U32, pairs)
    T = plan["block_tile"]
    r = np.random.default_rng(1306)
    bad = []
    for n in (T - 1, T, T + 1):
        for zeros in sorted({0, 1, 31, 32, 33, n // 2, n - 33, n - 1, n}):
            for placement in ("random", "reversed", "alternating"):
                keys = np.ones(n, dtype=np.uint32)
                if placement == "random":
                    keys[r.choice(n, size=zeros, replace=False)] = 0
                elif placement == "reversed":
                    keys[n - zeros:] = 0
                else:
                    idx = np.arange(0, n, 2)[:zeros]
                    idx = np.concatenate([idx, np.arange(1, n, 2)[: zeros - idx.size]])
                    keys[idx] = 0
                vals = np.arange(n, dtype=np.uint32) if pairs else None
                kd = to_dev(keys)
                ko = torch.empty_like(kd)
                vd = to_dev(vals) if pairs else None
                vo = torch.empty_like(vd) if pairs else None
                if pairs:
                    bcf.bcf_sort_pairs(ko, vo, kd, vd, kt=bcf.BCF_U32)
                else:
                    bcf.bcf_sort_keys(ko, kd, kt=bcf.BCF_U32)
                torch.cuda.synchronize()
                ek, ev = oracle.sort(keys, vals)
                ok = np.array_equal(from_dev(ko, np.uint32), ek)
                if pairs:
                    ok = ok and np.array_equal(from_dev(vo, np.uint32), ev)
                if not ok:
                    bad.append((n, zeros, placement))
    assert bcf.bcf_last_device_error() == 0
    assert not bad, f"0-1 tiles that differ from the oracle: {bad}"
