"""The benchmark's own input generators and output checks, on CPU tensors.

bench.py draws the large-sort grid's inputs on the device and checks every
output there (sorted order, payloads a permutation that follows its keys,
stability).  These tests run the same functions on CPU tensors: each law
produces what it states, a correct stable sort passes the check, and planted
mistakes -- a swapped pair, an unstable tie, a payload that left its key, a
changed key -- fail it.
"""
from __future__ import annotations

import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

DEV = torch.device("cpu")
N = 1 << 14


def reference_sort(k, key, pairs):
    """Stable sort by the key order through numpy (test reference only)."""
    o = bench.order_bits(torch, k, key).numpy()
    perm = np.argsort(o, kind="stable")
    ko = k[torch.from_numpy(perm)]
    vo = torch.from_numpy(perm.astype(np.int32)) if pairs else None
    return ko, vo


@pytest.mark.parametrize("key", ["u32", "f32", "u64"])
@pytest.mark.parametrize("dist", bench.GRID_DISTS)
def test_generated_laws(key, dist):
    k = bench.device_keys(torch, DEV, dist, key, N)
    assert k.numel() == N and k.dtype == (torch.int64 if key == "u64" else torch.int32)
    o = bench.order_bits(torch, k, key)
    if dist == "sorted":
        assert bool((o[1:] >= o[:-1]).all())
    if dist == "reverse":
        assert bool((o[1:] <= o[:-1]).all())
    if dist == "distinct16":
        assert torch.unique(k).numel() <= 16
    if dist == "gaussian" and key == "u32":
        u = (k.to(torch.int64) & 0xFFFFFFFF).double()
        assert abs(u.mean().item() - 2.0**31) < 4 * 2.0**28 / N**0.5
        assert abs(u.std().item() / 2.0**28 - 1) < 0.05
    if dist == "zipf":
        # rank 1 (key 0) is the most frequent symbol: P(1) = 1 / H(2^20, 1.1)
        h = float((torch.arange(1, (1 << 20) + 1, dtype=torch.float64) ** -1.1).sum())
        share = float((k == 0).double().mean()) if key != "f32" else float((k == 0).double().mean())
        assert abs(share - 1 / h) < 0.05
    # the same seed gives the same input
    assert torch.equal(k, bench.device_keys(torch, DEV, dist, key, N))


@pytest.mark.parametrize("key", ["u32", "f32", "u64"])
def test_check_accepts_a_stable_sort_and_rejects_planted_mistakes(key):
    k = bench.device_keys(torch, DEV, "distinct16", key, N)  # many ties
    ko, vo = reference_sort(k, key, True)
    assert bench.check_sorted_pairs(torch, k, ko, vo, key)
    ko1, _ = reference_sort(k, key, False)
    assert bench.check_sorted_pairs(torch, k, ko1, None, key)
    o = bench.order_bits(torch, ko, key)
    # an unstable tie: two payloads of equal keys swapped
    i = int(torch.nonzero(o[1:] == o[:-1])[0])
    bad = vo.clone()
    bad[i], bad[i + 1] = vo[i + 1], vo[i]
    assert not bench.check_sorted_pairs(torch, k, ko, bad, key)
    # two different keys out of order (their payloads move with them)
    j = int(torch.nonzero(o[1:] != o[:-1])[0])
    kb, vb = ko.clone(), vo.clone()
    kb[j], kb[j + 1] = ko[j + 1], ko[j]
    vb[j], vb[j + 1] = vo[j + 1], vo[j]
    assert not bench.check_sorted_pairs(torch, k, kb, vb, key)
    assert not bench.check_sorted_pairs(torch, k, kb, None, key)
    # a payload that left its key
    vc = vo.clone()
    vc[0], vc[-1] = vo[-1], vo[0]
    assert not bench.check_sorted_pairs(torch, k, ko, vc, key)
    # keys only: a key replaced by another value of the input (order kept)
    kc = ko1.clone()
    kc[0] = kc[1]
    if not torch.equal(kc, ko1):
        assert not bench.check_sorted_pairs(torch, k, kc, None, key)


def segmented_reference(k, offs, pairs):
    """Stable per-segment sort by unsigned key order (test reference only)."""
    o = (k.to(torch.int64) & 0xFFFFFFFF).numpy()
    perm = np.concatenate([a + np.argsort(o[a:b], kind="stable")
                           for a, b in zip(offs[:-1], offs[1:])]).astype(np.int64)
    ko = k[torch.from_numpy(perm)]
    return ko, (torch.from_numpy(perm.astype(np.int32)) if pairs else None)


def test_segmented_check_accepts_a_stable_segmented_sort_and_rejects_mistakes():
    r = np.random.default_rng(3)
    sizes = np.array([0, 1, 5, 0, 300, 1000, 2, 4000, 17, 0])
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(offs[-1])
    k = torch.from_numpy(r.integers(-2**31, 2**31, size=n).astype(np.int32))
    k[100:400] = 7  # ties inside one segment
    od = torch.from_numpy(offs)
    ko, vo = segmented_reference(k, offs, True)
    ko1, _ = segmented_reference(k, offs, False)
    assert bench.check_segmented(torch, k, ko, vo, od, chunk=1000)
    assert bench.check_segmented(torch, k, ko1, None, od, chunk=1000)
    # one sort of everything: order across segment borders is not required,
    # but keys must stay in their segments
    glob = k[torch.from_numpy(np.argsort((k.to(torch.int64) & 0xFFFFFFFF).numpy(),
                                         kind="stable"))]
    assert not bench.check_segmented(torch, k, glob, None, od, chunk=1000)
    # an unstable tie
    o = ko.to(torch.int64) & 0xFFFFFFFF
    i = int(torch.nonzero(o[1:] == o[:-1])[0])
    bad = vo.clone()
    bad[i], bad[i + 1] = vo[i + 1], vo[i]
    assert not bench.check_segmented(torch, k, ko, bad, od, chunk=1000)
    # two keys of one segment out of order (payloads move with them)
    j = int(torch.nonzero((o[1:] != o[:-1]))[5])
    kb, vb = ko.clone(), vo.clone()
    kb[j], kb[j + 1] = ko[j + 1], ko[j]
    vb[j], vb[j + 1] = vo[j + 1], vo[j]
    assert not bench.check_segmented(torch, k, kb, vb, od, chunk=1000)
    assert not bench.check_segmented(torch, k, kb, None, od, chunk=1000)
    # a key that moved to the neighbouring segment (each segment stays sorted)
    s = 5  # [306, 1306)
    a, b = int(offs[s]), int(offs[s + 1])
    kc = ko1.clone()
    kc[a] = ko1[a - 1]
    kc[a:b] = torch.from_numpy(np.sort(kc[a:b].numpy().view(np.uint32)).view(np.int32))
    assert not bench.check_segmented(torch, k, kc, None, od, chunk=1000)
    # a payload that points into another segment, with its key
    vc, kd2 = vo.clone(), ko.clone()
    vc[a], kd2[a] = vo[a - 1], ko[a - 1]
    assert not bench.check_segmented(torch, k, kd2, vc, od, chunk=1000)
