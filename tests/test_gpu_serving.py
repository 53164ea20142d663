"""The continuous-batching server: every result is the same in the mix as on
its own (bit-exact; the oracle agrees on a sample), in batched and in plain
mode, under arena pressure, for sort and merge requests, keys and pairs."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import from_dev

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


def make_mix(count, seed, lo=1 << 8, hi=1 << 18, merges=True):
    r = workloads.rng(seed)
    sizes = workloads.log_uniform_sizes(r, count, lo, hi)
    pairs = r.random(count) < 0.3
    ops = np.where(merges & (r.random(count) < 0.15), 1, 0)
    arrivals = np.sort(r.uniform(0, 0.05, size=count))  # a burst: requests overlap
    return sizes, pairs, ops, arrivals


def run_mix(bcf, mode, arena_bytes, sizes, pairs, ops, arrivals, seed=0):
    from paper_1306_5076_gb300 import serve

    n_tot = int(sizes.sum())
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    keys = torch.randint(-2**31, 2**31 - 1, (n_tot,), dtype=torch.int32, device="cuda",
                         generator=g)
    # merge requests need sorted runs: sort each of their runs in place first
    runs_of = {}
    rr = workloads.rng(seed + 1)
    for i in np.flatnonzero(ops == 1):
        n = int(sizes[i])
        k = int(rr.integers(1, 6))
        cuts = np.sort(rr.integers(0, n + 1, size=k - 1))
        ro = [0] + [int(c) for c in cuts] + [n]
        runs_of[i] = ro
        a = int(offs[i])
        for j in range(k):
            seg = keys[a + ro[j]:a + ro[j + 1]]
            if seg.numel():
                seg.copy_(torch.sort((seg.to(torch.int64) & 0xFFFFFFFF), stable=True).values
                          .to(torch.int64).to(torch.int32))
    vals = torch.arange(n_tot, dtype=torch.int32, device="cuda")
    # disjoint, 16-byte aligned slices: each request starts at the cumulative
    # sum of the previous sizes rounded up to 4 keys
    pad = np.concatenate([[0], np.cumsum((sizes + 3) // 4 * 4)]).astype(np.int64)
    kin = torch.zeros(int(pad[-1]) + int(sizes[-1]) + 8, dtype=torch.int32, device="cuda")
    vin = torch.zeros_like(kin)
    for i in range(len(sizes)):
        kin[pad[i]:pad[i] + sizes[i]] = keys[offs[i]:offs[i + 1]]
        vin[pad[i]:pad[i] + sizes[i]] = vals[offs[i]:offs[i + 1]]
    kout = torch.zeros_like(kin)
    vout = torch.zeros_like(vin)
    arena = torch.empty(arena_bytes, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    srv = serve.Server(arena, mode=mode, streams=4, small_max=1 << 14)

    def make(i):
        a, n = int(pad[i]), int(sizes[i])
        kw = dict(kt=0, n=n, keys_in=kin[a:].data_ptr(), keys_out=kout[a:].data_ptr())
        if pairs[i]:
            kw.update(vals_in=vin[a:].data_ptr(), vals_out=vout[a:].data_ptr())
        if ops[i] == 1:
            kw.update(op=1, run_offsets=runs_of[i])
        return kw

    res = serve.replay(srv, list(arrivals), make)
    torch.cuda.synchronize()
    srv.close()
    assert all(s == 0 for s in res["status"])
    return kin, vin, kout, vout, pad, res


def check_against_solo(bcf, kin, vin, kout, vout, pad, sizes, pairs, ops, oracle_every=7):
    for i in range(len(sizes)):
        a, n = int(pad[i]), int(sizes[i])
        ki = kin[a:a + n]
        ko = torch.empty_like(ki)
        if pairs[i]:
            vo = torch.empty_like(ki)
            bcf.bcf_sort_pairs(ko, vo, ki, vin[a:a + n].clone(), kt=0)
        else:
            bcf.bcf_sort_keys(ko, ki, kt=0)
        torch.cuda.synchronize()
        assert torch.equal(ko, kout[a:a + n]), f"request {i} keys differ from the solo sort"
        if pairs[i]:
            assert torch.equal(vo, vout[a:a + n]), f"request {i} values differ"
        if i % oracle_every == 0:
            kn = from_dev(ki, np.uint32)
            vn = from_dev(vin[a:a + n], np.uint32) if pairs[i] else None
            ek, ev = oracle.sort(kn, vn)
            assert np.array_equal(from_dev(kout[a:a + n], np.uint32), ek)
            if pairs[i]:
                assert np.array_equal(from_dev(vout[a:a + n], np.uint32), ev)


@pytest.mark.parametrize("mode", [0, 1])
def test_every_result_same_alone_and_in_the_mix(bcf, mode):
    sizes, pairs, ops, arrivals = make_mix(240, 51)
    out = run_mix(bcf, mode, 1 << 30, sizes, pairs, ops, arrivals)
    check_against_solo(bcf, *out[:5], sizes, pairs, ops)
    st = out[5]["stats"]
    if mode == 0:
        assert st["launched_batches"] > 0  # small requests were coalesced


def test_arena_pressure_defers_but_completes(bcf):
    sizes, pairs, ops, arrivals = make_mix(120, 52, hi=1 << 17)
    # room for about one large request at a time
    out = run_mix(bcf, 0, 24 << 20, sizes, pairs, ops, arrivals)
    check_against_solo(bcf, *out[:5], sizes, pairs, ops, oracle_every=11)
    assert out[5]["stats"]["arena_peak"] <= 24 << 20


def test_submit_errors(bcf):
    from paper_1306_5076_gb300 import serve

    arena = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    srv = serve.Server(arena)
    x = torch.zeros(1 << 20, dtype=torch.int32, device="cuda")
    with pytest.raises(bcf.BcfError) as ei:  # payload on one side only
        srv.submit(tag=0, kt=0, n=16, keys_in=x.data_ptr(), keys_out=x.data_ptr(),
                   vals_in=x.data_ptr())
    assert ei.value.status == 1
    with pytest.raises(bcf.BcfError) as ei:  # a large request that can never fit
        srv.submit(tag=1, kt=0, n=1 << 20, keys_in=x.data_ptr(), keys_out=x.data_ptr())
    assert ei.value.status == 2
    srv.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_mixed_key_types_and_directions(bcf, mode):
    """Requests of every key type and both directions, interleaved in one burst:
    batches are formed per (key type, direction, payload), and every result
    equals the oracle's."""
    from paper_1306_5076_gb300 import serve
    from tests.gpu_util import bits, kt_of, to_dev

    r = workloads.rng(53)
    count = 150
    kinds = list(workloads.DTYPES)
    reqs = []
    for i in range(count):
        dtype = kinds[int(r.integers(0, len(kinds)))]
        n = int(workloads.log_uniform_sizes(r, 1, 1, 1 << 15)[0])
        keys = workloads.keys("uniform" if i % 3 else "distinct16", dtype, n, seed=600 + i)
        vals = workloads.row_index(n) if r.random() < 0.4 else None
        desc = bool(r.random() < 0.5)
        kd = to_dev(keys)
        vd = None if vals is None else to_dev(vals)
        reqs.append(dict(keys=keys, vals=vals, desc=desc, kd=kd, vd=vd,
                         ko=torch.empty_like(kd), vo=None if vd is None else torch.empty_like(vd)))
    arena = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    srv = serve.Server(arena, mode=mode, streams=4, small_max=1 << 14)

    def make(i):
        q = reqs[i]
        kw = dict(kt=kt_of(q["keys"]), n=q["keys"].size, keys_in=q["kd"].data_ptr(),
                  keys_out=q["ko"].data_ptr(), descending=q["desc"])
        if q["vd"] is not None:
            kw.update(vals_in=q["vd"].data_ptr(), vals_out=q["vo"].data_ptr())
        return kw

    res = serve.replay(srv, [0.0] * count, make)
    torch.cuda.synchronize()
    srv.close()
    assert all(s == 0 for s in res["status"])
    for i, q in enumerate(reqs):
        ek, ev = oracle.sort(q["keys"], q["vals"], descending=q["desc"])
        gk = from_dev(q["ko"], q["keys"].dtype)
        assert np.array_equal(bits(gk), bits(ek)), f"request {i} ({q['keys'].dtype}) keys differ"
        if ev is not None:
            assert np.array_equal(from_dev(q["vo"], np.uint32), ev), f"request {i} values differ"
