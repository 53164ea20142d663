"""Parity of the GPU colored prefix sums (through the C ABI) with the CPU
oracle -- bit-exact (integer sums modulo 2^32).

Sizes span one and many tiles with ragged tails; 1 to 64 colors; both
shared-memory layouts (conflict-free and the conflicting baseline); inclusive
and exclusive; uniform, skewed and run-structured colors; in place; pointers
16 but not 32 bytes aligned; invalid colors; host-side argument errors; and the
full benchmark size.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads

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


def dev_u32(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to("cuda")


def dev_u8(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint8)).to("cuda")


def host_u32(t):
    return t.cpu().numpy().view(np.uint32)


def gpu_cps(bcf, values, colors, d, exclusive=False, layout=0, inplace=False):
    vd, cd = dev_u32(values), dev_u8(colors)
    out = vd if inplace else torch.empty_like(vd)
    bcf.bcf_colored_prefix_sums(out, vd, cd, d, exclusive=exclusive, layout=layout)
    torch.cuda.synchronize()
    return host_u32(out)


def check(bcf, values, colors, d, exclusive=False, layout=0, inplace=False):
    exp = oracle.colored_prefix_sums(values, colors, d, exclusive=exclusive)
    got = gpu_cps(bcf, values, colors, d, exclusive, layout, inplace)
    bad = np.flatnonzero(got != exp)
    assert bad.size == 0, f"{bad.size} outputs differ, first {bad[:6]}: {got[bad[:3]]} vs {exp[bad[:3]]}"
    assert bcf.bcf_last_device_error() == 0


SIZES = [1, 15, 16, 17, 63, 64, 65, 4097, 16383, 16384, 16385, 3 * 16384 + 5, (1 << 20) + 3]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("d", [1, 3, 16, 33, 64])
@pytest.mark.parametrize("layout", [0, 1])
def test_sizes_colors_layouts(bcf, n, d, layout):
    values, colors = workloads.colored_elements(n, d, seed=n + d)
    for excl in (False, True):
        check(bcf, values, colors, d, excl, layout)


@pytest.mark.parametrize("law", ["uniform", "skewed", "runs"])
@pytest.mark.parametrize("d", [2, 16, 32])
def test_color_laws(bcf, law, d):
    values, colors = workloads.colored_elements((1 << 21) + 77, d, seed=7, law=law)
    for layout in (0, 1):
        check(bcf, values, colors, d, False, layout)


def test_one_color_long_carry_chain(bcf):
    """d = 1 and all values 1: out[i] = i + 1 across ~256 tiles (every tile
    depends on the look-back through all its predecessors)."""
    n = (1 << 22) + 9
    values = np.ones(n, np.uint32)
    colors = np.zeros(n, np.uint8)
    got = gpu_cps(bcf, values, colors, 1)
    assert np.array_equal(got, np.arange(1, n + 1, dtype=np.uint32))


def test_in_place(bcf):
    values, colors = workloads.colored_elements(100_003, 16, seed=8)
    check(bcf, values, colors, 16, False, 0, inplace=True)
    check(bcf, values, colors, 16, True, 1, inplace=True)


def test_pointers_16_but_not_32_byte_aligned(bcf):
    n = 3 * 16384 + 40
    values, colors = workloads.colored_elements(n, 8, seed=9)
    vbuf = torch.zeros(n + 8, dtype=torch.int32, device="cuda")
    obuf = torch.zeros(n + 8, dtype=torch.int32, device="cuda")
    cbuf = torch.zeros(n + 32, dtype=torch.uint8, device="cuda")
    vbuf[4:4 + n] = dev_u32(values)
    cbuf[16:16 + n] = dev_u8(colors)
    vd, od, cd = vbuf[4:4 + n], obuf[4:4 + n], cbuf[16:16 + n]
    assert vd.data_ptr() % 32 == 16 and od.data_ptr() % 32 == 16
    bcf.bcf_colored_prefix_sums(od, vd, cd, 8)
    torch.cuda.synchronize()
    assert np.array_equal(host_u32(od), oracle.colored_prefix_sums(values, colors, 8))
    assert not obuf[:4].any() and not obuf[4 + n:].any()


def test_invalid_color_is_reported(bcf):
    n = 10_000
    values, colors = workloads.colored_elements(n, 4, seed=10)
    colors[[5, 4097, 9999]] = 4  # >= d
    # (n spans the first tile's steps and threads)
    got = gpu_cps(bcf, values, colors, 4)
    assert bcf.bcf_last_device_error() == 1  # BCF_EINVAL
    assert bcf.bcf_last_device_error() == 0  # cleared
    bad = colors >= 4
    v2, c2 = values.copy(), colors.copy()
    v2[bad] = 0
    c2[bad] = 0
    exp = oracle.colored_prefix_sums(v2, c2, 4)
    exp[bad] = 0
    assert np.array_equal(got, exp)


def test_host_side_errors(bcf):
    v = torch.zeros(64, dtype=torch.int32, device="cuda")
    c = torch.zeros(64, dtype=torch.uint8, device="cuda")
    o = torch.zeros_like(v)
    for d in (0, 65):
        with pytest.raises(bcf.BcfError) as ei:
            bcf.bcf_colored_prefix_sums(o, v, c, d)
        assert ei.value.status == 1
    with pytest.raises(bcf.BcfError) as ei:  # misaligned values
        bcf.bcf_colored_prefix_sums(o[:60], v[1:61], c[:60], 4)
    assert ei.value.status == 1
    with pytest.raises(bcf.BcfError) as ei:  # workspace too small
        bcf.bcf_colored_prefix_sums(o, v, c, 4, ws=torch.zeros(16, dtype=torch.uint8,
                                                               device="cuda"))
    assert ei.value.status == 2
    # n == 0 is a no-op
    bcf.bcf_colored_prefix_sums(o[:0], v[:0], c[:0], 4)
    assert bcf.bcf_last_device_error() == 0


def test_full_size_bench_config_against_oracle(bcf):
    """The benchmark's workload (2^29 elements, 16 colors, uniform), both
    layouts, compared with the oracle on every element."""
    n = 1 << 29
    values, colors = workloads.colored_elements(n, 16, seed=29)
    exp = oracle.colored_prefix_sums(values, colors, 16)
    vd, cd = dev_u32(values), dev_u8(colors)
    out = torch.empty_like(vd)
    for layout in (0, 1):
        out.zero_()
        bcf.bcf_colored_prefix_sums(out, vd, cd, 16, layout=layout)
        torch.cuda.synchronize()
        assert np.array_equal(host_u32(out), exp)
