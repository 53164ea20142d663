"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module generates INPUTS only.  It holds none of the sorting method's
arithmetic: no comparison, no key transform, no sort.  Sorted inputs are built
from cumulative exponential spacings (the order statistics of n uniforms are
the normalised partial sums of n+1 exponentials), so they are non-decreasing
by construction.

Distributions follow the paper's data sets (Sec. 4: random keys in
[0, 10^6], distinct = a shuffle of 1..n, 0-1, and defined duplicates = k copies
of n/k keys) plus the large-sort workload family: uniform, Gaussian, sorted,
reverse sorted, 16 distinct values and Zipf(1.1) over 2^20 symbols, for u32,
u64 and f32 keys and the signed / double extension types i32, i64 and f64.  Payloads are the u32 row index.  Every generator takes an
explicit seed; the recipe of each is stated in its docstring.
"""
from __future__ import annotations

import math

import numpy as np

DTYPES = {"u32": np.uint32, "u64": np.uint64, "f32": np.float32, "i32": np.int32,
          "i64": np.int64, "f64": np.float64, "u16": np.uint16, "i16": np.int16}
DISTRIBUTIONS = ("uniform", "gaussian", "sorted", "reverse", "distinct16", "zipf")
PAPER_SETS = ("random1e6", "distinct", "zero_one", "dup2", "dup16", "dup2250")

_GOLDEN32 = 0x9E3779B1
_GOLDEN64 = 0x9E3779B97F4A7C15


def rng(seed: int) -> np.random.Generator:
    """PCG64 generator for ``seed``."""
    return np.random.default_rng(seed)


def large_sort_seed(dist: str, dtype: str, n: int) -> int:
    """Seed of the large-sort workload: 1000*dist_id + 10*dtype_id + log2(n)."""
    dist_id = DISTRIBUTIONS.index(dist)
    dtype_id = list(DTYPES).index(dtype)
    return 1000 * dist_id + 10 * dtype_id + int(round(math.log2(max(n, 1))))


def _uniform_bits(g, n, dtype):
    """Uniform random bit patterns of the key width, viewed as ``dtype``."""
    if DTYPES[dtype]().itemsize == 2:
        u = g.integers(0, 2**16, size=n, dtype=np.uint64).astype(np.uint16)
        return u.view(DTYPES[dtype])
    if DTYPES[dtype]().itemsize == 8:
        u = g.integers(0, 2**64, size=n, dtype=np.uint64, endpoint=False)
        return u.view(DTYPES[dtype])
    u = g.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
    return u.view(DTYPES[dtype])


def _from_u32(u: np.ndarray, dtype: str) -> np.ndarray:
    """u32 workload values carried to ``dtype`` by a monotone map: u64 widens,
    f32 rounds to float32, i32 / i64 / f64 subtract 2^31 (so half the values are
    negative), u16 keeps the top 16 bits and i16 those minus 2^15."""
    if dtype == "u32":
        return u
    if dtype in ("u16", "i16"):
        h = (u >> np.uint32(16)).astype(np.uint16)
        return h if dtype == "u16" else (h ^ np.uint16(0x8000)).view(np.int16)
    if dtype == "u64":
        return u.astype(np.uint64)
    if dtype == "f32":
        return u.astype(np.float32)
    s = u.astype(np.int64) - (1 << 31)
    return s.astype(DTYPES[dtype])


def sorted_uniform_u64(g, n: int, hi: float) -> np.ndarray:
    """n non-decreasing integers distributed as sorted uniforms on [0, hi).

    Built from exponential spacings: S_i = E_1 + ... + E_i, U_(i) = S_i / S_{n+1}.
    """
    if n == 0:
        return np.zeros(0, dtype=np.uint64)
    e = g.exponential(1.0, size=n + 1)
    s = np.cumsum(e)
    u = s[:-1] / s[-1]
    x = np.floor(u * hi)
    x = np.minimum(x, np.nextafter(hi, 0))
    # float64 keeps the sequence monotone; the conversion is exact below 2^53
    # and monotone (round-toward-zero of a monotone sequence) above.
    out = x.astype(np.uint64)
    return np.maximum.accumulate(out)


def sorted_keys(g, n: int, dtype: str) -> np.ndarray:
    """Non-decreasing keys of ``dtype``: u64 sorted over [0, 2^64), i64 the same
    values with the top bit flipped (x - 2^63); the other types are the sorted
    u32 values carried over by :func:`_from_u32`."""
    if dtype in ("u64", "i64"):
        u = sorted_uniform_u64(g, n, 2.0**64)
        return u if dtype == "u64" else (u ^ np.uint64(1 << 63)).view(np.int64)
    u = sorted_uniform_u64(g, n, 2.0**32).astype(np.uint32)
    return _from_u32(u, dtype)


def gaussian_u32(g, n: int) -> np.ndarray:
    """rint(N(2^31, 2^28)) clamped to [0, 2^32 - 1]."""
    x = np.rint(g.normal(2.0**31, 2.0**28, size=n))
    return np.clip(x, 0, 2.0**32 - 1).astype(np.uint64).astype(np.uint32)


def zipf_ranks(g, n: int, s: float = 1.1, symbols: int = 1 << 20) -> np.ndarray:
    """Ranks r in [1, symbols] with P(r) proportional to r^-s (inverse CDF)."""
    w = np.arange(1, symbols + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = g.random(n)
    return np.minimum(np.searchsorted(cdf, u, side="left"), symbols - 1).astype(np.uint64) + 1


def keys(dist: str, dtype: str, n: int, seed: int | None = None) -> np.ndarray:
    """Keys of the large-sort workload family (``dist`` in DISTRIBUTIONS).

    uniform   : uniform random bit patterns of the key width (u32 / u64 /
                i32 / i64 over their full range; f32 / f64 with NaNs,
                infinities, subnormals and both zeros included, to exercise
                the total order).
    gaussian  : u32 = rint(N(2^31, 2^28)) clamped; u64 = the same values
                widened; f32 = float32 of the same values (many ties); i32 /
                i64 / f64 = the same values minus 2^31.
    sorted    : non-decreasing by construction (exponential spacings).
    (u16 / i16 carry the u32 values over by their top 16 bits, the gaussian
    and sorted laws included.)
    reverse   : ``sorted`` read backwards.
    distinct16: 16 values drawn from the uniform law, each element picks one.
    zipf      : rank r ~ Zipf(1.1) over 2^20 symbols, key = (r-1)*golden mod
                2^64 (u64; its bits for i64) or mod 2^32 (u32; f32 = float32
                of it; i32 = its bits; f64 = its value minus 2^31; u16 / i16 =
                its low 16 bits).
    """
    if seed is None:
        seed = large_sort_seed(dist, dtype, n)
    g = rng(seed)
    if dist == "uniform":
        return _uniform_bits(g, n, dtype)
    if dist == "gaussian":
        return _from_u32(gaussian_u32(g, n), dtype)
    if dist == "sorted":
        return sorted_keys(g, n, dtype)
    if dist == "reverse":
        return np.ascontiguousarray(sorted_keys(g, n, dtype)[::-1])
    if dist == "distinct16":
        pool = _uniform_bits(g, 16, dtype)
        return pool[g.integers(0, 16, size=n)]
    if dist == "zipf":
        r = zipf_ranks(g, n) - 1
        if dtype in ("u64", "i64"):
            return (r * np.uint64(_GOLDEN64)).view(DTYPES[dtype])  # wraps mod 2^64
        u = ((r * np.uint64(_GOLDEN32)) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
        if dtype in ("u16", "i16"):  # the low 16 bits: the symbol's identity mod 2^16
            return (u & np.uint32(0xFFFF)).astype(np.uint16).view(DTYPES[dtype])
        return u.view(np.int32) if dtype == "i32" else _from_u32(u, dtype)
    raise ValueError(f"unknown distribution {dist!r}")


def paper_keys(name: str, n: int, seed: int = 7) -> np.ndarray:
    """The paper's correctness data sets (Sec. 4), as u32 keys.

    random1e6: uniform in [0, 10^6]; distinct: a shuffle of 1..n; zero_one:
    uniform 0/1; dupK: K copies of each of n/K distinct keys, shuffled.
    """
    g = rng(seed)
    if name == "random1e6":
        return g.integers(0, 10**6 + 1, size=n).astype(np.uint32)
    if name == "distinct":
        return g.permutation(np.arange(1, n + 1, dtype=np.uint32))
    if name == "zero_one":
        return g.integers(0, 2, size=n).astype(np.uint32)
    if name.startswith("dup"):
        k = int(name[3:])
        distinct = max(1, -(-n // k))  # ceil(n / k); the last key may have fewer copies
        # distinct by construction: an odd multiplier is a bijection mod 2^32
        off = np.uint64(g.integers(0, 2**32))
        base = ((np.arange(distinct, dtype=np.uint64) * np.uint64(_GOLDEN32) + off)
                & np.uint64(0xFFFFFFFF)).astype(np.uint32)
        return g.permutation(np.repeat(base, k)[:n])
    raise ValueError(f"unknown paper data set {name!r}")


def row_index(n: int) -> np.ndarray:
    """Payload v[i] = i (u32)."""
    return np.arange(n, dtype=np.uint32)


def log_uniform_sizes(g, count: int, lo: float, hi: float) -> np.ndarray:
    """floor(exp(U(ln lo, ln(hi + 1)))) clamped to [lo, hi]."""
    x = np.floor(np.exp(g.uniform(math.log(lo), math.log(hi + 1), size=count)))
    return np.clip(x, lo, hi).astype(np.int64)


def run_lengths(k: int, total: int, seed: int | None = None,
                lo: int = 1 << 10, hi: int = 1 << 24) -> np.ndarray:
    """k run lengths drawn log-uniform in [lo, hi], rescaled to sum to ``total``.

    Rescaling uses cumulative rounding (lengths are the differences of the
    rounded partial sums of the scaled draws), so the lengths sum to ``total``
    exactly; every length is >= lo when k * lo <= total, else >= 1.  (For k = 2
    and 16 a total of 2^27 forces lengths above 2^24; that is unavoidable and
    reported by callers.)
    """
    if seed is None:
        seed = 3000 + k
    g = rng(seed)
    w = np.exp(g.uniform(math.log(lo), math.log(hi), size=k))
    floor_min = lo if k * lo <= total else 1
    spare = total - k * floor_min
    bounds = np.rint(np.cumsum(w) / w.sum() * spare).astype(np.int64)
    bounds[-1] = spare
    lens = np.diff(np.concatenate([[0], bounds]))
    return lens + floor_min


def sorted_runs(k: int, total: int, dtype: str = "u32", seed: int | None = None):
    """k sorted runs (lengths from :func:`run_lengths`) concatenated.

    Returns ``(keys, offsets)`` with offsets of length k+1.
    """
    if seed is None:
        seed = 3000 + k
    lens = run_lengths(k, total, seed)
    g = rng(seed + 1)
    parts = [sorted_keys(g, int(m), dtype) for m in lens]
    offs = np.zeros(k + 1, dtype=np.uint64)
    offs[1:] = np.cumsum(lens)
    return np.concatenate(parts) if parts else np.zeros(0, DTYPES[dtype]), offs


def segment_sizes(count: int = 100_000, hi: int = 1 << 18, seed: int = 4000) -> np.ndarray:
    """Segment sizes clamp(floor(exp(U(ln 1, ln(hi + 1)))), 1, hi)."""
    return log_uniform_sizes(rng(seed), count, 1, hi)


def segments(count: int, hi: int, dtype: str = "u32", seed: int = 4000):
    """Uniform keys in ``count`` segments of log-uniform size in [1, hi].

    Returns ``(keys, offsets)``.
    """
    sizes = segment_sizes(count, hi, seed)
    offs = np.zeros(count + 1, dtype=np.uint64)
    offs[1:] = np.cumsum(sizes)
    return _uniform_bits(rng(seed + 1), int(offs[-1]), dtype), offs


def request_trace(rate_hz: float = 2000.0, duration_s: float = 10.0, lo: int = 1 << 8,
                  hi: int = 1 << 24, pairs_fraction: float = 0.3, seed: int = 5000):
    """Open-loop request trace: Poisson arrivals, log-uniform sizes, 30 % pairs.

    Returns a dict of numpy arrays: ``t`` (arrival seconds), ``n`` (keys),
    ``pairs`` (bool).
    """
    g = rng(seed)
    gaps = g.exponential(1.0 / rate_hz, size=int(rate_hz * duration_s * 1.5) + 16)
    t = np.cumsum(gaps)
    t = t[t < duration_s]
    n = log_uniform_sizes(g, t.size, lo, hi)
    pairs = g.random(t.size) < pairs_fraction
    return {"t": t, "n": n, "pairs": pairs}


def colored_elements(n: int, d: int, seed: int = 6000, law: str = "uniform"):
    """Inputs of the colored prefix sums (Appendix A): ``values`` uniform u32
    over the full range (so sums wrap modulo 2^32) and ``colors`` u8 in [0, d).

    law "uniform": every color equally likely; "skewed": color c drawn with
    probability proportional to 2^-c (a few colors dominate); "runs": runs of
    one color with geometric lengths (mean 64).
    """
    g = rng(seed)
    values = g.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
    if law == "uniform":
        colors = g.integers(0, d, size=n)
    elif law == "skewed":
        p = 2.0 ** -np.arange(d)
        colors = g.choice(d, size=n, p=p / p.sum())
    elif law == "runs":
        lens = g.geometric(1.0 / 64, size=n // 8 + 2)
        cols = g.integers(0, d, size=lens.size)
        colors = np.repeat(cols, lens)[:n]
        if colors.size < n:
            colors = np.concatenate([colors, np.zeros(n - colors.size, np.int64)])
    else:
        raise ValueError(f"unknown color law {law!r}")
    return values, colors.astype(np.uint8)
