"""The server's device-arena allocator (bcf_arena_*) against a plain Python
model of first fit with a coalescing free list (CPU only: host bookkeeping,
no device memory)."""
from __future__ import annotations

import numpy as np

from paper_1306_5076_gb300 import build


def aligned(x):
    return (max(x, 1) + 255) // 256 * 256


class Model:
    def __init__(self, nbytes):
        self.free = [(0, nbytes // 256 * 256)]  # sorted (offset, size)
        self.used = 0

    def alloc(self, sz):
        sz = aligned(sz)
        for i, (o, s) in enumerate(self.free):
            if s >= sz:
                if s == sz:
                    self.free.pop(i)
                else:
                    self.free[i] = (o + sz, s - sz)
                self.used += sz
                return o
        return None

    def release(self, off, sz):
        sz = aligned(sz)
        self.used -= sz
        self.free.append((off, sz))
        self.free.sort()
        merged = []
        for o, s in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + s)
            else:
                merged.append((o, s))
        self.free = merged

    def largest(self):
        return max((s for _, s in self.free), default=0)


def test_arena_matches_first_fit_model():
    build.build()
    from paper_1306_5076_gb300.serve import Arena

    r = np.random.default_rng(3)
    total = 1 << 24
    a, m = Arena(total), Model(total)
    live = []
    for step in range(4000):
        if live and (r.random() < 0.45 or len(live) > 200):
            j = int(r.integers(len(live)))
            off, sz = live.pop(j)
            a.free(off, sz)
            m.release(off, sz)
        else:
            sz = int(r.integers(1, 1 << 18))
            got, exp = a.alloc(sz), m.alloc(sz)
            assert got == exp, (step, got, exp)
            if got is not None:
                live.append((got, sz))
        used, largest = a.usage()
        assert used == m.used and largest == m.largest()
    for off, sz in live:
        a.free(off, sz)
    assert a.usage() == (0, total)  # everything coalesced back into one block


def test_arena_exhaustion_and_exact_fit():
    build.build()
    from paper_1306_5076_gb300.serve import Arena

    a = Arena(4096)
    offs = [a.alloc(1024) for _ in range(4)]
    assert offs == [0, 1024, 2048, 3072]
    assert a.alloc(1) is None
    a.free(1024, 1024)
    a.free(2048, 1024)
    assert a.usage() == (2048, 2048)
    assert a.alloc(2048) == 1024


def test_arena_refuses_double_free_and_wrong_ranges():
    build.build()
    from paper_1306_5076_gb300 import _native

    lib = _native.load()
    import ctypes

    h = ctypes.c_void_p()
    assert lib.bcf_arena_create(1 << 20, ctypes.byref(h)) == 0
    off = ctypes.c_uint64()
    assert lib.bcf_arena_alloc(h, 1000, ctypes.byref(off)) == 0
    first = off.value
    assert lib.bcf_arena_alloc(h, 5000, ctypes.byref(off)) == 0
    second = off.value
    used, largest = ctypes.c_uint64(), ctypes.c_uint64()
    assert lib.bcf_arena_usage(h, ctypes.byref(used), ctypes.byref(largest)) == 0
    before = (used.value, largest.value)
    assert lib.bcf_arena_free(h, first + 256, 1000) == 1  # not the start of an allocation
    assert lib.bcf_arena_free(h, first, 4096) == 1  # wrong size
    assert lib.bcf_arena_free(h, (1 << 20) - 256, 256) == 1  # a free range
    assert lib.bcf_arena_usage(h, ctypes.byref(used), ctypes.byref(largest)) == 0
    assert (used.value, largest.value) == before  # nothing changed
    assert lib.bcf_arena_free(h, first, 1000) == 0
    assert lib.bcf_arena_free(h, first, 1000) == 1  # double free
    assert lib.bcf_arena_free(h, second, 5000) == 0
    assert lib.bcf_arena_usage(h, ctypes.byref(used), ctypes.byref(largest)) == 0
    assert (used.value, largest.value) == (0, 1 << 20)
    assert lib.bcf_arena_destroy(h) == 0
