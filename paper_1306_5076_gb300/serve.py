"""Python side of the continuous-batching request server (C ABI: bcf_server_*).

``Server`` wraps the C server (argument marshalling only; admission, batching,
launching and completion tracking run in the C++ library).  ``Arena`` wraps
the library's first-fit allocator (host bookkeeping over a range).
``replay`` drives a server open-loop over a request trace: request i is
submitted once the server clock passes its scheduled arrival, the server is
stepped continuously, and latency is measured from the scheduled arrival to
the completion the server observed -- so waiting for admission, queueing and
batching all count.
"""
from __future__ import annotations

import ctypes
import statistics

from . import BcfError, _native

BCF_SERVE_BATCHED = _native.BCF_SERVE_BATCHED
BCF_SERVE_PLAIN = _native.BCF_SERVE_PLAIN


def _check(st, what):
    if st != 0:
        raise BcfError(st, what)


class Arena:
    """First-fit allocator over [0, bytes) (bcf_arena_*)."""

    def __init__(self, nbytes: int):
        self._lib = _native.load()
        self._h = ctypes.c_void_p()
        _check(self._lib.bcf_arena_create(nbytes, ctypes.byref(self._h)), "bcf_arena_create")

    def alloc(self, nbytes: int):
        off = ctypes.c_uint64()
        st = self._lib.bcf_arena_alloc(self._h, nbytes, ctypes.byref(off))
        return None if st != 0 else off.value

    def free(self, off: int, nbytes: int):
        _check(self._lib.bcf_arena_free(self._h, off, nbytes), "bcf_arena_free")

    def usage(self):
        used, largest = ctypes.c_uint64(), ctypes.c_uint64()
        _check(self._lib.bcf_arena_usage(self._h, ctypes.byref(used), ctypes.byref(largest)),
               "bcf_arena_usage")
        return used.value, largest.value

    def close(self):
        if self._h:
            self._lib.bcf_arena_destroy(self._h)
            self._h = ctypes.c_void_p()

    __del__ = close


class Server:
    """bcf_server_* over a caller-owned device arena (a CUDA uint8 tensor)."""

    def __init__(self, arena_tensor, mode=BCF_SERVE_BATCHED, streams=4, small_max=1 << 16,
                 batch_max_keys=1 << 22):
        self._lib = _native.load()
        self._arena = arena_tensor  # keep alive
        cfg = _native.BcfServerConfig(ctypes.c_void_p(arena_tensor.data_ptr()),
                                      arena_tensor.numel(), streams, mode, small_max,
                                      batch_max_keys)
        self._h = ctypes.c_void_p()
        _check(self._lib.bcf_server_create(ctypes.byref(cfg), ctypes.byref(self._h)),
               "bcf_server_create")
        self._keep = {}  # run-offset arrays of merge requests until completion
        self._buf = (_native.BcfCompletion * 4096)()

    def now(self) -> float:
        return self._lib.bcf_server_now(self._h)

    def submit(self, *, tag, kt, n, keys_in, keys_out, vals_in=None, vals_out=None,
               descending=False, op=0, run_offsets=None):
        """Queue one request; pointers are raw device addresses (ints)."""
        r = _native.BcfRequest()
        r.op, r.kt, r.descending, r.n = op, kt, int(descending), n
        r.keys_in, r.keys_out = keys_in, keys_out
        r.vals_in, r.vals_out = vals_in, vals_out
        r.tag = tag
        if run_offsets is not None:
            arr = (ctypes.c_uint64 * len(run_offsets))(*run_offsets)
            self._keep[tag] = arr
            r.run_offsets = ctypes.cast(arr, ctypes.c_void_p)
            r.k = len(run_offsets) - 1
        _check(self._lib.bcf_server_submit(self._h, ctypes.byref(r)), "bcf_server_submit")

    def step(self) -> int:
        inflight = ctypes.c_int()
        _check(self._lib.bcf_server_step(self._h, ctypes.byref(inflight)), "bcf_server_step")
        return inflight.value

    def poll(self):
        n = self._lib.bcf_server_poll(self._h, self._buf, len(self._buf))
        out = []
        for i in range(n):
            c = self._buf[i]
            self._keep.pop(c.tag, None)
            out.append((c.tag, c.status, c.submit_s, c.admit_s, c.done_s))
        return out

    def stats(self) -> dict:
        s = _native.BcfServerStats()
        _check(self._lib.bcf_server_stats(self._h, ctypes.byref(s)), "bcf_server_stats")
        return {f: getattr(s, f) for f, _ in s._fields_}

    def drain(self):
        _check(self._lib.bcf_server_drain(self._h), "bcf_server_drain")

    def close(self):
        if self._h:
            self._lib.bcf_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    __del__ = close


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[k]


def replay(server: Server, arrivals, make_request, release=None, max_wait_s=600.0):
    """Open-loop replay.  ``arrivals[i]`` is request i's arrival (seconds from
    the start); ``make_request(i)`` returns the submit() kwargs (or None to
    retry later, e.g. while its output buffer space is taken);
    ``release(i)`` is called when request i completed.  Returns a dict with
    per-request latencies (arrival -> completion), p50/p99 and the span."""
    n = len(arrivals)
    t0 = server.now()
    i = 0
    lat = [None] * n
    status = [None] * n
    done = 0
    last_done = t0
    while done < n:
        now = server.now() - t0
        while i < n and arrivals[i] <= now:
            kw = make_request(i)
            if kw is None:
                break
            server.submit(tag=i, **kw)
            i += 1
        server.step()
        for tag, st, _sub, _adm, dn in server.poll():
            lat[tag] = dn - (t0 + arrivals[tag])
            status[tag] = st
            last_done = max(last_done, dn)
            done += 1
            if release is not None:
                release(tag)
        if now > arrivals[-1] + max_wait_s:
            raise TimeoutError("replay did not finish")
    span = last_done - (t0 + arrivals[0])
    return {"latency_s": lat, "status": status, "p50_s": percentile(lat, 50),
            "p99_s": percentile(lat, 99), "mean_s": statistics.mean(lat), "span_s": span,
            "stats": server.stats()}
