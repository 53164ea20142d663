"""Benchmark: GB300 bank-conflict-free merge sort, one JSON line on rank 0.

Workload (one "step" = one full sort through the C ABI): 2^28 uint32 keys,
uniform over [0, 2^32), seed 28 (the large-sort workload family's seed rule,
1000 * distribution + 10 * key type + log2 n),
ascending, keys only -- the configuration the >= 60 %-of-HBM-roofline-per-merge-
pass target is stated on.  Inputs are resident in HBM before the timed region;
1 GiB of keys is far larger than the 129 MB L2, so no flush is needed between
steps.

  value        keys sorted per second, whole job (all ranks)
  roofline     the merge-pass kernel: algorithmic bytes per launch (one read
               and one write of every key) / its mean CUDA-event duration,
               against the measured HBM copy bandwidth
  e2e          the same sort from pinned HOST memory: H2D copy, sort, D2H copy
               timed per step
  cpu_baseline the CPU oracle (test infrastructure) on a bounded sample, all
               host cores
Multi-GPU: each rank sorts its own 2^28 keys (independent replicas; sorting
does not shard without an exchange step, which this library does not have).

--impl reference times the oracle itself on the host cores (bounded sample per
step) and prints the same line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "keys/s & % HBM roofline per pass (bit-exact); served vs plain p99 latency on one GB300"
LOG2N = 28
N = 1 << LOG2N  # the benchmark workload; --log2n shrinks it for profiling captures only
SAMPLE_LOG2N = 24  # oracle sample (CPU legs)
KEY_BYTES = 4


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def source_digest(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


MERGE_SOURCES = ["paper_1306_5076_gb300/csrc/bcf_merge.cu",
                 "paper_1306_5076_gb300/csrc/bcf_merge.cuh",
                 "paper_1306_5076_gb300/csrc/bcf_device.cuh",
                 "paper_1306_5076_gb300/csrc/bcf_internal.h"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "merge_kernel_u32_traffic.json.txt")


def merge_traffic_per_launch():
    """DRAM bytes of one full-size merge launch from the committed ncu summary,
    or None if the kernel sources changed since it was taken."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.loads(f.read())
    except Exception:
        return None
    if rec.get("source_digest") != source_digest(MERGE_SOURCES):
        return None
    return rec.get("bytes_per_full_launch")


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        """Start sampling every 50 ms; returns once the first sample arrived."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        t0 = time.time()
        while not self.lines and time.time() - t0 < 5:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def mark(self):
        """Index of the next sample: brackets the timed region."""
        return len(self.lines)

    def stop(self, first=0, last=None):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        window = self.lines[first:last] or self.lines[-1:]
        for ln in window:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist

        backend = "gloo" if args.impl == "reference" else "nccl"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def per_pass_ms(launch_list):
    """Each pass of the sort on its own, averaged over the timed steps: the
    launches of one step are a block sort, then a partition and a merge per
    merge pass (launch order, as the library records them)."""
    steps, cur = [], None
    for kind, ms in launch_list:
        if kind == "block_sort":
            cur = {"block_sort": ms, "partition": [], "merge": []}
            steps.append(cur)
        elif cur is not None and kind in ("partition", "merge"):
            cur[kind].append(ms)
    if not steps:
        return None
    n = min(len(s["merge"]) for s in steps)
    mean = lambda xs: sum(xs) / len(xs)  # noqa: E731
    return {"block_sort": mean([s["block_sort"] for s in steps]),
            "partition": [mean([s["partition"][i] for s in steps]) for i in range(n)],
            "merge": [mean([s["merge"][i] for s in steps]) for i in range(n)],
            "steps": len(steps)}


def max_over_ranks(torch, pg, x, dev):
    """The largest of every rank's x (the job's time is its slowest rank's);
    x itself when there is no process group."""
    if pg is None:
        return x
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_keys_per_s(world, n_per_rank, ms):
    """Whole-job throughput: every rank sorts its own n_per_rank keys (weak
    scaling, replicas), the job takes the slowest rank's ms."""
    return world * n_per_rank / (ms * 1e-3)


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


SINGLE_LOG2N = 22  # oracle sample for the single-threaded timing


def oracle_keys_per_s(sample_log2n=SAMPLE_LOG2N, reps=1, threads=None):
    """The CPU oracle as it stands, on a sample of the workload: all host cores
    (threads None) or the given number of threads."""
    import numpy as np

    import oracle
    import workloads

    n = 1 << sample_log2n
    keys = workloads.keys("uniform", "u32", n, seed=workloads.large_sort_seed("uniform", "u32", N))
    cores = cpu_cores() if threads is None else threads
    oracle.sort(keys[: 1 << 12], nthreads=cores)  # load the library outside the timing
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.sort(keys, nthreads=cores)
        times.append(time.perf_counter() - t0)
    del np
    return n / statistics.median(times), cores, n, times


def oracle_table():
    """The CPU oracle as it stands on bounded samples of every workload, one
    host core and all host cores: context for the GPU numbers (keys/s)."""
    import numpy as np

    import oracle
    import workloads

    cores = cpu_cores()

    def rate(fn, n, reps=3):
        fn()  # load the library, touch the inputs
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t0)
        return n / statistics.median(ts)

    out = {"cores": cores, "cpu_model": host_cpu_model()}
    k = workloads.keys("uniform", "u32", 1 << 20, seed=0)
    out["C1 2^20 u32 uniform"] = {"one_core": rate(lambda: oracle.sort(k), k.size),
                                  "all_cores": rate(lambda: oracle.sort(k, nthreads=cores), k.size)}
    n1, na = 1 << 22, 1 << 24
    for key in ("u32", "f32", "u64"):
        for dist in (GRID_DISTS if key == "u32" else ("uniform",)):
            k1 = workloads.keys(dist, key, n1)
            ka = workloads.keys(dist, key, na)
            for pairs in (False, True):
                v1 = np.arange(n1, dtype=np.uint32) if pairs else None
                va = np.arange(na, dtype=np.uint32) if pairs else None
                out[f"C2 {key}{'+u32' if pairs else ''} {dist}"] = {
                    "one_core": rate(lambda: oracle.sort(k1, v1), n1, reps=1),
                    "all_cores": rate(lambda: oracle.sort(ka, va, nthreads=cores), na, reps=1)}
    for kr in (2, 16, 256):
        keys, offs = workloads.sorted_runs(kr, n1)
        out[f"C3 merge k={kr}"] = {
            "one_core": rate(lambda: oracle.merge_runs(keys, None, offs), n1, reps=1),
            # merge_runs is defined as the stable sort of the concatenated runs
            "all_cores": rate(lambda: oracle.sort(keys, nthreads=cores), n1, reps=1)}
    keys, offs = workloads.segments(500, 1 << 18, "u32", seed=4000)
    out["C4 segmented (500 segments of the law)"] = {
        "one_core": rate(lambda: oracle.segmented_sort(keys, None, offs), keys.size, reps=1),
        "all_cores": None}
    out["samples"] = ("C1: the 2^20-key input itself; C2: 2^22 keys (one core) and 2^24 keys "
                      "(all cores) per case; C3: 2^22 keys in k runs; C4: 500 segments "
                      f"({int(offs[-1])} keys) of the 100,000-segment law")
    return out


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    times = []
    n = 1 << SAMPLE_LOG2N
    for i in range(args.warmup + args.steps):
        kps, cores, n, t = oracle_keys_per_s()
        if i >= args.warmup:
            times.extend(t)
    mean_t = statistics.mean(times)
    value = n / mean_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "keys/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_t * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": f"sort of 2^{SAMPLE_LOG2N} uniform u32 keys (a bounded sample "
                               f"of the 2^{LOG2N}-key workload), keys only, ascending",
                   "n": n, "key": "u32", "parallelism": "host threads"},
        "cpu_baseline": {"value": value, "unit": "keys/s", "cores": cores, "kind": "oracle",
                         "sample": f"2^{SAMPLE_LOG2N} keys of the same workload per step "
                                   f"(stable merge sort, C, {cores} threads)"},
        "e2e": {"value": value, "unit": "keys/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def serving_bench(torch, dev, seconds, rate=2000.0, seed=5000):
    """Served (continuous batching) vs plain (one launch chain per request,
    FIFO) on the same open-loop Poisson trace: sizes log-uniform in
    [2^8, 2^24] u32 keys, 30 % with u32 payloads, arena 40 GB.  Inputs are
    slices of a pool resident in HBM outside the arena; outputs go to a pool
    managed with the library's allocator.  Latency = completion observed by
    the server - scheduled arrival."""
    import numpy as np

    import workloads
    from paper_1306_5076_gb300 import serve

    tr = workloads.request_trace(rate_hz=rate, duration_s=seconds, seed=seed)
    t, sizes, pairs = tr["t"], tr["n"], tr["pairs"]
    pool = 1 << 27
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    kin = torch.randint(-2**31, 2**31 - 1, (pool,), dtype=torch.int32, device=dev, generator=g)
    vin = torch.arange(pool, dtype=torch.int32, device=dev)
    out_keys = 1 << 28
    kout = torch.empty(out_keys, dtype=torch.int32, device=dev)
    vout = torch.empty(out_keys, dtype=torch.int32, device=dev)
    arena = torch.empty(40 << 30, dtype=torch.uint8, device=dev)
    kin_ptr, vin_ptr = kin.data_ptr(), vin.data_ptr()
    kout_ptr, vout_ptr = kout.data_ptr(), vout.data_ptr()
    # untimed warm-up trace: every size band, with and without payloads, so
    # that no kernel is loaded or launched for the first time inside the trace
    w_sizes = np.array([1 << b for b in range(8, 25, 2)] * 2)
    w_pairs = np.repeat([False, True], w_sizes.size // 2)
    w_t = np.arange(w_sizes.size) * 2e-3

    def replay(mode, ts, szs, prs):
        srv = serve.Server(arena, mode=mode, streams=4, small_max=1 << 16)
        outs = serve.Arena(out_keys * 4)
        held = {}

        def make(i):
            n = int(szs[i])
            off = outs.alloc(n * 4)
            if off is None:
                return None  # output pool full: the request waits (its latency counts)
            held[i] = off
            src = ((i * 2654435761) % (pool - n)) & ~3
            kw = dict(kt=0, n=n, keys_in=kin_ptr + 4 * src, keys_out=kout_ptr + off)
            if prs[i]:
                kw.update(vals_in=vin_ptr + 4 * src, vals_out=vout_ptr + off)
            return kw

        def release(i):
            outs.free(held.pop(i), int(szs[i]) * 4)

        # no garbage-collector pause inside the trace (the host loop is part
        # of every request's latency)
        gc.collect()
        gc.disable()
        try:
            r = serve.replay(srv, list(ts), make, release)
        finally:
            gc.enable()
        srv.close()
        outs.close()
        return r

    res = {}
    for name, mode in (("served", serve.BCF_SERVE_BATCHED), ("plain", serve.BCF_SERVE_PLAIN)):
        torch.cuda.synchronize()
        replay(mode, w_t, w_sizes, w_pairs)
        torch.cuda.synchronize()
        r = replay(mode, t, sizes, pairs)
        keys = float(sizes.sum())
        lat = r["latency_s"]
        worst = max(range(len(lat)), key=lambda i: lat[i])
        res[name] = {"p50_ms": r["p50_s"] * 1e3, "p99_ms": r["p99_s"] * 1e3,
                     "mean_ms": r["mean_s"] * 1e3, "max_ms": lat[worst] * 1e3,
                     "worst_arrival_s": float(t[worst]), "keys_per_s": keys / r["span_s"],
                     "span_s": r["span_s"], "launch_units": r["stats"]["launched_units"],
                     "coalesced_batches": r["stats"]["launched_batches"],
                     "arena_peak_gb": r["stats"]["arena_peak"] / 1e9,
                     "errors": int(sum(1 for x in r["status"] if x != 0))}
    del arena, kin, vin, kout, vout
    return {"trace": f"Poisson {rate:g} req/s for {seconds:g} s, {len(t)} requests, "
                     "sizes log-uniform [2^8, 2^24] u32, 30 % pairs, seed 5000",
            "offered_keys_per_s": float(sizes.sum()) / seconds, **res}


def timed_ms(torch, stream, fn, warmup=3, reps=10):
    """Mean CUDA-event time of fn() on `stream` (inputs larger than L2)."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def key_types_bench(torch, dev, bcf, peak, log2n=LOG2N):
    """Keys-only and pairs sorts of 2^log2n uniform keys of every key type:
    whole-sort time and the merge pass against the HBM roofline."""
    import numpy as np

    import workloads

    n = 1 << log2n
    stream = torch.cuda.current_stream(dev)
    out = {}
    codes = {"u32": bcf.BCF_U32, "i32": bcf.BCF_I32, "f32": bcf.BCF_F32, "u64": bcf.BCF_U64,
             "i64": bcf.BCF_I64, "f64": bcf.BCF_F64, "u16": bcf.BCF_U16, "i16": bcf.BCF_I16}
    for name, kt in codes.items():
        for pairs in (False, True):
            if pairs and name not in ("u32", "u64"):
                continue
            keys = workloads.keys("uniform", name, n)
            kb = keys.dtype.itemsize
            kd = torch.from_numpy(keys.view({2: np.int16, 4: np.int32, 8: np.int64}[kb])).to(dev)
            ko = torch.empty_like(kd)
            vd = torch.arange(n, dtype=torch.int32, device=dev) if pairs else None
            vo = torch.empty_like(vd) if pairs else None
            ws = torch.empty(bcf.bcf_workspace_bytes(bcf.BCF_OP_SORT, n, 0, kt, pairs),
                             dtype=torch.uint8, device=dev)
            if pairs:
                fn = lambda: bcf.bcf_sort_pairs(ko, vo, kd, vd, kt=kt, ws=ws, stream=stream)  # noqa: E731
            else:
                fn = lambda: bcf.bcf_sort_keys(ko, kd, kt=kt, ws=ws, stream=stream)  # noqa: E731
            fn()
            torch.cuda.synchronize()
            bcf.bcf_profile_collect()
            bcf.bcf_profile_enable(True)
            ms = timed_ms(torch, stream, fn, warmup=2, reps=5)
            bcf.bcf_profile_enable(False)
            prof = bcf.bcf_profile_collect()
            m = prof["merge"]
            merge_ms = m["total_ms"] / max(m["launches"], 1)
            plan = bcf.bcf_sort_plan(n, kt, pairs)
            gbs = plan["bytes_per_pass"] / (merge_ms * 1e-3) / 1e9
            out[name + ("+u32" if pairs else "")] = {
                "ms": ms, "keys_per_s": n / (ms * 1e-3), "merge_pass_ms": merge_ms,
                "merge_pass_gbs": gbs, "merge_pass_frac": gbs / peak,
                "block_sort_ms": prof["block_sort"]["total_ms"] / max(
                    prof["block_sort"]["launches"], 1),
                "merge_passes": plan["merge_passes"]}
            del kd, ko, vd, vo, ws
            torch.cuda.empty_cache()
    # u32 keys with 64-bit payloads (bcf_sort_pairs_wide: pairs sort + row gather)
    keys = workloads.keys("uniform", "u32", n)
    kd = torch.from_numpy(keys.view(np.int32)).to(dev)
    ko = torch.empty_like(kd)
    vd = torch.arange(n, dtype=torch.int64, device=dev)
    vo = torch.empty_like(vd)
    ws = torch.empty(bcf.bcf_workspace_bytes(bcf._native.BCF_OP_SORT_WIDE, n, 0, bcf.BCF_U32, 1),
                     dtype=torch.uint8, device=dev)
    ms = timed_ms(torch, stream, lambda: bcf.bcf_sort_pairs_wide(
        ko, vo, kd, vd, kt=bcf.BCF_U32, ws=ws, stream=stream), warmup=2, reps=5)
    out["u32+u64"] = {"ms": ms, "keys_per_s": n / (ms * 1e-3),
                      "how": "pairs sort with u32 row indices, then a gather of the 8-byte rows"}
    del kd, ko, vd, vo, ws
    torch.cuda.empty_cache()
    return {"n": n, "distribution": "uniform", "results": out}


def cps_bench(torch, dev, bcf, peak, log2n=29, colors=(1, 2, 4, 8, 16, 32, 64)):
    """Colored prefix sums (Appendix A, the paper's Fig. 2 experiment): time
    against the number of colors, conflict-free layout vs the row-per-thread
    layout.  Algorithmic bytes: 4 (value) + 1 (color) + 4 (output) per element."""
    import workloads

    n = 1 << log2n
    stream = torch.cuda.current_stream(dev)
    vals_np, _ = workloads.colored_elements(n, 1, seed=29)
    vd = torch.from_numpy(vals_np.view("int32")).to(dev)
    od = torch.empty_like(vd)
    ws = torch.empty(bcf.bcf_workspace_bytes(bcf.BCF_OP_CPS, n, max(colors), bcf.BCF_U32, 0),
                     dtype=torch.uint8, device=dev)
    res = {"banked": {}, "rows": {}}
    for d in colors:
        g = torch.Generator(device=dev)
        g.manual_seed(d)
        cd = torch.randint(0, d, (n,), dtype=torch.uint8, device=dev, generator=g)
        for name, layout in (("banked", bcf.BCF_CPS_BANKED), ("rows", bcf.BCF_CPS_ROWS)):
            ms = timed_ms(torch, stream, lambda: bcf.bcf_colored_prefix_sums(
                od, vd, cd, d, layout=layout, ws=ws, stream=stream))
            gbs = 9 * n / (ms * 1e-3) / 1e9
            res[name][str(d)] = {"ms": ms, "elements_per_s": n / (ms * 1e-3), "gbs": gbs,
                                 "frac": gbs / peak}
        del cd
    if bcf.bcf_last_device_error() != 0:
        raise RuntimeError("colored prefix sums: device error word set")
    return {"n": n, "values": "uniform u32", "colors": "uniform u8 in [0, d)",
            "bytes_per_element": 9, **res}


def pb_bench(torch, dev, bcf, log2n=LOG2N):
    """Pivot buckets (BCFMergesortPB) against the merge passes on the paper's
    duplicate-heavy inputs and on distinct keys, and the automatic choice
    between them: whole-sort time, 2^log2n u32 keys, keys only and pairs."""
    import numpy as np

    import workloads

    n = 1 << log2n
    stream = torch.cuda.current_stream(dev)
    out = {}
    for name in ("distinct16", "zipf", "zero_one", "dup16", "uniform"):
        keys = (workloads.paper_keys(name, n) if name in workloads.PAPER_SETS
                else workloads.keys(name, "u32", n))
        kd = torch.from_numpy(keys.view(np.int32)).to(dev)
        ko = torch.empty_like(kd)
        for pairs in (False, True):
            vd = torch.arange(n, dtype=torch.int32, device=dev) if pairs else None
            vo = torch.empty_like(vd) if pairs else None
            ws = torch.empty(bcf.bcf_workspace_bytes(bcf.BCF_OP_SORT_PB, n, 0, bcf.BCF_U32, pairs),
                             dtype=torch.uint8, device=dev)
            row = {}
            for algo in ("merge", "pivot_buckets", "auto"):
                if pairs:
                    fn = lambda: bcf.bcf_sort_pairs(ko, vo, kd, vd, kt=bcf.BCF_U32, ws=ws,  # noqa: E731
                                                    stream=stream, algorithm=algo)
                else:
                    fn = lambda: bcf.bcf_sort_keys(ko, kd, kt=bcf.BCF_U32, ws=ws,  # noqa: E731
                                                   stream=stream, algorithm=algo)
                ms = timed_ms(torch, stream, fn, warmup=2, reps=5)
                row[algo] = {"ms": ms, "keys_per_s": n / (ms * 1e-3)}
            row["speedup"] = row["merge"]["ms"] / row["pivot_buckets"]["ms"]
            # the automatic choice against the faster of the two (1.0 = as fast)
            row["auto_vs_best"] = min(row["merge"]["ms"], row["pivot_buckets"]["ms"]) / row["auto"]["ms"]
            out[name + ("+u32" if pairs else "")] = row
            del vd, vo, ws
            torch.cuda.empty_cache()
        del kd, ko
    return {"n": n, "key": "u32", "results": out}


def check_segmented(torch, kin, kout, vout, od, chunk=1 << 27):
    """Exact device checks of a segmented sort of u32 keys (int32 bits) whose
    payloads, if any, are the input positions: every segment in order; with
    payloads, each payload lies in its output's segment, its input key equals
    the output key, and equal keys keep input order (together: the payloads
    are a permutation of the segment's positions); keys only, each segment
    keeps its multiset (two modular fingerprints per segment)."""
    n = kin.numel()
    nseg = od.numel() - 1
    P = 1000000007
    ends = od[1:].contiguous()
    fp = [torch.zeros(nseg, dtype=torch.int64, device=kin.device) for _ in range(4)]
    ok = True
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        e1 = min(n, c1 + 1)  # one element of overlap joins the chunks
        pos = torch.arange(c0, e1, dtype=torch.int64, device=kin.device)
        seg = torch.searchsorted(ends, pos, right=True)
        o = kout[c0:e1].to(torch.int64) & 0xFFFFFFFF
        same = seg[1:] == seg[:-1]
        ok = ok and bool((~same | (o[1:] >= o[:-1])).all().item())
        if vout is not None:
            v = vout[c0:e1].to(torch.int64) & 0xFFFFFFFF
            ok = ok and bool((v < n).all().item())
            vs = torch.searchsorted(ends, v.clamp(max=n - 1), right=True)
            ok = ok and bool((vs == seg).all().item())
            ok = ok and bool((kin[v.clamp(max=n - 1)] == kout[c0:e1]).all().item())
            ties = same & (o[1:] == o[:-1])
            ok = ok and bool((~ties | (v[1:] > v[:-1])).all().item())
        else:
            m = c1 - c0
            i = kin[c0:c1].to(torch.int64) & 0xFFFFFFFF
            for x, a, b in ((i, 0, 1), (o[:m], 2, 3)):
                xm = x % P
                fp[a].index_add_(0, seg[:m], xm)
                fp[b].index_add_(0, seg[:m], xm * xm % P)
    if vout is None:
        ok = ok and bool((fp[0] == fp[2]).all().item()) and bool(
            ((fp[1] % P) == (fp[3] % P)).all().item())
    return ok


def segmented_bench(torch, dev, bcf):
    """Row A6 on its workload: 100,000 segments of log-uniform size in [1, 2^18]
    (about 2.1e9 keys; seed 4000) and the 1 GiB variant ([1, 2^14]), uniform u32
    keys, keys only and with u32 payloads, one persistent launch replayed from a
    CUDA graph.  Bytes per key and pass: 2 x (key + payload)."""
    import numpy as np

    import workloads

    out = {}
    side = torch.cuda.Stream(dev)
    for label, hi in (("[1, 2^18]", 1 << 18), ("[1, 2^14] (1 GiB variant)", 1 << 14)):
        sizes = workloads.segment_sizes(100_000, hi, seed=4000)
        offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        n = int(offs[-1])
        g = torch.Generator(device=dev)
        g.manual_seed(4001)
        kd = torch.randint(-2**31, 2**31 - 1, (n,), dtype=torch.int32, device=dev, generator=g)
        ko = torch.empty_like(kd)
        od = torch.from_numpy(offs).to(dev)
        for pairs in (False, True):
            vd = torch.arange(n, dtype=torch.int32, device=dev) if pairs else None
            vo = torch.empty_like(vd) if pairs else None
            ws = torch.empty(bcf.bcf_workspace_bytes(bcf.BCF_OP_SEGMENTED, n, sizes.size,
                                                     bcf.BCF_U32, pairs),
                             dtype=torch.uint8, device=dev)

            def call():
                bcf.bcf_segmented_sort(ko, vo, kd, vd, od, kt=bcf.BCF_U32, ws=ws, stream=side)

            with torch.cuda.stream(side):
                call()
            side.synchronize()
            exact = check_segmented(torch, kd, ko, vo, od)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=side):
                call()
            ms = timed_ms(torch, torch.cuda.current_stream(dev), graph.replay, warmup=2, reps=5)
            # where the time goes: one direct call with the library's launch records
            bcf.bcf_profile_collect()
            bcf.bcf_profile_enable(True)
            with torch.cuda.stream(side):
                call()
            side.synchronize()
            bcf.bcf_profile_enable(False)
            prof = bcf.bcf_profile_collect()
            parts = {k: round(v["total_ms"], 3) for k, v in prof.items() if v["launches"]}
            out[f"{label}{' +u32' if pairs else ''}"] = {
                "segments": int(sizes.size), "keys": n, "ms": ms, "keys_per_s": n / (ms * 1e-3),
                "payload": "u32" if pairs else None, "exact": exact,
                "merges": "launches" if "merge" in parts else "worker",
                "parts_ms": parts}
            del vd, vo, ws, graph
            torch.cuda.empty_cache()
        del kd, ko, od
        torch.cuda.empty_cache()
    if bcf.bcf_last_device_error() != 0:
        raise RuntimeError("segmented sort: device error word set")
    return {"graph_replay": True, "results": out}


def merge_runs_bench(torch, dev, bcf, peak):
    """Row A5 on its workload: k in {2, 16, 256} sorted u32 runs, 2^27 keys in
    total, lengths log-uniform in [2^10, 2^24] rescaled to the total (seed
    3000 + k), merged into one output; keys only and with u32 payloads."""
    import numpy as np

    import workloads

    total = 1 << 27
    out = {}
    stream = torch.cuda.current_stream(dev)
    for k in (2, 16, 256):
        keys, offs = workloads.sorted_runs(k, total)
        kd = torch.from_numpy(keys.view(np.int32)).to(dev)
        ko = torch.empty_like(kd)
        offl = [int(x) for x in offs]
        for pairs in (False, True):
            vd = torch.arange(total, dtype=torch.int32, device=dev) if pairs else None
            vo = torch.empty_like(vd) if pairs else None
            ws = torch.empty(bcf.bcf_workspace_bytes(bcf.BCF_OP_MERGE, total, k, bcf.BCF_U32,
                                                     pairs), dtype=torch.uint8, device=dev)
            def call():
                bcf.bcf_merge_runs(ko, vo, kd, vd, offl, kt=bcf.BCF_U32, ws=ws, stream=stream)

            ms = timed_ms(torch, stream, call, warmup=2, reps=5)
            # where one call's device time goes (library events on the stream)
            torch.cuda.synchronize()
            bcf.bcf_profile_collect()
            bcf.bcf_profile_enable(True)
            call()
            torch.cuda.synchronize()
            bcf.bcf_profile_enable(False)
            prof = bcf.bcf_profile_collect()
            passes = int(np.ceil(np.log2(k)))
            gbs = passes * 2 * total * (4 + (4 if pairs else 0)) / (ms * 1e-3) / 1e9
            out[f"k={k}{' +u32' if pairs else ''}"] = {
                "ms": ms, "keys_per_s": total / (ms * 1e-3), "merge_passes": passes,
                "gbs_over_passes": gbs, "frac": gbs / peak,
                "partition_ms": prof["partition"]["total_ms"], "merge_ms": prof["merge"]["total_ms"]}
            del vd, vo, ws
            torch.cuda.empty_cache()
        del kd, ko
    return {"total_keys": total, "results": out}


def host_cpu_model():
    """The host CPU's model name as lscpu reports it (Grace on the GB300 host)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
    except Exception:
        return None
    fields = {}
    for ln in out.splitlines():
        if ":" in ln:
            k, v = ln.split(":", 1)
            fields[k.strip()] = v.strip()
    model = fields.get("Model name")
    vendor = fields.get("Vendor ID")
    arch = fields.get("Architecture")
    return ", ".join(x for x in (vendor, model, arch) if x) or None


# ---- the large-sort family (uniform, gaussian, sorted, reverse, distinct16,
# zipf) drawn on the device.  Same laws as workloads.keys (which the parity
# tests use), drawn with torch's seeded device generator instead of numpy, so
# that 2^28-key inputs take milliseconds to make.  Seed = the family's rule
# (1000 * distribution + 10 * key type + log2 n).
GRID_DISTS = ("uniform", "gaussian", "sorted", "reverse", "distinct16", "zipf")


def device_u32_values(torch, dev, dist, n, seed):
    """u32 values (as int64 in [0, 2^32)) of one distribution of the family."""
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    if dist == "uniform":
        return torch.randint(0, 1 << 32, (n,), dtype=torch.int64, device=dev, generator=g)
    if dist == "gaussian":
        x = torch.normal(2.0**31, 2.0**28, (n,), dtype=torch.float64, device=dev, generator=g)
        return x.round_().clamp_(0, 2.0**32 - 1).to(torch.int64)
    if dist in ("sorted", "reverse"):
        e = torch.empty(n + 1, dtype=torch.float64, device=dev).exponential_(1.0, generator=g)
        s = torch.cumsum(e, 0)
        x = torch.floor(s[:-1] / s[-1] * 2.0**32).clamp_(max=2.0**32 - 1).to(torch.int64)
        x = torch.cummax(x, 0).values  # exponential spacings: sorted by construction
        return x.flip(0) if dist == "reverse" else x
    if dist == "distinct16":
        pool = torch.randint(0, 1 << 32, (16,), dtype=torch.int64, device=dev, generator=g)
        return pool[torch.randint(0, 16, (n,), device=dev, generator=g)]
    if dist == "zipf":
        w = torch.arange(1, (1 << 20) + 1, dtype=torch.float64, device=dev).pow_(-1.1)
        cdf = torch.cumsum(w, 0)
        cdf /= cdf[-1].clone()
        u = torch.rand(n, dtype=torch.float64, device=dev, generator=g)
        r = torch.searchsorted(cdf, u).clamp_(max=(1 << 20) - 1)
        return (r * 0x9E3779B1) & 0xFFFFFFFF
    raise ValueError(dist)


def device_keys(torch, dev, dist, key, n):
    """Keys of the family for key type key in {u32, f32, u64}, as a tensor of the
    key width (int32 / int64 bits)."""
    import workloads

    seed = workloads.large_sort_seed(dist, key, n)
    if key == "u64" and dist in ("uniform", "distinct16"):
        g = torch.Generator(device=dev)
        g.manual_seed(seed)
        if dist == "uniform":
            return torch.randint(-2**63, 2**63 - 1, (n,), dtype=torch.int64, device=dev,
                                 generator=g)
        pool = torch.randint(-2**63, 2**63 - 1, (16,), dtype=torch.int64, device=dev, generator=g)
        return pool[torch.randint(0, 16, (n,), device=dev, generator=g)]
    if key == "u64" and dist == "zipf":
        g = torch.Generator(device=dev)
        g.manual_seed(seed)
        w = torch.arange(1, (1 << 20) + 1, dtype=torch.float64, device=dev).pow_(-1.1)
        cdf = torch.cumsum(w, 0)
        cdf /= cdf[-1].clone()
        u = torch.rand(n, dtype=torch.float64, device=dev, generator=g)
        r = torch.searchsorted(cdf, u).clamp_(max=(1 << 20) - 1)
        return r * 0x9E3779B97F4A7C15  # wraps mod 2^64
    if key == "f32" and dist in ("uniform", "distinct16"):
        key = "u32"  # random bit patterns: NaNs, infinities, subnormals and zeros included
        seed = workloads.large_sort_seed(dist, "f32", n)
    v = device_u32_values(torch, dev, dist, n, seed)
    if key == "u32":
        return (v - (v >> 31 << 32)).to(torch.int32)  # the same 32 bits
    if key == "u64":
        return v
    return v.to(torch.float32).view(torch.int32)  # f32: float32 of the u32 value


def order_bits(torch, k, key):
    """Keys as int64 whose signed order is the key order (totalOrder for f32)."""
    if key == "u64":
        return k ^ (-2**63)  # unsigned order as signed
    u = k.to(torch.int64) & 0xFFFFFFFF
    if key == "f32":
        neg = (u >> 31) == 1
        u = torch.where(neg, u ^ 0xFFFFFFFF, u | 0x80000000)
    return u


def check_sorted_pairs(torch, kin, kout, vout, key):
    """Exact device checks of a stable sort whose payloads are the input
    positions: keys in order, payloads a permutation, every payload's input key
    equals its output key (keys and values travel together), equal keys in
    input order.  Keys only (vout None): in order and the same multiset
    (two modular fingerprints)."""
    o = order_bits(torch, kout, key)
    ok = bool((o[1:] >= o[:-1]).all().item())
    if vout is None:
        i = order_bits(torch, kin, key)
        p = 1000000007
        ok = ok and bool(((i % p).sum() == (o % p).sum()).item()) and bool(
            (((i % p) * (i % p) % p).sum() == ((o % p) * (o % p) % p).sum()).item())
        return ok
    v = vout.to(torch.int64) & 0xFFFFFFFF
    n = v.numel()
    ok = ok and bool((torch.bincount(v, minlength=n) == 1).all().item())
    ok = ok and bool((kin[v] == kout).all().item())
    ties = o[1:] == o[:-1]
    ok = ok and bool((~ties | (v[1:] > v[:-1])).all().item())
    return ok


def c2_grid(torch, dev, bcf, peak, sizes=(24, 26, 28), reps=3):
    """The large-sort grid: n in 2^sizes x the six distributions x {u32, f32,
    u64} keys x {keys only, u32 payloads}: whole-sort ms, keys/s and the merge
    pass's mean time against the HBM roofline, every output checked exactly on
    the device."""
    stream = torch.cuda.current_stream(dev)
    codes = {"u32": bcf.BCF_U32, "f32": bcf.BCF_F32, "u64": bcf.BCF_U64}
    out = {}
    all_ok = True
    for lg in sizes:
        n = 1 << lg
        for key in ("u32", "f32", "u64"):
            kt = codes[key]
            ws = torch.empty(bcf.bcf_workspace_bytes(bcf.BCF_OP_SORT, n, 0, kt, True),
                             dtype=torch.uint8, device=dev)
            for dist in GRID_DISTS:
                kd = device_keys(torch, dev, dist, key, n)
                ko = torch.empty_like(kd)
                for pairs in (False, True):
                    vd = torch.arange(n, dtype=torch.int32, device=dev) if pairs else None
                    vo = torch.empty_like(vd) if pairs else None
                    if pairs:
                        fn = lambda: bcf.bcf_sort_pairs(ko, vo, kd, vd, kt=kt, ws=ws,  # noqa: E731
                                                        stream=stream)
                    else:
                        fn = lambda: bcf.bcf_sort_keys(ko, kd, kt=kt, ws=ws,  # noqa: E731
                                                       stream=stream)
                    fn()
                    torch.cuda.synchronize()
                    bcf.bcf_profile_collect()
                    bcf.bcf_profile_enable(True)
                    ms = timed_ms(torch, stream, fn, warmup=0, reps=reps)
                    bcf.bcf_profile_enable(False)
                    prof = bcf.bcf_profile_collect()
                    ok = check_sorted_pairs(torch, kd, ko, vo, key)
                    all_ok = all_ok and ok
                    plan = bcf.bcf_sort_plan(n, kt, pairs)
                    m = prof["merge"]
                    merge_ms = m["total_ms"] / max(m["launches"], 1)
                    frac = (plan["bytes_per_pass"] / (merge_ms * 1e-3) / 1e9 / peak
                            if m["launches"] else None)
                    out[f"2^{lg} {key}{'+u32' if pairs else ''} {dist}"] = {
                        "ms": round(ms, 4), "gkeys_s": round(n / (ms * 1e-3) / 1e9, 3),
                        "merge_frac": None if frac is None else round(frac, 3), "exact": ok}
                    del vd, vo
                del kd, ko
            del ws
            torch.cuda.empty_cache()
    return {"laws": "the workload family's six laws, drawn on the device (torch generator, "
                    "seed rule 1000*dist+10*key+log2n); u32 payload = input position",
            "all_exact": all_ok, "results": out}


def c1_latency(torch, dev, bcf, calls=60):
    """The small plain sort: 2^20 uniform u32 keys, seed 0, ascending, keys
    only: per-call latency of one bcf_sort_keys (one launch chain), each call
    timed alone with CUDA events and by the host clock (launch to completion
    seen by the host), median of the last calls - 10; and back-to-back
    throughput.  4 MiB of keys: L2-resident, so no roofline claim."""
    import numpy as np

    import workloads

    n = 1 << 20
    keys = workloads.keys("uniform", "u32", n, seed=0)
    kd = torch.from_numpy(keys.view(np.int32)).to(dev)
    ko = torch.empty_like(kd)
    ws = torch.empty(bcf.bcf_workspace_bytes(bcf.BCF_OP_SORT, n, 0, bcf.BCF_U32, False),
                     dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    ev, host = [], []
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    for _ in range(calls):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        a.record(stream)
        bcf.bcf_sort_keys(ko, kd, kt=bcf.BCF_U32, ws=ws, stream=stream)
        b.record(stream)
        b.synchronize()
        host.append((time.perf_counter() - t0) * 1e3)
        ev.append(a.elapsed_time(b))
    ev, host = ev[10:], host[10:]
    thr_ms = timed_ms(torch, stream, lambda: bcf.bcf_sort_keys(ko, kd, kt=bcf.BCF_U32, ws=ws,
                                                              stream=stream), warmup=3, reps=50)
    ok = check_sorted_pairs(torch, kd, ko, None, "u32")
    plan = bcf.bcf_sort_plan(n, bcf.BCF_U32, False)
    return {"n": n, "seed": 0, "launches_per_call": plan["launches"],
            "latency_ms_median": statistics.median(ev), "latency_ms_p90": sorted(ev)[int(0.9 * len(ev))],
            "host_latency_ms_median": statistics.median(host),
            "back_to_back_ms": thr_ms, "keys_per_s": n / (thr_ms * 1e-3),
            "calls_timed": len(ev), "exact": ok}


def profile_case(args):
    """A small case of one path, for ncu captures (inputs larger than L2, a
    few launches): 'cps' = colored prefix sums of 2^26 elements, 16 colors,
    both layouts, two launches each; 'pb' = pivot-bucket sort of 2^26
    16-distinct u32 keys, twice; 'seg' = segmented sort of 5,000 segments
    with sizes log-uniform over [1, 2^18] (about 1.05e8 u32 keys), twice;
    'seg_c4' = the segmented workload itself (100,000 segments, about 2.1e9
    u32 keys drawn on the device as the bench draws them), twice -- for a
    launch list only (one ncu pass per launch);
    'pairs' / 'u64' / 'u64p' = sort of 2^26 uniform keys, twice: u32 keys
    with u32 payloads, u64 keys, u64 keys with u32 payloads."""
    import numpy as np
    import torch

    import paper_1306_5076_gb300 as bcf
    import workloads

    dev = torch.device("cuda", 0)
    bcf._native.load()
    bcf.bcf_profile_set_smem_floor(args.smem_floor)
    n = 1 << 26
    if args.profile_case in ("pairs", "u64", "u64p"):
        kname = "u32" if args.profile_case == "pairs" else "u64"
        keys = workloads.keys("uniform", kname, n)
        kd = torch.from_numpy(keys.view(np.int32 if kname == "u32" else np.int64)).to(dev)
        ko = torch.empty_like(kd)
        kt = bcf.BCF_U32 if kname == "u32" else bcf.BCF_U64
        with_vals = args.profile_case != "u64"
        vd = torch.arange(n, dtype=torch.int32, device=dev) if with_vals else None
        vo = torch.empty_like(vd) if with_vals else None
        for _ in range(2):
            if with_vals:
                bcf.bcf_sort_pairs(ko, vo, kd, vd, kt=kt)
            else:
                bcf.bcf_sort_keys(ko, kd, kt=kt)
    elif args.profile_case == "cps":
        vals, cols = workloads.colored_elements(n, 16, seed=26)
        vd = torch.from_numpy(vals.view(np.int32)).to(dev)
        cd = torch.from_numpy(cols).to(dev)
        od = torch.empty_like(vd)
        for layout in (bcf.BCF_CPS_BANKED, bcf.BCF_CPS_ROWS):
            for _ in range(2):
                bcf.bcf_colored_prefix_sums(od, vd, cd, 16, layout=layout)
    elif args.profile_case == "pb":
        keys = workloads.keys("distinct16", "u32", n)
        kd = torch.from_numpy(keys.view(np.int32)).to(dev)
        ko = torch.empty_like(kd)
        for _ in range(2):
            bcf.bcf_sort_keys(ko, kd, kt=bcf.BCF_U32, algorithm="pivot_buckets")
    elif args.profile_case == "seg_c4":
        sizes = workloads.segment_sizes(100_000, 1 << 18, seed=4000)
        offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        n = int(offs[-1])
        g = torch.Generator(device=dev)
        g.manual_seed(4001)
        kd = torch.randint(-2**31, 2**31 - 1, (n,), dtype=torch.int32, device=dev, generator=g)
        ko = torch.empty_like(kd)
        od = torch.from_numpy(offs).to(dev)
        for _ in range(2):
            bcf.bcf_segmented_sort(ko, None, kd, None, od, kt=bcf.BCF_U32)
    else:
        keys, offs = workloads.segments(5_000, 1 << 18, "u32", seed=4000)
        n = keys.size
        kd = torch.from_numpy(keys.view(np.int32)).to(dev)
        ko = torch.empty_like(kd)
        od = torch.from_numpy(offs.astype(np.int64)).to(dev)
        for _ in range(2):
            bcf.bcf_segmented_sort(ko, None, kd, None, od, kt=bcf.BCF_U32)
    torch.cuda.synchronize()
    if bcf.bcf_last_device_error() != 0:
        raise RuntimeError("device error word set")
    print(json.dumps({"profile_case": args.profile_case, "n": n, "ok": True}))
    return 0


def summary_of(line, peak):
    """A compact digest of the sections, placed last in the JSON line so that a
    reader who keeps only its tail still sees every headline number."""
    r3 = lambda x: None if x is None else round(float(x), 3)  # noqa: E731
    s = {"sort_2p28_u32_ms": r3(line["ms_per_step"]),
         "merge_pass_frac": r3(line["roofline"]["frac"]),
         "e2e_gkeys_s": r3(line["e2e"]["value"] / 1e9)}
    pp = line.get("per_kernel_ms") or {}
    s["block_sort_ms"], s["partition_ms"] = r3(pp.get("block_sort")), r3(pp.get("partition"))
    cpu = line.get("cpu_baseline")
    if cpu:
        s["oracle_mkeys_s"] = {"all_cores": r3(cpu["value"] / 1e6), "cores": cpu["cores"],
                               "one_core": r3(cpu["single_thread"]["value"] / 1e6),
                               "cpu": cpu.get("cpu_model")}
    sv = line.get("serving")
    if sv:
        s["serving_p50_p99_ms"] = {
            f"{tr}_{mode}": [r3(sv[tr][mode]["p50_ms"]), r3(sv[tr][mode]["p99_ms"])]
            for tr in ("nominal", "stress_8x") for mode in ("served", "plain")}
        s["serving_gkeys_s"] = {f"{tr}_{mode}": r3(sv[tr][mode]["keys_per_s"] / 1e9)
                                for tr in ("nominal", "stress_8x") for mode in ("served", "plain")}
        s["serving_batches"] = {tr: sv[tr]["served"]["coalesced_batches"]
                                for tr in ("nominal", "stress_8x")}
    c1 = line.get("small_sort_2p20")
    if c1:
        s["c1_2p20"] = {"latency_ms": r3(c1["latency_ms_median"]),
                        "gkeys_s": r3(c1["keys_per_s"] / 1e9), "exact": c1["exact"]}
    g = line.get("large_sort_grid")
    if g:
        res = g["results"]
        s["c2_exact"] = g["all_exact"]
        s["c2_gkeys_s_min_max"] = {}
        for lg in (24, 26, 28):
            for kind in ("u32", "u32+u32", "f32", "f32+u32", "u64", "u64+u32"):
                v = [x["gkeys_s"] for k, x in res.items() if k.startswith(f"2^{lg} {kind} ")]
                if v:
                    s["c2_gkeys_s_min_max"][f"2^{lg} {kind}"] = [min(v), max(v)]
    kt = line.get("key_types")
    if kt:
        s["merge_pass_frac_by_key"] = {k: r3(v.get("merge_pass_frac"))
                                       for k, v in kt["results"].items() if "merge_pass_frac" in v}
    mr = line.get("merge_runs")
    if mr:
        s["merge_runs_frac"] = {k: r3(v["frac"]) for k, v in mr["results"].items()}
    sg = line.get("segmented")
    if sg:
        s["segmented_ms"] = {k: r3(v["ms"]) for k, v in sg["results"].items()}
        s["segmented_exact"] = all(v.get("exact", False) for v in sg["results"].values())
    pb = line.get("pivot_buckets")
    if pb:
        s["pivot_bucket_speedup"] = {k: r3(v["speedup"]) for k, v in pb["results"].items()}
        s["auto_vs_best"] = {k: r3(v["auto_vs_best"]) for k, v in pb["results"].items()}
    cps = line.get("colored_prefix_sums")
    if cps:
        s["cps_frac_banked"] = {d: r3(v["frac"]) for d, v in cps["banked"].items()}
    s["peak_gbs"] = peak
    return s


def run_gpu(args, world, rank, local, pg):
    import numpy as np
    import torch

    import paper_1306_5076_gb300 as bcf
    import workloads

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    bcf._native.load()
    bcf.bcf_profile_set_smem_floor(args.smem_floor)
    seed = workloads.large_sort_seed("uniform", "u32", N) + 7919 * rank
    keys_np = workloads.keys("uniform", "u32", N, seed=seed)
    host_in = torch.from_numpy(keys_np.view(np.int32)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    kd = host_in.to(dev)
    ko = torch.empty_like(kd)
    ws = torch.empty(bcf.bcf_workspace_bytes(bcf.BCF_OP_SORT, N, 0, bcf.BCF_U32, False),
                     dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    plan = bcf.bcf_sort_plan(N, bcf.BCF_U32, False)

    def step():
        bcf.bcf_sort_keys(ko, kd, kt=bcf.BCF_U32, ws=ws, stream=stream)

    def barrier():
        if pg is not None:
            pg.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- device-resident timed region (Python's garbage collector paused: the
    # host loop enqueues every step, and a collection pause would idle the GPU)
    gc.collect()
    gc.disable()
    # Two regions of the same steps.  The first, the headline, runs the calls
    # as a user makes them (the library chains its launches); the second has
    # the launch profiler on, whose CUDA events around every kernel give the
    # per-kernel times of the roofline, and whose launches are plain (an event
    # between two kernels ends the chaining).
    clocks = ClockSampler(local)
    bcf.bcf_profile_collect()  # drop anything pending
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    m0 = clocks.mark()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    m1 = clocks.mark()
    barrier()
    bcf.bcf_profile_enable(True)
    barrier()
    torch.cuda.synchronize()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(args.steps):
        step()
    p1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop(m0, m1)
    bcf.bcf_profile_enable(False)
    prof, launch_list = bcf.bcf_profile_collect_launches(64 * (args.steps + 1) + 64)
    gc.enable()
    ms = max_over_ranks(torch, pg, e0.elapsed_time(e1) / args.steps, dev)
    ms_profiled = max_over_ranks(torch, pg, p0.elapsed_time(p1) / args.steps, dev)
    passes = per_pass_ms(launch_list)

    # correctness of the timed output (bit-exact order check on the device:
    # sorted and same multiset fingerprint as the input)
    ku = ko.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
    ok_sorted = bool((ku[1:] >= ku[:-1]).all().item())
    fi = (kd.view(torch.int32).to(torch.int64) & 0xFFFFFFFF)
    ok_multiset = bool((fi.sum() == ku.sum()).item() and
                       ((fi * fi) % 1000000007).sum().item() == ((ku * ku) % 1000000007).sum().item())

    # ---- end to end through the public host-buffer call: every step copies its
    # input in from pinned host memory, sorts it and copies the result out
    # (bcf_sort_keys_host).  Steps go round-robin to E2E_STREAMS streams with
    # their own workspaces, so one step's copy-in, another's sort and a third's
    # copy-out overlap (copy engines both ways, SMs).
    E2E_STREAMS = 3
    e2e_steps = max(E2E_STREAMS, min(args.steps, 12))
    del ws
    torch.cuda.empty_cache()
    side = [torch.cuda.Stream(dev) for _ in range(E2E_STREAMS)]
    wss = [torch.empty(bcf.bcf_workspace_bytes(bcf._native.BCF_OP_SORT_HOST, N, 0, bcf.BCF_U32,
                                               False), dtype=torch.uint8, device=dev)
           for _ in range(E2E_STREAMS)]
    houts = [host_out] + [torch.empty_like(host_in).pin_memory() for _ in range(E2E_STREAMS - 1)]

    def e2e_step(i):
        j = i % E2E_STREAMS
        bcf.bcf_sort_keys_host(houts[j], host_in, kt=bcf.BCF_U32, ws=wss[j], stream=side[j],
                               device=dev)

    for i in range(E2E_STREAMS):  # warm-up
        e2e_step(i)
    torch.cuda.synchronize()
    barrier()
    # seven timed regions of e2e_steps steps each; the median is reported (a
    # host-side stall of 0.1-0.2 s in up to three regions -- the host loop
    # issues every step -- does not decide the number), and all seven are listed
    regions = []
    gc.collect()
    gc.disable()
    for _ in range(7):
        h0 = torch.cuda.Event(enable_timing=True)
        h1 = torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        for st in side:
            st.wait_event(h0)
        for i in range(e2e_steps):
            e2e_step(i)
        for st in side:
            stream.wait_stream(st)
        h1.record(stream)
        torch.cuda.synchronize()
        regions.append(h0.elapsed_time(h1) / e2e_steps)
    gc.enable()
    e2e_ms = max_over_ranks(torch, pg, statistics.median(regions), dev)
    # every stream's last result equals the device-timed sort's output
    ok_e2e = all(bool(torch.equal(h, ko.cpu())) for h in houts)

    # the host link of this machine, for reading the end-to-end number: plain
    # copies of the same pinned buffers, each way alone and both at once
    def copy_gbs(pairs_):
        sts = [torch.cuda.Stream(dev) for _ in pairs_]
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = None
        for _ in range(3):  # the fastest of three
            torch.cuda.synchronize()
            c0.record(stream)
            for st, (dst, src) in zip(sts, pairs_):
                st.wait_event(c0)
                with torch.cuda.stream(st):
                    dst.copy_(src, non_blocking=True)
            for st in sts:
                stream.wait_stream(st)
            c1.record(stream)
            torch.cuda.synchronize()
            t = c0.elapsed_time(c1)
            best = t if best is None else min(best, t)
        return sum(d.numel() * d.element_size() for d, _ in pairs_) / (best * 1e6)

    link = {"h2d_gbs": copy_gbs([(kd, host_in)]), "d2h_gbs": copy_gbs([(houts[0], ko)]),
            "both_gbs": copy_gbs([(kd, host_in), (houts[0], ko)]),
            "d2h_gbs_each_output": [copy_gbs([(h, ko)]) for h in houts]}
    del wss
    torch.cuda.empty_cache()

    serving = None
    if args.serve_seconds > 0:
        # the workload's trace (2000 req/s), then the same request mix at 8x the
        # rate, past what one launch chain per request can sustain
        serving = {"nominal": serving_bench(torch, dev, args.serve_seconds),
                   "stress_8x": serving_bench(torch, dev, min(2.0, args.serve_seconds),
                                              rate=16000.0)}

    peak, peak_kind = measured_peaks()
    extras = None
    if not args.no_extras:
        extras = {"small_sort_2p20": c1_latency(torch, dev, bcf),
                  "large_sort_grid": c2_grid(torch, dev, bcf, peak),
                  "key_types": key_types_bench(torch, dev, bcf, peak),
                  "colored_prefix_sums": cps_bench(torch, dev, bcf, peak),
                  "pivot_buckets": pb_bench(torch, dev, bcf),
                  "merge_runs": merge_runs_bench(torch, dev, bcf, peak),
                  "segmented": segmented_bench(torch, dev, bcf)}

    if rank != 0:
        return 0
    m = prof["merge"]
    merge_ms = m["total_ms"] / max(m["launches"], 1)
    achieved = plan["bytes_per_pass"] / (merge_ms * 1e-3) / 1e9
    bs = prof["block_sort"]
    part = prof["partition"]
    launches = sum(v["launches"] for v in prof.values())
    traffic = merge_traffic_per_launch()
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        kps, cores, n, t = oracle_keys_per_s()
        kps1, _, n1, t1 = oracle_keys_per_s(SINGLE_LOG2N, threads=1)
        cpu = {"value": kps, "unit": "keys/s", "cores": cores, "kind": "oracle",
               "sample": f"2^{SAMPLE_LOG2N} keys of the same workload, one stable merge sort "
                         f"(C, {cores} threads), {t[0]:.2f} s",
               "single_thread": {"value": kps1, "unit": "keys/s", "cores": 1,
                                 "sample": f"2^{SINGLE_LOG2N} keys of the same workload, "
                                           f"{t1[0]:.2f} s"},
               "cpu_model": host_cpu_model()}
    line = {
        "metric": METRIC,
        "value": job_keys_per_s(world, N, ms),
        "unit": "keys/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": f"sort of 2^{args.log2n} uniform u32 keys, keys only, ascending",
                   "n": N, "key": "u32", "payload": None, "seed": seed,
                   "block_tile": plan["block_tile"], "merge_tile": plan["merge_tile"],
                   "merge_passes": plan["merge_passes"],
                   "l2": "inputs (1 GiB) larger than L2 (129 MB); no flush",
                   "timing": "value from a region of plain calls; roofline, per_kernel_ms, "
                             "per_pass_ms and gpu_launches from a second region of the same "
                             "steps with the launch profiler's CUDA events around every kernel",
                   "ms_per_step_profiled": ms_profiled,
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "merge pass (bcf merge_kernel)",
                     "peak_kind": f"{peak_kind} hbm_gbs (copy read+write)",
                     "bytes_per_launch": plan["bytes_per_pass"],
                     "mean_launch_ms": merge_ms},
        "per_kernel_ms": {"block_sort": bs["total_ms"] / max(bs["launches"], 1),
                          "partition": part["total_ms"] / max(part["launches"], 1),
                          "merge": merge_ms},
        "per_pass_ms": passes,
        "gpu_launches": launches,
        "e2e": {"value": job_keys_per_s(world, N, e2e_ms), "unit": "keys/s",
                "h2d_bytes_per_step": N * KEY_BYTES, "d2h_bytes_per_step": N * KEY_BYTES,
                "api": "bcf_sort_keys_host, pinned host buffers", "streams": E2E_STREAMS,
                "steps": e2e_steps, "regions_ms_per_step": regions, "host_link": link},
        "clocks": clk,
        "checks": {"sorted": ok_sorted, "multiset": ok_multiset, "e2e_roundtrip": ok_e2e},
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if serving is not None:
        line["serving"] = serving
    if extras is not None:
        line.update(extras)
    line["summary"] = summary_of(line, peak)
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-case", choices=["cps", "pb", "seg", "seg_c4", "pairs", "u64", "u64p"],
                    help="run only a small case of one path (for ncu captures) and exit")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other key types, the colored prefix sums and the "
                         "pivot-bucket comparison")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="length of the served-vs-plain request trace (0: skip)")
    ap.add_argument("--oracle-table", action="store_true",
                    help="time the CPU oracle on bounded samples of every workload (one core and "
                         "all cores) and exit; no GPU is used")
    ap.add_argument("--smem-floor", type=int, default=0,
                    help="profiling only: minimum dynamic shared memory (bytes) of the block "
                         "sort and merge launches, e.g. 200000 for one CTA per SM")
    ap.add_argument("--log2n", type=int, default=LOG2N,
                    help="keys = 2^log2n (default 28, the benchmark workload; smaller values "
                         "are for ncu captures)")
    args = ap.parse_args()
    global N
    N = 1 << args.log2n
    if args.warmup < 3:
        args.warmup = 3
    if args.profile_case:
        return profile_case(args)
    if args.oracle_table:
        print(json.dumps({"oracle_table": oracle_table()}))
        return 0
    world, rank, local, pg = dist_setup(args)
    try:
        if args.impl == "reference":
            return run_reference(args, world, rank)
        return run_gpu(args, world, rank, local, pg)
    finally:
        if pg is not None:
            pg.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
