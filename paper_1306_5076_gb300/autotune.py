"""Autotuner: picks elements per thread (E), CTA size (NT) and merge tile per
key width, payload flag and size band by measurement on the GPU, and writes
the table the C library reads (``tuning/gb300.tsv``).

The paper tunes its parameters by hand (Sec. 4: p = 8 P_h = 128, M = w^2 =
1024).  Here every compiled configuration (``bcf_tuning_config``) that is
built for the key width / payload is timed through the C ABI on a synthetic
input of the band's probe size, and the fastest is kept.  The sort's output
never depends on the choice (tests/test_gpu_tuning.py checks that).

Usage (on a GPU): ``python -m paper_1306_5076_gb300.autotune [--quick]``.
"""
from __future__ import annotations

import argparse
import os
import statistics
import sys

import paper_1306_5076_gb300 as bcf

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "tuning", "gb300.tsv")

# (n_min, n_max, probe size) of each size band
BANDS = [(0, 1 << 18, 1 << 16), (1 << 18, 1 << 23, 1 << 21), (1 << 23, 1 << 26, 1 << 24),
         (1 << 26, 1 << 48, 1 << 27)]
KINDS = [(4, False), (4, True), (8, False), (8, True)]  # (key bytes, pairs)


def _configs(kind, kb, pairs):
    out = []
    i = 0
    while True:
        c = bcf.bcf_tuning_config(kind, i)
        if c is None:
            return out
        if bcf.bcf_tuning_supported(kind, i, kb, pairs):
            out.append((i, c))
        i += 1


def _inputs(torch, n, kb, pairs, seed=0):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    dt = torch.int32 if kb == 4 else torch.int64
    lo, hi = (-2**31, 2**31 - 1) if kb == 4 else (-2**63, 2**63 - 1)
    k = torch.randint(lo, hi, (n,), dtype=dt, device="cuda", generator=g)
    v = torch.arange(n, dtype=torch.int32, device="cuda") if pairs else None
    return k, v


def _time(torch, fn, reps):
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def tune_sort(torch, kb, pairs, reps, log):
    rows = []
    kt = bcf.BCF_U32 if kb == 4 else bcf.BCF_U64
    blocks, merges = _configs(0, kb, pairs), _configs(1, kb, pairs)
    for n_min, n_max, n in BANDS:
        k, v = _inputs(torch, n, kb, pairs)
        ko = torch.empty_like(k)
        vo = torch.empty_like(v) if pairs else None
        ws = torch.empty(bcf.bcf_workspace_bytes(bcf.BCF_OP_SORT, n, 0, kt, pairs),
                         dtype=torch.uint8, device="cuda")
        best = None
        for bi, (be, bnt) in blocks:
            for mi, (me, mnt) in merges:
                if me * mnt > 2 * be * bnt:
                    continue
                bcf.bcf_tuning_set([dict(op=bcf.BCF_OP_SORT, key_bytes=kb, has_vals=int(pairs),
                                         n_min=0, n_max=1 << 48, block_cfg=bi, merge_cfg=mi,
                                         seg_cfg=0)])
                if pairs:
                    fn = lambda: bcf.bcf_sort_pairs(ko, vo, k, v, kt=kt, ws=ws)  # noqa: E731
                else:
                    fn = lambda: bcf.bcf_sort_keys(ko, k, kt=kt, ws=ws)  # noqa: E731
                ms = _time(torch, fn, reps)
                log(f"sort kb={kb} pairs={int(pairs)} n=2^{n.bit_length()-1} "
                    f"block={be}x{bnt} merge={me}x{mnt}: {ms:.3f} ms")
                if best is None or ms < best[0]:
                    best = (ms, bi, mi)
        rows.append((bcf.BCF_OP_SORT, kb, int(pairs), n_min, n_max, best[1], best[2], 0))
        rows.append((bcf.BCF_OP_MERGE, kb, int(pairs), n_min, n_max, best[1], best[2], 0))
        del k, v, ko, vo, ws
    return rows


# (n_min, n_max, probes) of the segmented sort's size bands: small batches (as
# the request server coalesces them) and large ones; each probe is (segments,
# largest segment) of a log-uniform size law, and a band's candidates are
# ranked by their summed time over its probes (large batches of short and of
# long segments)
SEG_BANDS = [(0, 1 << 24, [(2000, 1 << 14)]),
             (1 << 24, 1 << 48, [(5000, 1 << 18), (50000, 1 << 14)])]


def tune_segmented(torch, kb, pairs, reps, log):
    """Per size band: the worker configuration and who runs the merge passes
    (merge_cfg -1: the worker; else launches of that merge configuration,
    whose tile must not exceed the sort tile)."""
    import numpy as np

    import workloads

    kt = bcf.BCF_U32 if kb == 4 else bcf.BCF_U64
    merges = _configs(1, kb, pairs)
    cands = []
    for si, (se, snt) in _configs(2, kb, pairs):
        cands.append((si, -1, f"{se}x{snt}", "worker"))
        cands += [(si, mi, f"{se}x{snt}", f"launches, {me * mnt}-key tiles")
                  for mi, (me, mnt) in merges if me * mnt <= se * snt]
    rows = []
    for n_min, n_max, probes in SEG_BANDS:
        total = {c: 0.0 for c in cands}
        for nseg, hi in probes:
            sizes = workloads.segment_sizes(nseg, hi, seed=4000)
            offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
            n = int(offs[-1])
            k, v = _inputs(torch, n, kb, pairs)
            ko = torch.empty_like(k)
            vo = torch.empty_like(v) if pairs else None
            od = torch.from_numpy(offs).to("cuda")
            ws = torch.empty(bcf.bcf_workspace_bytes(bcf.BCF_OP_SEGMENTED, n, nseg, kt, pairs),
                             dtype=torch.uint8, device="cuda")
            for c in cands:
                si, mi, shape, who = c
                bcf.bcf_tuning_set([dict(op=bcf.BCF_OP_SEGMENTED, key_bytes=kb,
                                         has_vals=int(pairs), n_min=0, n_max=1 << 48,
                                         block_cfg=0, merge_cfg=mi, seg_cfg=si)])
                ms = _time(torch, lambda: bcf.bcf_segmented_sort(ko, vo, k, v, od, kt=kt, ws=ws),
                           reps)
                log(f"segmented kb={kb} pairs={int(pairs)} n={n} cfg={shape} merges: {who}: "
                    f"{ms:.3f} ms")
                total[c] += ms
            del k, v, ko, vo, od, ws
        best = min(cands, key=lambda c: total[c])
        rows.append((bcf.BCF_OP_SEGMENTED, kb, int(pairs), n_min, n_max, 0, best[1], best[0]))
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true", help="fewer repetitions")
    ap.add_argument("--out", default=TABLE)
    ap.add_argument("--only", choices=("sort", "segmented"), default=None,
                    help="tune one operation; the other's rows are kept from --out")
    args = ap.parse_args(argv)
    import torch

    sys.path.insert(0, os.path.dirname(HERE))
    reps = 3 if args.quick else 7
    log = lambda m: print(m, flush=True)  # noqa: E731
    rows = []
    if args.only and os.path.exists(args.out):
        keep = {"sort": {bcf.BCF_OP_SEGMENTED}, "segmented": {bcf.BCF_OP_SORT, bcf.BCF_OP_MERGE}}
        for line in open(args.out):
            if line.strip() and not line.startswith("#"):
                r = tuple(int(x) for x in line.split())
                if r[0] in keep[args.only]:
                    rows.append(r)
    for kb, pairs in KINDS:
        if args.only in (None, "sort"):
            rows += tune_sort(torch, kb, pairs, reps, log)
        if args.only in (None, "segmented"):
            rows += tune_segmented(torch, kb, pairs, reps, log)
    rows.sort(key=lambda r: (r[1], r[2], r[0], r[3]))
    bcf.bcf_tuning_set(None)
    name = torch.cuda.get_device_name()
    with open(args.out, "w") as f:
        f.write(f"# bcfsort tuning table, measured by paper_1306_5076_gb300/autotune.py on {name}\n")
        f.write("# op key_bytes has_vals n_min n_max block_cfg merge_cfg seg_cfg\n")
        for r in rows:
            f.write(" ".join(str(x) for x in r) + "\n")
    print("wrote", args.out)


if __name__ == "__main__":
    main()
