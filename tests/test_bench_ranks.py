"""The benchmark's multi-rank host logic on CPU (gloo, world size 2).

Every GPU runs its own replica of the sort (the sort does not shard), so the
only cross-rank steps are the barriers around the timed region and the
max-over-ranks of each timing; the job's throughput is every rank's keys over
the slowest rank's time.  These run here with the gloo backend; the reference
arm is also launched the way the driver launches it, two ranks under
torch.distributed.run, where rank 0 alone times the oracle and prints the line.
"""
from __future__ import annotations

import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.max_over_ranks(torch, dist, 3.0 + 4.0 * rank, "cpu")
        e2e = bench.max_over_ranks(torch, dist, 9.0 - rank, "cpu")
        out.put((rank, ms, e2e, bench.job_keys_per_s(world, 1 << 20, ms)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, e2e, value in res:
        assert ms == 7.0 and e2e == 9.0  # the slowest rank's time on every rank
        assert value == pytest.approx(2 * (1 << 20) / 7e-3)


def test_single_process_has_no_reduction():
    assert bench.max_over_ranks(torch, None, 4.5, "cpu") == 4.5
    assert bench.job_keys_per_s(1, 1000, 2.0) == pytest.approx(5e5)


def test_reference_arm_under_torchrun_two_ranks(tmp_path):
    """Launched as the driver launches it: rank 0 times the oracle and prints
    one JSON line; rank 1 exits 0 without work."""
    import oracle

    oracle.build()  # compiled once here, not inside rank 0's timed steps
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "3"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_per_pass_times_from_the_launch_list():
    """Each merge pass's time, averaged over steps, from the library's launch list."""
    one = [("block_sort", 2.0)] + [x for i in range(3)
                                   for x in (("partition", 0.04), ("merge", 0.3 + 0.01 * i))]
    two = [("block_sort", 4.0)] + [x for i in range(3)
                                   for x in (("partition", 0.06), ("merge", 0.5 + 0.01 * i))]
    got = bench.per_pass_ms(one + two)
    assert got["steps"] == 2 and got["block_sort"] == pytest.approx(3.0)
    assert got["partition"] == pytest.approx([0.05] * 3)
    assert got["merge"] == pytest.approx([0.4, 0.41, 0.42])
    assert bench.per_pass_ms([]) is None
