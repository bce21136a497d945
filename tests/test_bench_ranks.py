"""The bench's multi-rank host logic, on CPU with gloo ranks (world size 2).

With N > 1 the bench runs one replica per rank (the path is timed as
independent replicas: one GPU per rank, no data-path collective).  What the
ranks share is host logic: a barrier around the timed region, the slowest
rank's time (max over ranks) for the whole-job value, and, for the reference
arm, rank 0 alone doing the work and printing the line.
"""
import argparse
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        slowest = bench.max_over_ranks(world, 10.0 + 5.0 * rank)
        buf = io.StringIO()
        with redirect_stdout(buf):
            if rank != 0:  # rank 0's reference line is checked in its own test
                bench.run_reference(argparse.Namespace(steps=1, warmup=0, workload=bench.WORKLOAD), world, rank)
        bench.barrier(world)
        out.put((rank, slowest, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [15.0, 15.0]  # both ranks see the maximum
    assert got[1][2] == ""  # rank 1 prints nothing in the reference arm


def test_reference_line_on_rank_0(orc):
    import bench

    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(argparse.Namespace(steps=1, warmup=0, workload=bench.WORKLOAD), 1, 0)
    lines = [ln for ln in buf.getvalue().splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "particles/s"
    assert d["higher_is_better"] is True and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(1, 3.5) == 3.5
    bench.barrier(1)
