"""Host logic of the multi-GPU path (replicas only): two gloo ranks on the CPU.

bench.py under torchrun runs one independent replica per GPU.  The only collectives are the barrier
and the maximum over ranks of the timed region; the job's throughput is the units all ranks processed
over that maximum.  This test runs world_size 2 with the gloo backend on 127.0.0.1 and checks:
- max_over_ranks gives every rank the slowest rank's time;
- job_rate counts the units of all ranks;
- the reference arm does its work and prints on rank 0 only (the other ranks return at once).
"""
import io
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


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [1.25, 2.5][rank]
        slowest = bench.max_over_ranks(dist, mine, device="cpu")
        dist.barrier()
        rate = bench.job_rate(world, 1000, slowest)
        # the reference arm: rank 1 returns without work or output
        buf = io.StringIO()
        args = type("A", (), dict(workload="small", steps=1, warmup=0))()
        if rank == 1:
            with redirect_stdout(buf):
                bench.run_reference(args)
        q.put((rank, slowest, rate, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2.5, 2.5]
    assert all(abs(o[2] - 2 * 1000 / 2.5) < 1e-9 for o in out)
    assert out[1][3] == ""  # rank 1 printed nothing


def test_oracle_pool_on_host_cores():
    """The CPU baseline's all-cores leg: spawned single-threaded processes time the oracle together and
    the step time is extrapolated from the slowest one."""
    sys.path.insert(0, ROOT)
    import bench
    pool = bench.OraclePool(procs=2)
    try:
        w = bench._workload("small")
        t, desc = pool.step(w, 256, 4096, seed=1)
    finally:
        pool.close()
    assert pool.procs == 2 and t > 0 and "2 single-threaded processes" in desc
