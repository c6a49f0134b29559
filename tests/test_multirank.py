"""The bench's multi-rank path on CPU: two gloo ranks (one process each, rendezvous on 127.0.0.1).
The single-DAG path runs one replica per rank, so what the ranks share is the timing: the slowest rank's
time and the whole-job rate over it; the reference arm runs on rank 0 only."""
import contextlib
import io
import os
import socket
import sys
import types

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local = 1.0 + rank  # rank r "took" 1 + r seconds
        slowest = bench.max_over_ranks(local, world, device="cpu")
        rate = bench.job_rate(100.0, world, slowest)
        # the reference arm: rank 0 alone runs (here with no steps), the others return at once, silent
        args = types.SimpleNamespace(workload="layered1m", steps=0, warmup=0)
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            if rank != 0:
                bench.run_reference(args, rank, world)
        dist.barrier()
        out[rank] = (slowest, rate, buf.getvalue())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        slowest, rate, printed = res[r]
        assert slowest == 2.0                 # max over ranks, the same on every rank
        assert rate == pytest.approx(100.0)   # 2 ranks x 100 units / 2 s
        assert printed == ""                  # rank 1's reference arm did nothing


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_rate(10.0, 1, 2.0) == 5.0
