"""Placement of a batch's graphs on several GPUs: longest-processing-time-first list scheduling
(Graham, 1969) against exhaustive search, and the bench's shards on two gloo ranks (CPU)."""
import itertools
import os
import socket
import sys

import numpy as np
import pytest

from paper_1502_07451_b300 import gen, shard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_lpt_places_every_item_once_and_within_graham_bound():
    rng = np.random.default_rng(5)
    for trial in range(60):
        n = int(rng.integers(1, 10))
        m = int(rng.integers(1, 4))
        w = [int(x) for x in rng.integers(1, 100, n)]
        parts = shard.lpt(w, m)
        assert sorted(i for p in parts for i in p) == list(range(n))
        assert all(p == sorted(p) for p in parts)
        loads = [sum(w[i] for i in p) for p in parts]
        best = min(max(sum(w[i] for i in range(n) if a[i] == q) for q in range(m))
                   for a in itertools.product(range(m), repeat=n))
        assert max(loads) * 3 * m <= best * (4 * m - 1)  # LPT <= (4/3 - 1/(3m)) OPT
        assert shard.lpt(w, m) == parts  # deterministic: every rank computes the same placement


def test_lpt_edge_cases():
    assert shard.lpt([], 3) == [[], [], []]
    assert shard.lpt([5, 5, 5], 1) == [[0, 1, 2]]
    assert shard.lpt([7], 4) == [[0], [], [], []]
    assert shard.lpt([3, 3, 3, 3], 2) == [[0, 2], [1, 3]]  # ties: lowest index first, to the lowest part
    with pytest.raises(ValueError):
        shard.lpt([1], 0)


def test_spec_edge_counts_match_the_built_graphs():
    spec = gen.batch_spec(120)
    for it in spec[::7]:
        assert gen.spec_edges(it) == gen.build_from_spec(it)["m"], it


def test_batch_shards_cover_the_recipe_and_balance_edges():
    sys.path.insert(0, ROOT)
    import bench
    spec1, total1 = bench.batch_shard(512, 0, 1)
    assert spec1 == gen.batch_spec(512) and total1 == 512
    world = 3
    shards = [bench.batch_shard(512, r, world) for r in range(world)]
    allspec = gen.batch_spec(512 * world)
    got = sorted(it for s, _ in shards for it in s)
    assert got == sorted(allspec) and all(t == 512 * world for _, t in shards)
    loads = [sum(gen.spec_edges(it) for it in s) for s, _ in shards]
    assert max(loads) <= 1.01 * min(loads)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        spec, total = bench.batch_shard(300, rank, world)
        edges = sum(gen.spec_edges(it) for it in spec)
        slowest = bench.max_over_ranks(edges, world, device="cpu")  # stands in for the slowest rank's time
        out[rank] = ([tuple(x if not isinstance(x, tuple) else list(x) for x in it) for it in spec], total, edges,
                     slowest)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_disjoint_shards():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    seeds = [sorted(it[2] for it in res[r][0]) for r in range(world)]
    assert not set(seeds[0]) & set(seeds[1])
    assert sorted(seeds[0] + seeds[1]) == list(range(600))
    assert res[0][1] == res[1][1] == 600
    assert res[0][3] == res[1][3] == max(res[0][2], res[1][2])
