"""The makespan on a fixed number of workers per side (gp_makespan_workers and its batched form)
against the oracle's list schedule: makespan and every finish time, bit-exact, through the C-ABI.

Cases: the testbed's 3 CPU + 1 GPU workers and other counts up to 32 workers, ties of ready time,
tasks of cost 0, parallel entries, hubs whose releases fill the waiting arrays, the splits the
partitioner gives and random ones, and the mixed batch in one launch."""
import numpy as np
import pytest

import oracle
import paper_1502_07451_b300 as gp
from paper_1502_07451_b300 import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("offsets", "cols", "edge_cost", "cpu_cost", "gpu_cost")


def dgraph(g):
    return {k: (torch.from_numpy(np.ascontiguousarray(v)).cuda() if k in KEYS else v) for k, v in g.items()}


def zero_cost_dag():
    rng = np.random.default_rng(5)
    n = 300
    edges = [(u, v) for u in range(n) for v in range(u + 1, min(n, u + 6)) if rng.random() < 0.5]
    edges += edges[:40]  # parallel entries
    cpu = rng.integers(0, 4, n).tolist()
    gpu = rng.integers(0, 3, n).tolist()
    return gen.from_edges(n, edges, cpu, gpu, rng.integers(0, 5, len(edges)).tolist())


FIXTURES = {
    "cholesky16": lambda: gen.cholesky(16),
    "lu10": lambda: gen.lu(10),
    "two_input38": lambda: gen.two_input_dag(38, 3, extra=2),
    "random2k": lambda: gen.random_dag(2000, 9000, 5),
    "layered_small": lambda: gen.layered(40, 150, 40000, 7),
    "hub1000": lambda: gen.from_edges(1001, [(0, i) for i in range(1, 1001)], [10] * 1001, [5] * 1001,
                                      list(range(1, 1001))),
    "zero_costs": zero_cost_dag,
}


@pytest.mark.parametrize("name", sorted(FIXTURES))
def test_makespan_workers_matches_oracle(name):
    g = FIXTURES[name]()
    n = g["n"]
    rng = np.random.default_rng(n)
    with gp.Graph(dgraph(g)) as G:
        split = torch.empty(n, dtype=torch.uint8, device="cuda")
        G.partition(split)
        parts = [split.cpu().numpy(), rng.integers(0, 2, n).astype(np.uint8), np.ones(n, np.uint8),
                 np.zeros(n, np.uint8)]
        for part in parts:
            dpart = torch.from_numpy(part).cuda()
            for pc, pg in ((3, 1), (1, 1), (8, 2), (16, 16), (31, 1)):
                fin = torch.full((n,), -1, dtype=torch.int64, device="cuda")
                ms = gp.gp_makespan_workers(G.h, dpart, pc, pg, fin)
                oms, ofin = oracle.makespan_workers(g, part, pc, pg, with_finish=True)
                assert ms == oms, (name, pc, pg)
                assert np.array_equal(fin.cpu().numpy(), ofin), (name, pc, pg)
        # host split and host finish buffer
        hf = np.zeros(n, np.int64)
        assert gp.gp_makespan_workers(G.h, parts[0], 3, 1, hf) == oracle.makespan_workers(g, parts[0], 3, 1)
        assert np.array_equal(hf, oracle.makespan_workers(g, parts[0], 3, 1, with_finish=True)[1])


def test_makespan_workers_hand_examples():
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "hand_examples.json")
    with open(path) as f:
        exs = json.load(f)["makespan_workers"]
    for ex in exs:
        g = gen.from_edges(ex["n"], ex["edges"], ex["cpu"], ex["gpu"], ex["w"])
        with gp.Graph(dgraph(g)) as G:
            fin = np.zeros(ex["n"], np.int64)
            ms = gp.gp_makespan_workers(G.h, np.array(ex["part"], np.uint8), ex["workers_cpu"], ex["workers_gpu"], fin)
            assert ms == ex["makespan"] and fin.tolist() == ex["finish"], ex["name"]


def test_makespan_workers_many_workers_is_the_longest_path():
    """16 + 16 workers on a DAG no level of which is wider than 16: the result is gp_makespan's."""
    g = gen.layered(30, 12, 900, 3)
    n = g["n"]
    part = np.random.default_rng(2).integers(0, 2, n).astype(np.uint8)
    with gp.Graph(dgraph(g)) as G:
        dpart = torch.from_numpy(part).cuda()
        assert gp.gp_makespan_workers(G.h, dpart, 16, 16) == G.makespan(dpart)


def test_batch_makespan_workers_matches_oracle():
    specs = gen.batch_spec(48, nmin=100, nmax=6000, base_seed=17)
    graphs = [gen.build_from_spec(it) for it in specs] + [gen.from_edges(0, [], [], [], []),
                                                           gen.from_edges(1, [], [7], [3], [])]
    Gs = [gp.Graph(dgraph(g)) for g in graphs]
    try:
        parts = [torch.zeros(max(g["n"], 1), dtype=torch.uint8, device="cuda") for g in graphs]
        gp.gp_batch_partition([G.h for G in Gs], parts)
        for pc, pg in ((3, 1), (2, 2)):
            got = gp.gp_batch_makespan_workers([G.h for G in Gs], parts, pc, pg)
            for i, g in enumerate(graphs):
                p = parts[i].cpu().numpy()[: g["n"]]
                assert got[i] == oracle.makespan_workers(g, p, pc, pg), (i, pc, pg)
                if g["n"]:
                    assert got[i] == gp.gp_makespan_workers(Gs[i].h, parts[i], pc, pg)
    finally:
        for G in Gs:
            G.close()


def test_makespan_workers_rejects_bad_arguments():
    g = gen.cholesky(4)
    with gp.Graph(dgraph(g)) as G:
        part = torch.zeros(g["n"], dtype=torch.uint8, device="cuda")
        for pc, pg in ((0, 1), (1, 0), (20, 13)):
            with pytest.raises(gp.GpError) as e:
                gp.gp_makespan_workers(G.h, part, pc, pg)
            assert e.value.status == gp.GP_ERR_INVALID
        part[2] = 2
        with pytest.raises(gp.GpError) as e:
            gp.gp_makespan_workers(G.h, part, 3, 1)
        assert e.value.status == gp.GP_ERR_INVALID
