"""gp_graph_create_deferred: the levels are built beside the caller's next calls, and every result is
the one gp_graph_create gives (partition, trace, makespan, finish times, level export, batch and
network paths); a cycle is reported by each call that needs the levels."""
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


def run(g, deferred, seed=0):
    with gp.Graph(dgraph(g), deferred=deferred) as G:
        part = torch.empty(max(g["n"], 1), dtype=torch.uint8, device="cuda")
        res = G.partition(part, -1.0, 0.03, seed)
        tr = G.trace()
        fin = torch.empty(max(g["n"], 1), dtype=torch.int64, device="cuda")
        ms = G.makespan(part[: g["n"]], fin[: g["n"]]) if g["n"] else 0
        info = G.info()
        lv = torch.empty(max(g["n"], 1), dtype=torch.int32, device="cuda")
        if g["n"]:
            gp.gp_graph_export(G.h, level=lv)
        return (part.cpu().numpy()[: g["n"]], res, tr, ms, fin.cpu().numpy()[: g["n"]], info,
                lv.cpu().numpy()[: g["n"]])


@pytest.mark.parametrize("name", ["cholesky16", "layered", "random", "chain", "hub"])
def test_deferred_equals_immediate(name):
    g = {"cholesky16": lambda: gen.cholesky(16), "layered": lambda: gen.layered(60, 500, 200000, 3),
         "random": lambda: gen.random_dag(3000, 12000, 5),
         "chain": lambda: gen.from_edges(2000, [(i, i + 1) for i in range(1999)], [3] * 2000, [2] * 2000, [1] * 1999),
         "hub": lambda: gen.from_edges(1001, [(0, i) for i in range(1, 1001)], [10] * 1001, [5] * 1001, [1] * 1000)}[name]()
    a = run(g, False, seed=2)
    b = run(g, True, seed=2)
    assert np.array_equal(a[0], b[0]) and a[1] == b[1] and a[2] == b[2]
    assert a[3] == b[3] and np.array_equal(a[4], b[4]) and a[5] == b[5] and np.array_equal(a[6], b[6])
    lev, nl = oracle.levels(g)
    assert b[5]["nlevels"] == nl and np.array_equal(b[6], lev)
    assert b[3] == oracle.makespan(g, b[0])


def test_deferred_cycle_is_reported_by_every_level_reader():
    g = gen.from_edges(4, [(0, 1), (1, 2), (2, 1), (2, 3)], [1, 2, 3, 4], [1, 1, 1, 1], [1, 1, 1, 1])
    dg = dgraph(g)
    h = gp.gp_graph_create_deferred(g["n"], g["m"], *[dg[k] for k in KEYS])
    try:
        part = torch.empty(4, dtype=torch.uint8, device="cuda")
        with pytest.raises(gp.GpError) as e:
            gp.gp_partition(h, -1.0, 0.03, 0, part)
        assert e.value.status == gp.GP_ERR_NOT_DAG
        with pytest.raises(gp.GpError) as e:
            gp.gp_makespan(h, torch.zeros(4, dtype=torch.uint8, device="cuda"))
        assert e.value.status == gp.GP_ERR_NOT_DAG
        with pytest.raises(gp.GpError) as e:
            gp.gp_graph_info(h)
        assert e.value.status == gp.GP_ERR_NOT_DAG
    finally:
        gp.gp_graph_destroy(h)
    # a self-loop is found at creation, as gp_graph_create finds it
    g2 = gen.from_edges(3, [(0, 1), (1, 1), (1, 2)], [1, 1, 1], [1, 1, 1], [1, 1, 1])
    with pytest.raises(gp.GpError) as e:
        gp.Graph(dgraph(g2), deferred=True)
    assert e.value.status == gp.GP_ERR_NOT_DAG == oracle.validate(g2)


def test_deferred_empty_and_destroy_before_use():
    empty = gen.from_edges(0, [], [], [], [])
    with gp.Graph(empty, deferred=True) as G:
        assert G.info()["nlevels"] == 0
        assert G.makespan(np.zeros(1, np.uint8)) == 0
    g = gen.layered(200, 1000, 1_600_000, 9)
    dg = dgraph(g)
    for _ in range(3):  # destroyed while its levels may still be in flight
        h = gp.gp_graph_create_deferred(g["n"], g["m"], *[dg[k] for k in KEYS])
        gp.gp_graph_destroy(h)


def test_deferred_handles_in_batch_and_network_paths():
    graphs = [gen.cholesky(8), gen.layered(30, 200, 20000, 4), gen.random_dag(1500, 6000, 2)]
    imm = [gp.Graph(dgraph(g)) for g in graphs]
    dfr = [gp.Graph(dgraph(g), deferred=True) for g in graphs]
    try:
        outs = []
        for hs in (imm, dfr):
            parts = [torch.empty(g["n"], dtype=torch.uint8, device="cuda") for g in graphs]
            res = gp.gp_batch_partition([x.h for x in hs], parts, seeds=[1, 2, 3], makespans=True)
            outs.append(([p.cpu().numpy() for p in parts], res))
        assert all(np.array_equal(a, b) for a, b in zip(outs[0][0], outs[1][0]))
        strip = lambda rs: [{k: v for k, v in r.items() if k != "ms"} for r in rs]  # timings differ
        assert strip(outs[0][1][0]) == strip(outs[1][1][0]) and outs[0][1][1] == outs[1][1][1]
        model = gp.gp_model_create(3)
        try:
            la = [torch.empty(g["n"], dtype=torch.float32, device="cuda") for g in graphs]
            lb = [torch.empty(g["n"], dtype=torch.float32, device="cuda") for g in graphs]
            for x, y, a, b in zip(imm, dfr, la, lb):
                gp.gp_model_forward(model, x.h, a)
                gp.gp_model_forward(model, y.h, b)
                assert torch.equal(a, b)
        finally:
            gp.gp_model_destroy(model)
    finally:
        for x in imm + dfr:
            x.close()


def test_deferred_network_right_after_creation():
    """The network sorts the in-rows in place; on a deferred handle it must first wait for the level
    work that reads them: logits and the learned split equal those of a synchronous handle."""
    g = gen.layered(200, 1000, 1_600_000, 11)
    model = gp.gp_model_create(5)
    try:
        outs = []
        for deferred in (False, True):
            with gp.Graph(dgraph(g), deferred=deferred) as G:
                logits = torch.empty(g["n"], dtype=torch.float32, device="cuda")
                gp.gp_model_forward(model, G.h, logits)
                part = torch.empty(g["n"], dtype=torch.uint8, device="cuda")
                res = gp.gp_partition_learned(G.h, model, part)
                fin = torch.empty(g["n"], dtype=torch.int64, device="cuda")
                ms = gp.gp_makespan(G.h, part, fin)
                outs.append((logits.cpu(), part.cpu().numpy(), {k: v for k, v in res.items() if k != "ms"}, ms,
                             fin.cpu().numpy()))
        a, b = outs
        assert torch.equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2] and a[3] == b[3]
        assert np.array_equal(a[4], b[4])
    finally:
        gp.gp_model_destroy(model)
