"""The batched path: many graphs in one persistent launch, every result equal to the
single-graph result and to the CPU oracle (bit-exact), for every schedule.

Inputs are the mixed batch recipe (tiled Cholesky, tiled LU, layered random DAGs of
log-uniform size), plus degenerate graphs.  All calls go through the C-ABI.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import paper_1502_07451_b300 as gp
from paper_1502_07451_b300 import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
RES_KEYS = ("cut", "load_cpu", "load_gpu", "bound_cpu", "bound_gpu", "feasible", "levels", "rounds", "coarsest_n")


def dgraph(g):
    return {k: (torch.from_numpy(np.ascontiguousarray(v)).cuda()
                if isinstance(v, np.ndarray) and k in ("offsets", "cols", "edge_cost", "cpu_cost", "gpu_cost")
                else v) for k, v in g.items()}


def mixed(count, nmax, seed=0):
    return [gen.build_from_spec(it) for it in gen.batch_spec(count, nmin=100, nmax=nmax, base_seed=seed)]


def run_batch(graphs, r_cpu=None, seeds=None, tol=0.03, host_parts=False, makespans=True):
    Gs = [gp.Graph(dgraph(g)) for g in graphs]
    try:
        if host_parts:
            parts = [np.zeros(max(g["n"], 1), np.uint8) for g in graphs]
        else:
            parts = [torch.zeros(max(g["n"], 1), dtype=torch.uint8, device="cuda") for g in graphs]
        res, ms = gp.gp_batch_partition([G.h for G in Gs], parts, r_cpu=r_cpu, tol=tol, seeds=seeds,
                                        makespans=makespans)
        out = [(p if host_parts else p.cpu().numpy())[: g["n"]].copy() for p, g in zip(parts, graphs)]
        return out, res, ms
    finally:
        for G in Gs:
            G.close()


def check_oracle(graphs, parts, res, ms, r_cpu=None, seeds=None, tol=0.03):
    for i, g in enumerate(graphs):
        r = -1.0 if r_cpu is None else r_cpu[i]
        s = 0 if seeds is None else seeds[i]
        p_ref, res_ref = oracle.partition(g, r, tol, s)
        assert np.array_equal(parts[i], p_ref[: g["n"]]), "graph %d split" % i
        for k in RES_KEYS:
            assert res[i][k] == res_ref[k], "graph %d %s: %d vs %d" % (i, k, res[i][k], res_ref[k])
        if ms is not None:
            assert ms[i] == oracle.makespan(g, p_ref), "graph %d makespan" % i


def test_mixed_batch_matches_oracle():
    graphs = mixed(40, 8000, seed=3)
    parts, res, ms = run_batch(graphs)
    check_oracle(graphs, parts, res, ms)


def test_batch_per_graph_ratio_and_seed():
    graphs = mixed(24, 4000, seed=11)
    r_cpu = [-1.0 if i % 3 == 0 else (0.05 * (i % 19)) for i in range(len(graphs))]
    seeds = [i * 7919 + 5 for i in range(len(graphs))]
    parts, res, ms = run_batch(graphs, r_cpu=r_cpu, seeds=seeds, tol=0.05)
    check_oracle(graphs, parts, res, ms, r_cpu=r_cpu, seeds=seeds, tol=0.05)


def test_batch_host_buffers_and_no_makespan():
    graphs = mixed(12, 3000, seed=5)
    parts, res, ms = run_batch(graphs, host_parts=True, makespans=False)
    assert ms is None
    check_oracle(graphs, parts, res, None)


def test_batch_degenerate_graphs():
    graphs = [
        gen.from_edges(0, [], [], [], []),
        gen.from_edges(1, [], [7], [3], []),
        gen.from_edges(2, [(0, 1)], [5, 5], [1, 1], [4]),
        gen.cholesky(4),                        # 20 tasks: no coarsening at all
        gen.two_input_dag(38, 3, extra=2),
        gen.from_edges(1001, [(0, i) for i in range(1, 1001)], [10] * 1001, [5] * 1001, [1] * 1000),  # hub
        gen.random_dag(300, 12000, 6),         # dense rows: the block-wide merge tiers
        gen.layered(30, 200, 30000, 9),
    ]
    # r_cpu 0: all-GPU without trials; 1: everything must leave the GPU
    r_cpu = [-1.0, -1.0, 0.0, 1.0, -1.0, -1.0, 0.3, -1.0]
    parts, res, ms = run_batch(graphs, r_cpu=r_cpu)
    check_oracle(graphs, parts, res, ms, r_cpu=r_cpu)


def test_schedules_leave_results_unchanged():
    graphs = mixed(30, 6000, seed=21)
    ref = run_batch(graphs)
    try:
        for i in range(gp.gp_batch_schedule_count()):
            gp.gp_batch_set_schedule(i)
            parts, res, ms = run_batch(graphs)
            for a, b in zip(parts, ref[0]):
                assert np.array_equal(a, b), gp.gp_batch_schedule_name(i)
            assert [{k: r[k] for k in RES_KEYS} for r in res] == [{k: r[k] for k in RES_KEYS} for r in ref[1]]
            assert ms == ref[2]
    finally:
        gp.gp_batch_set_schedule(-1)
    check_oracle(graphs, *ref)


def test_autotune_picks_a_schedule():
    graphs = mixed(16, 3000, seed=2)
    Gs = [gp.Graph(dgraph(g)) for g in graphs]
    try:
        best, ms = gp.gp_batch_autotune([G.h for G in Gs])
        assert 0 <= best < gp.gp_batch_schedule_count()
        assert len(ms) == gp.gp_batch_schedule_count() and all(t > 0 for t in ms)
        assert ms[best] == min(ms)
    finally:
        for G in Gs:
            G.close()
    parts, res, msp = run_batch(graphs)  # the tuned schedule gives the same results
    check_oracle(graphs, parts, res, msp)


def test_batch_equals_single_graph_path():
    graphs = mixed(20, 12000, seed=8)
    parts, res, ms = run_batch(graphs)
    for i, g in enumerate(graphs):
        with gp.Graph(dgraph(g)) as G:
            p = torch.zeros(max(g["n"], 1), dtype=torch.uint8, device="cuda")
            r = G.partition(p, -1.0, 0.03, 0)
            assert np.array_equal(p.cpu().numpy()[: g["n"]], parts[i])
            for k in RES_KEYS:
                assert r[k] == res[i][k]
            assert G.makespan(p[: g["n"]]) == ms[i]


def test_deferred_graphs_keep_their_results():
    """A workspace too small for the larger graphs: they are deferred to the single-graph path
    inside the same call, with unchanged results."""
    code = r'''
import sys, json
sys.path.insert(0, %r)
sys.path.insert(0, %r)
import numpy as np, torch
import paper_1502_07451_b300 as gp
from paper_1502_07451_b300 import gen
import oracle
graphs = [gen.build_from_spec(it) for it in gen.batch_spec(10, nmin=200, nmax=5000, base_seed=4)]
Gs = [gp.Graph({k: (torch.from_numpy(np.ascontiguousarray(v)).cuda() if isinstance(v, np.ndarray) and k in
       ("offsets", "cols", "edge_cost", "cpu_cost", "gpu_cost") else v) for k, v in g.items()}) for g in graphs]
parts = [torch.zeros(g["n"], dtype=torch.uint8, device="cuda") for g in graphs]
res, ms = gp.gp_batch_partition([G.h for G in Gs], parts, makespans=True)
bad = 0
for i, g in enumerate(graphs):
    p_ref, r_ref = oracle.partition(g)
    bad += int(not np.array_equal(parts[i].cpu().numpy(), p_ref))
    bad += int(res[i]["cut"] != r_ref["cut"]) + int(ms[i] != oracle.makespan(g, p_ref))
print(json.dumps({"bad": bad}))
''' % (ROOT, os.path.join(ROOT, "tests"))
    env = dict(os.environ, GP_BATCH_SLOT_LIMIT="600000")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    assert '"bad": 0' in out.stdout


def test_batch_invalid_arguments():
    g = gen.cholesky(5)
    with gp.Graph(dgraph(g)) as G:
        p = torch.zeros(g["n"], dtype=torch.uint8, device="cuda")
        for kw in [dict(tol=-0.1), dict(tol=1.5), dict(r_cpu=[1.5]), dict(r_cpu=[float("nan")])]:
            with pytest.raises(gp.GpError) as e:
                gp.gp_batch_partition([G.h], [p], **kw)
            assert e.value.status == gp.GP_ERR_INVALID
        with pytest.raises(gp.GpError):
            gp.gp_batch_partition([G.h], [None])
    L = gp.lib()
    assert L.gp_batch_partition(-1, None, None, 0.03, None, None, None, None, None) == gp.GP_ERR_INVALID
    assert L.gp_batch_partition(0, None, None, 0.03, None, None, None, None, None) == gp.GP_OK
    assert gp.lib().gp_batch_set_schedule(gp.gp_batch_schedule_count()) == gp.GP_ERR_INVALID


MODEL = os.path.join(ROOT, "paper_1502_07451_b300", "models", "mpnn3_h64.bin")


def test_batch_learned_equals_single_learned_and_oracle():
    """One network forward over the union of the graphs, then the persistent kernel in learned mode:
    every graph gets exactly gp_partition_learned's result, which is the oracle's given the logits."""
    graphs = mixed(24, 8000, seed=31) + [gen.cholesky(4), gen.from_edges(1, [], [7], [3], [])]
    r_cpu = [-1.0] * (len(graphs) - 3) + [0.2, 0.0, -1.0]
    model = gp.gp_model_load(MODEL)
    Gs = [gp.Graph(dgraph(g)) for g in graphs]
    try:
        parts = [torch.zeros(max(g["n"], 1), dtype=torch.uint8, device="cuda") for g in graphs]
        res, ms = gp.gp_batch_partition_learned([G.h for G in Gs], model, parts, r_cpu=r_cpu, makespans=True)
        for i, (g, G) in enumerate(zip(graphs, Gs)):
            n = g["n"]
            p1 = torch.zeros(max(n, 1), dtype=torch.uint8, device="cuda")
            r1 = gp.gp_partition_learned(G.h, model, p1, r_cpu=r_cpu[i])
            assert torch.equal(p1[:n], parts[i][:n]), i
            assert all(r1[k] == res[i][k] for k in RES_KEYS), i
            assert ms[i] == (G.makespan(p1[:n]) if n else 0)
            lg = torch.empty(max(n, 1), dtype=torch.float32, device="cuda")
            if n:
                gp.gp_model_forward(model, G.h, lg)
            op, orr = oracle.partition_learned(g, lg.cpu().numpy()[:n], r_cpu=r_cpu[i])
            assert np.array_equal(op, parts[i].cpu().numpy()[:n]), i
            assert all(orr[k] == res[i][k] for k in RES_KEYS), i
    finally:
        for G in Gs:
            G.close()
        gp.gp_model_destroy(model)


def test_batch_learned_host_buffers_and_schedules():
    graphs = mixed(10, 3000, seed=41)
    model = gp.gp_model_load(MODEL)
    Gs = [gp.Graph(dgraph(g)) for g in graphs]
    try:
        hp = [np.zeros(g["n"], np.uint8) for g in graphs]
        ref, _ = gp.gp_batch_partition_learned([G.h for G in Gs], model, hp)
        try:
            for si in range(gp.gp_batch_schedule_count()):
                gp.gp_batch_set_schedule(si)
                dp = [torch.zeros(g["n"], dtype=torch.uint8, device="cuda") for g in graphs]
                res, _ = gp.gp_batch_partition_learned([G.h for G in Gs], model, dp)
                for a, b in zip(hp, dp):
                    assert np.array_equal(a, b.cpu().numpy())
                assert [r["cut"] for r in res] == [r["cut"] for r in ref]
        finally:
            gp.gp_batch_set_schedule(-1)
    finally:
        for G in Gs:
            G.close()
        gp.gp_model_destroy(model)


def _export(h, g):
    n = g["n"]
    info = gp.gp_graph_info(h)
    o = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    a = torch.empty(max(info["a0"], 1), dtype=torch.int32, device="cuda")
    w = torch.empty(max(info["a0"], 1), dtype=torch.int64, device="cuda")
    lv = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    gp.gp_graph_export(h, o, a, w, lv)
    return info, o.cpu().numpy(), a.cpu().numpy()[:info["a0"]], w.cpu().numpy()[:info["a0"]], lv.cpu().numpy()[:n]


def _bad_graphs():
    ok = gen.cholesky(5)
    bad_col = dict(ok, cols=ok["cols"].copy())
    bad_col["cols"][3] = ok["n"] + 5
    neg_cost = dict(ok, cpu_cost=ok["cpu_cost"].copy())
    neg_cost["cpu_cost"][2] = -1
    cyclic = gen.from_edges(3, [(0, 1), (1, 2), (2, 0)], [1, 1, 1], [1, 1, 1], [1, 1, 1])
    selfloop = gen.from_edges(3, [(0, 1), (1, 1)], [1, 1, 1], [1, 1, 1], [1, 1])
    big = 2 ** 31 - 1
    overflow = gen.from_edges(3, [(0, 1)], [big, big, big], [1, 1, 1], [1])
    overflow2 = gen.from_edges(2 ** 9, [], [big] * (2 ** 9), [1] * (2 ** 9), [])
    bad_off = dict(ok, offsets=ok["offsets"].copy())
    bad_off["offsets"][4] = bad_off["offsets"][5] + 1
    return [bad_col, neg_cost, cyclic, selfloop, overflow, overflow2, bad_off]


@pytest.mark.parametrize("side", ["device", "host"])
def test_create_batch_equals_single_create(side):
    """Statuses, sums, levels, the symmetrised graph, and everything downstream (partition, makespan,
    the learned path) agree with gp_graph_create, DAG by DAG."""
    graphs = mixed(30, 12000, seed=51) + [gen.from_edges(0, [], [], [], []), gen.from_edges(1, [], [7], [3], []),
                                          gen.from_edges(1001, [(0, i) for i in range(1, 1001)], [10] * 1001,
                                                         [5] * 1001, [1] * 1000)] + _bad_graphs()
    src = [dgraph(g) for g in graphs] if side == "device" else graphs
    hs, sts = gp.gp_graph_create_batch(src)
    try:
        for i, g in enumerate(graphs):
            try:
                ref = gp.Graph(dgraph(g))
            except gp.GpError as e:
                assert sts[i] == e.status and hs[i] is None, i
                continue
            with ref:
                assert sts[i] == gp.GP_OK, (i, sts[i])
                ib, ob, ab, wb, lb = _export(hs[i], g)
                ir, orr, ar, wr, lr = _export(ref.h, g)
                assert ib == ir
                assert np.array_equal(ob, orr) and np.array_equal(ab, ar) and np.array_equal(wb, wr)
                assert np.array_equal(lb, lr)
                if g["n"] == 0:
                    continue
                p1 = torch.zeros(g["n"], dtype=torch.uint8, device="cuda")
                p2 = torch.zeros(g["n"], dtype=torch.uint8, device="cuda")
                r1 = gp.gp_partition(hs[i], -1.0, 0.03, 0, p1)
                r2 = ref.partition(p2)
                assert torch.equal(p1, p2) and all(r1[k] == r2[k] for k in RES_KEYS)
                assert gp.gp_makespan(hs[i], p1) == ref.makespan(p2)
    finally:
        for h in hs:
            if h is not None:
                gp.gp_graph_destroy(h)


def test_create_batch_handles_outlive_each_other():
    graphs = mixed(6, 2000, seed=61)
    hs, sts = gp.gp_graph_create_batch([dgraph(g) for g in graphs])
    assert all(st == gp.GP_OK for st in sts)
    # destroy every other handle; the rest stay usable (one shared block)
    for h in hs[::2]:
        gp.gp_graph_destroy(h)
    for i in range(1, len(graphs), 2):
        p = torch.zeros(graphs[i]["n"], dtype=torch.uint8, device="cuda")
        r = gp.gp_partition(hs[i], -1.0, 0.03, 0, p)
        op, orr = oracle.partition(graphs[i])
        assert np.array_equal(p.cpu().numpy(), op) and r["cut"] == orr["cut"]
        gp.gp_graph_destroy(hs[i])
