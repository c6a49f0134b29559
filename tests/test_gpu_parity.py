"""Parity of the CUDA path with the CPU oracle (bit-exact: every quantity is an integer).

Each step is compared on identical seeded inputs, then the whole
bipartitioner and the makespan on workloads that span several tiles and
ragged tails, degenerate graphs, long rows (all three row-merge tiers), and
the full-size layered DAG the benchmark times.  All calls go through the C-ABI.
"""
import json
import os

import numpy as np
import pytest

import oracle
import paper_1502_07451_b300 as gp
from paper_1502_07451_b300 import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def dev(a, dtype=None):
    a = np.ascontiguousarray(a if dtype is None else np.asarray(a, dtype=dtype))
    return torch.from_numpy(a).cuda()


def host(t):
    return t.cpu().numpy()


def dgraph(g):
    return {k: (dev(v) if isinstance(v, np.ndarray) and k in ("offsets", "cols", "edge_cost", "cpu_cost", "gpu_cost")
                else v) for k, v in g.items()}


def ucsr(n, edges):
    rows = [dict() for _ in range(n)]
    for u, v, w in edges:
        rows[u][v] = rows[u].get(v, 0) + w
        rows[v][u] = rows[v].get(u, 0) + w
    off = np.zeros(n + 1, np.int64)
    adj, W = [], []
    for v in range(n):
        for u in sorted(rows[v]):
            adj.append(u)
            W.append(rows[v][u])
        off[v + 1] = len(adj)
    return off, np.array(adj, np.int32), np.array(W, np.int64)


def gpu_partition(g, r_cpu=-1.0, tol=0.03, seed=0):
    with gp.Graph(dgraph(g)) as G:
        part = torch.empty(max(g["n"], 1), dtype=torch.uint8, device="cuda")
        res = G.partition(part, r_cpu, tol, seed)
        tr = G.trace()
        ms = G.makespan(part[: g["n"]]) if g["n"] else 0
        return host(part)[: g["n"]], res, tr, ms


FIXTURES = {
    "cholesky16": lambda: gen.cholesky(16),
    "cholesky4": lambda: gen.cholesky(4),
    "lu10": lambda: gen.lu(10),
    "two_input38": lambda: gen.two_input_dag(38, 3, extra=2),
    "random2k": lambda: gen.random_dag(2000, 9000, 5),
    "random300_dense": lambda: gen.random_dag(300, 12000, 6),
    "layered_small": lambda: gen.layered(40, 150, 40000, 7),
    "hub1000": lambda: gen.from_edges(1001, [(0, i) for i in range(1, 1001)], [10] * 1001, [5] * 1001, [1] * 1000),
}


# ---------------------------------------------------------------------------
# graph creation: symmetrisation and topological levels
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", sorted(FIXTURES))
def test_create_matches_oracle(name):
    g = FIXTURES[name]()
    off, adj, W = oracle.symmetrize(g)
    lev, nl = oracle.levels(g)
    with gp.Graph(dgraph(g)) as G:
        info = G.info()
        assert info["a0"] == len(adj) and info["nlevels"] == nl
        assert info["sum_cpu"] == int(g["cpu_cost"].sum()) and info["sum_gpu"] == int(g["gpu_cost"].sum())
        o = torch.empty(g["n"] + 1, dtype=torch.int64, device="cuda")
        a = torch.empty(max(len(adj), 1), dtype=torch.int32, device="cuda")
        w = torch.empty(max(len(adj), 1), dtype=torch.int64, device="cuda")
        lv = torch.empty(max(g["n"], 1), dtype=torch.int32, device="cuda")
        gp.gp_graph_export(G.h, o, a, w, lv)
        assert np.array_equal(host(o), off)
        assert np.array_equal(host(a)[: len(adj)], adj)
        assert np.array_equal(host(w)[: len(adj)], W)
        assert np.array_equal(host(lv)[: g["n"]], lev)


def test_create_is_repeatable():
    """Graph creation runs a cooperative kernel with grid barriers; repeated runs must agree."""
    for name in ("random2k", "layered_small", "cholesky16"):
        g = FIXTURES[name]()
        lev, nl = oracle.levels(g)
        for _ in range(12):
            with gp.Graph(dgraph(g)) as G:
                assert G.info()["nlevels"] == nl
                lv = torch.empty(g["n"], dtype=torch.int32, device="cuda")
                gp.gp_graph_export(G.h, level=lv)
                assert np.array_equal(host(lv), lev)


def test_levels_from_one_cta_to_the_cluster():
    """Kahn's levels: narrow levels in one CTA, then a 6,000-wide level where the cluster kernel takes
    over (its frontier records partly beyond the CTA's shared-memory capacity, read back from global
    memory), a 10,000-wide level and narrow levels after it; levels, partition and makespan against
    the oracle."""
    edges = [(i, i + 1) for i in range(9)]
    a0, na = 10, 6000
    c = a0 + na
    d0, nd = c + 1, 10000
    e = d0 + nd
    edges += [(9, a0 + j) for j in range(na)] + [(a0 + j, c) for j in range(na)]
    edges += [(c, d0 + j) for j in range(nd)] + [(d0 + j, e) for j in range(nd)] + [(e, e + 1), (e + 1, e + 2)]
    n = e + 3
    rng = np.random.default_rng(17)
    g = gen.from_edges(n, edges, rng.integers(1, 1000, n).tolist(), rng.integers(1, 1000, n).tolist(),
                       rng.integers(1, 100, len(edges)).tolist())
    lev, nl = oracle.levels(g)
    with gp.Graph(dgraph(g)) as G:
        assert G.info()["nlevels"] == nl == 16
        lv = torch.empty(n, dtype=torch.int32, device="cuda")
        gp.gp_graph_export(G.h, level=lv)
        assert np.array_equal(host(lv), lev)
    part, res, tr, ms = gpu_partition(g, seed=2)
    opart, ores = oracle.partition(g, seed=2)
    assert np.array_equal(part, opart) and {k: res[k] for k in ores} == ores
    assert ms == oracle.makespan(g, opart)


def test_long_rows_use_every_merge_tier():
    """Rows of <= 256 (warp), <= 8192 (block) and > 8192 raw entries (radix tier), with parallel edges."""
    k = 20000
    edges = [(0, i) for i in range(1, k)] + [(0, i) for i in range(1, 3000)] + [(i, k) for i in range(1, 600)]
    w = [1 + (i * 7919) % 1000 for i in range(len(edges))]
    g = gen.from_edges(k + 1, edges, [3] * (k + 1), [2] * (k + 1), w)
    off, adj, W = oracle.symmetrize(g)
    with gp.Graph(dgraph(g)) as G:
        o = torch.empty(g["n"] + 1, dtype=torch.int64, device="cuda")
        a = torch.empty(len(adj), dtype=torch.int32, device="cuda")
        ww = torch.empty(len(adj), dtype=torch.int64, device="cuda")
        gp.gp_graph_export(G.h, o, a, ww)
        assert np.array_equal(host(o), off) and np.array_equal(host(a), adj) and np.array_equal(host(ww), W)
    part, res, tr, ms = gpu_partition(g, seed=3)
    opart, ores, otr = oracle.partition(g, seed=3, trace=True)
    assert np.array_equal(part, opart)
    assert {k: res[k] for k in ores} == ores
    assert ms == oracle.makespan(g, opart)


# ---------------------------------------------------------------------------
# step parity
# ---------------------------------------------------------------------------

def level_graphs():
    """(name, n, off, adj, W, vC, vG, BC, BG) level graphs: level 0 of several DAGs and coarse levels."""
    out = []
    for name in ("cholesky16", "random2k", "layered_small", "random300_dense"):
        g = FIXTURES[name]()
        off, adj, W = oracle.symmetrize(g)
        vC, vG = g["cpu_cost"].astype(np.int64), g["gpu_cost"].astype(np.int64)
        BC, BG = oracle.bounds(int(vC.sum()), int(vG.sum()))
        n = g["n"]
        out.append((name + "_l0", n, off, adj, W, vC, vG, BC, BG))
        for lvl in range(1, 3):
            m = oracle.match(n, off, adj, W, vC, vG, BC // 8, BG // 8, 0)
            m = oracle.match_twohop(n, off, adj, W, vC, vG, BC // 8, BG // 8, 0, m)
            cmap, off, adj, W, vC, vG = oracle.contract(n, off, adj, W, vC, vG, m)
            n = len(off) - 1
            out.append((name + "_l%d" % lvl, n, off, adj, W, vC, vG, BC, BG))
    return out


LEVELS = level_graphs()


@pytest.mark.parametrize("lv", LEVELS, ids=[x[0] for x in LEVELS])
def test_step_match_and_contract(lv):
    name, n, off, adj, W, vC, vG, BC, BG = lv
    d = [dev(off), dev(adj), dev(W), dev(vC), dev(vG)]
    for seed in (0, 17):
        # (two-hop pairing anchors the vertices the last round's confirm lists; with 0 rounds the anchor
        # pass runs over every vertex, with 1 the first round's confirm writes that list)
        for rounds, twohop in ((1, 0), (4, 0), (4, 1), (0, 1), (1, 1), (2, 1)):
            mate = torch.empty(n, dtype=torch.int32, device="cuda")
            gp.gp_step_match(n, *d, BC // 8, BG // 8, seed, rounds, twohop, mate)
            want = oracle.match(n, off, adj, W, vC, vG, BC // 8, BG // 8, seed, rounds)
            if twohop:
                want = oracle.match_twohop(n, off, adj, W, vC, vG, BC // 8, BG // 8, seed, want)
            assert np.array_equal(host(mate), want), (name, seed, rounds, twohop)
        cmap = torch.empty(n, dtype=torch.int32, device="cuda")
        coff = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        cadj = torch.empty(max(len(adj), 1), dtype=torch.int32, device="cuda")
        cW = torch.empty(max(len(adj), 1), dtype=torch.int64, device="cuda")
        cvC = torch.empty(n, dtype=torch.int64, device="cuda")
        cvG = torch.empty(n, dtype=torch.int64, device="cuda")
        nc, ac = gp.gp_step_contract(n, *d, mate, cmap, coff, cadj, cW, cvC, cvG)
        ocmap, ocoff, ocadj, ocW, ocvC, ocvG = oracle.contract(n, off, adj, W, vC, vG, want)
        assert nc == len(ocoff) - 1 and ac == len(ocadj)
        assert np.array_equal(host(cmap), ocmap)
        assert np.array_equal(host(coff)[: nc + 1], ocoff)
        # coarse rows are sets: compare each row sorted by neighbour
        ga, gw = host(cadj)[:ac], host(cW)[:ac]
        for c in range(nc):
            lo, hi = ocoff[c], ocoff[c + 1]
            o = np.argsort(ga[lo:hi], kind="stable")
            assert np.array_equal(ga[lo:hi][o], ocadj[lo:hi]) and np.array_equal(gw[lo:hi][o], ocW[lo:hi])
        assert np.array_equal(host(cvC)[:nc], ocvC) and np.array_equal(host(cvG)[:nc], ocvG)


@pytest.mark.parametrize("lv", [x for x in LEVELS if x[1] <= 3000], ids=[x[0] for x in LEVELS if x[1] <= 3000])
def test_step_gggp(lv):
    name, n, off, adj, W, vC, vG, BC, BG = lv
    d = [dev(off), dev(adj), dev(W), dev(vC), dev(vG)]
    for seed in (0, 5, 99):
        for bc, bg in ((BC, BG), (BC // 2, BG), (BC * 2, BG // 3)):
            part = torch.empty(n, dtype=torch.uint8, device="cuda")
            t = gp.gp_step_gggp(n, *d, bc, bg, seed, part)
            op, ot = oracle.gggp(n, off, adj, W, vC, vG, bc, bg, seed)
            assert t == ot and np.array_equal(host(part), op), (name, seed, bc, bg)
    for start in range(0, n, max(1, n // 7)):
        part = torch.empty(n, dtype=torch.uint8, device="cuda")
        cut = gp.gp_step_gggp_grow(n, *d, BC, BG, start, part)
        op, oc = oracle.gggp_grow(n, off, adj, W, vC, vG, BC, BG, start)
        assert cut == oc and np.array_equal(host(part), op), (name, start)


@pytest.mark.parametrize("lv", LEVELS, ids=[x[0] for x in LEVELS])
def test_step_refine(lv):
    name, n, off, adj, W, vC, vG, BC, BG = lv
    d = [dev(off), dev(adj), dev(W), dev(vC), dev(vG)]
    rng = np.random.default_rng(n)
    starts = [rng.integers(0, 2, n).astype(np.uint8), np.zeros(n, np.uint8), np.ones(n, np.uint8)]
    p0, _ = oracle.gggp(n, off, adj, W, vC, vG, BC, BG, 0)
    starts.append(p0)
    for i, p in enumerate(starts):
        for bc, bg in ((BC, BG), (BC + BC // 4, BG // 2)):
            part = dev(p)
            st = gp.gp_step_refine(n, *d, bc, bg, part)
            op, ost = oracle.refine(n, off, adj, W, vC, vG, bc, bg, p)
            assert np.array_equal(host(part), op), (name, i, bc, bg)
            assert st == ost, (name, i, st, ost)


def test_hand_examples_on_gpu():
    ex = json.load(open(os.path.join(GOLD, "hand_examples.json")))
    for e in ex["match"]:
        off, adj, W = ucsr(e["n"], e["edges"])
        mate = torch.empty(e["n"], dtype=torch.int32, device="cuda")
        gp.gp_step_match(e["n"], dev(off), dev(adj), dev(W), dev(e["vC"], np.int64), dev(e["vG"], np.int64),
                         e["cap_cpu"], e["cap_gpu"], 0, 4, 1, mate)
        assert host(mate).tolist() == e["mate"], e["name"]
    for e in ex["refine"]:
        off, adj, W = ucsr(e["n"], e["edges"])
        part = dev(np.array(e["part_in"], np.uint8))
        st = gp.gp_step_refine(e["n"], dev(off), dev(adj), dev(W), dev(e["vC"], np.int64), dev(e["vG"], np.int64),
                               e["bound_cpu"], e["bound_gpu"], part)
        assert host(part).tolist() == e["part_out"], e["name"]
        assert (st["rounds"], st["moves"], st["balanced"], st["bal_moves"]) == \
            (e["rounds"], e["moves"], e["balanced"], e["bal_moves"]), e["name"]
    for e in ex["gggp_grow"]:
        off, adj, W = ucsr(e["n"], e["edges"])
        for start, want in e["starts"].items():
            part = torch.empty(e["n"], dtype=torch.uint8, device="cuda")
            cut = gp.gp_step_gggp_grow(e["n"], dev(off), dev(adj), dev(W), dev(e["vC"], np.int64),
                                       dev(e["vG"], np.int64), e["bound_cpu"], e["bound_gpu"], int(start), part)
            assert host(part).tolist() == want["part"] and cut == want["cut"]
    for e in ex["makespan"]:
        g = gen.from_edges(e["n"], e["edges"], e["cpu"], e["gpu"], e["w"])
        with gp.Graph(dgraph(g)) as G:
            for c in e["cases"]:
                fin = torch.empty(e["n"], dtype=torch.int64, device="cuda")
                assert G.makespan(dev(np.array(c["part"], np.uint8)), fin) == c["makespan"]
                assert host(fin).tolist() == c["finish"]


# ---------------------------------------------------------------------------
# whole path
# ---------------------------------------------------------------------------

CASES = [("cholesky16", -1.0, 0.03, 0), ("cholesky16", 0.3, 0.03, 1), ("cholesky4", -1.0, 0.03, 2),
         ("lu10", -1.0, 0.05, 3), ("two_input38", -1.0, 0.03, 4), ("random2k", -1.0, 0.03, 5),
         ("random2k", 0.6, 0.01, 6), ("random300_dense", -1.0, 0.1, 7), ("layered_small", -1.0, 0.03, 8),
         ("layered_small", 0.0, 0.03, 9), ("layered_small", 1.0, 0.03, 10), ("hub1000", -1.0, 0.03, 11)]


@pytest.mark.parametrize("case", CASES, ids=["%s-r%s-t%s-s%d" % c for c in CASES])
def test_partition_and_makespan_parity(case):
    name, r, tol, seed = case
    g = FIXTURES[name]()
    part, res, tr, ms = gpu_partition(g, r, tol, seed)
    opart, ores, otr = oracle.partition(g, r, tol, seed, trace=True)
    assert np.array_equal(part, opart)
    assert {k: res[k] for k in ores} == ores
    for k in ("levels", "gggp_trial", "n", "a", "rounds", "moves", "balanced", "bal_moves"):
        assert tr[k] == otr[k], k
    oms, ofin = oracle.makespan(g, opart, with_finish=True)
    assert ms == oms
    with gp.Graph(dgraph(g)) as G:
        fin = torch.empty(g["n"], dtype=torch.int64, device="cuda")
        assert G.makespan(dev(opart), fin) == oms
        assert np.array_equal(host(fin), ofin)
        assert G.cut(dev(opart)) == oracle.cut(g, opart)


def test_makespan_random_mappings():
    for seed in range(6):
        g = gen.random_dag(3000 + 17 * seed, 12000, seed)
        rng = np.random.default_rng(seed)
        with gp.Graph(dgraph(g)) as G:
            for _ in range(3):
                p = rng.integers(0, 2, g["n"]).astype(np.uint8)
                fin = torch.empty(g["n"], dtype=torch.int64, device="cuda")
                ms = G.makespan(dev(p), fin)
                oms, ofin = oracle.makespan(g, p, with_finish=True)
                assert ms == oms and np.array_equal(host(fin), ofin)


def _long_range_chain(n, stride, seed):
    """A chain 0 -> 1 -> ... -> n-1 (one vertex per level) with extra edges from every stride-th
    vertex to vertices 9,000 to 11,000 positions later: predecessors further back than any ring."""
    rng = np.random.default_rng(seed)
    edges = [(i, i + 1) for i in range(n - 1)]
    for u in range(0, n - 11000, stride):
        edges.append((u, u + int(rng.integers(9000, 11000))))
    ne = len(edges)
    return gen.from_edges(n, edges, rng.integers(1, 1000, n).tolist(), rng.integers(1, 1000, n).tolist(),
                          rng.integers(1, 5000, ne).tolist())


def test_makespan_kernels_agree_with_oracle():
    """Every makespan kernel against the oracle (by default: the cluster kernel with a distributed-
    shared-memory ring of recent finish times, exchanged by st.async, where every level fits it; a
    cooperative grid with its own bounded grid barrier where levels are wider than a cluster's groups;
    GP_MAKESPAN_KERNEL=cluster: one cluster reading every predecessor from global memory) on graphs that
    reach each branch: levels narrow enough for the ring, levels too wide for it, predecessors beyond
    the ring, one-vertex levels, several lanes per vertex, levels wider than the groups."""
    graphs = [gen.layered(30, 1000, 240000, 1), gen.layered(12, 3000, 300000, 2), gen.layered(6, 5000, 200000, 9),
              gen.layered(5, 12000, 400000, 12),  # wider than the ring and a cluster's groups: the grid kernel
              gen.layered(4, 1500, 60000, 3), gen.random_dag(3000, 12000, 4), gen.random_dag(300, 12000, 6),
              _long_range_chain(30000, 97, 5), FIXTURES["hub1000"](), gen.cholesky(16)]
    old = os.environ.get("GP_MAKESPAN_KERNEL")
    try:
        for i, g in enumerate(graphs):
            rng = np.random.default_rng(100 + i)
            p = rng.integers(0, 2, g["n"]).astype(np.uint8)
            oms, ofin = oracle.makespan(g, p, with_finish=True)
            with gp.Graph(dgraph(g)) as G:
                for kern in ("default", "cluster"):
                    os.environ["GP_MAKESPAN_KERNEL"] = kern
                    fin = torch.empty(g["n"], dtype=torch.int64, device="cuda")
                    assert G.makespan(dev(p), fin) == oms, (i, kern)
                    assert np.array_equal(host(fin), ofin), (i, kern)
                    assert G.makespan(dev(p)) == oms, (i, kern)
    finally:
        if old is None:
            os.environ.pop("GP_MAKESPAN_KERNEL", None)
        else:
            os.environ["GP_MAKESPAN_KERNEL"] = old


def test_host_buffers_end_to_end():
    g = FIXTURES["random2k"]()
    with gp.Graph(g) as G:  # numpy inputs: host pointers
        part = np.zeros(g["n"], np.uint8)
        res = G.partition(part, -1.0, 0.03, 0)
        fin = np.zeros(g["n"], np.int64)
        ms = G.makespan(part, fin)
    opart, ores = oracle.partition(g)
    oms, ofin = oracle.makespan(g, opart, with_finish=True)
    assert np.array_equal(part, opart) and res["cut"] == ores["cut"]
    assert ms == oms and np.array_equal(fin, ofin)


def test_deterministic_repeat():
    g = FIXTURES["layered_small"]()
    a = gpu_partition(g, seed=4)
    b = gpu_partition(g, seed=4)
    assert np.array_equal(a[0], b[0]) and a[1]["cut"] == b[1]["cut"] and a[3] == b[3]


def test_degenerate_graphs():
    empty = gen.from_edges(0, [], [], [], [])
    with gp.Graph(empty) as G:
        res = G.partition(np.zeros(1, np.uint8))
        assert res["feasible"] == 1 and res["cut"] == 0
        assert G.makespan(np.zeros(1, np.uint8)) == 0
    for g in (gen.from_edges(1, [], [5], [3], []), gen.from_edges(3, [(0, 1), (1, 2)], [0, 0, 0], [0, 0, 0], [0, 0]),
              gen.from_edges(5, [], [4, 1, 7, 2, 9], [1, 1, 1, 1, 1], [])):
        part, res, tr, ms = gpu_partition(g)
        opart, ores = oracle.partition(g)
        assert np.array_equal(part, opart) and {k: res[k] for k in ores} == ores
        assert ms == oracle.makespan(g, opart)


def test_validation_status_matches_oracle():
    ok = gen.from_edges(3, [(0, 1), (1, 2)], [1, 1, 1], [1, 1, 1], [1, 1])

    def mod(**kw):
        g = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in ok.items()}
        g.update({k: np.asarray(v, dtype=ok[k].dtype) for k, v in kw.items()})
        return g

    bad = [mod(offsets=[0, 2, 1, 2]), mod(offsets=[1, 1, 2, 2]), mod(cols=[1, 3]), mod(cols=[1, -1]),
           mod(edge_cost=[1, -1]), mod(cpu_cost=[1, -1, 1]), mod(cols=[0, 2]),
           gen.from_edges(3, [(0, 1), (1, 2), (2, 0)], [1, 1, 1], [1, 1, 1], [1, 1, 1]),
           dict(gen.from_edges(3, [(0, 1), (1, 2), (2, 0)], [1, 1, 1], [1, 1, 1], [1, 1, 1]),
                edge_cost=np.array([1, -1, 1], np.int32))]
    for g in bad:
        want = oracle.validate(g)
        with pytest.raises(gp.GpError) as e:
            gp.Graph(dgraph(g))
        assert e.value.status == want
    with gp.Graph(dgraph(ok)) as G:
        with pytest.raises(gp.GpError) as e:
            G.makespan(dev(np.array([0, 2, 1], np.uint8)))
        assert e.value.status == gp.GP_ERR_INVALID
        with pytest.raises(gp.GpError):
            G.partition(torch.empty(3, dtype=torch.uint8, device="cuda"), r_cpu=1.5)


# ---------------------------------------------------------------------------
# the benchmark workload at full size
# ---------------------------------------------------------------------------

def test_full_size_layered_1m_bit_exact():
    """1,000 layers x 1,000 vertices, 8M edges: the whole path, as the benchmark runs it, against the
    oracle on the same input (partition, every result field, per-level trace, makespan, finish times)."""
    g = gen.config_layered_1m()
    part, res, tr, ms = gpu_partition(g)
    opart, ores, otr = oracle.partition(g, trace=True)
    assert np.array_equal(part, opart)
    assert {k: res[k] for k in ores} == ores
    assert tr["n"] == otr["n"] and tr["a"] == otr["a"] and tr["rounds"] == otr["rounds"]
    assert ms == oracle.makespan(g, opart)
