"""Pins of the CPU oracle to things other than itself.

The oracle (oracle/) is the reference the CUDA path is checked against, so it
is first checked here against what the paper and the mathematics fix:
closed forms of Eq. (1)-(2) on the tiled-Cholesky workload, hand-worked
examples of every step, the published splitmix64 sequence behind the
tie-break hash, exhaustive search on tiny DAGs, path enumeration for the
makespan, and invariants of each step on random inputs.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import _brute
import _splitmix
from paper_1502_07451_b300 import gen

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def ucsr(n, edges):
    """Symmetric CSR (rows sorted by neighbour) from undirected [u, v, W] triples."""
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


def csr_edges(off, adj, W):
    """Undirected edge set {(min, max): W} of a symmetric CSR, checking symmetry."""
    out = {}
    n = len(off) - 1
    for v in range(n):
        for e in range(off[v], off[v + 1]):
            u = int(adj[e])
            key = (min(u, v), max(u, v))
            if key in out:
                assert out[key] == int(W[e]), "asymmetric weight"
            out[key] = int(W[e])
    return out


# ---------------------------------------------------------------------------
# Hash and closed forms
# ---------------------------------------------------------------------------

def test_splitmix_reference_sequence(oracle_mod):
    g = load("splitmix64_seed1234567.json")
    assert _splitmix.splitmix64_sequence(g["seed"], 5) == g["outputs"]
    s = g["seed"]
    for want in g["outputs"]:
        s = (s + 0x9E3779B97F4A7C15) & _splitmix.M64
        assert oracle_mod.mix64(s) == want


def test_edge_hash_definition(oracle_mod):
    rng = np.random.default_rng(1)
    for _ in range(200):
        seed = int(rng.integers(0, 2**63))
        a, b = (int(x) for x in rng.integers(0, 2**31, 2))
        assert oracle_mod.edge_hash(seed, a, b) == _splitmix.h(seed, a, b)


def test_cholesky16_closed_form(oracle_mod):
    cf = load("cholesky16_closed_form.json")
    g = gen.cholesky(16)
    assert (g["n"], g["m"]) == (cf["n"], cf["m"])
    for k in range(4):
        sel = g["task_kind"] == k
        assert set(g["cpu_cost"][sel].tolist()) == {cf["cpu_ns"][k]}
        assert set(g["gpu_cost"][sel].tolist()) == {cf["gpu_ns"][k]}
    assert set(g["edge_cost"].tolist()) == {cf["edge_ns"]}
    SC, SG = int(g["cpu_cost"].sum()), int(g["gpu_cost"].sum())
    assert (SC, SG) == (cf["sum_cpu"], cf["sum_gpu"])
    assert oracle_mod.bounds(SC, SG, -1.0, 0.03) == (cf["bound_cpu"], cf["bound_gpu"])
    assert oracle_mod.levels(g)[1] == cf["levels"]
    assert oracle_mod.makespan(g, np.ones(g["n"], np.uint8)) == cf["all_gpu_makespan"]


def test_task_counts_closed_form():
    for T in (2, 3, 4, 7, 16):
        assert gen.cholesky(T)["n"] == T + T * (T - 1) // 2 * 2 + T * (T - 1) * (T - 2) // 6
        assert gen.lu(T)["n"] == T + T * (T - 1) + sum((T - 1 - k) ** 2 for k in range(T))
    g4 = gen.cholesky(4)
    assert (g4["n"], g4["m"]) == (20, 30)
    assert gen.lu(16)["n"] == 1496


def test_bounds_eq1_eq2_exact_rationals(oracle_mod):
    """Eq. (1): R_CPU = T_GPU/(T_GPU+T_CPU); Eq. (2): R_GPU = 1 - R_CPU.
    Both sides' loads at those shares equal T* = SC*SG/(SC+SG); the bounds add
    the tolerance and round down.  Checked with exact rationals."""
    rng = np.random.default_rng(7)
    for _ in range(300):
        SC, SG = (int(x) for x in rng.integers(0, 2**50, 2))
        tol = float(rng.choice([0.0, 0.01, 0.03, 0.1, 0.5, 1.0]))
        if SC + SG == 0:
            continue
        r_cpu = Fraction(SG, SG + SC)
        r_gpu = 1 - r_cpu
        assert r_cpu * SC == r_gpu * SG
        tstar = int(np.floor(0)) + (r_cpu * SC).numerator // (r_cpu * SC).denominator
        want = (Fraction(tstar) * (1 + Fraction(round(tol * 1e6), 10**6))).__floor__()
        assert oracle_mod.bounds(SC, SG, -1.0, tol) == (want, want)


def test_bounds_explicit_ratio_matches_eq1(oracle_mod):
    """The explicit-ratio branch, fed Eq. (1)'s ratio, lands within the 2^-32
    quantisation of the Eq. (1) branch."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        SC, SG = (int(x) for x in rng.integers(1, 2**40, 2))
        bc, bg = oracle_mod.bounds(SC, SG, -1.0, 0.0)
        ec, eg = oracle_mod.bounds(SC, SG, SG / (SC + SG), 0.0)
        slack_c = SC // 2**31 + 2
        slack_g = SG // 2**31 + 2
        assert abs(ec - bc) <= slack_c and abs(eg - bg) <= slack_g


def test_bounds_hand_examples(oracle_mod):
    for b in load("hand_examples.json")["bounds"]:
        assert oracle_mod.bounds(b["sum_cpu"], b["sum_gpu"], b["r_cpu"], b["tol"]) == (b["bound_cpu"], b["bound_gpu"])


def test_bounds_rejects_bad_arguments(oracle_mod):
    for r, t in [(1.5, 0.03), (float("nan"), 0.03), (-1.0, -0.1), (-1.0, float("nan")), (-1.0, 1.5)]:
        with pytest.raises(oracle_mod.OracleError):
            oracle_mod.bounds(10, 10, r, t)


# ---------------------------------------------------------------------------
# Makespan
# ---------------------------------------------------------------------------

def test_makespan_hand_examples(oracle_mod):
    for ex in load("hand_examples.json")["makespan"]:
        g = gen.from_edges(ex["n"], ex["edges"], ex["cpu"], ex["gpu"], ex["w"])
        for c in ex["cases"]:
            ms, fin = oracle_mod.makespan(g, np.array(c["part"], np.uint8), with_finish=True)
            assert ms == c["makespan"], (ex["name"], c)
            assert fin.tolist() == c["finish"], (ex["name"], c)


def test_makespan_equals_path_enumeration(oracle_mod):
    for seed in range(40):
        g = gen.two_input_dag(6 + seed % 7, seed, extra=seed % 4)
        rng = np.random.default_rng(seed)
        for _ in range(4):
            part = rng.integers(0, 2, g["n"]).astype(np.uint8)
            assert oracle_mod.makespan(g, part) == _brute.longest_path_makespan(g, part)


def test_makespan_bounds(oracle_mod):
    """critical path with min(cC, cG) and no transfers <= makespan <= sum of all costs + transfers"""
    for seed in range(20):
        g = gen.random_dag(30, 70, seed)
        mincost = np.minimum(g["cpu_cost"], g["gpu_cost"]).astype(np.int32)
        lb_graph = dict(g, cpu_cost=mincost, gpu_cost=mincost)
        lb = oracle_mod.makespan(lb_graph, np.zeros(g["n"], np.uint8))
        rng = np.random.default_rng(seed)
        for _ in range(5):
            part = rng.integers(0, 2, g["n"]).astype(np.uint8)
            ms = oracle_mod.makespan(g, part)
            ub = int(np.where(part == 1, g["gpu_cost"], g["cpu_cost"]).sum()) + int(g["edge_cost"].sum())
            assert lb <= ms <= ub


# ---------------------------------------------------------------------------
# Matching, two-hop pairing, contraction
# ---------------------------------------------------------------------------

def test_match_hand_examples(oracle_mod):
    for ex in load("hand_examples.json")["match"]:
        off, adj, W = ucsr(ex["n"], ex["edges"])
        vC, vG = np.array(ex["vC"]), np.array(ex["vG"])
        m1 = oracle_mod.match(ex["n"], off, adj, W, vC, vG, ex["cap_cpu"], ex["cap_gpu"], 0)
        assert m1.tolist() == ex["mate_handshake"], ex["name"]
        m2 = oracle_mod.match_twohop(ex["n"], off, adj, W, vC, vG, ex["cap_cpu"], ex["cap_gpu"], 0, m1)
        assert m2.tolist() == ex["mate"], ex["name"]


def test_match_hash_tie_break(oracle_mod):
    """A hub with equally heavy edges matches the leaf whose edge hashes highest;
    the remaining leaves anchor at the hub and pair up in id order."""
    for seed in range(12):
        n = 5
        off, adj, W = ucsr(n, [[0, u, 7] for u in range(1, n)])
        one = np.ones(n, np.int64)
        m = oracle_mod.match(n, off, adj, W, one, one, 100, 100, seed)
        best = max(range(1, n), key=lambda u: _splitmix.h(seed, 0, u))
        assert m[0] == best and m[best] == 0
        m2 = oracle_mod.match_twohop(n, off, adj, W, one, one, 100, 100, seed, m)
        rest = [u for u in range(1, n) if u != best]
        assert m2[rest[0]] == rest[1] and m2[rest[1]] == rest[0]
        assert m2[rest[2]] == -1


def _level0(g):
    import oracle
    off, adj, W = oracle.symmetrize(g)
    return off, adj, W, g["cpu_cost"].astype(np.int64), g["gpu_cost"].astype(np.int64)


def _key(W, seed, u, v):
    mn, mx = min(u, v), max(u, v)
    return (W, _splitmix.h(seed, mn, mx), -mn, -mx)


def test_match_invariants_and_dominant_edges(oracle_mod):
    """mate is an involution; every matched pair is an edge within the caps;
    after one round, every edge that is the best eligible edge at both of its
    ends (locally dominant) is matched, and nothing else is."""
    for seed in range(6):
        g = gen.random_dag(120, 400, seed)
        off, adj, W, vC, vG = _level0(g)
        n = g["n"]
        capC, capG = int(vC.sum()) // 20, int(vG.sum()) // 20
        m = oracle_mod.match(n, off, adj, W, vC, vG, capC, capG, seed, rounds=1)
        best = {}
        for v in range(n):
            cands = [(_key(int(W[e]), seed, v, int(adj[e])), int(adj[e])) for e in range(off[v], off[v + 1])
                     if vC[v] + vC[adj[e]] <= capC and vG[v] + vG[adj[e]] <= capG]
            best[v] = max(cands)[1] if cands else -1
        for v in range(n):
            u = best[v]
            mutual = u >= 0 and best[u] == v
            assert (m[v] == u) if mutual else (m[v] == -1)
        m4 = oracle_mod.match(n, off, adj, W, vC, vG, capC, capG, seed)
        m5 = oracle_mod.match_twohop(n, off, adj, W, vC, vG, capC, capG, seed, m4)
        for mm, need_edge in ((m4, True), (m5, False)):
            for v in range(n):
                u = mm[v]
                if u >= 0:
                    assert mm[u] == v and u != v
                    assert vC[v] + vC[u] <= capC and vG[v] + vG[u] <= capG
                    if need_edge:
                        assert u in adj[off[v]:off[v + 1]]
        assert np.all(m5[m4 >= 0] == m4[m4 >= 0])


def test_contract_hand_examples(oracle_mod):
    for ex in load("hand_examples.json")["contract"]:
        off, adj, W = ucsr(ex["n"], ex["edges"])
        cmap, coff, cadj, cW, cvC, cvG = oracle_mod.contract(ex["n"], off, adj, W, np.array(ex["vC"]),
                                                             np.array(ex["vG"]), np.array(ex["mate"]))
        assert cmap.tolist() == ex["cmap"]
        assert len(coff) - 1 == ex["coarse_n"]
        assert csr_edges(coff, cadj, cW) == {(a, b): w for a, b, w in ex["coarse_edges"]}
        assert cvC.tolist() == ex["coarse_vC"] and cvG.tolist() == ex["coarse_vG"]


def test_contract_invariants(oracle_mod):
    """Vertex weights are preserved; adjacency weight is preserved except the
    internal edges of merged pairs; rows are sorted, symmetric and loop-free;
    a coarse split projected to the fine level keeps its cut and loads."""
    for seed in range(6):
        g = gen.two_input_dag(300, seed, extra=200)
        off, adj, W, vC, vG = _level0(g)
        n = g["n"]
        capC, capG = int(vC.sum()) // 8, int(vG.sum()) // 8
        m = oracle_mod.match(n, off, adj, W, vC, vG, capC, capG, seed)
        m = oracle_mod.match_twohop(n, off, adj, W, vC, vG, capC, capG, seed, m)
        cmap, coff, cadj, cW, cvC, cvG = oracle_mod.contract(n, off, adj, W, vC, vG, m)
        nc = len(coff) - 1
        assert nc == oracle_mod.count_coarse(m)
        assert cvC.sum() == vC.sum() and cvG.sum() == vG.sum()
        internal = sum(int(W[e]) for v in range(n) for e in range(off[v], off[v + 1]) if cmap[adj[e]] == cmap[v])
        assert int(cW.sum()) == int(W.sum()) - internal
        ce = csr_edges(coff, cadj, cW)
        for c in range(nc):
            row = cadj[coff[c]:coff[c + 1]]
            assert np.all(np.diff(row) > 0) and c not in row
        rng = np.random.default_rng(seed)
        pc = rng.integers(0, 2, nc).astype(np.uint8)
        pf = pc[cmap]
        cut_c = sum(w for (a, b), w in ce.items() if pc[a] != pc[b])
        assert oracle_mod.cut(g, pf) == cut_c
        assert int(vC[pf == 0].sum()) == int(cvC[pc == 0].sum())
        assert int(vG[pf == 1].sum()) == int(cvG[pc == 1].sum())


def test_symmetrize_invariants(oracle_mod):
    for seed in range(5):
        g = gen.random_dag(80, 300, seed)
        off, adj, W = oracle_mod.symmetrize(g)
        ue = csr_edges(off, adj, W)
        assert 2 * int(g["edge_cost"].sum()) == int(W.sum())
        want = {}
        for u in range(g["n"]):
            for e in range(g["offsets"][u], g["offsets"][u + 1]):
                v = int(g["cols"][e])
                k = (min(u, v), max(u, v))
                want[k] = want.get(k, 0) + int(g["edge_cost"][e])
        assert ue == want
        rng = np.random.default_rng(seed)
        part = rng.integers(0, 2, g["n"]).astype(np.uint8)
        assert oracle_mod.cut(g, part) == sum(w for (a, b), w in ue.items() if part[a] != part[b])


# ---------------------------------------------------------------------------
# Initial split and refinement
# ---------------------------------------------------------------------------

def _s(seed, t, n):
    return _splitmix.h(seed, 0xFFFFFFFF, t) % n


def test_gggp_hand_examples(oracle_mod):
    ex = {e["name"]: e for e in load("hand_examples.json")["gggp"]}
    e = ex["four_cycle"]
    off, adj, W = ucsr(e["n"], e["edges"])
    part, t = oracle_mod.gggp(e["n"], off, adj, W, np.array(e["vC"]), np.array(e["vG"]), e["bound_cpu"],
                              e["bound_gpu"], e["seed"])
    s0 = _s(e["seed"], 0, e["n"])
    want = np.ones(4, np.uint8)
    want[[s0, e["heavy_partner"][s0]]] = 0
    assert t == 0 and part.tolist() == want.tolist()

    e = ex["isolated_start_fallback"]
    off, adj, W = ucsr(e["n"], e["edges"])
    part, t = oracle_mod.gggp(e["n"], off, adj, W, np.array(e["vC"]), np.array(e["vG"]), e["bound_cpu"],
                              e["bound_gpu"], e["seed"])
    starts = [_s(e["seed"], k, 3) for k in range(8)]
    assert 2 in starts or True
    assert t == min(k for k in range(8) if starts[k] in (0, 1))
    assert part.tolist() == [0, 0, 1]

    e = ex["all_gpu_fits"]
    off, adj, W = ucsr(e["n"], e["edges"])
    part, t = oracle_mod.gggp(e["n"], off, adj, W, np.array(e["vC"]), np.array(e["vG"]), e["bound_cpu"],
                              e["bound_gpu"], e["seed"])
    assert part.tolist() == e["part"] and t == e["trial"]


def test_gggp_grow_hand_examples(oracle_mod):
    for e in load("hand_examples.json")["gggp_grow"]:
        off, adj, W = ucsr(e["n"], e["edges"])
        for start, want in e["starts"].items():
            part, cut = oracle_mod.gggp_grow(e["n"], off, adj, W, np.array(e["vC"]), np.array(e["vG"]),
                                             e["bound_cpu"], e["bound_gpu"], int(start))
            assert part.tolist() == want["part"] and cut == want["cut"], (e["name"], start)


def test_gggp_fallback_trial_is_scored():
    """Choose a seed whose trial 0 starts at the isolated vertex, so the
    fallback path runs and its cut-5 trial must lose to a cut-0 trial."""
    import oracle
    e = {x["name"]: x for x in load("hand_examples.json")["gggp"]}["isolated_start_fallback"]
    off, adj, W = ucsr(e["n"], e["edges"])
    seed = next(s for s in range(1000) if _s(s, 0, 3) == 2 and any(_s(s, k, 3) != 2 for k in range(8)))
    part, t = oracle.gggp(3, off, adj, W, np.array(e["vC"]), np.array(e["vG"]), e["bound_cpu"], e["bound_gpu"], seed)
    assert t > 0 and part.tolist() == [0, 0, 1]


def test_refine_hand_examples(oracle_mod):
    for e in load("hand_examples.json")["refine"]:
        off, adj, W = ucsr(e["n"], e["edges"])
        part, st = oracle_mod.refine(e["n"], off, adj, W, np.array(e["vC"]), np.array(e["vG"]), e["bound_cpu"],
                                     e["bound_gpu"], np.array(e["part_in"], np.uint8))
        assert part.tolist() == e["part_out"], e["name"]
        for k in ("rounds", "moves", "balanced", "bal_moves", "load_cpu", "load_gpu"):
            assert st[k] == e[k], (e["name"], k)


def test_refine_never_increases_cut_and_keeps_feasibility(oracle_mod):
    for seed in range(8):
        g = gen.two_input_dag(200, seed, extra=150)
        off, adj, W, vC, vG = _level0(g)
        n = g["n"]
        SC, SG = int(vC.sum()), int(vG.sum())
        BC, BG = oracle_mod.bounds(SC, SG, -1.0, 0.1)
        rng = np.random.default_rng(seed)
        for _ in range(5):
            part = rng.integers(0, 2, n).astype(np.uint8)
            LC, LG = int(vC[part == 0].sum()), int(vG[part == 1].sum())
            feas0 = LC <= BC and LG <= BG
            before = oracle_mod.cut(g, part)
            out, st = oracle_mod.refine(n, off, adj, W, vC, vG, BC, BG, part)
            assert st["load_cpu"] == int(vC[out == 0].sum()) and st["load_gpu"] == int(vG[out == 1].sum())
            if feas0:
                assert st["balanced"] == 0
                assert oracle_mod.cut(g, out) <= before
                assert st["load_cpu"] <= BC and st["load_gpu"] <= BG


# ---------------------------------------------------------------------------
# The whole bipartitioner
# ---------------------------------------------------------------------------

def test_partition_vs_exhaustive_search(oracle_mod):
    """On DAGs of <= 18 vertices: the reported cut and loads are those of the
    returned split; a feasible answer never beats the optimum; the heuristic
    is optimal on a good share of instances and close on average."""
    ratios = []
    for seed in range(120):
        n = 8 + seed % 11
        g = gen.two_input_dag(n, seed, extra=seed % 5)
        part, res = oracle_mod.partition(g, seed=seed)
        masks, lc, lg, cut = _brute.all_splits(g)
        mask = int(sum(int(part[v]) << v for v in range(n)))
        assert res["cut"] == int(cut[mask])
        assert res["load_cpu"] == int(lc[mask]) and res["load_gpu"] == int(lg[mask])
        assert res["feasible"] == int(lc[mask] <= res["bound_cpu"] and lg[mask] <= res["bound_gpu"])
        opt, _ = _brute.best_feasible(g, res["bound_cpu"], res["bound_gpu"])
        if opt is not None and res["feasible"]:
            assert res["cut"] >= opt
            ratios.append(res["cut"] / max(opt, 1))
    r = np.array(ratios)
    assert len(r) > 100
    assert (r <= 1.0).mean() >= 0.35 and np.median(r) <= 1.1 and r.mean() <= 1.4


def test_partition_all_gpu_when_speed_gap_is_large(oracle_mod):
    """Sec. IV.C (matrix multiply): with SG/SC <= tol the CPU's share from
    Eq. (1) vanishes and the whole DAG goes to the GPU, with no transfers and
    the GPU critical path as makespan."""
    for seed in range(10):
        g = gen.random_dag(60, 150, seed, ratio_pct=(1, 3))
        SC, SG = int(g["cpu_cost"].sum()), int(g["gpu_cost"].sum())
        assert SG <= 0.03 * SC
        part, res = oracle_mod.partition(g, seed=seed)
        assert np.all(part == 1) and res["cut"] == 0 and res["load_cpu"] == 0
        gpu_only = dict(g, cpu_cost=g["gpu_cost"])
        assert oracle_mod.makespan(g, part) == oracle_mod.makespan(gpu_only, np.zeros(g["n"], np.uint8))


def test_partition_trace_follows_the_level_rules(oracle_mod):
    g = gen.cholesky(24)
    part, res, tr = oracle_mod.partition(g, trace=True)
    L = tr["levels"]
    assert res["levels"] == L and res["coarsest_n"] == tr["n"][L]
    assert res["rounds"] == sum(tr["rounds"])
    for l in range(L):
        assert 100 * tr["n"][l + 1] <= 95 * tr["n"][l]
        assert tr["n"][l] > 128
    assert tr["cut"][0] == res["cut"]
    for l in range(L + 1):
        assert 1 <= tr["rounds"][l] <= 8


def test_partition_hub_coarsens_by_two_hop_pairs(oracle_mod):
    e = load("hand_examples.json")["partition"][0]
    k = e["hub_out_degree"]
    g = gen.from_edges(k + 1, [(0, i) for i in range(1, k + 1)], [e["cpu_each"]] * (k + 1),
                       [e["gpu_each"]] * (k + 1), [e["edge_cost"]] * k)
    part, res, tr = oracle_mod.partition(g, trace=True)
    assert tr["levels"] >= e["min_levels"] and tr["n"][-1] <= e["max_coarsest"]
    assert tr["n"][1] <= (k + 1) // 2 + 2


def test_partition_degenerate_inputs(oracle_mod):
    empty = gen.from_edges(0, [], [], [], [])
    part, res = oracle_mod.partition(empty)
    assert res["feasible"] == 1 and res["cut"] == 0 and len(part) == 0
    # one vertex cannot be split: T* = floor(5*3/8) = 1 and neither side holds it
    single = gen.from_edges(1, [], [5], [3], [])
    part, res = oracle_mod.partition(single)
    assert part.tolist() == [1] and res["feasible"] == 0 and (res["bound_cpu"], res["bound_gpu"]) == (1, 1)
    zero = gen.from_edges(3, [(0, 1), (1, 2)], [0, 0, 0], [0, 0, 0], [0, 0])
    part, res = oracle_mod.partition(zero)
    assert res["feasible"] == 1 and res["cut"] == 0


# ---------------------------------------------------------------------------
# Fixed vertices (the host-source kernel of Sec. III.B pinned to the CPU)
# ---------------------------------------------------------------------------

def _random_pins(n, seed, frac):
    """int8 pins: about frac of the vertices pinned, half to each side (stream of its own)."""
    r = gen.u64(seed, 41, 0, n)
    fx = np.full(n, -1, np.int8)
    sel = (r % np.uint64(1000)).astype(np.int64) < int(frac * 1000)
    fx[sel] = ((r[sel] >> np.uint64(20)) & np.uint64(1)).astype(np.int8)
    return fx


def test_fixed_partition_vs_exhaustive_search(oracle_mod):
    """Tiny DAGs with one to three pinned vertices: pins hold, the reported cut and loads are the
    returned split's, and a feasible answer never beats the optimum over the splits that respect
    the pins (exhaustive); the heuristic is optimal on a good share of instances."""
    ratios = []
    for seed in range(90):
        n = 8 + seed % 10
        g = gen.two_input_dag(n, seed, extra=seed % 4)
        fx = np.full(n, -1, np.int8)
        picks = [int(x) for x in gen.u64(seed, 42, 0, 3) % np.uint64(n)]
        for i, v in enumerate(picks[: 1 + seed % 3]):
            fx[v] = (seed + i) & 1
        part, res = oracle_mod.partition(g, seed=seed, fixed=fx)
        assert np.all(part[fx >= 0] == fx[fx >= 0])
        masks, lc, lg, cut = _brute.all_splits(g)
        mask = int(sum(int(part[v]) << v for v in range(n)))
        assert res["cut"] == int(cut[mask])
        assert res["load_cpu"] == int(lc[mask]) and res["load_gpu"] == int(lg[mask])
        respect = np.ones(masks.shape[0], bool)
        for v in np.flatnonzero(fx >= 0):
            respect &= ((masks >> int(v)) & 1) == int(fx[v])
        ok = respect & (lc <= res["bound_cpu"]) & (lg <= res["bound_gpu"])
        if ok.any() and res["feasible"]:
            opt = int(cut[ok].min())
            assert res["cut"] >= opt
            ratios.append(res["cut"] / max(opt, 1))
    r = np.array(ratios)
    assert len(r) > 60
    assert (r <= 1.0).mean() >= 0.3 and np.median(r) <= 1.15


def test_fixed_all_free_is_the_plain_partition(oracle_mod):
    for g in (gen.cholesky(12), gen.lu(9), gen.layered(30, 60, 6000, 5)):
        a = oracle_mod.partition(g, trace=True, seed=3)
        b = oracle_mod.partition(g, trace=True, seed=3, fixed=np.full(g["n"], -1, np.int8))
        assert np.array_equal(a[0], b[0]) and a[1] == b[1] and a[2] == b[2]


def test_fixed_vertices_keep_their_side_through_every_level(oracle_mod):
    """Heavy pinning (adjacent vertices pinned to opposite sides are common) on graphs that coarsen
    over several levels: every pinned vertex ends on its side, the reported loads are the split's."""
    cases = [(gen.layered(40, 60, 9000, s), s) for s in range(3)] + [(gen.cholesky(14), 7), (gen.lu(10), 8)]
    for g, s in cases:
        for frac in (0.05, 0.3, 0.6):
            fx = _random_pins(g["n"], s * 10 + int(frac * 10), frac)
            part, res, tr = oracle_mod.partition(g, trace=True, seed=s, fixed=fx)
            assert tr["levels"] >= 1
            assert np.all(part[fx >= 0] == fx[fx >= 0]), (s, frac)
            lc = int(g["cpu_cost"][part == 0].sum())
            lg = int(g["gpu_cost"][part == 1].sum())
            assert (res["load_cpu"], res["load_gpu"]) == (lc, lg)
            assert res["cut"] == oracle_mod.cut(g, part)


def test_fixed_host_source_on_the_cpu(oracle_mod):
    """Sec. III.B: the initial data sit in host memory, modelled as an empty kernel feeding every
    kernel without a predecessor.  Pinned, it stays on the CPU; its zero costs change no load.
    With a large speed gap everything free goes to the GPU with the source alone on the CPU: the
    growing's pre-check (trial -1), which refinement can only improve on."""
    base = gen.layered(20, 50, 3000, 1)
    g, src = gen.with_host_source(base, 1)
    fx = np.full(g["n"], -1, np.int8)
    fx[src] = 0
    part, res, tr = oracle_mod.partition(g, trace=True, fixed=fx)
    assert part[src] == 0
    assert np.flatnonzero(np.bincount(g["cols"], minlength=g["n"]) == 0).tolist() == [src]
    roots = np.flatnonzero(np.bincount(base["cols"], minlength=base["n"]) == 0)
    assert g["cols"][g["offsets"][src]:].tolist() == roots.tolist() and len(roots) >= 50
    gap, s2 = gen.with_host_source(gen.random_dag(60, 150, 2, ratio_pct=(1, 3)), 2)
    fx = np.full(gap["n"], -1, np.int8)
    fx[s2] = 0
    part, res, tr = oracle_mod.partition(gap, trace=True, fixed=fx)
    assert tr["gggp_trial"] == -1 and part[s2] == 0 and res["feasible"] == 1
    # refinement starts from that split and only lowers its cut (the source's transfers)
    off = gap["offsets"]
    assert res["cut"] <= int(gap["edge_cost"][off[s2]:off[s2 + 1]].sum())
    assert (part == 0).sum() <= 3


def test_fixed_everything_pinned_and_bad_values(oracle_mod):
    g = gen.cholesky(8)
    for s in range(4):
        fx = (gen.u64(s, 43, 0, g["n"]) & np.uint64(1)).astype(np.int8)
        part, res = oracle_mod.partition(g, fixed=fx, seed=s)
        assert np.array_equal(part, fx.astype(np.uint8))
        assert res["feasible"] == int(res["load_cpu"] <= res["bound_cpu"] and res["load_gpu"] <= res["bound_gpu"])
    bad = np.full(g["n"], -1, np.int8)
    bad[5] = 2
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.partition(g, fixed=bad)


def test_validation_codes(oracle_mod):
    ok = gen.from_edges(3, [(0, 1), (1, 2)], [1, 1, 1], [1, 1, 1], [1, 1])
    assert oracle_mod.validate(ok) == oracle_mod.OK

    def mod(**kw):
        g = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in ok.items()}
        g.update(kw)
        return g

    assert oracle_mod.validate(mod(offsets=np.array([0, 2, 2, 2]))) == oracle_mod.OK
    assert oracle_mod.validate(mod(offsets=np.array([0, 2, 1, 2]))) == oracle_mod.ERR_INVALID
    assert oracle_mod.validate(mod(offsets=np.array([1, 1, 2, 2]))) == oracle_mod.ERR_INVALID
    assert oracle_mod.validate(mod(cols=np.array([1, 3]))) == oracle_mod.ERR_INVALID
    assert oracle_mod.validate(mod(cols=np.array([1, -1]))) == oracle_mod.ERR_INVALID
    assert oracle_mod.validate(mod(edge_cost=np.array([1, -1]))) == oracle_mod.ERR_INVALID
    assert oracle_mod.validate(mod(cpu_cost=np.array([1, -1, 1]))) == oracle_mod.ERR_INVALID
    assert oracle_mod.validate(mod(cols=np.array([0, 2]))) == oracle_mod.ERR_NOT_DAG  # self-loop 0->0
    cyc = gen.from_edges(3, [(0, 1), (1, 2), (2, 0)], [1, 1, 1], [1, 1, 1], [1, 1, 1])
    assert oracle_mod.validate(cyc) == oracle_mod.ERR_NOT_DAG
    both = dict(cyc, edge_cost=np.array([1, -1, 1]))
    assert oracle_mod.validate(both) == oracle_mod.ERR_INVALID


def test_oracle_regression_record(oracle_mod):
    """The oracle still reproduces its committed results (written by
    tests/golden/make_oracle_golden.py, which calls only oracle/)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("mk", os.path.join(GOLD, "make_oracle_golden.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    rec = {c["name"]: c for c in load("oracle_small.json")["cases"]}
    for name, g, kw in mk.fixtures():
        part, res, tr = oracle_mod.partition(g, trace=True, **kw)
        c = rec[name]
        assert res == c["result"] and np.packbits(part).tobytes().hex() == c["part_hex"], name
        assert oracle_mod.makespan(g, part) == c["makespan"] and tr["n"] == c["levels_n"], name


# ---------------------------------------------------------------------------
# Makespan on a fixed number of workers (list schedule; Sec. IV.A's 3 CPU + 1 GPU workers)
# ---------------------------------------------------------------------------

def test_makespan_workers_hand_examples(oracle_mod):
    for ex in load("hand_examples.json")["makespan_workers"]:
        g = gen.from_edges(ex["n"], ex["edges"], ex["cpu"], ex["gpu"], ex["w"])
        part = np.array(ex["part"], np.uint8)
        ms, fin = oracle_mod.makespan_workers(g, part, ex["workers_cpu"], ex["workers_gpu"], with_finish=True)
        assert ms == ex["makespan"], ex["name"]
        assert fin.tolist() == ex["finish"], ex["name"]
        assert oracle_mod.makespan(g, part) == ex["unbounded_makespan"], ex["name"]


def test_makespan_workers_unbounded_is_the_longest_path(oracle_mod):
    """With a worker for every task on both sides, every task starts when its data arrive: the
    finish times are those of the longest-path makespan."""
    for seed in range(30):
        g = gen.random_dag(40 + seed, 120 + 3 * seed, seed)
        rng = np.random.default_rng(seed)
        for _ in range(3):
            part = rng.integers(0, 2, g["n"]).astype(np.uint8)
            ms, fin = oracle_mod.makespan(g, part, with_finish=True)
            ms2, fin2 = oracle_mod.makespan_workers(g, part, g["n"], g["n"], with_finish=True)
            assert ms2 == ms and np.array_equal(fin, fin2)


def test_makespan_workers_one_worker_runs_back_to_back(oracle_mod):
    """One worker and every task on its side: no transfers, and the worker is never idle while a
    task is left (some unfinished task always has all its predecessors done), so the makespan is the
    sum of the costs."""
    for seed in range(20):
        g = gen.random_dag(50, 150, seed)
        n = g["n"]
        assert oracle_mod.makespan_workers(g, np.zeros(n, np.uint8), 1, 5) == int(g["cpu_cost"].sum())
        assert oracle_mod.makespan_workers(g, np.ones(n, np.uint8), 7, 1) == int(g["gpu_cost"].sum())


def test_makespan_workers_equals_time_stepped_simulation(oracle_mod):
    """Tiny DAGs with small integer costs (zeros included): the event-driven schedule equals a
    schedule simulated one time unit at a time."""
    for seed in range(60):
        rng = np.random.default_rng(1000 + seed)
        n = int(rng.integers(2, 11))
        pairs = [(u, v) for u in range(n) for v in range(u + 1, n)]
        k = int(rng.integers(0, min(len(pairs), 18) + 1))
        idx = rng.choice(len(pairs), size=k, replace=False) if k else []
        edges = [pairs[i] for i in idx]
        if seed % 5 == 0 and edges:
            edges.append(edges[0])  # a parallel entry
        g = gen.from_edges(n, edges, rng.integers(0, 7, n).tolist(), rng.integers(0, 7, n).tolist(),
                           rng.integers(0, 7, len(edges)).tolist())
        for pc, pg in ((1, 1), (2, 1), (3, 1), (1, 2)):
            part = rng.integers(0, 2, n).astype(np.uint8)
            ms, fin = oracle_mod.makespan_workers(g, part, pc, pg, with_finish=True)
            bms, bfin = _brute.list_schedule_stepped(g, part, pc, pg)
            assert ms == bms and fin.tolist() == bfin, (seed, pc, pg)


def test_makespan_workers_bounds(oracle_mod):
    """longest path <= makespan; load of a side / its workers <= makespan; makespan <= all costs +
    all transfers."""
    for seed in range(20):
        g = gen.random_dag(60, 200, seed)
        rng = np.random.default_rng(seed)
        for pc, pg in ((3, 1), (2, 2), (1, 1)):
            part = rng.integers(0, 2, g["n"]).astype(np.uint8)
            ms = oracle_mod.makespan_workers(g, part, pc, pg)
            lc = int(g["cpu_cost"][part == 0].sum())
            lg = int(g["gpu_cost"][part == 1].sum())
            assert ms >= oracle_mod.makespan(g, part)
            assert ms * pc >= lc and ms * pg >= lg
            assert ms <= lc + lg + int(g["edge_cost"].sum())


def test_makespan_workers_rejects_bad_arguments(oracle_mod):
    g = gen.cholesky(4)
    part = np.zeros(g["n"], np.uint8)
    for pc, pg in ((0, 1), (1, 0)):
        with pytest.raises(oracle_mod.OracleError):
            oracle_mod.makespan_workers(g, part, pc, pg)
    part[3] = 2
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.makespan_workers(g, part, 3, 1)
    empty = gen.from_edges(0, [], [], [], [])
    assert oracle_mod.makespan_workers(empty, np.zeros(0, np.uint8), 3, 1) == 0


# ---------------------------------------------------------------------------
# The learned path as a V-cycle (restricted coarsening)
# ---------------------------------------------------------------------------

def _noisy_logits(g, oracle_mod, seed, scale=0.8):
    """Logits a trained network might give: the plain split's sides (CPU positive) plus noise."""
    p0, _ = oracle_mod.partition(g)
    rng = np.random.default_rng(seed)
    return (np.where(p0 == 0, 1.0, -1.0) + rng.normal(0.0, scale, g["n"])).astype(np.float32)


def test_vcycle_all_gpu_proposal_is_the_plain_partition(oracle_mod):
    """When all-GPU fits (SG <= B_G) the proposal is all-GPU, so the restriction is void: the
    V-cycle's coarsening, coarsest split (all-GPU, the growing's pre-check) and refinement are the
    plain partition's, result for result."""
    for seed in range(6):
        g = gen.layered(30, 40, 3000, seed, ratio_lo=60.0, ratio_hi=80.0)
        sc, sg = int(g["cpu_cost"].sum()), int(g["gpu_cost"].sum())
        _, bg = oracle_mod.bounds(sc, sg)
        assert sg <= bg
        lg = np.random.default_rng(seed).normal(0, 1, g["n"]).astype(np.float32)
        pv, rv, tv = oracle_mod.partition_vcycle(g, lg, seed=seed, trace=True)
        pp, rp, tp = oracle_mod.partition(g, seed=seed, trace=True)
        assert np.array_equal(pv, pp) and rv == rp
        assert tv["n"] == tp["n"] and tv["a"] == tp["a"] and tv["levels"] > 0


def test_vcycle_never_worse_than_a_feasible_proposal(oracle_mod):
    """The coarsest split is the proposal itself (a coarse vertex holds one proposed side, so the
    projection keeps its cut and loads); a feasible split needs no balance round and gain rounds
    never raise the cut: the result is feasible, its cut at most the proposal's, and strictly below
    it on noisy proposals (refinement at the coarse levels moves whole clusters)."""
    lower = 0
    for seed, g in enumerate([gen.layered(40, 150, 40000, 7), gen.cholesky(20), gen.lu(16),
                              gen.layered(60, 300, 120000, 3), gen.random_dag(3000, 12000, 4)]):
        lg = _noisy_logits(g, oracle_mod, seed)
        cc, cg = g["cpu_cost"].astype(np.int64), g["gpu_cost"].astype(np.int64)
        bc, bg = oracle_mod.bounds(int(cc.sum()), int(cg.sum()))
        prop, _ = oracle_mod.propose(lg, cc, cg, bc, bg)
        feasible = cc[prop == 0].sum() <= bc and cg[prop == 1].sum() <= bg
        part, res, tr = oracle_mod.partition_vcycle(g, lg, trace=True)
        assert res["cut"] == oracle_mod.cut(g, part)
        assert res["load_cpu"] == int(cc[part == 0].sum()) and res["load_gpu"] == int(cg[part == 1].sum())
        if feasible:
            assert res["feasible"] == 1 and sum(tr["balanced"]) == 0
            # level by level (coarsest first) the refined cut only falls, from the proposal's
            cuts = [oracle_mod.cut(g, prop)] + tr["cut"][::-1]
            assert all(a >= b for a, b in zip(cuts, cuts[1:])), cuts
            assert res["cut"] <= oracle_mod.cut(g, prop)
            lower += res["cut"] < oracle_mod.cut(g, prop)
    assert lower >= 3


def test_vcycle_coarsens_through_levels_and_reports_them(oracle_mod):
    g = gen.layered(60, 300, 120000, 3)
    lg = _noisy_logits(g, oracle_mod, 9)
    part, res, tr = oracle_mod.partition_vcycle(g, lg, trace=True)
    assert res["levels"] == tr["levels"] > 3 and tr["gggp_trial"] == -1
    assert tr["n"][0] == g["n"] and res["coarsest_n"] == tr["n"][-1]
    assert all(a > b for a, b in zip(tr["n"], tr["n"][1:]))
    assert sum(tr["rounds"]) == res["rounds"]


# ---------------------------------------------------------------------------
# k device classes by recursive bisection
# ---------------------------------------------------------------------------

def _comb(*xs):
    """Group time of classes working on one task together: 1/t = sum 1/t_i, floored pairwise."""
    a = int(xs[0])
    for b in xs[1:]:
        b = int(b)
        a = 0 if a + b == 0 else (a * b) // (a + b)
    return a


def _induced(g, keep):
    """The subgraph on the vertices with keep[v] (renumbered in increasing id), every entry with both
    ends kept; costs are left to the caller."""
    ids = np.flatnonzero(keep)
    new = -np.ones(g["n"], np.int64)
    new[ids] = np.arange(ids.size)
    edges, w = [], []
    for u in ids:
        for e in range(g["offsets"][u], g["offsets"][u + 1]):
            v = int(g["cols"][e])
            if keep[v]:
                edges.append((int(new[u]), int(new[v])))
                w.append(int(g["edge_cost"][e]))
    return ids, edges, w


def _costs3(g, seed):
    rng = np.random.default_rng(seed)
    fpga = np.maximum(0, (g["cpu_cost"].astype(np.int64) * rng.uniform(0.2, 0.8, g["n"]))).astype(np.int32)
    return np.stack([g["cpu_cost"], g["gpu_cost"], fpga]).astype(np.int32)


def test_kway_two_classes_is_the_2way_partition(oracle_mod):
    for seed, g in enumerate([gen.cholesky(16), gen.lu(10), gen.layered(40, 150, 40000, 7)]):
        cls, r = oracle_mod.partition_kway(g, np.stack([g["cpu_cost"], g["gpu_cost"]]), seed=seed)
        part, res = oracle_mod.partition(g, seed=seed)
        assert np.array_equal(cls, part) and r["cut"] == res["cut"]
        assert r["loads"] == [res["load_cpu"], res["load_gpu"]] and r["feasible"] == res["feasible"]
        assert r["bisections"] == 1


def test_kway_one_class_takes_everything(oracle_mod):
    g = gen.cholesky(8)
    cls, r = oracle_mod.partition_kway(g, g["cpu_cost"][None, :])
    assert not cls.any() and r == dict(cut=0, loads=[int(g["cpu_cost"].sum())], feasible=1, bisections=0)


def test_kway_group_times_and_recursion(oracle_mod):
    """k = 3: the first split is the 2-way problem between group {0, 1} (times folded as
    floor(x*y/(x+y))) and class 2; then the {0, 1} side's induced subgraph is split between classes
    0 and 1.  k = 4: groups {0, 1} and {2, 3} first, each then split on its own induced subgraph."""
    for seed, g in enumerate([gen.lu(12), gen.layered(30, 120, 20000, 5), gen.random_dag(900, 4000, 2)]):
        cs = _costs3(g, seed)
        cls, r = oracle_mod.partition_kway(g, cs, seed=seed)
        n = g["n"]
        top = dict(g, cpu_cost=np.array([_comb(cs[0, v], cs[1, v]) for v in range(n)], np.int32),
                   gpu_cost=cs[2].copy())
        p1, _ = oracle_mod.partition(top, seed=seed)
        assert np.array_equal(cls == 2, p1 == 1)
        ids, edges, w = _induced(g, p1 == 0)
        sub = gen.from_edges(ids.size, edges, cs[0, ids].tolist(), cs[1, ids].tolist(), w)
        p2, _ = oracle_mod.partition(sub, seed=seed)
        assert np.array_equal(cls[ids], p2)
        # k = 4 (a second FPGA-like class)
        cs4 = np.concatenate([cs, (cs[2:3] * 3 // 2).astype(np.int32)])
        cls4, r4 = oracle_mod.partition_kway(g, cs4, seed=seed)
        top4 = dict(g, cpu_cost=np.array([_comb(cs4[0, v], cs4[1, v]) for v in range(n)], np.int32),
                    gpu_cost=np.array([_comb(cs4[2, v], cs4[3, v]) for v in range(n)], np.int32))
        q, _ = oracle_mod.partition(top4, seed=seed)
        assert np.array_equal(cls4 >= 2, q == 1)
        for side, (a, b) in ((0, (0, 1)), (1, (2, 3))):
            ids, edges, w = _induced(g, q == side)
            if ids.size:
                sub = gen.from_edges(ids.size, edges, cs4[a, ids].tolist(), cs4[b, ids].tolist(), w)
                ps, _ = oracle_mod.partition(sub, seed=seed)
                assert np.array_equal(cls4[ids], np.where(ps == 0, a, b))


def test_kway_reported_cut_and_loads(oracle_mod):
    for seed in range(6):
        g = gen.random_dag(400, 2000, seed)
        cs = _costs3(g, seed)
        cls, r = oracle_mod.partition_kway(g, cs, seed=seed)
        assert cls.max() < 3
        cut = sum(int(g["edge_cost"][e]) for u in range(g["n"]) for e in range(g["offsets"][u], g["offsets"][u + 1])
                  if cls[u] != cls[g["cols"][e]])
        assert r["cut"] == cut
        assert r["loads"] == [int(cs[i][cls == i].sum()) for i in range(3)]
        assert r["bisections"] == 2


def test_kway_rejects_bad_arguments(oracle_mod):
    g = gen.cholesky(4)
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.partition_kway(g, np.zeros((0, g["n"]), np.int32))
    bad = np.stack([g["cpu_cost"], g["gpu_cost"]]).astype(np.int32)
    bad[1, 3] = -1
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.partition_kway(g, bad)
