"""Bit-exact parity on the three largest workloads, against the oracle's recorded results.

The oracle takes minutes of host time on these workloads, so `tests/golden/make_large_golden.py`
(which calls only oracle/ and the input generators) records every result field, the makespan and
the SHA-256 of each split; here the CUDA path runs the same inputs through the C-ABI and must give
the same records:

  - the layered DAG of 1,000 layers x 16,000 vertices and 128M edges (int64 offsets): the
    single-graph path, plus the learned path against the oracle's proposal rule and refinement run
    on the network's logits;
  - the 4,096-graph mix (every graph of the recipe, 100..50,000 vertices), batched in one
    persistent launch, with makespans;
  - tiled Cholesky T = 64 under seeds 0..1023, batched; and the learned batch of 1,024 such graphs
    against the oracle's learned path on the network's logits.
"""
import hashlib
import json
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle
import paper_1502_07451_b300 as gp
from paper_1502_07451_b300 import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden")
MODEL = os.path.join(os.path.dirname(HERE), "paper_1502_07451_b300", "models", "mpnn3_h64.bin")
KEYS = ("offsets", "cols", "edge_cost", "cpu_cost", "gpu_cost")
FIELDS = ("cut", "load_cpu", "load_gpu", "bound_cpu", "bound_gpu", "feasible", "levels", "rounds", "coarsest_n")


def sha(part, nhex=64):
    return hashlib.sha256(np.ascontiguousarray(part, dtype=np.uint8).tobytes()).hexdigest()[:nhex]


def table(name):
    """Rows of a per-graph oracle table as dicts keyed by its "# columns:" line (numbers as int)."""
    cols, rows = None, []
    with open(os.path.join(GOLD, name)) as f:
        for ln in f:
            if ln.startswith("# columns:"):
                cols = ln[len("# columns:"):].split()
            elif not ln.startswith("#"):
                vals = ln.split()
                rows.append({k: (int(v) if k not in ("kind", "param", "sha256") else v) for k, v in zip(cols, vals)})
    return rows


def want_of(row):
    return {k: row[k] for k in FIELDS + ("makespan",)}


def _build(items):
    return [gen.build_from_spec(it) for it in items]


def test_layered16m_matches_oracle_record():
    """The whole single-graph path on 16M vertices / 128M edges: split digest, every result field,
    the per-level vertex and entry counts, and the makespan, as the oracle recorded them."""
    with open(os.path.join(GOLD, "layered16m_oracle.json")) as f:
        want = json.load(f)
    g = gen.config_layered_16m()
    n = g["n"]
    assert (n, g["m"]) == (want["n"], want["m"])
    assert int(g["cpu_cost"].astype(np.int64).sum()) == want["cpu_cost_sum"]
    dg = {k: torch.from_numpy(g[k]).cuda() for k in KEYS}
    with gp.Graph(dict(dg, n=n, m=g["m"])) as G:
        part = torch.empty(n, dtype=torch.uint8, device="cuda")
        res = G.partition(part)
        tr = G.trace()
        ms = G.makespan(part)
        p = part.cpu().numpy()
        assert {k: res[k] for k in FIELDS} == want["result"]
        assert tr["n"] == want["trace_n"] and tr["a"] == want["trace_a"] and tr["rounds"] == want["trace_rounds"]
        assert sha(p) == want["sha256"]
        assert ms == want["makespan"]
        assert gp.gp_makespan_workers(G.h, part, 3, 1) == want["makespan_w31"]
        # the learned path on the same handle: the oracle's proposal rule and level-0 refinement,
        # given the network's logits, must reproduce its split bit for bit
        model = gp.gp_model_load(MODEL)
        try:
            logits = torch.empty(n, dtype=torch.float32, device="cuda")
            gp.gp_model_forward(model, G.h, logits)
            rl = gp.gp_partition_learned(G.h, model, part)
            pl = part.cpu().numpy()
        finally:
            gp.gp_model_destroy(model)
        lg = logits.cpu().numpy()
        assert np.isfinite(lg).all()
        opl, orl = oracle.partition_learned(g, lg)
        assert all(rl[k] == orl[k] for k in orl)
        assert np.array_equal(pl, opl)


def test_full_batch_4096_matches_oracle_records():
    """Every graph of the 4,096-graph mix, batched in one persistent launch with makespans: split
    digest, every result field and the makespan equal the oracle's record of that graph."""
    rows = table("batch4096_oracle.txt")
    spec = gen.batch_spec(4096)
    assert len(rows) == len(spec) == 4096
    nproc = max(1, min(16, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(nproc) as pool:
        chunks = pool.map(_build, [spec[i::nproc] for i in range(nproc)])
    graphs = [None] * len(spec)
    for i, part in enumerate(chunks):
        for j, g in enumerate(part):
            graphs[i + j * nproc] = g
    src = [dict({k: torch.from_numpy(np.ascontiguousarray(g[k])).cuda() for k in KEYS}, n=g["n"], m=g["m"])
           for g in graphs]
    hs, sts = gp.gp_graph_create_batch(src)
    try:
        assert all(st == gp.GP_OK for st in sts)
        parts = [torch.zeros(max(g["n"], 1), dtype=torch.uint8, device="cuda") for g in graphs]
        res, mks = gp.gp_batch_partition(hs, parts, makespans=True)
        bad = []
        for i, (g, row) in enumerate(zip(graphs, rows)):
            assert row["i"] == i and (row["n"], row["m"]) == (g["n"], g["m"])
            got = dict({k: res[i][k] for k in FIELDS}, makespan=mks[i])
            if got != want_of(row) or sha(parts[i].cpu().numpy()[: g["n"]], 32) != row["sha256"]:
                bad.append(i)
        assert not bad, "graphs differing from the oracle: %s" % bad[:20]
        # the same splits on 3 CPU workers and 1 GPU worker (one launch, a warp per graph)
        msw = gp.gp_batch_makespan_workers(hs, parts, 3, 1)
        bad = [i for i, row in enumerate(rows) if msw[i] != row["makespan_w31"]]
        assert not bad, "list-schedule makespans differing from the oracle: %s" % bad[:20]
    finally:
        for h in hs:
            gp.gp_graph_destroy(h)


def test_cholesky64_seeds_and_learned_batch_match_oracle():
    """1,024 handles of tiled Cholesky T = 64: the plain batch under seeds 0..1023 equals the
    oracle's record of each seed; the learned batch equals the oracle's learned path on the
    network's logits (the same DAG, so the same logits and the same split for every handle)."""
    rows = table("cholesky64_seeds_oracle.txt")
    assert len(rows) == 1024
    g = gen.cholesky(64)
    n, m = g["n"], g["m"]
    dg = {k: torch.from_numpy(g[k]).cuda() for k in KEYS}
    hs = [gp.gp_graph_create(n, m, *[dg[k] for k in KEYS]) for _ in range(1024)]
    model = gp.gp_model_load(MODEL)
    try:
        parts = [torch.zeros(n, dtype=torch.uint8, device="cuda") for _ in range(1024)]
        res, mks = gp.gp_batch_partition(hs, parts, seeds=list(range(1024)), makespans=True)
        bad = []
        for s, row in enumerate(rows):
            assert row["seed"] == s
            got = dict({k: res[s][k] for k in FIELDS}, makespan=mks[s])
            if got != want_of(row) or sha(parts[s].cpu().numpy(), 32) != row["sha256"]:
                bad.append(s)
        assert not bad, "seeds differing from the oracle: %s" % bad[:20]
        msw = gp.gp_batch_makespan_workers(hs, parts, 3, 1)
        bad = [s for s, row in enumerate(rows) if msw[s] != row["makespan_w31"]]
        assert not bad, "list-schedule makespans differing from the oracle: %s" % bad[:20]
        logits = torch.empty(n, dtype=torch.float32, device="cuda")
        gp.gp_model_forward(model, hs[0], logits)
        opl, orl = oracle.partition_learned(g, logits.cpu().numpy())
        oms = oracle.makespan(g, opl)
        lres, lmks = gp.gp_batch_partition_learned(hs, model, parts, makespans=True)
        for i in range(1024):
            assert all(lres[i][k] == orl[k] for k in orl), i
            assert lmks[i] == oms
            assert np.array_equal(parts[i].cpu().numpy(), opl), i
    finally:
        gp.gp_model_destroy(model)
        for h in hs:
            gp.gp_graph_destroy(h)
