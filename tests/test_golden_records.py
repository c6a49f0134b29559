"""The recorded oracle results of the largest workloads (tests/golden/*_oracle.*) are the
oracle's: a sample of their rows is recomputed here from the input generators and the oracle, and
the 16M record is checked against Eq. (1)-(2) and its own fields.  CPU only."""
import hashlib
import json
import os

import numpy as np

import oracle
from paper_1502_07451_b300 import gen

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FIELDS = ("cut", "load_cpu", "load_gpu", "bound_cpu", "bound_gpu", "feasible", "levels", "rounds", "coarsest_n")


def rows(name):
    cols, out = None, []
    with open(os.path.join(GOLD, name)) as f:
        for ln in f:
            if ln.startswith("# columns:"):
                cols = ln[len("# columns:"):].split()
            elif not ln.startswith("#"):
                out.append(dict(zip(cols, ln.split())))
    return out


def check_row(g, seed, row):
    part, res = oracle.partition(g, -1.0, 0.03, seed)
    assert [res[k] for k in FIELDS] == [int(row[k]) for k in FIELDS]
    assert oracle.makespan(g, part) == int(row["makespan"])
    assert oracle.makespan_workers(g, part, 3, 1) == int(row["makespan_w31"])
    assert hashlib.sha256(part.tobytes()).hexdigest()[:32] == row["sha256"]


def test_batch_records_sample_recomputed():
    spec = gen.batch_spec(4096)
    table = rows("batch4096_oracle.txt")
    assert len(table) == 4096
    small = sorted(range(4096), key=lambda i: int(table[i]["n"]))[:12]
    for i in sorted(set(small) | {0, 1, 2, 1000, 2047}):
        kind, p, s = spec[i]
        row = table[i]
        assert int(row["i"]) == i and row["kind"] == kind and int(row["graph_seed"]) == s
        g = gen.build_from_spec(spec[i])
        assert (int(row["n"]), int(row["m"])) == (g["n"], g["m"])
        check_row(g, 0, row)


def test_cholesky64_records_sample_recomputed():
    table = rows("cholesky64_seeds_oracle.txt")
    assert [int(r["seed"]) for r in table] == list(range(1024))
    g = gen.cholesky(64)
    for s in (0, 1, 511, 1023):
        check_row(g, s, table[s])


def test_layered16m_record_is_consistent():
    with open(os.path.join(GOLD, "layered16m_oracle.json")) as f:
        rec = json.load(f)
    r = rec["result"]
    assert (rec["n"], rec["m"]) == (16_000_000, 128_000_000)
    assert (r["bound_cpu"], r["bound_gpu"]) == oracle.bounds(rec["cpu_cost_sum"], rec["gpu_cost_sum"])
    assert r["feasible"] == int(r["load_cpu"] <= r["bound_cpu"] and r["load_gpu"] <= r["bound_gpu"])
    assert r["levels"] == len(rec["trace_n"]) - 1 and rec["trace_n"][0] == rec["n"]
    assert rec["trace_n"][-1] == r["coarsest_n"] and sum(rec["trace_rounds"]) == r["rounds"]
    assert all(a > b for a, b in zip(rec["trace_n"], rec["trace_n"][1:]))
    assert len(rec["sha256"]) == 64 and rec["makespan"] > 0 and np.isfinite(rec["oracle_s"])
    assert rec["makespan_w31"] >= rec["makespan"]
