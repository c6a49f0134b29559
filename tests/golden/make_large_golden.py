"""Writes the oracle's results on the three largest workloads, as digests:

  layered16m_oracle.json      the layered DAG of 1,000 layers x 16,000 vertices and 128M edges
                              (int64 offsets), seed 0, ratio from Eq. (1), 3% tolerance
  batch4096_oracle.txt        the 4,096-graph mix (tiled Cholesky, tiled LU, layered; 100..50,000
                              vertices), every graph with seed 0
  cholesky64_seeds_oracle.txt tiled Cholesky T = 64 (45,760 tasks), seeds 0..1023

Each record holds every field of the oracle's result, its makespan (as many workers as needed), its
makespan on 3 CPU workers and 1 GPU worker (the list schedule; Sec. IV.A's testbed) and the SHA-256
of its split (n bytes, 0 = CPU, 1 = GPU), so that a test can compare a split of any size without
storing it.  The per-graph tables name their columns in a "# columns:" line.
Calls only oracle/ and the input generators (spawned workers, one graph per task); rerun it, and
say why in the commit, only when the oracle's arithmetic changes on purpose.  Takes about six
minutes on eight host cores (the 16M graph: one minute to build, four and a half in the oracle).

  python tests/golden/make_large_golden.py [layered16m] [batch] [cholesky64]
"""
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FIELDS = ("cut", "load_cpu", "load_gpu", "bound_cpu", "bound_gpu", "feasible", "levels", "rounds", "coarsest_n")


def digest(part, nhex=64) -> str:
    """SHA-256 of the split's bytes (hex; the per-graph tables keep its first 32 digits)."""
    import numpy as np
    return hashlib.sha256(np.ascontiguousarray(part, dtype=np.uint8).tobytes()).hexdigest()[:nhex]


def record(g, seed):
    import oracle
    part, res = oracle.partition(g, -1.0, 0.03, seed)
    ms = oracle.makespan(g, part) if g["n"] else 0
    msw = oracle.makespan_workers(g, part, 3, 1)
    return dict(res, makespan=ms, makespan_w31=msw, sha256=digest(part, 32))


def _batch_item(args):
    i, item = args
    from paper_1502_07451_b300 import gen
    g = gen.build_from_spec(item)
    r = record(g, 0)
    return i, item, g["n"], g["m"], r


def _chol_seed(seed):
    from paper_1502_07451_b300 import gen
    g = gen.cholesky(64)
    return seed, record(g, seed)


def _layered16m(_):
    from paper_1502_07451_b300 import gen
    import oracle
    t0 = time.time()
    g = gen.config_layered_16m(0)
    t1 = time.time()
    part, res, tr = oracle.partition(g, -1.0, 0.03, 0, trace=True)
    t2 = time.time()
    ms = oracle.makespan(g, part)
    msw = oracle.makespan_workers(g, part, 3, 1)
    return dict(result=res, makespan=ms, makespan_w31=msw, sha256=digest(part), trace_n=tr["n"], trace_a=tr["a"],
                trace_rounds=tr["rounds"], gggp_trial=tr["gggp_trial"], n=g["n"], m=g["m"],
                cpu_cost_sum=int(g["cpu_cost"].astype("int64").sum()),
                gpu_cost_sum=int(g["gpu_cost"].astype("int64").sum()),
                build_s=round(t1 - t0, 1), oracle_s=round(t2 - t1, 1))


def line(fields):
    return " ".join(str(x) for x in fields)


def main(which):
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(8, os.cpu_count() or 1)) as pool:
        big = pool.map_async(_layered16m, [0]) if "layered16m" in which else None
        if "batch" in which:
            from paper_1502_07451_b300 import gen
            spec = gen.batch_spec(4096)
            rows = sorted(pool.imap_unordered(_batch_item, list(enumerate(spec)), chunksize=4))
            with open(os.path.join(HERE, "batch4096_oracle.txt"), "w") as f:
                f.write("# oracle on the 4,096-graph mix (batch_spec(4096), base seed 0), partition seed 0, ratio from\n"
                        "# Eq. (1), tolerance 3%; one line per graph in recipe order; sha256 = first 32 hex digits\n"
                        "# columns: i kind param graph_seed n m " + " ".join(FIELDS) + " makespan makespan_w31 sha256\n")
                for i, item, n, m, r in rows:
                    kind, p, gs = item
                    ps = "%dx%d" % p if kind == "layered" else str(p)
                    f.write(line([i, kind, ps, gs, n, m] + [r[k] for k in FIELDS] +
                                 [r["makespan"], r["makespan_w31"], r["sha256"]]) + "\n")
            print("batch done", flush=True)
        if "cholesky64" in which:
            rows = sorted(pool.imap_unordered(_chol_seed, range(1024), chunksize=8))
            with open(os.path.join(HERE, "cholesky64_seeds_oracle.txt"), "w") as f:
                f.write("# oracle on tiled Cholesky T = 64 (45,760 tasks, 131,040 edges), ratio from Eq. (1),\n"
                        "# tolerance 3%, partition seeds 0..1023; one line per seed; sha256 = first 32 hex digits\n"
                        "# columns: seed " + " ".join(FIELDS) + " makespan makespan_w31 sha256\n")
                for seed, r in rows:
                    f.write(line([seed] + [r[k] for k in FIELDS] + [r["makespan"], r["makespan_w31"], r["sha256"]]) + "\n")
            print("cholesky64 done", flush=True)
        if big is not None:
            rec = big.get()[0]
            rec = dict(cite="oracle on the layered DAG of 1,000 layers x 16,000 vertices, 128,000,000 edges, seed 0 "
                            "(partition seed 0, ratio from Eq. (1), tolerance 3%); sha256 over the split's n bytes",
                       args=dict(r_cpu=-1.0, tol=0.03, seed=0), **rec)
            with open(os.path.join(HERE, "layered16m_oracle.json"), "w") as f:
                json.dump(rec, f, indent=1)
                f.write("\n")
            print("layered16m done", rec["oracle_s"], flush=True)


if __name__ == "__main__":
    main(set(sys.argv[1:]) or {"layered16m", "batch", "cholesky64"})
