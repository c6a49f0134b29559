"""Writes oracle_small.json: the oracle's full results on small seeded
fixtures.  Calls only oracle/ and the input generators; rerun it (and say why
in the commit) only when the oracle's arithmetic changes on purpose."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1502_07451_b300 import gen  # noqa: E402


def fixtures():
    yield "cholesky16", gen.cholesky(16), dict(r_cpu=-1.0, tol=0.03, seed=0)
    yield "lu12", gen.lu(12), dict(r_cpu=-1.0, tol=0.03, seed=1)
    yield "two_input38", gen.two_input_dag(38, 5, extra=2), dict(r_cpu=-1.0, tol=0.03, seed=2)
    yield "random500", gen.random_dag(500, 1500, 3), dict(r_cpu=-1.0, tol=0.05, seed=3)
    yield "random500_r30", gen.random_dag(500, 1500, 3), dict(r_cpu=0.3, tol=0.03, seed=4)


def main():
    out = {"cite": "oracle results on seeded fixtures (regression record of the oracle's own arithmetic)", "cases": []}
    for name, g, kw in fixtures():
        part, res, tr = oracle.partition(g, trace=True, **kw)
        ms = oracle.makespan(g, part)
        out["cases"].append(dict(name=name, args=kw, result=res, makespan=ms,
                                 part_hex=np.packbits(part).tobytes().hex(), levels_n=tr["n"],
                                 rounds=tr["rounds"], gggp_trial=tr["gggp_trial"]))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_small.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
