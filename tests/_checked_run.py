"""Run by tests/test_checked.py in a child process with GP_LIBRARY=checked: the whole path through the
checked library (every gathered index tested in-kernel) on small and medium inputs, against the oracle,
twice (the second run must give identical bytes), with no failed index test; then the self-test of the
mechanism.  Prints "checked ok" at the end."""
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import oracle  # noqa: E402
import paper_1502_07451_b300 as gp  # noqa: E402
from paper_1502_07451_b300 import gen  # noqa: E402

assert os.environ.get("GP_LIBRARY") == "checked"
assert gp.library_path().endswith("libgp_checked.so"), gp.library_path()
KEYS = ("offsets", "cols", "edge_cost", "cpu_cost", "gpu_cost")
FIELDS = ("cut", "load_cpu", "load_gpu", "bound_cpu", "bound_gpu", "feasible", "levels", "rounds", "coarsest_n")


def dev(g):
    return {k: (torch.from_numpy(np.ascontiguousarray(v)).cuda() if k in KEYS else v) for k, v in g.items()}


def one_pass(g):
    n = g["n"]
    out = {}
    with gp.Graph(dev(g)) as G:
        part = torch.empty(n, dtype=torch.uint8, device="cuda")
        res = G.partition(part)
        out["part"] = part.cpu().numpy()
        out["res"] = {k: res[k] for k in FIELDS}
        out["ms"] = G.makespan(part)
        out["msw"] = gp.gp_makespan_workers(G.h, part, 3, 1)
        fin = torch.empty(n, dtype=torch.int64, device="cuda")
        G.makespan(part, fin)
        out["fin"] = fin.cpu().numpy()
    return out


graphs = [gen.cholesky(16), gen.lu(10), gen.two_input_dag(38, 3, extra=2), gen.random_dag(2000, 9000, 5),
          gen.layered(40, 600, 90000, 2), gen.config_layered_1m()]
for g in graphs:
    a = one_pass(g)
    b = one_pass(g)
    for k in ("part", "fin"):
        assert np.array_equal(a[k], b[k]), k  # a second run gives the same bytes
    assert a["res"] == b["res"] and a["ms"] == b["ms"] and a["msw"] == b["msw"]
    opart, ores = oracle.partition(g)
    assert np.array_equal(a["part"], opart) and a["res"] == ores
    oms, ofin = oracle.makespan(g, opart, with_finish=True)
    assert a["ms"] == oms and np.array_equal(a["fin"], ofin)
    assert a["msw"] == oracle.makespan_workers(g, opart, 3, 1)
    assert gp.gp_checked_site(True) == 0, g["n"]

# the batch path and k-way on a small mix
specs = gen.batch_spec(24, nmin=100, nmax=4000, base_seed=7)
small = [gen.build_from_spec(it) for it in specs]
Gs = [gp.Graph(dev(g)) for g in small]
parts = [torch.zeros(max(g["n"], 1), dtype=torch.uint8, device="cuda") for g in small]
res, mks = gp.gp_batch_partition([G.h for G in Gs], parts, makespans=True)
for i, g in enumerate(small):
    opart, ores = oracle.partition(g)
    assert np.array_equal(parts[i].cpu().numpy()[: g["n"]], opart) and {k: res[i][k] for k in FIELDS} == ores
for G in Gs:
    G.close()
g = gen.layered(40, 150, 40000, 7)
cs = gen.kway_costs(g, 3, 0)
cls = np.zeros(g["n"], np.uint8)
r = gp.gp_partition_kway(g, cs, cls)
ocls, orr = oracle.partition_kway(g, cs)
assert np.array_equal(cls, ocls) and r == orr
assert gp.gp_checked_site(True) == 0

# the mechanism itself: a gather through an out-of-range index behind its test is skipped and recorded
gp.gp_selftest_checked()
assert gp.gp_checked_site(True) == 99
assert gp.gp_checked_site(True) == 0
print("checked ok")
