"""Fixed vertices on the GPU (gp_partition_fixed) against the oracle, bit-exact.

Sec. III.B roots every initial kernel at an empty kernel whose data sit in host memory; pinning that
vertex to the CPU, and more generally any vertex to either side, changes the matching (pinned to
different sides never merge), the coarse pins, the growing (starts from the pinned split, moves free
vertices only, pre-check on the split with every free vertex on the GPU) and refinement (pinned
vertices never move).  Each case compares the split, every result field and the per-level trace
with the oracle on the same seeded input and pins; the pinned sets are dense enough that adjacent
vertices pinned to opposite sides are common, and the graphs reach the one-CTA, cluster and
whole-grid refinement stages.
"""
import numpy as np
import pytest

import oracle
import paper_1502_07451_b300 as gp
from paper_1502_07451_b300 import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TRACE_KEYS = ("levels", "gggp_trial", "n", "a", "rounds", "moves", "balanced", "bal_moves")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def dgraph(g):
    return {k: (dev(v) if k in ("offsets", "cols", "edge_cost", "cpu_cost", "gpu_cost") else v) for k, v in g.items()}


def pins(n, seed, frac):
    r = gen.u64(seed, 44, 0, n)
    fx = np.full(n, -1, np.int8)
    sel = (r % np.uint64(1000)).astype(np.int64) < int(frac * 1000)
    fx[sel] = ((r[sel] >> np.uint64(20)) & np.uint64(1)).astype(np.int8)
    return fx


def host_source(g, seed):
    h, s = gen.with_host_source(g, seed)
    fx = np.full(h["n"], -1, np.int8)
    fx[s] = 0
    return h, fx


def check(g, fx, r=-1.0, tol=0.03, seed=0, fixed_on_host=False):
    n = g["n"]
    with gp.Graph(dgraph(g)) as G:
        part = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
        res = G.partition(part, r, tol, seed, fixed=fx if fixed_on_host else dev(fx))
        tr = G.trace()
        p = part.cpu().numpy()[:n]
    opart, ores, otr = oracle.partition(g, r, tol, seed, trace=True, fixed=fx)
    assert np.array_equal(p, opart)
    assert {k: res[k] for k in ores} == ores
    for k in TRACE_KEYS:
        assert tr[k] == otr[k], k
    assert np.all(p[fx >= 0] == fx[fx >= 0])
    return res, tr


CASES = {
    "cholesky16_p10": lambda: (gen.cholesky(16), pins(816, 1, 0.1)),
    "lu10_p30": lambda: (gen.lu(10), pins(gen.lu_tasks(10), 2, 0.3)),
    "random2k_p20": lambda: (gen.random_dag(2000, 9000, 5), pins(2000, 3, 0.2)),
    "layered6k_p2": lambda: (gen.layered(40, 150, 40000, 7), pins(6000, 4, 0.02)),
    "layered6k_p30": lambda: (gen.layered(40, 150, 40000, 7), pins(6000, 5, 0.3)),
    "layered6k_p60": lambda: (gen.layered(40, 150, 40000, 7), pins(6000, 6, 0.6)),
    "layered50k_p10": lambda: (gen.layered(100, 500, 200000, 8), pins(50000, 7, 0.1)),
    "hub1000": lambda: (gen.from_edges(1001, [(0, i) for i in range(1, 1001)], [10] * 1001, [5] * 1001, [1] * 1000),
                        np.array([0] + [1, -1] * 500, np.int8)),
    "host_source_layered6k": lambda: host_source(gen.layered(40, 150, 40000, 9), 9),
    "host_source_speed_gap": lambda: host_source(gen.random_dag(600, 2000, 2, ratio_pct=(1, 3)), 2),
    "all_pinned": lambda: (gen.cholesky(8), (gen.u64(0, 45, 0, 120) & np.uint64(1)).astype(np.int8)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_fixed_partition_parity(name):
    g, fx = CASES[name]()
    res, tr = check(g, fx, seed=len(name))
    if name == "host_source_speed_gap":
        assert tr["gggp_trial"] == -1  # the pre-check on the pinned split, decided in the growing kernel


@pytest.mark.parametrize("r,tol", [(0.3, 0.03), (0.0, 0.03), (1.0, 0.05)])
def test_fixed_explicit_ratios(r, tol):
    g = gen.layered(40, 150, 40000, 7)
    check(g, pins(6000, 11, 0.2), r, tol, seed=3)


def test_fixed_host_buffer_and_all_free():
    g = gen.layered(30, 100, 15000, 12)
    fx = pins(g["n"], 12, 0.25)
    a = check(g, fx, fixed_on_host=True)
    b = check(g, fx)
    assert a == b
    # no pins: exactly gp_partition
    with gp.Graph(dgraph(g)) as G:
        p1 = torch.empty(g["n"], dtype=torch.uint8, device="cuda")
        p2 = torch.empty_like(p1)
        r1 = G.partition(p1, seed=4)
        r2 = G.partition(p2, seed=4, fixed=dev(np.full(g["n"], -1, np.int8)))
        r3 = gp.gp_partition_fixed(G.h, None, -1.0, 0.03, 4, p2)
        assert torch.equal(p1, p2) and r1 == r2 == r3


def test_fixed_bad_values_and_empty_graph():
    g = gen.cholesky(6)
    bad = np.full(g["n"], -1, np.int8)
    bad[7] = 3
    with gp.Graph(dgraph(g)) as G:
        part = torch.empty(g["n"], dtype=torch.uint8, device="cuda")
        with pytest.raises(gp.GpError) as e:
            G.partition(part, fixed=dev(bad))
        assert e.value.status == gp.GP_ERR_INVALID
        bad[7] = -2
        with pytest.raises(gp.GpError):
            G.partition(part, fixed=bad)
        res = G.partition(part, fixed=dev(np.zeros(g["n"], np.int8)))  # the handle stays usable
        assert torch.all(part == 0) and res["load_gpu"] == 0
    empty = gen.from_edges(0, [], [], [], [])
    with gp.Graph(dgraph(empty)) as G:
        res = G.partition(torch.empty(1, dtype=torch.uint8, device="cuda"), fixed=np.zeros(1, np.int8))
        assert res["feasible"] == 1


def test_fixed_host_source_layered_1m_bit_exact():
    """The benchmark's 1,000 x 1,000 layered DAG with the host vertex (every kernel without a
    predecessor reads from it), pinned to the CPU: split, results and trace against the oracle."""
    g, fx = host_source(gen.config_layered_1m(), 0)
    res, tr = check(g, fx)
    assert tr["levels"] >= 10
