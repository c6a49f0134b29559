"""k device classes by recursive bisection (gp_partition_kway) against the oracle: every vertex's
class, the cut, every class's load and the feasibility flag, bit-exact, through the C-ABI.

k = 2 must be the 2-way partition; k = 3 and 4 exercise the group times, the induced subgraphs and
the recursion; k = 1, an empty side, host and device buffers, and the validation precedence."""
import numpy as np
import pytest

import oracle
import paper_1502_07451_b300 as gp
from paper_1502_07451_b300 import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("offsets", "cols", "edge_cost")


def classes(g, k, seed):
    """Times of k classes: the CPU and GPU times, then accelerator-like classes derived from them."""
    rng = np.random.default_rng(seed)
    cs = [g["cpu_cost"].astype(np.int64), g["gpu_cost"].astype(np.int64)]
    for i in range(2, k):
        f = rng.uniform(0.1, 0.9, g["n"]) if i % 2 == 0 else rng.uniform(0.5, 3.0, g["n"])
        cs.append(np.floor(cs[i % 2] * f).astype(np.int64))
    return np.ascontiguousarray(np.stack(cs[:k]).astype(np.int32))


def run(g, cs, device=True, tol=0.03, seed=0):
    n = g["n"]
    if device:
        d = {k: torch.from_numpy(np.ascontiguousarray(g[k])).cuda() for k in KEYS}
        d.update(n=n, m=g["m"])
        dcs = torch.from_numpy(cs).cuda()
        out = torch.full((max(n, 1),), 255, dtype=torch.uint8, device="cuda")
        r = gp.gp_partition_kway(d, dcs, out, tol=tol, seed=seed)
        return out.cpu().numpy()[:n], r
    out = np.full(max(n, 1), 255, np.uint8)
    r = gp.gp_partition_kway(g, cs, out, tol=tol, seed=seed)
    return out[:n], r


FIXTURES = {
    "cholesky16": lambda: gen.cholesky(16),
    "lu12": lambda: gen.lu(12),
    "layered_small": lambda: gen.layered(40, 150, 40000, 7),
    "random2k": lambda: gen.random_dag(2000, 9000, 5),
    "layered100k": lambda: gen.layered(100, 1000, 800000, 3),
}


@pytest.mark.parametrize("name", sorted(FIXTURES))
@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_kway_matches_oracle(name, k):
    g = FIXTURES[name]()
    cs = classes(g, k, k)
    cls, r = run(g, cs, seed=k)
    ocls, orr = oracle.partition_kway(g, cs, seed=k)
    assert np.array_equal(cls, ocls)
    assert r == orr


def test_kway_two_classes_is_gp_partition():
    g = gen.lu(10)
    cs = np.ascontiguousarray(np.stack([g["cpu_cost"], g["gpu_cost"]]).astype(np.int32))
    cls, r = run(g, cs, device=False)
    with gp.Graph({k: torch.from_numpy(np.ascontiguousarray(v)).cuda() if isinstance(v, np.ndarray) else v
                   for k, v in g.items()}) as G:
        part = torch.empty(g["n"], dtype=torch.uint8, device="cuda")
        res = G.partition(part)
    assert np.array_equal(cls, part.cpu().numpy())
    assert r["cut"] == res["cut"] and r["loads"] == [res["load_cpu"], res["load_gpu"]]


def test_kway_edge_cases():
    g = gen.cholesky(6)
    one = np.ascontiguousarray(g["cpu_cost"][None, :].astype(np.int32))
    cls, r = run(g, one)
    assert not cls.any() and r == oracle.partition_kway(g, one)[1]
    # a class that wins nothing: its times are far above the others'
    cs = classes(g, 3, 1)
    cs[2] = np.int32(2_000_000_000)
    cls, r = run(g, cs, device=False)
    ocls, orr = oracle.partition_kway(g, cs)
    assert np.array_equal(cls, ocls) and r == orr
    empty = gen.from_edges(0, [], [], [], [])
    cls, r = run(empty, np.zeros((3, 0), np.int32), device=False)
    assert r == oracle.partition_kway(empty, np.zeros((3, 0), np.int32))[1]


def test_kway_validation_precedence():
    g = gen.cholesky(4)
    n = g["n"]
    cs = classes(g, 3, 0)
    for bad_k in (np.zeros((0, n), np.int32),):
        with pytest.raises(gp.GpError) as e:
            run(g, bad_k, device=False)
        assert e.value.status == gp.GP_ERR_INVALID
    neg = cs.copy()
    neg[2, 5] = -1
    cyc = gen.from_edges(3, [(0, 1), (1, 2), (2, 0)], [1, 1, 1], [1, 1, 1], [1, 1, 1])
    cases = [(g, neg), (g, cs, 1.5), (cyc, np.ones((2, 3), np.int32)),
             (cyc, np.array([[1, 1, 1], [1, -1, 1]], np.int32))]
    for case in cases:
        gg, cc = case[0], case[1]
        tol = case[2] if len(case) > 2 else 0.03
        with pytest.raises(oracle.OracleError) as oe:
            oracle.partition_kway(gg, cc, tol=tol)
        with pytest.raises(gp.GpError) as e:
            run(gg, cc, device=False, tol=tol)
        assert e.value.status == oe.value.status
