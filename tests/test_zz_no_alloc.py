"""gp_makespan_noalloc: the makespan for callers that cannot allocate device memory.

It must give exactly what gp_makespan gives (integer results, so equality is
the tolerance), on two calls in a row (the second one finds the first one's
leftovers in the shared scratch array), and refuse graphs over its limit.
This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import paper_1502_07451_b300 as gp
from paper_1502_07451_b300 import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("offsets", "cols", "edge_cost", "cpu_cost", "gpu_cost")


def to_device(g):
    return {k: (torch.from_numpy(np.ascontiguousarray(v)).cuda() if k in KEYS else v) for k, v in g.items()}


@pytest.mark.parametrize("make", [lambda: gen.cholesky(16), lambda: gen.layered(60, 500, 120000, 4),
                                  lambda: gen.random_dag(5000, 30000, 9)])
def test_noalloc_makespan_equals_makespan_twice(make):
    g = make()
    n = g["n"]
    rng = np.random.default_rng(n)
    with gp.Graph(to_device(g)) as G:
        parts = [torch.from_numpy(rng.integers(0, 2, n).astype(np.uint8)).cuda(),
                 torch.ones(n, dtype=torch.uint8, device="cuda")]
        for part in parts:
            fin_ref = torch.empty(n, dtype=torch.int64, device="cuda")
            want = G.makespan(part, fin_ref)
            for _ in range(2):
                fin = torch.full((n,), -1, dtype=torch.int64, device="cuda")
                got = gp.gp_makespan_noalloc(G.h, part, fin)
                assert got == want
                assert torch.equal(fin, fin_ref)
            assert gp.gp_makespan_noalloc(G.h, part) == want


def test_noalloc_rejects_what_it_cannot_hold():
    n = gp.MAKESPAN_NOALLOC_MAX_N + 1
    g = gen.from_edges(n, [], np.ones(n, np.int64), np.ones(n, np.int64), [])
    with gp.Graph(to_device(g)) as G:
        part = torch.zeros(n, dtype=torch.uint8, device="cuda")
        assert G.makespan(part) == 1
        with pytest.raises(gp.GpError) as e:
            gp.gp_makespan_noalloc(G.h, part)
        assert e.value.status == gp.GP_ERR_INVALID
    small = gen.cholesky(4)
    with gp.Graph(to_device(small)) as G:
        with pytest.raises(gp.GpError):
            gp.gp_makespan_noalloc(G.h, np.ones(small["n"], np.uint8))  # host memory is refused
