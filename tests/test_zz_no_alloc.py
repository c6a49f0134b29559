"""gp_makespan_noalloc: the makespan for callers that cannot allocate device memory.

Some hosts give all device memory to their own allocator and let no one else allocate, and some
loops must not stall on an allocation; this entry point serves them from a scratch array compiled
into the library.  It must give exactly what gp_makespan gives (integer results, so equality is
the tolerance) and what the oracle gives, on two calls in a row (the second one finds the first
one's leftovers in the shared scratch array), on each makespan kernel (the shared-memory ring, the
cluster kernel, the cooperative grid kernel of wide levels), allocate nothing, and refuse graphs
over its limit.  This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import oracle
import paper_1502_07451_b300 as gp
from paper_1502_07451_b300 import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("offsets", "cols", "edge_cost", "cpu_cost", "gpu_cost")

CASES = {
    "cholesky16": lambda: gen.cholesky(16),
    "layered_narrow": lambda: gen.layered(60, 500, 120000, 4),
    "random5k": lambda: gen.random_dag(5000, 30000, 9),
    # 12,000-wide levels: wider than the ring, so the cooperative grid kernel runs
    "layered_wide": lambda: gen.layered(5, 12000, 400000, 12),
}


def to_device(g):
    return {k: (torch.from_numpy(np.ascontiguousarray(v)).cuda() if k in KEYS else v) for k, v in g.items()}


def pool_bytes():
    """(used, reserved) bytes of the current device's memory pool, which the library allocates from,
    and the device's free bytes."""
    from cuda.bindings import driver as cu
    err, dev = cu.cuCtxGetDevice()
    assert err == cu.CUresult.CUDA_SUCCESS
    err, pool = cu.cuDeviceGetMemPool(dev)
    assert err == cu.CUresult.CUDA_SUCCESS
    out = []
    for attr in (cu.CUmemPool_attribute.CU_MEMPOOL_ATTR_USED_MEM_CURRENT,
                 cu.CUmemPool_attribute.CU_MEMPOOL_ATTR_RESERVED_MEM_CURRENT):
        err, v = cu.cuMemPoolGetAttribute(pool, attr)
        assert err == cu.CUresult.CUDA_SUCCESS
        out.append(int(v))
    torch.cuda.synchronize()
    out.append(torch.cuda.mem_get_info()[0])
    return tuple(out)


@pytest.fixture(params=["auto", "cluster"])
def makespan_kernel(request, monkeypatch):
    if request.param == "cluster":
        monkeypatch.setenv("GP_MAKESPAN_KERNEL", "cluster")
    else:
        monkeypatch.delenv("GP_MAKESPAN_KERNEL", raising=False)
    return request.param


@pytest.mark.parametrize("name", sorted(CASES))
def test_noalloc_makespan_equals_makespan_twice(name, makespan_kernel):
    g = CASES[name]()
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
        ms, ofin = oracle.makespan(g, parts[0].cpu().numpy(), with_finish=True)
        fin = torch.empty(n, dtype=torch.int64, device="cuda")
        assert gp.gp_makespan_noalloc(G.h, parts[0], fin) == ms
        assert np.array_equal(fin.cpu().numpy(), ofin)


def test_noalloc_full_size_layered_1m_against_oracle():
    """The 1M-vertex workload (within the 2^20 limit): the split gp_partition gives, evaluated twice
    without allocation, equals the oracle's makespan and finish times and gp_makespan's."""
    g = gen.config_layered_1m()
    n = g["n"]
    with gp.Graph(to_device(g)) as G:
        part = torch.empty(n, dtype=torch.uint8, device="cuda")
        G.partition(part)
        want = G.makespan(part)
        ms, ofin = oracle.makespan(g, part.cpu().numpy(), with_finish=True)
        assert want == ms
        for _ in range(2):
            fin = torch.full((n,), -1, dtype=torch.int64, device="cuda")
            assert gp.gp_makespan_noalloc(G.h, part, fin) == ms
            assert np.array_equal(fin.cpu().numpy(), ofin)


@pytest.mark.parametrize("name", ["cholesky16", "layered_wide"])
def test_noalloc_allocates_nothing(name):
    """After a warm-up call, further calls change neither the pool's used or reserved bytes nor the
    device's free memory."""
    g = CASES[name]()
    n = g["n"]
    with gp.Graph(to_device(g)) as G:
        part = torch.from_numpy(np.random.default_rng(1).integers(0, 2, n).astype(np.uint8)).cuda()
        fin = torch.empty(n, dtype=torch.int64, device="cuda")
        want = G.makespan(part)
        assert gp.gp_makespan_noalloc(G.h, part, fin) == want  # warm-up (first call on the device)
        before = pool_bytes()
        for _ in range(3):
            assert gp.gp_makespan_noalloc(G.h, part, fin) == want
        after = pool_bytes()
        assert after == before, (before, after)


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
