"""Host-side fault injection (GP_FAULT): an allocation that fails as out of memory or as a failed
runtime call, and a partition that reports an expired device wait, each come back as their status
through the C-ABI; nothing is done to the GPU, and the next call (fault switched off) succeeds and
matches the oracle, so the context stays usable."""
import numpy as np
import pytest

import oracle
import paper_1502_07451_b300 as gp
from paper_1502_07451_b300 import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("offsets", "cols", "edge_cost", "cpu_cost", "gpu_cost")


@pytest.mark.parametrize("fault,status", [("oom", gp.GP_ERR_OOM), ("cuda", gp.GP_ERR_CUDA),
                                          ("timeout", gp.GP_ERR_TIMEOUT)])
def test_injected_fault_is_reported_and_the_context_stays_usable(fault, status, monkeypatch):
    g = gen.layered(40, 600, 90000, 2)  # levels above 16,384 vertices: the grid refinement runs
    dg = {k: (torch.from_numpy(np.ascontiguousarray(v)).cuda() if k in KEYS else v) for k, v in g.items()}
    with gp.Graph(dg) as G:
        part = torch.empty(g["n"], dtype=torch.uint8, device="cuda")
        monkeypatch.setenv("GP_FAULT", fault)
        with pytest.raises(gp.GpError) as e:
            G.partition(part)
        assert e.value.status == status
        monkeypatch.delenv("GP_FAULT")
        res = G.partition(part)
        opart, ores = oracle.partition(g)
        assert np.array_equal(part.cpu().numpy(), opart)
        assert {k: res[k] for k in ores} == ores
