"""The tensor-core GEMM of the learned proposal (tcgen05, BF16 inputs, FP32 accumulation in tensor
memory) against a plain FP32 product of the same BF16 values.

Products of BF16 values are exact in FP32, so the only difference is the summation order:
the bound is K * 2^-23 * sum |a||b| per entry (FP32 accumulation)."""
import numpy as np
import pytest

import paper_1502_07451_b300 as gp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 64, 192), (1000, 64, 192), (77, 192, 64), (4097, 192, 64),
                                   (129, 64, 64), (1, 64, 192), (300000, 64, 192)])
def test_mma_bf16_matches_fp32_reference(M, N, K):
    g = torch.Generator(device="cpu").manual_seed(M * 131 + N * 7 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(K, N, generator=g).to(torch.bfloat16).cuda()
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    gp.gp_step_mma_bf16(A, B, C)
    ref = A.double() @ B.double()
    bound = K * 2.0 ** -22 * (A.double().abs() @ B.double().abs()) + 1e-30
    err = (C.double() - ref).abs()
    assert torch.isfinite(C).all()
    assert (err <= bound).all(), float((err / bound).max())


def test_mma_rejects_bad_shapes():
    A = torch.zeros(8, 48, dtype=torch.bfloat16, device="cuda")
    B = torch.zeros(48, 64, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(8, 64, dtype=torch.float32, device="cuda")
    with pytest.raises(gp.GpError) as e:
        gp.gp_step_mma_bf16(A, B, C)
    assert e.value.status == gp.GP_ERR_INVALID
    with pytest.raises(gp.GpError):
        gp.gp_step_mma_bf16(A.cpu(), B.cpu(), C.cpu())


def test_grid_barrier_wait_gives_up_and_the_context_stays_usable():
    """The grid barrier of the wide-level makespan and the large-level refinement: with one CTA that
    never arrives, the other's bounded wait gives up (GP_ERR_TIMEOUT), and a partition that uses the
    barrier then runs normally."""
    import time
    import oracle
    from paper_1502_07451_b300 import gen
    L = gp.lib()
    t0 = time.perf_counter()
    assert L.gp_selftest_grid_wait_timeout(None) == gp.GP_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    g = gen.layered(40, 600, 90000, 3)  # levels above 16,384 vertices: the grid refinement runs
    dg = {k: torch.from_numpy(g[k]).cuda() for k in ("offsets", "cols", "edge_cost", "cpu_cost", "gpu_cost")}
    with gp.Graph(dict(dg, n=g["n"], m=g["m"])) as G:
        part = torch.empty(g["n"], dtype=torch.uint8, device="cuda")
        res = G.partition(part)
    opart, ores = oracle.partition(g)
    assert np.array_equal(part.cpu().numpy(), opart) and res["cut"] == ores["cut"]


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """A device wait on an mbarrier that nothing arrives at gives up after its limit and reports
    GP_ERR_TIMEOUT; tensor memory is released and the next product runs normally."""
    L = gp.lib()
    assert L.gp_selftest_wait_timeout(50, None) == gp.GP_ERR_TIMEOUT
    assert L.gp_selftest_wait_timeout(0, None) == gp.GP_ERR_INVALID
    A = torch.randn(256, 192).to(torch.bfloat16).cuda()
    B = torch.randn(192, 64).to(torch.bfloat16).cuda()
    C = torch.empty(256, 64, device="cuda")
    gp.gp_step_mma_bf16(A, B, C)
    assert torch.allclose(C.double(), A.double() @ B.double(), rtol=1e-3, atol=1e-3)
