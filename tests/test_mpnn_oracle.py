"""Pins of the learned proposal's CPU oracle: the FP64 network (oracle/mpnn.py) and the proposal
rule (og_propose / og_partition_learned).

The network's gradient is pinned by central finite differences of its own loss; its forward pass
by a hand-worked chain where the weights isolate one aggregation direction at a time, and by
relabelling invariance.  The proposal rule by hand examples of the prefix, the float total order
and the rejection of NaN."""
import numpy as np
import pytest

import oracle
from oracle import mpnn
from paper_1502_07451_b300 import gen


def rand_params(seed, scale=0.3):
    return np.random.RandomState(seed).randn(mpnn.NPARAMS) * scale


def test_param_count_matches_layout():
    assert mpnn.NPARAMS == 37505
    p = rand_params(0)
    assert np.array_equal(mpnn.pack(mpnn.unpack(p)), p)


@pytest.mark.parametrize("seed", [1, 2])
def test_gradient_matches_central_differences(seed):
    g = gen.random_dag(24, 60, seed)
    S = mpnn.structure(g)
    P = rand_params(seed)
    y = (np.random.RandomState(seed + 7).rand(g["n"]) < 0.3).astype(float)
    loss, grad = mpnn.loss_and_grad(P, S, y)
    rs = np.random.RandomState(seed + 11)
    idx = np.concatenate([rs.choice(mpnn.NPARAMS, 300, replace=False), np.arange(mpnn.NPARAMS - 65, mpnn.NPARAMS)])
    eps = 1e-6
    num = np.empty(idx.shape[0])
    for t, i in enumerate(idx):
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += eps
        Pm[i] -= eps
        num[t] = (mpnn.loss_and_grad(Pp, S, y)[0] - mpnn.loss_and_grad(Pm, S, y)[0]) / (2 * eps)
    err = np.abs(num - grad[idx])
    assert np.all(err <= 1e-6 + 1e-4 * np.abs(num)), float(err.max())
    assert np.abs(grad).sum() > 0


def _chain_graph():
    # a -> b -> c with distinct costs; no parallel entries
    return gen.from_edges(3, [(0, 1), (1, 2)], [1000, 2000, 4000], [10, 20, 40], [100, 300])


def _select_params(in_w, out_w):
    """h0 = feature 0 (log1p(cpu)/16) in unit 0; layer 1 puts in_w * ain[0] + out_w * aout[0] into
    unit 0; layers 2 and 3 pass unit 0 through; logit = unit 0.  All values stay >= 0, so no ReLU
    clips them."""
    P = {name: np.zeros(shape) for name, shape in mpnn.SHAPES}
    P["W_in"][0, 0] = 1.0
    P["W1"][64 + 0, 0] = in_w
    P["W1"][128 + 0, 0] = out_w
    P["W2"][0, 0] = 1.0
    P["W3"][0, 0] = 1.0
    P["w_o"][0] = 1.0
    return mpnn.pack(P)


def test_forward_direction_and_normalisation_by_hand():
    g = _chain_graph()
    S = mpnn.structure(g)
    x0 = np.log1p([1000.0, 2000.0, 4000.0]) / 16
    e1, e2 = np.log1p(100.0) / 16, np.log1p(300.0) / 16
    # predecessors only: ain_a = 0, ain_b = e1 x0_a, ain_c = e2 x0_b (in-degree 1 each)
    logit, _ = mpnn.forward(_select_params(1.0, 0.0), S)
    assert np.allclose(logit, [0.0, e1 * x0[0], e2 * x0[1]], rtol=1e-14, atol=0)
    # successors only: aout_a = e1 x0_b, aout_b = e2 x0_c, aout_c = 0
    logit, _ = mpnn.forward(_select_params(0.0, 1.0), S)
    assert np.allclose(logit, [e1 * x0[1], e2 * x0[2], 0.0], rtol=1e-14, atol=0)


def test_forward_fan_in_is_a_mean_and_parallel_entries_count():
    # u0 -> v, u1 -> v, u1 -> v (parallel): in-degree 3
    g = gen.from_edges(3, [(0, 2), (1, 2), (1, 2)], [1000, 3000, 5000], [1, 1, 1], [50, 70, 90])
    S = mpnn.structure(g)
    x0 = np.log1p([1000.0, 3000.0, 5000.0]) / 16
    e = np.log1p([50.0, 70.0, 90.0]) / 16
    logit, _ = mpnn.forward(_select_params(1.0, 0.0), S)
    assert np.isclose(logit[2], (e[0] * x0[0] + e[1] * x0[1] + e[2] * x0[1]) / 3, rtol=1e-14)
    logit, _ = mpnn.forward(_select_params(0.0, 1.0), S)
    assert np.isclose(logit[1], (e[1] + e[2]) * x0[2] / 2, rtol=1e-14)


def test_forward_is_relabelling_equivariant():
    g = gen.random_dag(40, 120, 3)
    n = g["n"]
    perm = np.random.RandomState(5).permutation(n)  # old id -> new id
    src = np.repeat(np.arange(n), np.diff(g["offsets"]))
    edges = list(zip(perm[src].tolist(), perm[g["cols"]].tolist()))
    cpu = np.empty(n, np.int64)
    gpu = np.empty(n, np.int64)
    cpu[perm] = g["cpu_cost"]
    gpu[perm] = g["gpu_cost"]
    order = np.lexsort((perm[g["cols"]], perm[src]))
    h = gen.from_edges(n, [edges[i] for i in order], cpu, gpu, g["edge_cost"][order])
    P = rand_params(9)
    la, _ = mpnn.forward(P, mpnn.structure(g))
    lb, _ = mpnn.forward(P, mpnn.structure(h))
    assert np.allclose(lb[perm], la, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------------------
# the proposal rule
# ---------------------------------------------------------------------------

def test_propose_prefix_rule_by_hand():
    # order by logit desc: v2 (3.0), v0 (2.0), v3 (2.0, larger id), v1 (-1.0)
    logits = np.array([2.0, -1.0, 3.0, 2.0], np.float32)
    vC = np.array([4, 1, 5, 3])
    vG = np.array([2, 1, 2, 1])  # SG = 6
    # B_C = 9: prefix CPU loads 5, 9, 12 -> kC = 2; B_G = 3: GPU loads 6, 4, 2 -> kG = 2
    part, k = oracle.propose(logits, vC, vG, 9, 3)
    assert k == 2 and part.tolist() == [0, 1, 0, 1]
    # B_G = 5: GPU load 4 after one vertex -> kG = 1 < kC
    part, k = oracle.propose(logits, vC, vG, 9, 5)
    assert k == 1 and part.tolist() == [1, 1, 0, 1]
    # B_C = 4: the first vertex (CPU 5) does not fit -> kC = 0
    part, k = oracle.propose(logits, vC, vG, 4, 0)
    assert k == 0 and part.tolist() == [1, 1, 1, 1]
    # everything fits on the GPU: nothing moves
    part, k = oracle.propose(logits, vC, vG, 100, 6)
    assert k == 0


def test_propose_float_total_order_and_nan():
    # -0.0 sorts below +0.0; -inf last; +inf first
    logits = np.array([-0.0, 0.0, -np.inf, np.inf, -1e-45], np.float32)
    vC = np.ones(5, np.int64)
    vG = np.ones(5, np.int64)
    part, k = oracle.propose(logits, vC, vG, 2, 3)  # kC = 2, kG = 2
    assert k == 2 and part.tolist() == [1, 0, 1, 0, 1]  # +inf (3), +0.0 (1)
    part, k = oracle.propose(logits, vC, vG, 3, 2)  # kC = 3, kG = 3: then -0.0 (0)
    assert k == 3 and part.tolist() == [0, 0, 1, 0, 1]
    with pytest.raises(RuntimeError):
        oracle.propose(np.array([0.0, np.nan], np.float32), np.ones(2), np.ones(2), 1, 1)


def test_learned_path_result_fields():
    g = gen.cholesky(6)
    logits = np.random.RandomState(0).randn(g["n"]).astype(np.float32)
    part, res = oracle.partition_learned(g, logits)
    assert res["levels"] == 0 and res["coarsest_n"] == g["n"]
    assert res["cut"] == oracle.cut(g, part)
    cC = g["cpu_cost"]
    cG = g["gpu_cost"]
    assert res["load_cpu"] == int(cC[part == 0].sum()) and res["load_gpu"] == int(cG[part == 1].sum())
    # the refinement only improves on the proposal's cut when the proposal is feasible
    p0, _ = oracle.propose(logits, cC, cG, res["bound_cpu"], res["bound_gpu"])
    if cC[p0 == 0].sum() <= res["bound_cpu"] and cG[p0 == 1].sum() <= res["bound_gpu"]:
        assert res["cut"] <= oracle.cut(g, p0)
