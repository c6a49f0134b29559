"""The learned proposal on the GPU: the network against the FP64 oracle (BF16 tolerance), the
learned path against the oracle given the same logits (bit-exact), training, checkpoints, and
what the trained network gains over the method without it.

The layer products run in BF16 with FP32 accumulation: inputs carry a relative rounding error of
2^-9, so logits and gradients are compared within a few percent (logits: max error <= 3% of the
logit scale; gradients: cosine >= 0.999 and relative L2 error <= 2e-2), the bound stated for the
network.  Everything downstream of the logits is integer and must match exactly."""
import os
import tempfile

import numpy as np
import pytest

import oracle
from oracle import mpnn
import paper_1502_07451_b300 as gp
from paper_1502_07451_b300 import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("cut", "load_cpu", "load_gpu", "bound_cpu", "bound_gpu", "feasible", "levels", "rounds", "coarsest_n")


def dgraph(g):
    return {k: (torch.from_numpy(np.ascontiguousarray(v)).cuda()
                if isinstance(v, np.ndarray) and k in ("offsets", "cols", "edge_cost", "cpu_cost", "gpu_cost")
                else v) for k, v in g.items()}


class Model:
    def __init__(self, seed=0, params=None):
        self.h = gp.gp_model_create(seed)
        if params is not None:
            gp.gp_model_set_params(self.h, params)

    def close(self):
        if self.h is not None:
            gp.gp_model_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def structure_of(g, G):
    lev, nl = oracle.levels(g)
    return mpnn.structure(g, lev, nl)


def gpu_logits(M, G, n):
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    gp.gp_model_forward(M.h, G.h, out)
    return out.cpu().numpy().astype(np.float64)


GRAPHS = {
    "cholesky8": lambda: gen.cholesky(8),
    "lu6": lambda: gen.lu(6),
    "random500": lambda: gen.random_dag(500, 3000, 4),
    "layered3k": lambda: gen.layered(30, 100, 12000, 5),
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_forward_matches_oracle(name):
    g = GRAPHS[name]()
    with gp.Graph(dgraph(g)) as G, Model(seed=3) as M:
        P = gp.gp_model_get_params(M.h).astype(np.float64)
        ref, _ = mpnn.forward(P, structure_of(g, G))
        got = gpu_logits(M, G, g["n"])
    scale = max(1.0, float(np.abs(ref).max()))
    assert np.abs(got - ref).max() <= 0.03 * scale, float(np.abs(got - ref).max())
    assert np.corrcoef(got, ref)[0, 1] > 0.999


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_gradient_matches_oracle(name):
    g = GRAPHS[name]()
    labels, _ = oracle.partition(g)
    with gp.Graph(dgraph(g)) as G, Model(seed=5) as M:
        P = gp.gp_model_get_params(M.h).astype(np.float64)
        loss, grad = gp.gp_model_grad(M.h, G.h, torch.from_numpy(labels).cuda())
    rl, rg = mpnn.loss_and_grad(P, structure_of(g, G), mpnn.labels_from_part(labels))
    assert abs(loss - rl) <= 2e-2 * max(1.0, abs(rl))
    grad = grad.astype(np.float64)
    cos = grad @ rg / (np.linalg.norm(grad) * np.linalg.norm(rg))
    rel = np.linalg.norm(grad - rg) / np.linalg.norm(rg)
    assert cos >= 0.999 and rel <= 2e-2, (cos, rel)
    # every block of the parameter vector
    o = 0
    for nm, shape in mpnn.SHAPES:
        k = int(np.prod(shape))
        a, b = grad[o:o + k], rg[o:o + k]
        if np.linalg.norm(b) > 1e-9:
            assert np.linalg.norm(a - b) <= 5e-2 * np.linalg.norm(b) + 1e-7, nm
        o += k


def test_forward_is_deterministic():
    g = gen.layered(50, 200, 40000, 8)
    with gp.Graph(dgraph(g)) as G, Model(seed=1) as M:
        a = gpu_logits(M, G, g["n"])
        b = gpu_logits(M, G, g["n"])
    assert np.array_equal(a, b)


@pytest.mark.parametrize("name", sorted(GRAPHS) + ["layered_big"])
def test_learned_path_matches_oracle_given_logits(name):
    g = GRAPHS[name]() if name in GRAPHS else gen.layered(200, 500, 400000, 12)
    with gp.Graph(dgraph(g)) as G, Model(seed=7) as M:
        logits = torch.empty(g["n"], dtype=torch.float32, device="cuda")
        gp.gp_model_forward(M.h, G.h, logits)
        part = torch.empty(g["n"], dtype=torch.uint8, device="cuda")
        res = gp.gp_partition_learned(G.h, M.h, part)          # logits from the network
        part2 = torch.empty(g["n"], dtype=torch.uint8, device="cuda")
        res2 = gp.gp_partition_learned(G.h, None, part2, logits=logits)  # the same logits, passed in
        ref_part, ref = oracle.partition_learned(g, logits.cpu().numpy())
    assert np.array_equal(part.cpu().numpy(), ref_part)
    assert np.array_equal(part2.cpu().numpy(), ref_part)
    for k in KEYS:
        assert res[k] == ref[k] and res2[k] == ref[k], k


def test_learned_path_edge_cases():
    g = gen.cholesky(10)
    n = g["n"]
    with gp.Graph(dgraph(g)) as G:
        cases = {
            "ties": np.zeros(n, np.float32),
            "signed_zero": np.where(np.arange(n) % 2 == 0, -0.0, 0.0).astype(np.float32),
            "infinite": np.where(np.arange(n) % 3 == 0, np.inf, -np.inf).astype(np.float32),
            "ramp": np.arange(n, dtype=np.float32) * 1e-3,
        }
        for nm, lg in cases.items():
            for r in (-1.0, 0.0, 1.0, 0.3):
                part = torch.empty(n, dtype=torch.uint8, device="cuda")
                res = gp.gp_partition_learned(G.h, None, part, logits=torch.from_numpy(lg).cuda(), r_cpu=r)
                ref_part, ref = oracle.partition_learned(g, lg, r_cpu=r)
                assert np.array_equal(part.cpu().numpy(), ref_part), (nm, r)
                assert all(res[k] == ref[k] for k in KEYS), (nm, r)
        bad = np.zeros(n, np.float32)
        bad[5] = np.nan
        with pytest.raises(gp.GpError) as e:
            gp.gp_partition_learned(G.h, None, torch.empty(n, dtype=torch.uint8, device="cuda"),
                                    logits=torch.from_numpy(bad).cuda())
        assert e.value.status == gp.GP_ERR_INVALID
        # host buffers
        hp = np.zeros(n, np.uint8)
        lg = np.random.RandomState(1).randn(n).astype(np.float32)
        gp.gp_partition_learned(G.h, None, hp, logits=lg)
        assert np.array_equal(hp, oracle.partition_learned(g, lg)[0])


def _train_set(count, seed):
    spec = gen.batch_spec(count, nmin=400, nmax=6000, base_seed=seed)
    return [gen.build_from_spec(it) for it in spec]


def test_training_is_deterministic_and_checkpoints_roundtrip():
    gs = _train_set(6, 100)
    Gs = [gp.Graph(dgraph(g)) for g in gs]
    labs = []
    for G in Gs:
        p = torch.empty(G.n, dtype=torch.uint8, device="cuda")
        G.partition(p)
        labs.append(p)
    try:
        finals = []
        for rep in range(2):
            with Model(seed=11) as M:
                for step in range(12):
                    i = step % len(Gs)
                    gp.gp_model_train_step(M.h, Gs[i].h, labs[i], 3e-3)
                finals.append(gp.gp_model_get_params(M.h).copy())
                if rep == 0:
                    d = tempfile.mkdtemp()
                    path = os.path.join(d, "m.bin")
                    gp.gp_model_save(M.h, path)
                    M2 = gp.gp_model_load(path)
                    try:
                        assert np.array_equal(gp.gp_model_get_params(M2), finals[0])
                        l1 = torch.empty(Gs[0].n, device="cuda")
                        l2 = torch.empty(Gs[0].n, device="cuda")
                        gp.gp_model_forward(M.h, Gs[0].h, l1)
                        gp.gp_model_forward(M2, Gs[0].h, l2)
                        assert torch.equal(l1, l2)
                        # the optimiser state travels too: one more step gives the same parameters
                        gp.gp_model_train_step(M.h, Gs[1].h, labs[1], 3e-3)
                        gp.gp_model_train_step(M2, Gs[1].h, labs[1], 3e-3)
                        assert np.array_equal(gp.gp_model_get_params(M.h), gp.gp_model_get_params(M2))
                    finally:
                        gp.gp_model_destroy(M2)
                    # the checksum: a flipped byte, a truncated or a longer file are refused
                    raw = open(path, "rb").read()
                    for bad in (raw[:100] + bytes([raw[100] ^ 1]) + raw[101:], raw[:-5], raw + b"\0"):
                        with open(path, "wb") as f:
                            f.write(bad)
                        with pytest.raises(gp.GpError) as e:
                            gp.gp_model_load(path)
                        assert e.value.status == gp.GP_ERR_INVALID
                    # a version-1 file (no checksum) still loads, with the same parameters
                    with open(path, "wb") as f:
                        f.write(raw[:8] + (1).to_bytes(4, "little") + raw[12:-8])
                    M3 = gp.gp_model_load(path)
                    try:
                        assert np.array_equal(gp.gp_model_get_params(M3), finals[0])
                    finally:
                        gp.gp_model_destroy(M3)
        assert np.array_equal(finals[0], finals[1])  # same seed, same data: same parameters
    finally:
        for G in Gs:
            G.close()


def test_trained_network_gains_over_the_method_without_it():
    """Train on generated DAGs labelled by the plain method, then on held-out DAGs compare the
    learned path (network proposal + flat refinement) with the same flat refinement started from
    the untrained network's proposal, and report the plain multilevel path beside them."""
    train = _train_set(48, 2000)
    held = [gen.layered(40, 250, 80000, 9000 + i) for i in range(3)] + [gen.cholesky(24), gen.lu(20)]
    Gs = [gp.Graph(dgraph(g)) for g in train]
    Hs = [gp.Graph(dgraph(g)) for g in held]
    try:
        labs = []
        for G in Gs:
            p = torch.empty(G.n, dtype=torch.uint8, device="cuda")
            G.partition(p)
            labs.append(p)
        with Model(seed=21) as M0, Model(seed=21) as M:
            losses = []
            for ep in range(6):
                for i in range(len(Gs)):
                    losses.append(gp.gp_model_train_step(M.h, Gs[i].h, labs[i], 2e-3))
            assert np.mean(losses[-len(Gs):]) < 0.8 * np.mean(losses[:len(Gs)])
            tot = {"trained": 0, "untrained": 0, "plain": 0}
            for g, H in zip(held, Hs):
                part = torch.empty(g["n"], dtype=torch.uint8, device="cuda")
                r_t = gp.gp_partition_learned(H.h, M.h, part)
                r_u = gp.gp_partition_learned(H.h, M0.h, part)
                r_p = H.partition(part)
                tot["trained"] += r_t["cut"]
                tot["untrained"] += r_u["cut"]
                tot["plain"] += r_p["cut"]
                print("held-out n=%d: trained %d untrained %d plain %d (feasible %d/%d/%d)" % (
                    g["n"], r_t["cut"], r_u["cut"], r_p["cut"], r_t["feasible"], r_u["feasible"], r_p["feasible"]))
            print("total cut", tot)
            assert tot["trained"] < tot["untrained"]
    finally:
        for G in Gs + Hs:
            G.close()


def test_network_is_deterministic_across_handles():
    """Two handles of the same DAG fill their in-rows in different orders; the network sorts them
    before its first read, so the logits agree bit for bit."""
    g = gen.layered(60, 300, 70000, 13)
    with gp.Graph(dgraph(g)) as G1, gp.Graph(dgraph(g)) as G2, Model(seed=4) as M:
        a = gpu_logits(M, G1, g["n"])
        b = gpu_logits(M, G2, g["n"])
    assert np.array_equal(a, b)


# ---------------------------------------------------------------------------
# The learned path as a V-cycle (restricted coarsening, refinement at every level)
# ---------------------------------------------------------------------------

TRAINED = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1502_07451_b300",
                       "models", "mpnn3_h64.bin")


@pytest.mark.parametrize("name", sorted(GRAPHS) + ["layered_big", "cholesky24", "lu16"])
def test_vcycle_matches_oracle_given_logits(name):
    """Split, every result field and the per-level trace equal the oracle's V-cycle run on the
    network's logits (the trained checkpoint), for the network's own logits and passed-in ones."""
    extra = {"layered_big": lambda: gen.layered(200, 500, 400000, 12), "cholesky24": lambda: gen.cholesky(24),
             "lu16": lambda: gen.lu(16)}
    g = GRAPHS[name]() if name in GRAPHS else extra[name]()
    n = g["n"]
    model = gp.gp_model_load(TRAINED)
    try:
        with gp.Graph(dgraph(g)) as G:
            logits = torch.empty(n, dtype=torch.float32, device="cuda")
            gp.gp_model_forward(model, G.h, logits)
            part = torch.empty(n, dtype=torch.uint8, device="cuda")
            res = gp.gp_partition_learned_vcycle(G.h, model, part, seed=3)
            tr = G.trace()
            part2 = np.zeros(n, np.uint8)
            res2 = gp.gp_partition_learned_vcycle(G.h, None, part2, logits=logits.cpu().numpy(), seed=3)
    finally:
        gp.gp_model_destroy(model)
    ref_part, ref, otr = oracle.partition_vcycle(g, logits.cpu().numpy(), seed=3, trace=True)
    assert np.array_equal(part.cpu().numpy(), ref_part)
    assert np.array_equal(part2, ref_part)
    for k in KEYS:
        assert res[k] == ref[k] and res2[k] == ref[k], k
    assert tr["n"] == otr["n"] and tr["a"] == otr["a"] and tr["rounds"] == otr["rounds"]
    assert tr["gggp_trial"] == -1


def test_vcycle_ratio_branches_and_noisy_logits():
    g = gen.layered(60, 300, 120000, 3)
    n = g["n"]
    p0, _ = oracle.partition(g)
    rng = np.random.default_rng(4)
    lg = (np.where(p0 == 0, 1.0, -1.0) + rng.normal(0, 0.8, n)).astype(np.float32)
    with gp.Graph(dgraph(g)) as G:
        for r in (-1.0, 0.0, 0.2, 1.0):
            part = torch.empty(n, dtype=torch.uint8, device="cuda")
            res = gp.gp_partition_learned_vcycle(G.h, None, part, logits=torch.from_numpy(lg).cuda(), r_cpu=r)
            ref_part, ref = oracle.partition_vcycle(g, lg, r_cpu=r)
            assert np.array_equal(part.cpu().numpy(), ref_part), r
            assert all(res[k] == ref[k] for k in KEYS), r
        bad = lg.copy()
        bad[7] = np.nan
        with pytest.raises(gp.GpError) as e:
            gp.gp_partition_learned_vcycle(G.h, None, torch.empty(n, dtype=torch.uint8, device="cuda"),
                                           logits=torch.from_numpy(bad).cuda())
        assert e.value.status == gp.GP_ERR_INVALID
