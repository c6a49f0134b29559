"""CPU oracle of the learned proposal's message-passing network (test infrastructure, FP64).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg may use this module;
the library never does.  It states the network, its loss and its gradient in plain numpy /
scipy.sparse, in float64, as the definition the GPU kernels are checked against (the GPU computes
the layer products in BF16 with FP32 accumulation, the rest in FP32).

The paper has no network: it is a project addition that proposes the initial split (the paper's
split comes from METIS, Sec. III.A).  Definition:

  features of vertex v (5):  log1p(cpu_cost)/16, log1p(gpu_cost)/16, log1p(in-degree)/4,
                             log1p(out-degree)/4, level / max(1, levels - 1)
  edge feature of a directed entry u->v:  e = log1p(transfer cost)/16
  h0 = relu(x W_in + b_in)
  for l = 1, 2, 3:
     ain_v  = sum over entries u->v of e * h_u, divided by max(1, in-degree of v)
     aout_v = sum over entries v->u of e * h_u, divided by max(1, out-degree of v)
     h_l = relu([h_{l-1} | ain | aout] W_l + b_l)          (W_l: 192 x 64)
  logit_v = h3_v . w_o + b_o
  loss = mean over v of softplus(logit_v) - y_v logit_v, y_v = 1 when the label puts v on the CPU.

Parameters travel as one float32 vector in the order W_in, b_in, W1, b1, W2, b2, W3, b3, w_o, b_o
(row-major matrices), the same order as the library's gp_model_get_params.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

HID = 64
NFEAT = 5
SHAPES = [("W_in", (NFEAT, HID)), ("b_in", (HID,)),
          ("W1", (3 * HID, HID)), ("b1", (HID,)),
          ("W2", (3 * HID, HID)), ("b2", (HID,)),
          ("W3", (3 * HID, HID)), ("b3", (HID,)),
          ("w_o", (HID,)), ("b_o", (1,))]
NPARAMS = int(sum(int(np.prod(s)) for _, s in SHAPES))


def unpack(flat):
    flat = np.asarray(flat, dtype=np.float64)
    assert flat.shape == (NPARAMS,)
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = flat[o:o + k].reshape(shape)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in SHAPES])


def structure(g, level=None, nlev=None):
    """Features and the two normalised aggregation matrices of a DAG given as out-CSR arrays."""
    import oracle
    n = int(g["n"])
    off = np.asarray(g["offsets"], np.int64)
    cols = np.asarray(g["cols"], np.int64)
    w = np.asarray(g["edge_cost"], np.float64)
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(off))
    dst = cols
    outdeg = np.diff(off).astype(np.float64)
    indeg = np.bincount(dst, minlength=n).astype(np.float64)
    if level is None:
        level, nlev = oracle.levels(g)
    X = np.stack([np.log1p(np.asarray(g["cpu_cost"], np.float64)) / 16.0,
                  np.log1p(np.asarray(g["gpu_cost"], np.float64)) / 16.0,
                  np.log1p(indeg) / 4.0, np.log1p(outdeg) / 4.0,
                  np.asarray(level, np.float64) / max(1, nlev - 1)], axis=1)
    e = np.log1p(w) / 16.0
    A_in = sp.csr_matrix((e / np.maximum(1.0, indeg[dst]), (dst, src)), shape=(n, n))
    A_out = sp.csr_matrix((e / np.maximum(1.0, outdeg[src]), (src, dst)), shape=(n, n))
    return {"n": n, "X": X, "A_in": A_in, "A_out": A_out}


def forward(params, S):
    P = unpack(params) if not isinstance(params, dict) else params
    cache = {}
    z = S["X"] @ P["W_in"] + P["b_in"]
    h = np.maximum(z, 0.0)
    cache["z0"] = z
    cache["h0"] = h
    for l in (1, 2, 3):
        c = np.concatenate([h, S["A_in"] @ h, S["A_out"] @ h], axis=1)
        z = c @ P["W%d" % l] + P["b%d" % l]
        h = np.maximum(z, 0.0)
        cache["c%d" % l] = c
        cache["z%d" % l] = z
        cache["h%d" % l] = h
    logit = h @ P["w_o"] + P["b_o"][0]
    cache["logit"] = logit
    return logit, cache


def softplus(x):
    return np.logaddexp(0.0, x)


def loss_and_grad(params, S, y):
    """Mean binary cross-entropy with logits and its gradient (flat, float64)."""
    P = unpack(params) if not isinstance(params, dict) else params
    y = np.asarray(y, np.float64)
    n = S["n"]
    logit, c = forward(P, S)
    loss = float(np.mean(softplus(logit) - y * logit))
    dlogit = (1.0 / (1.0 + np.exp(-logit)) - y) / n
    G = {}
    G["w_o"] = c["h3"].T @ dlogit
    G["b_o"] = np.array([dlogit.sum()])
    dh = np.outer(dlogit, P["w_o"])
    for l in (3, 2, 1):
        dz = dh * (c["z%d" % l] > 0)
        G["W%d" % l] = c["c%d" % l].T @ dz
        G["b%d" % l] = dz.sum(axis=0)
        dc = dz @ P["W%d" % l].T
        dh = dc[:, :HID] + S["A_in"].T @ dc[:, HID:2 * HID] + S["A_out"].T @ dc[:, 2 * HID:]
    dz = dh * (c["z0"] > 0)
    G["W_in"] = S["X"].T @ dz
    G["b_in"] = dz.sum(axis=0)
    return loss, pack(G)


def labels_from_part(part):
    """Training target: 1 where the plain method put the vertex on the CPU (side 0)."""
    return (np.asarray(part) == 0).astype(np.float64)
