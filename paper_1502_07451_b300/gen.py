"""Seeded synthetic task-DAG generators.

These are input recipes only: they build the weighted DAGs that both the CUDA
path and the CPU oracle consume, and hold none of the partitioning or makespan
arithmetic.  Every random draw comes from one counter-based generator, the
splitmix64 output function (Vigna, public domain) applied to
``base(seed, stream) + (i + 1) * 0x9E3779B97F4A7C15``; value ``i`` of a stream
therefore depends only on ``(seed, stream, i)``.

A graph is returned as a dict of numpy arrays:
  n, m         vertex / directed-edge counts
  offsets      int64[n+1]  out-CSR row pointers
  cols         int32[m]    successor of each edge (rows sorted by successor)
  edge_cost    int32[m]    transfer time of the edge, ns (direction-free, §III.B)
  cpu_cost     int32[n]    kernel time on the CPU, ns
  gpu_cost     int32[n]    kernel time on the GPU, ns

Vertex weights are the two measured kernel times and edge weights the PCIe
transfer time, as the paper's scheduler weights its DAG (§III.B).  The paper
measures them; here they come from a flop/byte cost model (tiled factorisation
DAGs) or from seeded distributions (layered random DAGs).
"""
from __future__ import annotations

import functools
import math

import numpy as np

_MASK = (1 << 64) - 1
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_S30, _S27, _S31 = np.uint64(30), np.uint64(27), np.uint64(31)

INT32_MAX = 2**31 - 1


def _mix(z: np.ndarray) -> np.ndarray:
    z = z ^ (z >> _S30)
    z = z * _M1
    z = z ^ (z >> _S27)
    z = z * _M2
    return z ^ (z >> _S31)


def _base(seed: int, stream: int) -> np.uint64:
    x = (int(seed) ^ ((int(stream) + 1) * 0xD1B54A32D192ED03)) & _MASK
    return _mix(np.array([x], dtype=np.uint64))[0]


def u64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Values start..start+count-1 of stream ``stream`` under ``seed`` (uint64)."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    return _mix(_base(seed, stream) + idx * _GAMMA)


def uniform(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits."""
    return (u64(seed, stream, start, count) >> np.uint64(11)).astype(np.float64) * (2.0**-53)


def randint(seed: int, stream: int, start: int, count: int, lo: int, hi: int) -> np.ndarray:
    """Integers in [lo, hi] (inclusive) as int64, by reduction modulo the range."""
    span = np.uint64(hi - lo + 1)
    return (u64(seed, stream, start, count) % span).astype(np.int64) + lo


def _csr_from_edges(n: int, src: np.ndarray, dst: np.ndarray):
    """Sort edges by (src, dst) and build out-CSR row pointers."""
    order = np.lexsort((dst, src))
    src = src[order].astype(np.int64)
    dst = dst[order].astype(np.int32)
    counts = np.bincount(src, minlength=n).astype(np.int64)
    offsets = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    return offsets, dst


def _pack(n, offsets, cols, edge_cost, cpu_cost, gpu_cost, **meta):
    g = dict(
        n=int(n),
        m=int(cols.shape[0]),
        offsets=np.ascontiguousarray(offsets, dtype=np.int64),
        cols=np.ascontiguousarray(cols, dtype=np.int32),
        edge_cost=np.ascontiguousarray(edge_cost, dtype=np.int32),
        cpu_cost=np.ascontiguousarray(cpu_cost, dtype=np.int32),
        gpu_cost=np.ascontiguousarray(gpu_cost, dtype=np.int32),
    )
    g.update(meta)
    return g


# --------------------------------------------------------------------------
# Tiled dense factorisation task graphs with a flop / byte cost model.
#   CPU time  = flops at 50 GFLOP/s       -> (flops + 25) // 50        ns
#   GPU time  = flops at 1 TFLOP/s + 20us -> (flops + 500) // 1000 + 20000 ns
#   transfer  = one b x b FP64 tile over 12 GB/s -> (8 b^2 + 6) // 12 ns
# --------------------------------------------------------------------------

def tile_costs(flops: int):
    return (flops + 25) // 50, (flops + 500) // 1000 + 20000


def tile_edge_cost(b: int) -> int:
    return (8 * b * b + 6) // 12


def cholesky(T: int, b: int = 512):
    """Right-looking tiled Cholesky (lower) task DAG on a T x T tile grid.

    Tasks: POTRF(k); TRSM(k,i), SYRK(k,i) for i > k; GEMM(k,i,j) for k < j < i.
    Task count T + T(T-1) + T(T-1)(T-2)/6; every task writes one tile and each
    dependency moves one tile.
    """
    ids = {}
    kinds = []

    def add(key, kind):
        ids[key] = len(kinds)
        kinds.append(kind)

    for k in range(T):
        add(("P", k), 0)
        for i in range(k + 1, T):
            add(("T", k, i), 1)
        for i in range(k + 1, T):
            add(("S", k, i), 2)
        for i in range(k + 1, T):
            for j in range(k + 1, i):
                add(("G", k, i, j), 3)
    src, dst = [], []

    def edge(a, c):
        src.append(ids[a])
        dst.append(ids[c])

    for k in range(T):
        for i in range(k + 1, T):
            edge(("P", k), ("T", k, i))
            edge(("T", k, i), ("S", k, i))
            for j in range(k + 1, i):
                edge(("T", k, i), ("G", k, i, j))
                edge(("T", k, j), ("G", k, i, j))
            # SYRK(k,i) updates tile (i,i): next writer is SYRK(k+1,i) or POTRF(i)
            edge(("S", k, i), ("P", i) if i == k + 1 else ("S", k + 1, i))
            for j in range(k + 1, i):
                # GEMM(k,i,j) updates tile (i,j): next writer TRSM(j,i) or GEMM(k+1,i,j)
                edge(("G", k, i, j), ("T", j, i) if j == k + 1 else ("G", k + 1, i, j))
    n = len(kinds)
    b3 = b * b * b
    flops = np.array([b3 // 3, b3, b3, 2 * b3], dtype=np.int64)[np.array(kinds)]
    cpu = (flops + 25) // 50
    gpu = (flops + 500) // 1000 + 20000
    offsets, cols = _csr_from_edges(n, np.array(src), np.array(dst))
    w = np.full(cols.shape[0], tile_edge_cost(b), dtype=np.int32)
    return _pack(n, offsets, cols, w, cpu, gpu, kind="cholesky", T=T, b=b,
                 task_kind=np.array(kinds, dtype=np.int8))


def lu(T: int, b: int = 512):
    """Right-looking tiled LU (no pivoting) task DAG on a T x T tile grid.

    Tasks: GETRF(k); TRSM_L(k,j) for the row panel j > k; TRSM_U(k,i) for the
    column panel i > k; GEMM(k,i,j) for i, j > k.
    Task count T + T(T-1) + (T-1)T(2T-1)/6.
    """
    ids = {}
    kinds = []

    def add(key, kind):
        ids[key] = len(kinds)
        kinds.append(kind)

    for k in range(T):
        add(("F", k), 0)
        for j in range(k + 1, T):
            add(("R", k, j), 1)
        for i in range(k + 1, T):
            add(("C", k, i), 1)
        for i in range(k + 1, T):
            for j in range(k + 1, T):
                add(("G", k, i, j), 2)
    src, dst = [], []

    def edge(a, c):
        src.append(ids[a])
        dst.append(ids[c])

    def writer_of(k, i, j):
        # task at step k that next writes tile (i, j), for i, j >= k
        if i == k and j == k:
            return ("F", k)
        if i == k:
            return ("R", k, j)
        if j == k:
            return ("C", k, i)
        return ("G", k, i, j)

    for k in range(T):
        for j in range(k + 1, T):
            edge(("F", k), ("R", k, j))
        for i in range(k + 1, T):
            edge(("F", k), ("C", k, i))
        for i in range(k + 1, T):
            for j in range(k + 1, T):
                edge(("C", k, i), ("G", k, i, j))
                edge(("R", k, j), ("G", k, i, j))
                edge(("G", k, i, j), writer_of(k + 1, i, j))
    n = len(kinds)
    b3 = b * b * b
    flops = np.array([(2 * b3) // 3, b3, 2 * b3], dtype=np.int64)[np.array(kinds)]
    cpu = (flops + 25) // 50
    gpu = (flops + 500) // 1000 + 20000
    offsets, cols = _csr_from_edges(n, np.array(src), np.array(dst))
    w = np.full(cols.shape[0], tile_edge_cost(b), dtype=np.int32)
    return _pack(n, offsets, cols, w, cpu, gpu, kind="lu", T=T, b=b,
                 task_kind=np.array(kinds, dtype=np.int8))


def cholesky_tasks(T: int) -> int:
    return T + T * (T - 1) + T * (T - 1) * (T - 2) // 6


def lu_tasks(T: int) -> int:
    return T + T * (T - 1) + (T - 1) * T * (2 * T - 1) // 6


# --------------------------------------------------------------------------
# Layered random DAGs with lognormal kernel times.
# --------------------------------------------------------------------------

def _lognormal_costs(n: int, seed: int, mu: float, sigma: float, ratio_lo: float, ratio_hi: float):
    u1 = uniform(seed, 4, 0, n)
    u2 = uniform(seed, 5, 0, n)
    z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)  # Box-Muller
    cpu = np.clip(np.rint(np.exp(mu + sigma * z)), 1, INT32_MAX).astype(np.int64)
    r = ratio_lo + (ratio_hi - ratio_lo) * uniform(seed, 6, 0, n)
    gpu = np.maximum(1, np.rint(cpu / r)).astype(np.int64)
    return cpu, gpu


def _first_distinct(keys: np.ndarray, m: int):
    """The first m distinct values of `keys` in draw order (a later repeat of a value is skipped),
    sorted; (None, number of distinct values) if there are fewer than m.  Found with one plain sort
    of all keys (repeats are rare) and a stable sort of the repeated values' occurrences only."""
    s = np.sort(keys)
    rep = s[1:] == s[:-1]
    distinct = int(keys.shape[0] - np.count_nonzero(rep))
    if distinct < m:
        return None, distinct
    if not rep.any():
        return np.sort(keys[:m]), distinct
    dup_vals = np.unique(s[1:][rep])
    pos = np.minimum(np.searchsorted(dup_vals, keys), dup_vals.shape[0] - 1)
    occ = np.flatnonzero(dup_vals[pos] == keys)  # every occurrence of a repeated value, in draw order
    order = np.argsort(keys[occ], kind="stable")
    ko = keys[occ][order]
    later = np.concatenate([[False], ko[1:] == ko[:-1]])  # not the value's first occurrence
    valid = np.ones(keys.shape[0], dtype=bool)
    valid[occ[order][later]] = False
    keep = np.flatnonzero(valid)[:m]
    return np.sort(keys[keep]), distinct


def layered(layers: int, width: int, m: int, seed: int, span: int = 4, wmax: int = 10000,
            mu: float = 10.0, sigma: float = 1.0, ratio_lo: float = 2.0, ratio_hi: float = 40.0):
    """Layered random DAG: ``layers`` x ``width`` vertices, ``m`` distinct edges.

    Vertex ``v`` sits in layer ``v // width``.  Each edge draws its source
    uniformly over layers 0..layers-2, its target layer uniformly among the
    next ``min(span, layers-1-src_layer)`` layers and its target uniformly
    within that layer; repeated (src, dst) pairs are dropped and more edges are
    drawn until ``m`` distinct pairs exist (first occurrences in draw order).
    CPU time lognormal(mu, sigma) clamped to [1, 2^31-1] ns; GPU time = CPU
    time / U(ratio_lo, ratio_hi), at least 1; transfer time U{1..wmax} ns.
    """
    n = layers * width
    if layers < 2 or width < 1:
        raise ValueError("layered DAG needs >= 2 layers and width >= 1")
    max_edges = 0
    for ls in range(layers - 1):
        max_edges += width * width * min(span, layers - 1 - ls)
    if m > max_edges:
        raise ValueError("more edges requested than distinct pairs exist")
    keys = np.empty(0, dtype=np.int64)
    drawn = 0
    need = m
    while True:
        cnt = int(need * 1.02) + 1024
        r0 = u64(seed, 0, drawn, cnt)
        r1 = u64(seed, 1, drawn, cnt)
        r2 = u64(seed, 2, drawn, cnt)
        drawn += cnt
        src = (r0 % np.uint64((layers - 1) * width)).astype(np.int64)
        ls = src // width
        maxspan = np.minimum(span, layers - 1 - ls).astype(np.uint64)
        lt = ls + 1 + (r1 % maxspan).astype(np.int64)
        dst = lt * width + (r2 % np.uint64(width)).astype(np.int64)
        keys = np.concatenate([keys, src * n + dst])
        sel, distinct = _first_distinct(keys, m)
        if sel is not None:
            break
        need = m - distinct
    src = sel // n
    dst = (sel % n).astype(np.int32)
    counts = np.bincount(src, minlength=n).astype(np.int64)
    offsets = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    w = randint(seed, 3, 0, m, 1, wmax).astype(np.int32)
    cpu, gpu = _lognormal_costs(n, seed, mu, sigma, ratio_lo, ratio_hi)
    return _pack(n, offsets, dst, w, cpu, gpu, kind="layered", layers=layers, width=width)


# --------------------------------------------------------------------------
# Small integer-only DAGs used as test fixtures (stable across machines).
# --------------------------------------------------------------------------

def random_dag(n: int, m: int, seed: int, cmin: int = 1000, cmax: int = 100000,
               ratio_pct=(10, 100), wmax: int = 50000):
    """Uniform random DAG on ``n`` vertices with ``m`` distinct edges i -> j, i < j.

    Integer-only draws: CPU time U{cmin..cmax}, GPU time = CPU time * U{ratio_pct} / 100
    (at least 1), transfer time U{1..wmax}.
    """
    max_edges = n * (n - 1) // 2
    if m > max_edges:
        raise ValueError("too many edges")
    keys = []
    seen = set()
    i = 0
    while len(keys) < m:
        r = u64(seed, 0, i, 2)
        i += 2
        a = int(r[0] % np.uint64(n))
        b = int(r[1] % np.uint64(n))
        if a == b:
            continue
        s, d = (a, b) if a < b else (b, a)
        if (s, d) in seen:
            continue
        seen.add((s, d))
        keys.append((s, d))
    src = np.array([k[0] for k in keys], dtype=np.int64)
    dst = np.array([k[1] for k in keys], dtype=np.int64)
    offsets, cols = _csr_from_edges(n, src, dst)
    w = randint(seed, 3, 0, m, 1, wmax)
    cpu = randint(seed, 4, 0, n, cmin, cmax)
    pct = randint(seed, 5, 0, n, ratio_pct[0], ratio_pct[1])
    gpu = np.maximum(1, cpu * pct // 100)
    return _pack(n, offsets, cols, w, cpu, gpu, kind="random")


def two_input_dag(n: int, seed: int, extra: int = 0, **kw):
    """DAG in which every vertex v >= 2 reads two distinct earlier outputs
    (vertex 1 reads vertex 0), plus ``extra`` random forward edges; the shape
    of the paper's generated test task (§IV.A: kernels with two inputs and one
    output)."""
    src, dst = [], []
    seen = set()
    for v in range(1, n):
        k = min(2, v)
        picks = []
        j = 0
        while len(picks) < k:
            r = int(u64(seed, 7, v * 64 + j, 1)[0] % np.uint64(v))
            j += 1
            if r not in picks:
                picks.append(r)
        for u in picks:
            src.append(u)
            dst.append(v)
            seen.add((u, v))
    j = 0
    added = 0
    while added < extra:
        r = u64(seed, 8, j, 2)
        j += 2
        a = int(r[0] % np.uint64(n))
        b = int(r[1] % np.uint64(n))
        if a == b:
            continue
        s, d = (a, b) if a < b else (b, a)
        if (s, d) in seen:
            continue
        seen.add((s, d))
        src.append(s)
        dst.append(d)
        added += 1
    offsets, cols = _csr_from_edges(n, np.array(src, dtype=np.int64), np.array(dst, dtype=np.int64))
    m = cols.shape[0]
    cmin = kw.get("cmin", 1000)
    cmax = kw.get("cmax", 100000)
    lo, hi = kw.get("ratio_pct", (10, 100))
    w = randint(seed, 3, 0, m, 1, kw.get("wmax", 50000))
    cpu = randint(seed, 4, 0, n, cmin, cmax)
    gpu = np.maximum(1, cpu * randint(seed, 5, 0, n, lo, hi) // 100)
    return _pack(n, offsets, cols, w, cpu, gpu, kind="two_input")


def from_edges(n: int, edges, cpu_cost, gpu_cost, edge_cost):
    """Build a graph from an explicit edge list [(u, v), ...] and cost lists
    (edge costs in the order of ``edges``)."""
    edges = list(edges)
    src = np.array([e[0] for e in edges], dtype=np.int64)
    dst = np.array([e[1] for e in edges], dtype=np.int64)
    w = np.array(edge_cost, dtype=np.int64)
    if src.shape[0]:
        order = np.lexsort((dst, src))
        src, dst, w = src[order], dst[order], w[order]
    counts = np.bincount(src, minlength=n).astype(np.int64) if n else np.zeros(0, np.int64)
    offsets = np.zeros(n + 1, dtype=np.int64)
    if n:
        np.cumsum(counts, out=offsets[1:])
    return _pack(n, offsets, dst.astype(np.int32), w, np.array(cpu_cost, dtype=np.int64),
                 np.array(gpu_cost, dtype=np.int64), kind="explicit")


def with_host_source(g, seed: int, wmax: int = 10000):
    """The DAG with the paper's host vertex added (Sec. III.B): every kernel without a predecessor
    gets an edge from one empty kernel (CPU and GPU time 0) that stands for the initial data in host
    memory.  The new vertex is ``n`` (the last id); its edges' transfer times are U{1..wmax} ns
    (stream 40).  Returns (graph, source id)."""
    n, m = int(g["n"]), int(g["m"])
    off = np.asarray(g["offsets"], dtype=np.int64)
    cols = np.asarray(g["cols"], dtype=np.int32)
    indeg = np.bincount(cols, minlength=n) if m else np.zeros(n, np.int64)
    roots = np.flatnonzero(indeg == 0).astype(np.int32)
    k = roots.shape[0]
    offsets = np.empty(n + 2, dtype=np.int64)
    offsets[: n + 1] = off
    offsets[n + 1] = m + k
    w = np.concatenate([np.asarray(g["edge_cost"], dtype=np.int32),
                        randint(seed, 40, 0, k, 1, wmax).astype(np.int32)])
    cpu = np.concatenate([np.asarray(g["cpu_cost"], dtype=np.int32), np.zeros(1, np.int32)])
    gpu = np.concatenate([np.asarray(g["gpu_cost"], dtype=np.int32), np.zeros(1, np.int32)])
    meta = {k2: v for k2, v in g.items() if k2 not in ("n", "m", "offsets", "cols", "edge_cost", "cpu_cost",
                                                      "gpu_cost")}
    meta["host_source"] = n
    return _pack(n + 1, offsets, np.concatenate([cols, roots]), w, cpu, gpu, **meta), n


# --------------------------------------------------------------------------
# Workload recipes.
# --------------------------------------------------------------------------

def config_cholesky16():
    """Tiled Cholesky, T = 16 (816 tasks, 2,040 dependencies), 512 x 512 FP64 tiles."""
    return cholesky(16)


def config_layered_1m(seed: int = 0):
    """Layered random DAG, 1,000 layers of 1,000 vertices, 8M distinct edges."""
    return layered(1000, 1000, 8_000_000, seed)


def config_layered_16m(seed: int = 0):
    """Layered random DAG, 1,000 layers of 16,000 vertices, 128M distinct edges."""
    return layered(1000, 16000, 128_000_000, seed)


def kway_costs(g, k: int, seed: int = 0):
    """Times of k device classes for the k-way split (int32 [k, n]): class 0 the CPU time, class 1 the
    GPU time, and each further class an accelerator derived from them with per-task speed factors
    (stream 50 + i): even classes CPU time x U(0.1, 0.9) (an FPGA-like part faster than the CPU on
    every task), odd classes GPU time x U(0.5, 3.0), floored."""
    n = g["n"]
    out = [np.asarray(g["cpu_cost"], np.int64), np.asarray(g["gpu_cost"], np.int64)]
    for i in range(2, k):
        u = uniform(seed, 50 + i, 0, n)
        f = 0.1 + 0.8 * u if i % 2 == 0 else 0.5 + 2.5 * u
        out.append(np.floor(out[i % 2] * f).astype(np.int64))
    return np.ascontiguousarray(np.stack(out[:k]).astype(np.int32))


def nearest_T(target: int, tasks_fn, lo: int, hi: int) -> int:
    best = lo
    for T in range(lo, hi + 1):
        if abs(tasks_fn(T) - target) < abs(tasks_fn(best) - target):
            best = T
    return best


def batch_spec(count: int = 4096, nmin: int = 100, nmax: int = 50000, base_seed: int = 0, tmax: int = 40):
    """Recipe of the mixed batch: graph i has a log-uniform target size in
    [nmin, nmax] and kind i mod 3 (tiled Cholesky T=4..tmax, tiled LU T=2..tmax,
    layered of width ~sqrt(n) with 8 edges per vertex)."""
    u = uniform(base_seed, 9, 0, count)
    target = np.exp(math.log(nmin) + (math.log(nmax) - math.log(nmin)) * u)
    spec = []
    for i in range(count):
        t = int(round(target[i]))
        kind = i % 3
        if kind == 0:
            spec.append(("cholesky", nearest_T(t, cholesky_tasks, 4, tmax), base_seed + i))
        elif kind == 1:
            spec.append(("lu", nearest_T(t, lu_tasks, 2, tmax), base_seed + i))
        else:
            width = max(2, int(round(math.sqrt(t))))
            layers = max(2, int(round(t / width)))
            spec.append(("layered", (layers, width), base_seed + i))
    return spec


def spec_edges(item) -> int:
    """Directed edge count of a batch item's graph (the tiled graphs are built once per T, the
    layered count is the recipe's)."""
    kind, p, _ = item
    if kind in ("cholesky", "lu"):
        return int(_tiled(kind, p)["m"])
    layers, width = p
    cap = 0
    for ls in range(layers - 1):
        cap += width * width * min(4, layers - 1 - ls)
    return min(8 * layers * width, cap)


@functools.lru_cache(maxsize=None)
def _tiled(kind: str, T: int):
    return cholesky(T) if kind == "cholesky" else lu(T)


def build_from_spec(item):
    """The graph of one batch item.  Tiled Cholesky / LU graphs depend on T only and are built
    once per T (the returned arrays are shared: treat them as read-only)."""
    kind, p, seed = item
    if kind in ("cholesky", "lu"):
        return _tiled(kind, p)
    layers, width = p
    n = layers * width
    cap = 0
    for ls in range(layers - 1):
        cap += width * width * min(4, layers - 1 - ls)
    return layered(layers, width, min(8 * n, cap), seed)
