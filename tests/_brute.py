"""Exhaustive 2-way splits of tiny DAGs (independent of the oracle's code).

Enumerates all 2^n assignments as bit masks (bit v = 1: vertex v on the GPU)
and evaluates, with numpy over all masks at once, the loads on both sides and
the cut transfer cost, straight from the problem statement: minimise the sum
of transfer costs of edges whose ends lie on different sides subject to both
loads staying within their bounds.
"""
import numpy as np


def all_splits(g):
    n = g["n"]
    assert n <= 22
    masks = np.arange(1 << n, dtype=np.int64)
    load_cpu = np.zeros(1 << n, dtype=np.int64)
    load_gpu = np.zeros(1 << n, dtype=np.int64)
    for v in range(n):
        bit = (masks >> v) & 1
        load_gpu += bit * int(g["gpu_cost"][v])
        load_cpu += (1 - bit) * int(g["cpu_cost"][v])
    cut = np.zeros(1 << n, dtype=np.int64)
    off, cols, w = g["offsets"], g["cols"], g["edge_cost"]
    for u in range(n):
        for e in range(off[u], off[u + 1]):
            v = int(cols[e])
            cut += (((masks >> u) ^ (masks >> v)) & 1) * int(w[e])
    return masks, load_cpu, load_gpu, cut


def best_feasible(g, bound_cpu, bound_gpu):
    """(optimal cut, mask) over feasible splits, or (None, None)."""
    masks, lc, lg, cut = all_splits(g)
    ok = (lc <= bound_cpu) & (lg <= bound_gpu)
    if not ok.any():
        return None, None
    i = np.argmin(np.where(ok, cut, np.iinfo(np.int64).max))
    return int(cut[i]), int(masks[i])


def longest_path_makespan(g, part):
    """Makespan by enumerating every source-to-sink path (tiny DAGs only)."""
    n = g["n"]
    off, cols, w = g["offsets"], g["cols"], g["edge_cost"]
    cost = [int(g["gpu_cost"][v]) if part[v] else int(g["cpu_cost"][v]) for v in range(n)]
    indeg = np.zeros(n, dtype=np.int64)
    for e in range(g["m"]):
        indeg[cols[e]] += 1
    best = 0
    stack = [(v, cost[v]) for v in range(n) if indeg[v] == 0]
    while stack:
        v, t = stack.pop()
        best = max(best, t)
        for e in range(off[v], off[v + 1]):
            u = int(cols[e])
            stack.append((u, t + (int(w[e]) if part[u] != part[v] else 0) + cost[u]))
    return best


def list_schedule_stepped(g, part, workers_cpu, workers_gpu):
    """The list schedule on P_C CPU and P_G GPU workers, simulated one time unit at a time (integer
    costs; tiny graphs only).  At every integer time t: tasks that end at t end and release the
    successors whose predecessors have all ended, then every idle worker takes the released task of
    its side with the smallest (data arrival, id) among those whose data have arrived; a task of cost 0
    ends at once, so both steps repeat until nothing changes at t.  Returns (makespan, finish list)."""
    n = g["n"]
    off, cols, w = g["offsets"], g["cols"], g["edge_cost"]
    cost = [int(g["gpu_cost"][v]) if part[v] else int(g["cpu_cost"][v]) for v in range(n)]
    npred = [0] * n
    for e in range(int(off[n])):
        npred[int(cols[e])] += 1
    arrive = [0] * n
    released = {v for v in range(n) if npred[v] == 0}
    started = set()
    ended = set()
    end = [None] * n
    idle = [workers_cpu, workers_gpu]
    t = 0
    limit = sum(cost) + int(np.asarray(w).sum()) + 1
    while len(ended) < n:
        assert t <= limit, "no progress"
        changed = True
        while changed:
            changed = False
            for u in range(n):
                if u in started and u not in ended and end[u] == t:
                    ended.add(u)
                    idle[part[u]] += 1
                    changed = True
                    for e in range(int(off[u]), int(off[u + 1])):
                        v = int(cols[e])
                        arrive[v] = max(arrive[v], t + (int(w[e]) if part[u] != part[v] else 0))
                        npred[v] -= 1
                        if npred[v] == 0:
                            released.add(v)
            for s in (0, 1):
                while idle[s] > 0:
                    ready = [(arrive[v], v) for v in released if part[v] == s and v not in started and arrive[v] <= t]
                    if not ready:
                        break
                    _, v = min(ready)
                    started.add(v)
                    end[v] = t + cost[v]
                    idle[s] -= 1
                    changed = True
        t += 1
    return (max(end) if n else 0), end
