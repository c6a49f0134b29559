"""CPU oracle of the multilevel CPU/GPU task-DAG bipartitioner (test infrastructure).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this package; the library path never does.  It wraps the plain C
implementation in ``gp_oracle.c`` (single-threaded, step by step) with ctypes
and numpy, and shares no code with the CUDA implementation.

Each wrapper names the paper passage or the algorithm step it follows; see the
comments in ``gp_oracle.c`` for the full statement of each step.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gp_oracle.c")
_HDR = os.path.join(_HERE, "gp_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, ERR_INVALID, ERR_NOT_DAG, ERR_OOM, ERR_OVERFLOW = 0, 1, 2, 3, 6
MAX_LEVELS = 48
MATCH_ROUNDS = 4
CAP_DIV = 8
COARSEST = 128
TRIALS = 8
REFINE_ROUNDS = 8

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gp_oracle.c into liboracle.so with gcc (plain C, -O2)."""
    stale = (not os.path.exists(_LIB)) or max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)) > os.path.getmtime(_LIB)
    if force or stale:
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-std=gnu11", "-O2", "-Wall", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Result(C.Structure):
    _fields_ = [("cut", C.c_int64), ("load_cpu", C.c_int64), ("load_gpu", C.c_int64),
                ("bound_cpu", C.c_int64), ("bound_gpu", C.c_int64),
                ("feasible", C.c_int32), ("levels", C.c_int32), ("rounds", C.c_int32),
                ("coarsest_n", C.c_int32)]

    def as_dict(self):
        return {f[0]: int(getattr(self, f[0])) for f in self._fields_}


_L1 = MAX_LEVELS + 1


class Trace(C.Structure):
    _fields_ = [("levels", C.c_int32), ("gggp_trial", C.c_int32),
                ("n", C.c_int64 * _L1), ("a", C.c_int64 * _L1), ("rounds", C.c_int32 * _L1),
                ("moves", C.c_int64 * _L1), ("balanced", C.c_int32 * _L1),
                ("bal_moves", C.c_int64 * _L1), ("cut", C.c_int64 * _L1)]

    def as_dict(self):
        L = self.levels
        return dict(levels=L, gggp_trial=self.gggp_trial,
                    n=list(self.n[:L + 1]), a=list(self.a[:L + 1]), rounds=list(self.rounds[:L + 1]),
                    moves=list(self.moves[:L + 1]), balanced=list(self.balanced[:L + 1]),
                    bal_moves=list(self.bal_moves[:L + 1]), cut=list(self.cut[:L + 1]))


class RefineStats(C.Structure):
    _fields_ = [("rounds", C.c_int32), ("balanced", C.c_int32), ("moves", C.c_int64),
                ("bal_moves", C.c_int64), ("load_cpu", C.c_int64), ("load_gpu", C.c_int64)]


_P = C.c_void_p
_I64 = C.c_int64


def lib():
    """The loaded oracle library.  GP_ORACLE_LIB names another build of the
    same source to load instead (used by the mutation tests)."""
    global _lib
    with _lock:
        if _lib is None:
            alt = os.environ.get("GP_ORACLE_LIB")
            if alt:
                L = C.CDLL(alt)
            else:
                build()
                L = C.CDLL(_LIB)
            L.og_mix64.restype = C.c_uint64
            L.og_mix64.argtypes = [C.c_uint64]
            L.og_hash.restype = C.c_uint64
            L.og_hash.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32]
            L.og_validate.argtypes = [_I64, _I64, _P, _P, _P, _P, _P]
            L.og_bounds.argtypes = [_I64, _I64, C.c_double, C.c_double, _P, _P]
            L.og_symmetrize.argtypes = [_I64, _I64, _P, _P, _P, _P, _P, _P, _P]
            L.og_match.argtypes = [_I64, _P, _P, _P, _P, _P, _I64, _I64, C.c_uint64, C.c_int32, _P]
            L.og_match_twohop.argtypes = [_I64, _P, _P, _P, _P, _P, _I64, _I64, C.c_uint64, _P]
            L.og_count_coarse.restype = _I64
            L.og_count_coarse.argtypes = [_I64, _P]
            L.og_contract.argtypes = [_I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]
            L.og_gggp_grow.argtypes = [_I64, _P, _P, _P, _P, _P, _I64, _I64, _I64, _P, _P]
            L.og_gggp.argtypes = [_I64, _P, _P, _P, _P, _P, _I64, _I64, C.c_uint64, _P, _P]
            L.og_refine.argtypes = [_I64, _P, _P, _P, _P, _P, _I64, _I64, _P, _P]
            L.og_partition.argtypes = [_I64, _I64, _P, _P, _P, _P, _P, C.c_double, C.c_double,
                                       C.c_uint64, _P, _P, _P]
            L.og_partition_fixed.argtypes = [_I64, _I64, _P, _P, _P, _P, _P, _P, C.c_double, C.c_double,
                                             C.c_uint64, _P, _P, _P]
            L.og_cut.argtypes = [_I64, _P, _P, _P, _P, _P]
            L.og_levels.argtypes = [_I64, _I64, _P, _P, _P, _P]
            L.og_makespan.argtypes = [_I64, _I64, _P, _P, _P, _P, _P, _P, _P, _P]
            L.og_partition_vcycle.argtypes = [_I64, _I64, _P, _P, _P, _P, _P, _P, C.c_double, C.c_double,
                                              C.c_uint64, _P, _P, _P]
            L.og_partition_kway.argtypes = [_I64, _I64, _P, _P, _P, C.c_int32, _P, C.c_double, C.c_uint64, _P, _P,
                                            _P, _P, _P]
            L.og_makespan_workers.argtypes = [_I64, _I64, _P, _P, _P, _P, _P, _P, _I64, _I64, _P, _P]
            L.og_propose.argtypes = [_I64, _P, _P, _P, _I64, _I64, _P, _P]
            L.og_partition_learned.argtypes = [_I64, _I64, _P, _P, _P, _P, _P, _P, C.c_double, C.c_double,
                                               _P, _P]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class OracleError(RuntimeError):
    def __init__(self, status, where):
        super().__init__("%s returned status %d" % (where, status))
        self.status = status


def _check(st, where):
    if st != OK:
        raise OracleError(st, where)


def _graph_arrays(g):
    return (_c(g["offsets"], np.int64), _c(g["cols"], np.int32), _c(g["edge_cost"], np.int32),
            _c(g["cpu_cost"], np.int32), _c(g["gpu_cost"], np.int32))


# ---------------------------------------------------------------------------
# Wrappers, one per step.
# ---------------------------------------------------------------------------

def mix64(z: int) -> int:
    return int(lib().og_mix64(z))


def edge_hash(seed: int, a: int, b: int) -> int:
    """h(seed, a, b), the matching tie-break hash."""
    return int(lib().og_hash(seed, a, b))


def validate(g) -> int:
    """Status of the input checks (INVALID > OVERFLOW > NOT_DAG precedence)."""
    off, cols, w, cc, cg = _graph_arrays(g)
    return int(lib().og_validate(g["n"], g["m"], _p(off), _p(cols), _p(w), _p(cc), _p(cg)))


def bounds(sum_cpu: int, sum_gpu: int, r_cpu: float = -1.0, tol: float = 0.03):
    """(B_C, B_G) from Eq. (1)-(2), or from an explicit CPU share r_cpu >= 0."""
    bc, bg = C.c_int64(), C.c_int64()
    _check(lib().og_bounds(sum_cpu, sum_gpu, r_cpu, tol, C.byref(bc), C.byref(bg)), "og_bounds")
    return int(bc.value), int(bg.value)


def symmetrize(g):
    """Undirected level-0 graph (offsets, adj, W) of the DAG (transfer cost is direction-free)."""
    off, cols, w, _, _ = _graph_arrays(g)
    n, m = g["n"], g["m"]
    uoff = np.zeros(n + 1, np.int64)
    uadj = np.zeros(2 * m + 1, np.int32)
    uW = np.zeros(2 * m + 1, np.int64)
    a = C.c_int64()
    _check(lib().og_symmetrize(n, m, _p(off), _p(cols), _p(w), _p(uoff), _p(uadj), _p(uW), C.byref(a)),
           "og_symmetrize")
    a = int(a.value)
    return uoff, uadj[:a].copy(), uW[:a].copy()


def match(n, off, adj, W, vC, vG, cap_cpu, cap_gpu, seed, rounds=MATCH_ROUNDS):
    """Handshake heavy-edge matching (mate array, -1 = unmatched)."""
    off, adj, W = _c(off, np.int64), _c(adj, np.int32), _c(W, np.int64)
    vC, vG = _c(vC, np.int64), _c(vG, np.int64)
    mate = np.zeros(max(n, 1), np.int32)
    _check(lib().og_match(n, _p(off), _p(adj), _p(W), _p(vC), _p(vG), cap_cpu, cap_gpu, seed, rounds,
                          _p(mate)), "og_match")
    return mate[:n]


def match_twohop(n, off, adj, W, vC, vG, cap_cpu, cap_gpu, seed, mate):
    """Two-hop pairing of vertices left unmatched, grouped by their anchor (best neighbour)."""
    off, adj, W = _c(off, np.int64), _c(adj, np.int32), _c(W, np.int64)
    vC, vG = _c(vC, np.int64), _c(vG, np.int64)
    mate = np.array(mate, dtype=np.int32, copy=True)
    if mate.shape[0] == 0:
        mate = np.zeros(1, np.int32)
    _check(lib().og_match_twohop(n, _p(off), _p(adj), _p(W), _p(vC), _p(vG), cap_cpu, cap_gpu, seed,
                                 _p(mate)), "og_match_twohop")
    return mate[:n]


def count_coarse(mate) -> int:
    mate = _c(mate, np.int32)
    return int(lib().og_count_coarse(mate.shape[0], _p(mate)))


def contract(n, off, adj, W, vC, vG, mate):
    """Contraction: (cmap, coarse offsets, adj, W, vC, vG)."""
    off, adj, W = _c(off, np.int64), _c(adj, np.int32), _c(W, np.int64)
    vC, vG, mate = _c(vC, np.int64), _c(vG, np.int64), _c(mate, np.int32)
    a = adj.shape[0]
    cmap = np.zeros(max(n, 1), np.int32)
    coff = np.zeros(n + 1, np.int64)
    cadj = np.zeros(a + 1, np.int32)
    cW = np.zeros(a + 1, np.int64)
    cvC = np.zeros(max(n, 1), np.int64)
    cvG = np.zeros(max(n, 1), np.int64)
    nc, ac = C.c_int64(), C.c_int64()
    _check(lib().og_contract(n, _p(off), _p(adj), _p(W), _p(vC), _p(vG), _p(mate), _p(cmap), C.byref(nc),
                             _p(coff), _p(cadj), _p(cW), _p(cvC), _p(cvG), C.byref(ac)), "og_contract")
    nc, ac = int(nc.value), int(ac.value)
    return cmap[:n], coff[:nc + 1].copy(), cadj[:ac].copy(), cW[:ac].copy(), cvC[:nc].copy(), cvG[:nc].copy()


def gggp_grow(n, off, adj, W, vC, vG, bound_cpu, bound_gpu, start):
    """One greedy graph-growing trial from ``start``: (part, cut)."""
    off, adj, W = _c(off, np.int64), _c(adj, np.int32), _c(W, np.int64)
    vC, vG = _c(vC, np.int64), _c(vG, np.int64)
    part = np.zeros(max(n, 1), np.uint8)
    cut = C.c_int64()
    _check(lib().og_gggp_grow(n, _p(off), _p(adj), _p(W), _p(vC), _p(vG), bound_cpu, bound_gpu, start,
                              _p(part), C.byref(cut)), "og_gggp_grow")
    return part[:n], int(cut.value)


def gggp(n, off, adj, W, vC, vG, bound_cpu, bound_gpu, seed):
    """Greedy graph-growing initial split: (part, winning trial or -1)."""
    off, adj, W = _c(off, np.int64), _c(adj, np.int32), _c(W, np.int64)
    vC, vG = _c(vC, np.int64), _c(vG, np.int64)
    part = np.zeros(max(n, 1), np.uint8)
    t = C.c_int32()
    _check(lib().og_gggp(n, _p(off), _p(adj), _p(W), _p(vC), _p(vG), bound_cpu, bound_gpu, seed, _p(part),
                         C.byref(t)), "og_gggp")
    return part[:n], int(t.value)


def refine(n, off, adj, W, vC, vG, bound_cpu, bound_gpu, part):
    """Balance round (if infeasible) + gain rounds at one level: (part, stats dict)."""
    off, adj, W = _c(off, np.int64), _c(adj, np.int32), _c(W, np.int64)
    vC, vG = _c(vC, np.int64), _c(vG, np.int64)
    p = np.array(part, dtype=np.uint8, copy=True)
    if p.shape[0] == 0:
        p = np.zeros(1, np.uint8)
    st = RefineStats()
    _check(lib().og_refine(n, _p(off), _p(adj), _p(W), _p(vC), _p(vG), bound_cpu, bound_gpu, _p(p),
                           C.byref(st)), "og_refine")
    return p[:n], {f[0]: int(getattr(st, f[0])) for f in RefineStats._fields_}


def partition(g, r_cpu: float = -1.0, tol: float = 0.03, seed: int = 0, trace: bool = False, fixed=None):
    """The whole bipartitioner: (part, result dict[, trace dict]).  fixed: None, or int8 per vertex
    (0 pinned to the CPU, 1 to the GPU, -1 free)."""
    off, cols, w, cc, cg = _graph_arrays(g)
    n = g["n"]
    part = np.zeros(max(n, 1), np.uint8)
    res = Result()
    tr = Trace()
    tr_p = C.byref(tr) if trace else None
    if fixed is None:
        _check(lib().og_partition(n, g["m"], _p(off), _p(cols), _p(w), _p(cc), _p(cg), r_cpu, tol, seed,
                                  _p(part), C.byref(res), tr_p), "og_partition")
    else:
        fx = _c(fixed, np.int8)
        if fx.shape[0] != n:
            raise ValueError("fixed must hold one value per vertex")
        if n == 0:
            fx = np.zeros(1, np.int8)
        _check(lib().og_partition_fixed(n, g["m"], _p(off), _p(cols), _p(w), _p(cc), _p(cg), _p(fx), r_cpu, tol,
                                        seed, _p(part), C.byref(res), tr_p), "og_partition_fixed")
    if trace:
        return part[:n], res.as_dict(), tr.as_dict()
    return part[:n], res.as_dict()


def propose(logits, vC, vG, bound_cpu, bound_gpu):
    """Learned proposal: vertices by (logit desc, id asc) under the total order of the float bits;
    the first k = min(kC, kG) go to the CPU.  Returns (part, k)."""
    lg = _c(logits, np.float32)
    n = lg.shape[0]
    vC = _c(vC, np.int64)
    vG = _c(vG, np.int64)
    part = np.zeros(max(n, 1), np.uint8)
    k = C.c_int64()
    _check(lib().og_propose(n, _p(lg), _p(vC), _p(vG), int(bound_cpu), int(bound_gpu), _p(part), C.byref(k)),
           "og_propose")
    return part[:n], int(k.value)


def partition_learned(g, logits, r_cpu: float = -1.0, tol: float = 0.03):
    """The learned path from given logits: proposal, then refinement at level 0 only."""
    off, cols, w, cc, cg = _graph_arrays(g)
    n = g["n"]
    lg = _c(logits, np.float32)
    if lg.shape[0] == 0:
        lg = np.zeros(1, np.float32)
    part = np.zeros(max(n, 1), np.uint8)
    res = Result()
    _check(lib().og_partition_learned(n, g["m"], _p(off), _p(cols), _p(w), _p(cc), _p(cg), _p(lg), r_cpu, tol,
                                      _p(part), C.byref(res)), "og_partition_learned")
    return part[:n], res.as_dict()


def partition_vcycle(g, logits, r_cpu: float = -1.0, tol: float = 0.03, seed: int = 0, trace: bool = False):
    """The learned path as a V-cycle: the proposal from the logits restricts the matching to
    same-side pairs, the coarsest split is the proposed sides, and every level is refined on the way
    back.  Returns (part, result dict[, trace dict])."""
    off, cols, w, cc, cg = _graph_arrays(g)
    n = g["n"]
    lg = _c(logits, np.float32)
    if lg.shape[0] == 0:
        lg = np.zeros(1, np.float32)
    part = np.zeros(max(n, 1), np.uint8)
    res = Result()
    tr = Trace()
    _check(lib().og_partition_vcycle(n, g["m"], _p(off), _p(cols), _p(w), _p(cc), _p(cg), _p(lg), r_cpu, tol,
                                     seed, _p(part), C.byref(res), C.byref(tr) if trace else None),
           "og_partition_vcycle")
    if trace:
        return part[:n], res.as_dict(), tr.as_dict()
    return part[:n], res.as_dict()


def cut(g, part) -> int:
    """Sum of transfer costs of directed edges whose ends are on different sides."""
    off, cols, w, _, _ = _graph_arrays(g)
    part = _c(part, np.uint8)
    c = C.c_int64()
    _check(lib().og_cut(g["n"], _p(off), _p(cols), _p(w), _p(part), C.byref(c)), "og_cut")
    return int(c.value)


def levels(g):
    """Topological levels (longest hop count from a source) and their number."""
    off, cols, _, _, _ = _graph_arrays(g)
    n = g["n"]
    lev = np.zeros(max(n, 1), np.int32)
    nl = C.c_int32()
    _check(lib().og_levels(n, g["m"], _p(off), _p(cols), _p(lev), C.byref(nl)), "og_levels")
    return lev[:n], int(nl.value)


def makespan(g, part, with_finish: bool = False):
    """Makespan of the mapping (max-plus longest path with cut-edge transfers)."""
    off, cols, w, cc, cg = _graph_arrays(g)
    n = g["n"]
    part = _c(part, np.uint8)
    if part.shape[0] == 0:
        part = np.zeros(1, np.uint8)
    fin = np.zeros(max(n, 1), np.int64)
    ms = C.c_int64()
    _check(lib().og_makespan(n, g["m"], _p(off), _p(cols), _p(w), _p(cc), _p(cg), _p(part), _p(fin),
                             C.byref(ms)), "og_makespan")
    if with_finish:
        return int(ms.value), fin[:n]
    return int(ms.value)


def makespan_workers(g, part, workers_cpu: int = 3, workers_gpu: int = 1, with_finish: bool = False):
    """Makespan of the mapping on a fixed number of workers per side (Sec. IV.A's testbed: 3 CPU
    worker cores, 1 GPU worker): the list schedule of og_makespan_workers."""
    off, cols, w, cc, cg = _graph_arrays(g)
    n = g["n"]
    part = _c(part, np.uint8)
    if part.shape[0] == 0:
        part = np.zeros(1, np.uint8)
    fin = np.zeros(max(n, 1), np.int64)
    ms = C.c_int64()
    _check(lib().og_makespan_workers(n, g["m"], _p(off), _p(cols), _p(w), _p(cc), _p(cg), _p(part),
                                     int(workers_cpu), int(workers_gpu), _p(fin), C.byref(ms)),
           "og_makespan_workers")
    if with_finish:
        return int(ms.value), fin[:n]
    return int(ms.value)


def partition_kway(g, costs, tol: float = 0.03, seed: int = 0):
    """k device classes by recursive bisection: costs is int32 [k, n] (v's time on class i).  Returns
    (cls uint8[n], dict(cut, loads (list of k), feasible, bisections))."""
    off, cols, w, _, _ = _graph_arrays(g)
    n = g["n"]
    cs = np.ascontiguousarray(np.asarray(costs, dtype=np.int32))
    k = int(cs.shape[0])
    if cs.ndim != 2 or cs.shape[1] != n:
        raise ValueError("costs must be [k, n]")
    flat = cs.reshape(-1) if cs.size else np.zeros(1, np.int32)
    cls = np.zeros(max(n, 1), np.uint8)
    cut_ = C.c_int64()
    loads = np.zeros(max(k, 1), np.int64)
    feas = C.c_int32()
    nb = C.c_int32()
    _check(lib().og_partition_kway(n, g["m"], _p(off), _p(cols), _p(w), k, _p(flat), tol, seed, _p(cls),
                                   C.byref(cut_), _p(loads), C.byref(feas), C.byref(nb)), "og_partition_kway")
    return cls[:n], dict(cut=int(cut_.value), loads=[int(x) for x in loads[:k]], feasible=int(feas.value),
                         bisections=int(nb.value))
