"""B300-native multilevel CPU/GPU bipartitioner for weighted task DAGs.

Python binding of the C-ABI in ``include/gp.h``: argument marshalling only.
Every step of the path runs in the CUDA library ``libgp.so`` (sm_103a),
built in-tree by ``build.py``; if it cannot be built or loaded, every call
raises.  Arrays may be torch tensors (CUDA or CPU) or numpy arrays; device
tensors are passed as device pointers, everything else as host pointers.

The method (Wu, Lohmann, Schroeder-Preikschat, Sec. III.B, Eq. (1)-(2)):
split a DAG with per-vertex CPU/GPU kernel times and per-edge transfer times
into a CPU side and a GPU side under load bounds from the workload ratio,
minimising the transfer cost of cut edges; then evaluate the makespan.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

GP_OK, GP_ERR_INVALID, GP_ERR_NOT_DAG, GP_ERR_OOM, GP_ERR_CUDA, GP_ERR_TIMEOUT, GP_ERR_OVERFLOW = range(7)
MAX_LEVELS = 48

_lock = threading.Lock()
_lib = None


class GpError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = "%s failed: %s (status %d)" % (where, status_string(status) if _lib else "?", status)
        super().__init__(msg)
        self.status = status


class Result(C.Structure):
    _fields_ = [("cut", C.c_int64), ("load_cpu", C.c_int64), ("load_gpu", C.c_int64),
                ("bound_cpu", C.c_int64), ("bound_gpu", C.c_int64), ("feasible", C.c_int32),
                ("levels", C.c_int32), ("rounds", C.c_int32), ("coarsest_n", C.c_int32),
                ("alg_bytes", C.c_int64), ("ms", C.c_float * 8)]

    def as_dict(self):
        d = {f[0]: int(getattr(self, f[0])) for f in self._fields_ if f[0] != "ms"}
        d["ms"] = [float(x) for x in self.ms]
        return d


_L1 = MAX_LEVELS + 1


class Trace(C.Structure):
    _fields_ = [("levels", C.c_int32), ("gggp_trial", C.c_int32), ("n", C.c_int64 * _L1),
                ("a", C.c_int64 * _L1), ("rounds", C.c_int32 * _L1), ("moves", C.c_int64 * _L1),
                ("balanced", C.c_int32 * _L1), ("bal_moves", C.c_int64 * _L1)]

    def as_dict(self):
        L = self.levels
        return dict(levels=L, gggp_trial=self.gggp_trial, n=list(self.n[:L + 1]), a=list(self.a[:L + 1]),
                    rounds=list(self.rounds[:L + 1]), moves=list(self.moves[:L + 1]),
                    balanced=list(self.balanced[:L + 1]), bal_moves=list(self.bal_moves[:L + 1]))


_P = C.c_void_p
_I64 = C.c_int64
_I32 = C.c_int32
_U64 = C.c_uint64
_D = C.c_double


def lib():
    """The loaded libgp.so (built in-tree on first use if missing or older than its sources)."""
    global _lib
    with _lock:
        if _lib is None:
            # GP_LIBRARY=checked loads the checked build (every gathered index tested in-kernel)
            path = _build.build(checked=os.environ.get("GP_LIBRARY") == "checked")
            L = C.CDLL(path)
            sig = {
                "gp_graph_create": [_I64, _I64, _P, _P, _P, _P, _P, C.c_int, _P, C.POINTER(_P)],
                "gp_graph_create_deferred": [_I64, _I64, _P, _P, _P, _P, _P, C.c_int, _P, C.POINTER(_P)],
                "gp_graph_destroy": [_P],
                "gp_graph_info": [_P, _P, _P, _P, _P, _P, _P],
                "gp_graph_export": [_P, _P, _P, _P, _P, _P],
                "gp_bounds": [_I64, _I64, _D, _D, _P, _P],
                "gp_partition": [_P, _D, _D, _U64, _P, _P, _P],
                "gp_partition_fixed": [_P, _P, _D, _D, _U64, _P, _P, _P],
                "gp_last_trace": [_P, _P],
                "gp_makespan": [_P, _P, _P, _P, _P],
                "gp_cut": [_P, _P, _P, _P],
                "gp_makespan_noalloc": [_P, _P, _P, _P, _P],
                "gp_makespan_workers": [_P, _P, _I32, _I32, _P, _P, _P],
                "gp_selftest_checked": [_P],
                "gp_partition_kway": [_I64, _I64, _P, _P, _P, _I32, _P, C.c_int, _D, _U64, _P, _P, _P, _P, _P, _P],
                "gp_batch_makespan_workers": [_I32, _P, _P, _I32, _I32, _P, _P],
                "gp_step_match": [_I64, _P, _P, _P, _P, _P, _I64, _I64, _U64, _I32, _I32, _P, _P],
                "gp_step_contract": [_I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P],
                "gp_step_gggp": [_I64, _P, _P, _P, _P, _P, _I64, _I64, _U64, _P, _P, _P],
                "gp_step_gggp_grow": [_I64, _P, _P, _P, _P, _P, _I64, _I64, _I64, _P, _P, _P],
                "gp_step_refine": [_I64, _P, _P, _P, _P, _P, _I64, _I64, _P, _P, _P],
                "gp_prof_enable": [C.c_int],
                "gp_prof_reset": [],
                "gp_prof_read": [C.c_int, _P, _P, _P],
                "gp_batch_partition": [_I32, _P, _P, _D, _P, _P, _P, _P, _P],
                "gp_batch_set_schedule": [_I32],
                "gp_batch_autotune": [_I32, _P, _P, _D, _P, _P, _P, _P],
                "gp_step_mma_bf16": [_I64, _I32, _I32, _P, _P, _P, _P],
                "gp_model_create": [_U64, C.POINTER(_P)],
                "gp_model_destroy": [_P],
                "gp_model_get_params": [_P, _P],
                "gp_model_set_params": [_P, _P],
                "gp_model_save": [_P, C.c_char_p],
                "gp_model_load": [C.c_char_p, C.POINTER(_P)],
                "gp_model_forward": [_P, _P, _P, _P],
                "gp_model_grad": [_P, _P, _P, _P, _P, _P],
                "gp_model_train_step": [_P, _P, _P, C.c_float, _P, _P],
                "gp_partition_learned": [_P, _P, _P, _D, _D, _P, _P, _P],
                "gp_partition_learned_vcycle": [_P, _P, _P, _D, _D, _U64, _P, _P, _P],
                "gp_batch_partition_learned": [_I32, _P, _P, _P, _D, _P, _P, _P, _P],
                "gp_graph_create_batch": [_I32, _P, _P, _P, _P, _P, _P, _P, C.c_int, _P, _P, _P],
                "gp_selftest_wait_timeout": [_I32, _P],
                "gp_selftest_grid_wait_timeout": [_P],
            }
            for name, args in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = C.c_int
            L.gp_status_string.argtypes = [C.c_int]
            L.gp_status_string.restype = C.c_char_p
            L.gp_kernel_name.argtypes = [C.c_int]
            L.gp_kernel_name.restype = C.c_char_p
            L.gp_launch_count.argtypes = []
            L.gp_launch_count.restype = C.c_int64
            L.gp_model_param_count.argtypes = []
            L.gp_model_param_count.restype = C.c_int64
            L.gp_batch_schedule_count.argtypes = []
            L.gp_batch_schedule_count.restype = C.c_int32
            L.gp_batch_schedule_name.argtypes = [_I32]
            L.gp_batch_schedule_name.restype = C.c_char_p
            L.gp_checked_site.argtypes = [_I32]
            L.gp_checked_site.restype = C.c_int32
            _lib = L
    return _lib


def library_path() -> str:
    """The library file lib() loads (libgp.so, or libgp_checked.so with GP_LIBRARY=checked)."""
    return _build.LIB_CHECKED if os.environ.get("GP_LIBRARY") == "checked" else _build.LIB


def status_string(st: int) -> str:
    return lib().gp_status_string(st).decode()


def _check(st: int, where: str):
    if st != GP_OK:
        raise GpError(st, where)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, is_device) of a torch tensor / numpy array / None."""
    if x is None:
        return None, False
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), bool(x.is_cuda)
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data, False
    raise TypeError("expected a torch tensor or a numpy array, got %r" % type(x))


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------------------
# C-ABI, same names
# ---------------------------------------------------------------------------

def _create(fn, name, n, m, arrs, stream):
    ptrs = [_ptr(a) for a in arrs]
    kinds = {dev for (_, dev) in ptrs}
    if len(kinds) != 1:
        raise ValueError("all five arrays must live on the same side (host or device)")
    h = _P()
    st = fn(int(n), int(m), *[p for p, _ in ptrs], 1 if kinds.pop() else 0, _stream(stream), C.byref(h))
    _check(st, name)
    return h


def gp_graph_create(n, m, offsets, cols, edge_cost, cpu_cost, gpu_cost, stream=None):
    """Copy a DAG (out-CSR + costs) to the device and validate it; returns the handle."""
    return _create(lib().gp_graph_create, "gp_graph_create", n, m, [offsets, cols, edge_cost, cpu_cost, gpu_cost],
                   stream)


def gp_graph_create_deferred(n, m, offsets, cols, edge_cost, cpu_cost, gpu_cost, stream=None):
    """gp_graph_create whose topological levels are computed beside the caller's next work; a cycle
    is reported (GP_ERR_NOT_DAG) by the first call that needs the levels."""
    return _create(lib().gp_graph_create_deferred, "gp_graph_create_deferred", n, m,
                   [offsets, cols, edge_cost, cpu_cost, gpu_cost], stream)


def gp_graph_create_batch(graphs, stream=None):
    """gp_graph_create for many DAGs in one persistent launch.  graphs: dicts as for Graph (all
    arrays on the host, or all on the device).  Returns (handles, statuses); a handle is None where
    its status is not GP_OK."""
    count = len(graphs)
    keys = ("offsets", "cols", "edge_cost", "cpu_cost", "gpu_cost")
    ptrs = [[_ptr(g[k]) for k in keys] for g in graphs]
    kinds = {dev for row in ptrs for (p, dev) in row if p is not None}
    if len(kinds) > 1:
        raise ValueError("all arrays must live on the same side (host or device)")
    kind = 1 if kinds and kinds.pop() else 0
    arr = lambda t, vals: (t * max(count, 1))(*vals)
    n = arr(C.c_int64, [int(g["n"]) for g in graphs])
    m = arr(C.c_int64, [int(g["m"]) for g in graphs])
    cols = [arr(_P, [row[j][0] for row in ptrs]) for j in range(5)]
    out = (_P * max(count, 1))()
    st = (C.c_int * max(count, 1))()
    _check(lib().gp_graph_create_batch(count, n, m, *cols, kind, _stream(stream), out, st), "gp_graph_create_batch")
    handles = [(_P(out[i]) if st[i] == GP_OK else None) for i in range(count)]
    return handles, [int(st[i]) for i in range(count)]


def gp_graph_destroy(h):
    _check(lib().gp_graph_destroy(h), "gp_graph_destroy")


def gp_graph_info(h):
    v = [C.c_int64(), C.c_int64(), C.c_int64(), C.c_int32(), C.c_int64(), C.c_int64()]
    _check(lib().gp_graph_info(h, *[C.byref(x) for x in v]), "gp_graph_info")
    return dict(n=v[0].value, m=v[1].value, a0=v[2].value, nlevels=v[3].value, sum_cpu=v[4].value,
                sum_gpu=v[5].value)


def gp_graph_export(h, off=None, adj=None, W=None, level=None, stream=None):
    _check(lib().gp_graph_export(h, _ptr(off)[0], _ptr(adj)[0], _ptr(W)[0], _ptr(level)[0], _stream(stream)),
           "gp_graph_export")


def gp_bounds(sum_cpu, sum_gpu, r_cpu=-1.0, tol=0.03):
    bc, bg = C.c_int64(), C.c_int64()
    _check(lib().gp_bounds(int(sum_cpu), int(sum_gpu), float(r_cpu), float(tol), C.byref(bc), C.byref(bg)),
           "gp_bounds")
    return int(bc.value), int(bg.value)


def gp_partition(h, r_cpu, tol, seed, part_out, stream=None):
    res = Result()
    _check(lib().gp_partition(h, float(r_cpu), float(tol), int(seed), _ptr(part_out)[0], C.byref(res),
                              _stream(stream)), "gp_partition")
    return res.as_dict()


def gp_partition_fixed(h, fixed, r_cpu, tol, seed, part_out, stream=None):
    """gp_partition with pinned vertices: fixed = int8 per vertex (0 CPU, 1 GPU, -1 free), host or
    device, or None (all free)."""
    if fixed is not None and str(getattr(fixed, "dtype", "")) not in ("int8", "torch.int8"):
        raise TypeError("fixed must be an int8 array")
    res = Result()
    _check(lib().gp_partition_fixed(h, _ptr(fixed)[0], float(r_cpu), float(tol), int(seed), _ptr(part_out)[0],
                                    C.byref(res), _stream(stream)), "gp_partition_fixed")
    return res.as_dict()


def gp_last_trace(h):
    t = Trace()
    _check(lib().gp_last_trace(h, C.byref(t)), "gp_last_trace")
    return t.as_dict()


def gp_makespan(h, part, finish_out=None, stream=None):
    ms = C.c_int64()
    _check(lib().gp_makespan(h, _ptr(part)[0], C.byref(ms), _ptr(finish_out)[0], _stream(stream)), "gp_makespan")
    return int(ms.value)


def gp_partition_kway(g, costs, cls_out, tol=0.03, seed=0, stream=None):
    """k device classes by recursive bisection.  g: dict with n, m, offsets, cols, edge_cost (all host
    or all device); costs: int32 [k, n] (same memory kind); cls_out: uint8[n] (device or host).
    Returns dict(cut, loads (list of k), feasible, bisections)."""
    n, m = int(g["n"]), int(g["m"])
    k = int(costs.shape[0])
    ptrs = [_ptr(g[key]) for key in ("offsets", "cols", "edge_cost")] + [_ptr(costs)]
    kinds = {p[1] for p in ptrs if p[0]}
    if len(kinds) > 1:
        raise ValueError("CSR arrays and costs must all be host or all be device memory")
    kind = kinds.pop() if kinds else 0
    cut = C.c_int64()
    loads = (C.c_int64 * max(k, 1))()
    feas = C.c_int32()
    nb = C.c_int32()
    _check(lib().gp_partition_kway(n, m, ptrs[0][0], ptrs[1][0], ptrs[2][0], k, ptrs[3][0], kind, float(tol), int(seed),
                                   _ptr(cls_out)[0], C.byref(cut), loads, C.byref(feas), C.byref(nb), _stream(stream)),
           "gp_partition_kway")
    return dict(cut=int(cut.value), loads=[int(loads[i]) for i in range(k)], feasible=int(feas.value),
                bisections=int(nb.value))


def gp_makespan_workers(h, part, workers_cpu=3, workers_gpu=1, finish_out=None, stream=None):
    """Makespan of the mapping on a fixed number of workers per side (a list schedule; the paper's
    testbed has 3 CPU workers and 1 GPU worker)."""
    ms = C.c_int64()
    _check(lib().gp_makespan_workers(h, _ptr(part)[0], int(workers_cpu), int(workers_gpu), C.byref(ms),
                                     _ptr(finish_out)[0], _stream(stream)), "gp_makespan_workers")
    return int(ms.value)


def gp_batch_makespan_workers(handles, parts, workers_cpu=3, workers_gpu=1, stream=None):
    """gp_makespan_workers for many graphs in one launch; returns the makespans (list)."""
    count, hs, _, _ = _batch_args(handles, None, None)
    if len(parts) != count:
        raise ValueError("one split buffer per graph")
    pp = (_P * max(count, 1))(*[_ptr(p)[0] for p in parts])
    ms = (C.c_int64 * max(count, 1))()
    _check(lib().gp_batch_makespan_workers(count, hs, pp, int(workers_cpu), int(workers_gpu), ms, _stream(stream)),
           "gp_batch_makespan_workers")
    return [int(ms[i]) for i in range(count)]


MAKESPAN_NOALLOC_MAX_N = 1 << 20


def gp_makespan_noalloc(h, part, finish_out=None, stream=None):
    """gp_makespan without any device allocation (scratch compiled into the library).

    For callers that cannot allocate device memory (a host allocator that owns all of it, a
    latency-critical loop).  ``part`` and ``finish_out`` must be device tensors; at most
    MAKESPAN_NOALLOC_MAX_N vertices; the call synchronises ``stream``; calls that overlap on one
    GPU race on the shared scratch.  The first call on a device (and the first after a reset of
    its context) resolves the scratch address: make it before any stream capture.
    """
    ms = C.c_int64()
    st = lib().gp_makespan_noalloc(h, _ptr(part)[0], C.byref(ms), _ptr(finish_out)[0], _stream(stream))
    if st == GP_ERR_INVALID:
        raise GpError(st, "gp_makespan_noalloc (device buffers required, at most %d vertices, handle on the "
                          "current device)" % MAKESPAN_NOALLOC_MAX_N)
    _check(st, "gp_makespan_noalloc")
    return int(ms.value)


def gp_cut(h, part, stream=None):
    c = C.c_int64()
    _check(lib().gp_cut(h, _ptr(part)[0], C.byref(c), _stream(stream)), "gp_cut")
    return int(c.value)


def gp_step_match(n, off, adj, W, vC, vG, cap_cpu, cap_gpu, seed, rounds, twohop, mate_out, stream=None):
    _check(lib().gp_step_match(int(n), _ptr(off)[0], _ptr(adj)[0], _ptr(W)[0], _ptr(vC)[0], _ptr(vG)[0],
                               int(cap_cpu), int(cap_gpu), int(seed), int(rounds), int(twohop),
                               _ptr(mate_out)[0], _stream(stream)), "gp_step_match")


def gp_step_contract(n, off, adj, W, vC, vG, mate, cmap_out, coff, cadj, cW, cvC, cvG, stream=None):
    nc, ac = C.c_int64(), C.c_int64()
    _check(lib().gp_step_contract(int(n), _ptr(off)[0], _ptr(adj)[0], _ptr(W)[0], _ptr(vC)[0], _ptr(vG)[0],
                                  _ptr(mate)[0], _ptr(cmap_out)[0], _ptr(coff)[0], _ptr(cadj)[0], _ptr(cW)[0],
                                  _ptr(cvC)[0], _ptr(cvG)[0], C.byref(nc), C.byref(ac), _stream(stream)),
           "gp_step_contract")
    return int(nc.value), int(ac.value)


def gp_step_gggp(n, off, adj, W, vC, vG, bound_cpu, bound_gpu, seed, part_out, stream=None):
    t = C.c_int32()
    _check(lib().gp_step_gggp(int(n), _ptr(off)[0], _ptr(adj)[0], _ptr(W)[0], _ptr(vC)[0], _ptr(vG)[0],
                              int(bound_cpu), int(bound_gpu), int(seed), _ptr(part_out)[0], C.byref(t),
                              _stream(stream)), "gp_step_gggp")
    return int(t.value)


def gp_step_gggp_grow(n, off, adj, W, vC, vG, bound_cpu, bound_gpu, start, part_out, stream=None):
    c = C.c_int64()
    _check(lib().gp_step_gggp_grow(int(n), _ptr(off)[0], _ptr(adj)[0], _ptr(W)[0], _ptr(vC)[0], _ptr(vG)[0],
                                   int(bound_cpu), int(bound_gpu), int(start), _ptr(part_out)[0], C.byref(c),
                                   _stream(stream)), "gp_step_gggp_grow")
    return int(c.value)


def gp_step_refine(n, off, adj, W, vC, vG, bound_cpu, bound_gpu, part, stream=None):
    st = (C.c_int64 * 6)()
    _check(lib().gp_step_refine(int(n), _ptr(off)[0], _ptr(adj)[0], _ptr(W)[0], _ptr(vC)[0], _ptr(vG)[0],
                                int(bound_cpu), int(bound_gpu), _ptr(part)[0], st, _stream(stream)),
           "gp_step_refine")
    return dict(rounds=st[0], balanced=st[1], moves=st[2], bal_moves=st[3], load_cpu=st[4], load_gpu=st[5])


def _batch_args(handles, r_cpu, seeds):
    count = len(handles)
    hs = (_P * max(count, 1))(*[h.value if isinstance(h, _P) else h for h in handles])
    rc = None if r_cpu is None else (_D * max(count, 1))(*[float(x) for x in r_cpu])
    sd = None if seeds is None else (_U64 * max(count, 1))(*[int(x) for x in seeds])
    return count, hs, rc, sd


def gp_batch_partition(handles, parts, r_cpu=None, tol=0.03, seeds=None, makespans=False, stream=None):
    """Partition many graphs in one call (one persistent launch); returns (results, makespans).

    handles: graph handles; parts: one uint8 buffer per graph (device tensors or host arrays);
    r_cpu / seeds: per-graph lists or None (-1 / 0 for all).  makespans=True also evaluates the
    makespan of every final split.
    """
    count, hs, rc, sd = _batch_args(handles, r_cpu, seeds)
    if len(parts) != count:
        raise ValueError("one split buffer per graph")
    pp = (_P * max(count, 1))(*[_ptr(p)[0] for p in parts])
    res = (Result * max(count, 1))()
    ms = (C.c_int64 * max(count, 1))() if makespans else None
    _check(lib().gp_batch_partition(count, hs, rc, float(tol), sd, pp, res, ms, _stream(stream)),
           "gp_batch_partition")
    out = [res[i].as_dict() for i in range(count)]
    return out, ([int(ms[i]) for i in range(count)] if makespans else None)


def gp_batch_partition_learned(handles, model, parts, r_cpu=None, tol=0.03, makespans=False, stream=None):
    """The learned path for many graphs: one network forward over their union, then the persistent
    batch kernel (proposal + refinement of level 0 per graph).  Returns (results, makespans)."""
    count, hs, rc, _ = _batch_args(handles, r_cpu, None)
    if len(parts) != count:
        raise ValueError("one split buffer per graph")
    pp = (_P * max(count, 1))(*[_ptr(p)[0] for p in parts])
    res = (Result * max(count, 1))()
    ms = (C.c_int64 * max(count, 1))() if makespans else None
    _check(lib().gp_batch_partition_learned(count, hs, model, rc, float(tol), pp, res, ms, _stream(stream)),
           "gp_batch_partition_learned")
    out = [res[i].as_dict() for i in range(count)]
    return out, ([int(ms[i]) for i in range(count)] if makespans else None)


def gp_batch_schedule_count() -> int:
    return int(lib().gp_batch_schedule_count())


def gp_batch_schedule_name(i: int):
    r = lib().gp_batch_schedule_name(int(i))
    return r.decode() if r is not None else None


def gp_batch_set_schedule(i: int):
    _check(lib().gp_batch_set_schedule(int(i)), "gp_batch_set_schedule")


def gp_batch_autotune(handles, r_cpu=None, tol=0.03, seeds=None, stream=None):
    """Time every batch schedule on this batch, keep the fastest; returns (best, ms per schedule)."""
    count, hs, rc, sd = _batch_args(handles, r_cpu, seeds)
    k = gp_batch_schedule_count()
    best = C.c_int32()
    ms = (C.c_float * k)()
    _check(lib().gp_batch_autotune(count, hs, rc, float(tol), sd, C.byref(best), ms, _stream(stream)),
           "gp_batch_autotune")
    return int(best.value), [float(ms[i]) for i in range(k)]


def gp_step_mma_bf16(A, B, C, stream=None):
    """C = A . B on the tensor cores (BF16 in, FP32 accumulate); device tensors, (N, K) in
    {(64, 192), (192, 64), (64, 64)}."""
    M, K = A.shape
    N = B.shape[1]
    _check(lib().gp_step_mma_bf16(int(M), int(N), int(K), _ptr(A)[0], _ptr(B)[0], _ptr(C)[0], _stream(stream)),
           "gp_step_mma_bf16")


MPNN_PARAMS = 37505


def gp_model_create(seed=0):
    h = _P()
    _check(lib().gp_model_create(int(seed), C.byref(h)), "gp_model_create")
    return h


def gp_model_destroy(m):
    _check(lib().gp_model_destroy(m), "gp_model_destroy")


def gp_model_get_params(m):
    out = np.zeros(MPNN_PARAMS, np.float32)
    _check(lib().gp_model_get_params(m, out.ctypes.data), "gp_model_get_params")
    return out


def gp_model_set_params(m, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.shape != (MPNN_PARAMS,):
        raise ValueError("expected %d parameters" % MPNN_PARAMS)
    _check(lib().gp_model_set_params(m, p.ctypes.data), "gp_model_set_params")


def gp_model_save(m, path):
    _check(lib().gp_model_save(m, str(path).encode()), "gp_model_save")


def gp_model_load(path):
    h = _P()
    _check(lib().gp_model_load(str(path).encode(), C.byref(h)), "gp_model_load")
    return h


def gp_model_forward(m, g, logits_out, stream=None):
    _check(lib().gp_model_forward(m, g, _ptr(logits_out)[0], _stream(stream)), "gp_model_forward")


def gp_model_grad(m, g, labels, stream=None):
    grad = np.zeros(MPNN_PARAMS, np.float32)
    loss = C.c_double()
    _check(lib().gp_model_grad(m, g, _ptr(labels)[0], grad.ctypes.data, C.byref(loss), _stream(stream)),
           "gp_model_grad")
    return float(loss.value), grad


def gp_model_train_step(m, g, labels, lr, stream=None):
    loss = C.c_double()
    _check(lib().gp_model_train_step(m, g, _ptr(labels)[0], float(lr), C.byref(loss), _stream(stream)),
           "gp_model_train_step")
    return float(loss.value)


def gp_partition_learned(g, model, part_out, logits=None, r_cpu=-1.0, tol=0.03, stream=None):
    res = Result()
    _check(lib().gp_partition_learned(g, model, _ptr(logits)[0], float(r_cpu), float(tol), _ptr(part_out)[0],
                                      C.byref(res), _stream(stream)), "gp_partition_learned")
    return res.as_dict()


def gp_partition_learned_vcycle(g, model, part_out, logits=None, r_cpu=-1.0, tol=0.03, seed=0, stream=None):
    """The learned path as a V-cycle: the proposal restricts the matching to same-side pairs, the
    coarsest split is the proposed sides, and every level is refined on the way back."""
    res = Result()
    _check(lib().gp_partition_learned_vcycle(g, model, _ptr(logits)[0], float(r_cpu), float(tol), int(seed),
                                             _ptr(part_out)[0], C.byref(res), _stream(stream)),
           "gp_partition_learned_vcycle")
    return res.as_dict()


def gp_checked_site(clear: bool = True) -> int:
    """Checked build: the site of the first failed in-kernel index test since the last clear (0: none);
    -1 in the unchecked build."""
    return int(lib().gp_checked_site(1 if clear else 0))


def gp_selftest_checked(stream=None):
    """Checked build: one gather through an out-of-range index behind its test (site 99)."""
    _check(lib().gp_selftest_checked(_stream(stream)), "gp_selftest_checked")


def gp_launch_count() -> int:
    return int(lib().gp_launch_count())


def gp_prof_enable(on: bool):
    _check(lib().gp_prof_enable(1 if on else 0), "gp_prof_enable")


def gp_prof_reset():
    _check(lib().gp_prof_reset(), "gp_prof_reset")


def gp_prof_read(kernel: int):
    n, ms, b = C.c_int64(), C.c_double(), C.c_int64()
    _check(lib().gp_prof_read(int(kernel), C.byref(n), C.byref(ms), C.byref(b)), "gp_prof_read")
    return dict(launches=int(n.value), total_ms=float(ms.value), alg_bytes=int(b.value))


def gp_kernel_name(kernel: int):
    r = lib().gp_kernel_name(int(kernel))
    return r.decode() if r is not None else None


def kernel_families():
    out = []
    k = 0
    while True:
        name = gp_kernel_name(k)
        if name is None:
            return out
        out.append(name)
        k += 1


# ---------------------------------------------------------------------------
# Convenience: a handle that owns its device graph
# ---------------------------------------------------------------------------

class Graph:
    """Device copy of a DAG given as a dict of arrays (see gen.py), torch or numpy."""

    def __init__(self, g, stream=None, deferred=False):
        self.n, self.m = int(g["n"]), int(g["m"])
        create = gp_graph_create_deferred if deferred else gp_graph_create
        self.h = create(self.n, self.m, g["offsets"], g["cols"], g["edge_cost"], g["cpu_cost"], g["gpu_cost"],
                        stream=stream)

    def info(self):
        return gp_graph_info(self.h)

    def partition(self, part_out, r_cpu=-1.0, tol=0.03, seed=0, stream=None, fixed=None):
        if fixed is not None:
            return gp_partition_fixed(self.h, fixed, r_cpu, tol, seed, part_out, stream)
        return gp_partition(self.h, r_cpu, tol, seed, part_out, stream)

    def makespan(self, part, finish_out=None, stream=None):
        return gp_makespan(self.h, part, finish_out, stream)

    def cut(self, part, stream=None):
        return gp_cut(self.h, part, stream)

    def trace(self):
        return gp_last_trace(self.h)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            gp_graph_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
