"""Benchmark: DAG edges partitioned per second on B300.

One step = the whole path on one DAG resident in HBM: gp_graph_create_deferred
from device CSR (validation, transpose, symmetrisation; the topological levels and
the level-ordered in-CSR on a side stream, beside the partition),
gp_partition (coarsening, initial split, refinement, cut), gp_makespan and
gp_graph_destroy.
Default workload (the largest single-GPU one): layered random DAG, 1,000 layers x
16,000 vertices, 128M edges (int64 offsets), lognormal CPU times, GPU = CPU /
U(2, 40), transfer U{1..10,000} ns, seed 0.  Its split, result fields and makespan
are compared with the oracle's recorded result (tests/golden/layered16m_oracle.json).

The line also carries objects: "layered1m" (the same step on 1,000 x 1,000
vertices, 8M edges, checked against the oracle run here), "fixed" (that DAG with
the paper's host vertex pinned to the CPU), "learned" / "learned_16m" (network
proposal + refinement; 16 held-out 1M DAGs against the plain path) and "batch"
(4,096 DAGs of log-uniform size 100..50,000 partitioned by gp_batch_partition in
one persistent launch replayed from a captured CUDA graph, against the plain path
in a loop).  --workload layered1m | batch | cholesky64x1024 makes another
workload the main line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload layered16m|layered1m|batch|cholesky64x1024]
                  [--no-batch] [--no-learned] [--no-cpu-baseline]

Under torchrun (N > 1) every rank runs an independent replica (the single-DAG
path does not shard); value = edges processed by all ranks / max rank time.
The L2 is flushed (256 MB write) between timed steps, outside the events.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "dag_edges_partitioned_per_sec"
UNIT = "edges/s"
WORKLOAD = "layered DAG 1,000 layers x 1,000 vertices, 8,000,000 edges, seed 0"
BATCH_METRIC = "dag_graphs_partitioned_per_sec"
BATCH_UNIT = "graphs/s"
BATCH_COUNT = 4096
BATCH_WORKLOAD = ("4,096 DAGs, log-uniform 100..50,000 vertices, kinds in turn tiled Cholesky (T 4..40), "
                  "tiled LU, layered (width ~sqrt(n), 8 edges per vertex to the next 1-4 layers); base seed 0")


MODEL_PATH = os.path.join(ROOT, "paper_1502_07451_b300", "models", "mpnn3_h64.bin")
CHOL_WORKLOAD = ("1,024 tiled Cholesky task DAGs, T = 64 (45,760 tasks and 131,040 edges each), learned proposal + "
                 "refinement + makespan per graph; the plain batched path uses seeds 0..1023")
HELD_OUT_SEEDS = tuple(range(1, 17))  # 16 held-out 1M-vertex layered DAGs


def _build_chunk(chunk):
    from paper_1502_07451_b300 import gen
    return [gen.build_from_spec(it) for it in chunk]


def _build_layered_1m(seed):
    from paper_1502_07451_b300 import gen
    return gen.config_layered_1m(seed)


def batch_shard(count, rank, world):
    """This rank's graphs of the batch: with one rank the recipe's `count` graphs; with `world` ranks
    (weak scaling: `count` graphs per GPU) the recipe's count * world graphs placed on the ranks by
    longest-processing-time first on their edge counts.  Returns (spec items, total graphs)."""
    from paper_1502_07451_b300 import gen, shard
    spec = gen.batch_spec(count * world)
    if world == 1:
        return spec, count
    mine = shard.lpt([gen.spec_edges(it) for it in spec], world)[rank]
    return [spec[i] for i in mine], count * world


class BatchGen:
    """Builds the batch's graphs in spawned worker processes (started before any CUDA call)."""

    def __init__(self, count=BATCH_COUNT, held=True, rank=0, world=1, batch=True):
        import multiprocessing as mp
        self.spec, self.total = batch_shard(count, rank, world)
        if not batch:
            self.spec = []
        self.count = len(self.spec)
        self.nproc = max(1, min(32, (os.cpu_count() or 4) // world))
        self.pool = mp.get_context("spawn").Pool(self.nproc)
        self.chunks = [self.spec[i::self.nproc] for i in range(self.nproc)]
        self.res = self.pool.map_async(_build_chunk, self.chunks)
        self.held = self.pool.map_async(_build_layered_1m, HELD_OUT_SEEDS if held else ())

    def held_out(self):
        return self.held.get()

    def wait(self):
        """Block until every graph is built, then end the workers (their results stay with the
        parent), so that no worker process competes with the timed regions."""
        self.res.wait()
        self.held.wait()
        self.close()

    def graphs(self):
        out = [None] * self.count
        for i, part in enumerate(self.res.get()):
            for j, g in enumerate(part):
                out[i + j * self.nproc] = g
        return out

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None


def profiled_traffic(family, workload="1m", alg_bytes_per_launch=None, schedule=None):
    """DRAM bytes per launch of `family` on `workload` ("1m", "16m" or "batch4096") from a committed ncu
    summary that covers this family and workload (and, where the summary names one, this batch
    schedule) and whose kernel sources are unchanged since the capture, else None.
    Returns (bytes, source file, how): a summary gives either the family's bytes per launch
    (traffic_bytes_per_launch, every launch of a step captured) or the DRAM / algorithmic ratio of one
    captured launch (traffic_ratio), which scales this run's algorithmic bytes per launch."""
    import hashlib
    import glob
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        kv = {}
        with open(path) as f:
            for line in f:
                if line.startswith("traffic_"):
                    k, _, v = line.partition(":")
                    kv[k.strip()] = v.strip()
        if kv.get("traffic_kernel") != family:
            continue
        if kv.get("traffic_workload", "1m") != workload:
            continue
        if kv.get("traffic_schedule", schedule) != schedule:
            continue
        h = hashlib.sha256()
        for src in kv.get("traffic_sources", "").split():
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
        if h.hexdigest() != kv.get("traffic_sources_sha256"):
            continue
        rel = os.path.relpath(path, ROOT)
        if "traffic_bytes_per_launch" in kv:
            return float(kv["traffic_bytes_per_launch"]), rel, "DRAM bytes of every launch of one step / launches"
        if "traffic_ratio" in kv and alg_bytes_per_launch:
            return (float(kv["traffic_ratio"]) * alg_bytes_per_launch, rel,
                    "DRAM / algorithmic bytes of the captured launch (%s) x this run's algorithmic bytes per launch"
                    % kv["traffic_ratio"])
    return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi's start-up (driver queries) stays out of the timed region: wait for its first sample
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for name, v in zip(names, p[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def physical_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        parts = [p for p in vis.split(",") if p.strip()]
        if local_rank < len(parts):
            return parts[local_rank].strip()
    return str(local_rank)


def oracle_step(g):
    import oracle
    t0 = time.perf_counter()
    part, res = oracle.partition(g)
    ms = oracle.makespan(g, part)
    return time.perf_counter() - t0, part, res, ms


def oracle_batch_sample(graphs, budget_s=12.0):
    """The oracle over the batch's graphs in order until about budget_s seconds of CPU work."""
    import oracle
    t0 = time.perf_counter()
    k = 0
    for g in graphs:
        part, _ = oracle.partition(g)
        oracle.makespan(g, part)
        k += 1
        if time.perf_counter() - t0 > budget_s:
            break
    return k, time.perf_counter() - t0


def _oracle_batch_worker(arg):
    """One host core's share of the batch: build its graphs (not timed), then run the oracle's
    partition + makespan over them in order until `budget` seconds of oracle time."""
    items, budget = arg
    import oracle
    from paper_1502_07451_b300 import gen
    oracle.lib()
    graphs = [gen.build_from_spec(it) for it in items]
    k, spent = 0, 0.0
    for g in graphs:
        t0 = time.perf_counter()
        part, _ = oracle.partition(g)
        oracle.makespan(g, part)
        spent += time.perf_counter() - t0
        k += 1
        if spent > budget:
            break
    return k, spent


def oracle_batch_all_cores(count=BATCH_COUNT, budget_s=12.0):
    """The oracle over the batch recipe on every host core: worker w takes graphs w, w + P, w + 2P, ...
    (P workers, spawned) until budget_s seconds of oracle time; value = graphs done by all workers /
    the slowest worker's oracle time."""
    import multiprocessing as mp
    from paper_1502_07451_b300 import gen
    spec = gen.batch_spec(count)
    nproc = max(1, min(64, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(nproc) as pool:
        out = pool.map(_oracle_batch_worker, [(spec[i::nproc], budget_s) for i in range(nproc)])
    done = sum(k for k, _ in out)
    slowest = max(t for _, t in out)
    return done / slowest, nproc, done, slowest


def run_reference_batch(args, rank, world):
    if rank != 0:
        return
    bg = BatchGen(256)
    graphs = bg.graphs()
    oracle_batch_sample(graphs[:2], 1e9)
    tot, done = 0.0, 0
    for _ in range(args.steps):
        k, dt = oracle_batch_sample(graphs, 20.0 / max(args.steps, 1))
        tot += dt
        done += k
    value = done / tot
    desc = "the first graphs of the batch recipe in order (%d graphs over %d steps), oracle partition + makespan" % (
        done, args.steps)
    line = {"metric": BATCH_METRIC, "value": value, "unit": BATCH_UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "sample": desc}, "impl": "reference",
            "cpu_baseline": {"value": value, "unit": BATCH_UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": BATCH_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def quiet_heap():
    """Collect the heap once, freeze it and switch the collector off, so that no garbage-collection pass
    over the (large) input graphs lands in a timed region."""
    import gc
    gc.collect()
    gc.freeze()
    gc.disable()  # and no pass at all until the line is printed (the bench allocates little meanwhile)


def max_over_ranks(x, world, device="cuda"):
    """The largest of the ranks' values (the slowest rank's time); x itself on one rank."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return world * units_per_rank / seconds


def run_reference(args, rank, world):
    """The oracle on the host cores, timed on a bounded sample of the workload (first 100 layers)."""
    from paper_1502_07451_b300 import gen
    if rank != 0:
        return
    if args.workload == "batch":
        run_reference_batch(args, rank, world)
        return
    if args.workload == "cholesky64x1024":
        g = gen.cholesky(64)
        oracle_step(g)
        tot = 0.0
        for i in range(args.steps):
            import oracle
            t0 = time.perf_counter()
            part, _ = oracle.partition(g, seed=i)
            oracle.makespan(g, part)
            tot += time.perf_counter() - t0
        value = args.steps / tot
        desc = "one tiled Cholesky T=64 DAG per step (seed = step), oracle partition + makespan"
        line = {"metric": BATCH_METRIC, "value": value, "unit": BATCH_UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
                "config": {"workload": CHOL_WORKLOAD, "sample": desc}, "impl": "reference",
                "cpu_baseline": {"value": value, "unit": BATCH_UNIT, "cores": 1, "kind": "oracle", "sample": desc},
                "e2e": {"value": value, "unit": BATCH_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    big = args.workload == "layered16m"
    sample = gen.layered(20, 16000, 2_560_000, 0) if big else gen.layered(100, 1000, 800_000, 0)
    for _ in range(args.warmup):
        oracle_step(sample)
    tot = 0.0
    for _ in range(args.steps):
        dt, _, _, _ = oracle_step(sample)
        tot += dt
    value = args.steps * sample["m"] / tot
    if big:
        desc = ("first 20 layers of the 16M workload recipe (320,000 vertices, 2,560,000 edges), oracle partition "
                "+ makespan")
        wl = "layered DAG 1,000 layers x 16,000 vertices, 128,000,000 edges (int64 offsets), seed 0"
    else:
        desc = "first 100 layers of the workload recipe (100,000 vertices, 800,000 edges), oracle partition + makespan"
        wl = WORKLOAD
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": wl, "sample": desc}, "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="layered16m",
                    choices=["layered16m", "layered1m", "batch", "cholesky64x1024"])
    ap.add_argument("--no-batch", action="store_true", help="skip the batch object of the layered lines")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned objects of the layered lines")
    ap.add_argument("--profile-case", default=None,
                    choices=["layered1m", "learned1m", "batch64", "batch4096", "layered4m", "layered16m"],
                    help="run one small invocation for a profiler (no timing, no JSON line contract)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.profile_case:
        run_profile_case(args.profile_case)
        return
    if args.workload == "cholesky64x1024":
        run_cholesky_line(args, rank, world, local_rank)
        return
    if args.workload == "batch":
        bgen = BatchGen(held=False, rank=rank, world=world)
        run_batch_line(args, rank, world, local_rank, bgen)
        return
    run_layered_line(args, rank, world, local_rank)


def _build_layered_16m(seed):
    from paper_1502_07451_b300 import gen
    return gen.config_layered_16m(seed)


def golden_16m_match(part, res, ms):
    """Whether the 16M workload's split, result fields and makespan equal the oracle's record of
    them (tests/golden/layered16m_oracle.json, written by a script that runs only the oracle)."""
    import hashlib
    path = os.path.join(ROOT, "tests", "golden", "layered16m_oracle.json")
    try:
        with open(path) as f:
            want = json.load(f)
    except OSError:
        return None
    ok = hashlib.sha256(np.ascontiguousarray(part).tobytes()).hexdigest() == want["sha256"]
    ok = ok and all(res[k] == v for k, v in want["result"].items()) and ms == want["makespan"]
    return bool(ok)


def measure_plain(g, K, W, stream, flush, world, sampler=None):
    """One step = gp_graph_create_deferred (device CSR) + gp_partition + gp_makespan +
    gp_graph_destroy on `g`.  W warm-ups, K timed steps (CUDA events on the stream, L2 flushed
    between steps), then the same K steps end to end from pinned host buffers, then a pass with
    events around every launch for the per-family roofline.  Returns a dict; "part" holds the
    split (host)."""
    import torch
    import torch.distributed as dist
    import paper_1502_07451_b300 as gp
    n, m = g["n"], g["m"]
    keys = ("offsets", "cols", "edge_cost", "cpu_cost", "gpu_cost")
    dg = {k: torch.from_numpy(g[k]).cuda() for k in keys}
    part = torch.empty(n, dtype=torch.uint8, device="cuda")

    def step():
        # the levels (read only by the makespan) are built on a side stream beside the partition
        h = gp.gp_graph_create_deferred(n, m, dg["offsets"], dg["cols"], dg["edge_cost"], dg["cpu_cost"],
                                        dg["gpu_cost"], stream=stream)
        res = gp.gp_partition(h, -1.0, 0.03, 0, part, stream)
        ms = gp.gp_makespan(h, part, None, stream)
        gp.gp_graph_destroy(h)
        return res, ms

    for _ in range(W):
        res, ms = step()
    torch.cuda.synchronize()

    # ---- timed device pass
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    launches0 = gp.gp_launch_count()
    total_ms = 0.0
    for _ in range(K):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        res, ms = step()
        b.record(stream)
        b.synchronize()
        total_ms += a.elapsed_time(b)
    torch.cuda.synchronize()
    launches = gp.gp_launch_count() - launches0
    clocks = sampler.stop() if sampler else None
    total_ms = max_over_ranks(total_ms, world)
    if world > 1:
        dist.barrier()
    value = job_rate(K * m, world, total_ms / 1e3)

    # ---- end to end through the C-ABI with pinned host buffers (H2D and D2H inside the timed region)
    hg = {k: torch.from_numpy(g[k]).pin_memory() for k in keys}
    hpart = torch.empty(n, dtype=torch.uint8).pin_memory()
    h2d = sum(int(hg[k].numel() * hg[k].element_size()) for k in keys)
    d2h = n + 8 + 8 * 28

    def e2e_step():
        h = gp.gp_graph_create_deferred(n, m, hg["offsets"], hg["cols"], hg["edge_cost"], hg["cpu_cost"],
                                        hg["gpu_cost"], stream=stream)
        r = gp.gp_partition(h, -1.0, 0.03, 0, hpart, stream)
        mk = gp.gp_makespan(h, hpart, None, stream)
        gp.gp_graph_destroy(h)
        return r, mk

    e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(K):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, world)
    e2e_value = job_rate(K * m, world, e2e_s)
    host_part = part.cpu().numpy()
    e2e_ok = bool(np.array_equal(hpart.numpy(), host_part))

    # ---- roofline: a second pass of the same K steps with CUDA events around every launch
    gp.gp_prof_reset()
    gp.gp_prof_enable(True)
    for _ in range(K):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()
    gp.gp_prof_enable(False)
    fams = gp.kernel_families()
    prof = {f: gp.gp_prof_read(i) for i, f in enumerate(fams)}
    gp.gp_prof_reset()
    hbm_peak, peak_kind = peaks()
    mem_fams = [f for f in fams if prof[f]["alg_bytes"] > 0]
    # the level traversal runs on a second stream beside the partition (deferred creation): it takes
    # device time but not step time, so the roofline kernel is the largest family of the critical path
    overlapped = {"levels"}
    dom = max((f for f in mem_fams if f not in overlapped), key=lambda f: prof[f]["total_ms"])
    dp = prof[dom]
    per_launch_bytes = dp["alg_bytes"] / max(dp["launches"], 1)
    per_launch_ms = dp["total_ms"] / max(dp["launches"], 1)
    achieved = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9
    share = {f: round(prof[f]["total_ms"] / max(sum(p["total_ms"] for p in prof.values()), 1e-9), 4)
             for f in fams if prof[f]["launches"]}
    # every family's achieved bandwidth (algorithmic bytes / event time), as a fraction of the peak
    by_family = {f: {"ms_per_step": round(prof[f]["total_ms"] / K, 4),
                     "achieved_gbs": round(prof[f]["alg_bytes"] / (prof[f]["total_ms"] * 1e-3) / 1e9, 1),
                     "frac": round(prof[f]["alg_bytes"] / (prof[f]["total_ms"] * 1e-3) / 1e9 / hbm_peak, 4)}
                 for f in mem_fams}
    return {"value": value, "ms_per_step": total_ms / K, "launches": int(launches), "clocks": clocks,
            "res": res, "makespan": ms, "part": host_part, "part_dev": part,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "e2e_ok": e2e_ok, "share": share, "by_family": by_family,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "peak_kind": peak_kind,
                         "alg_bytes_per_launch": per_launch_bytes, "launch_ms": per_launch_ms,
                         "launches": dp["launches"],
                         "overlapped_ms_per_step": {f: round(prof[f]["total_ms"] / K, 4) for f in overlapped
                                                    if f in prof}}}


WORKLOAD_16M = "layered DAG 1,000 layers x 16,000 vertices, 128,000,000 edges (int64 offsets), seed 0"
STEP = "gp_graph_create_deferred(device CSR) + gp_partition + gp_makespan + gp_graph_destroy"


def run_layered_line(args, rank, world, local_rank):
    """The layered lines: with --workload layered16m (the default) the 16M-vertex / 128M-edge DAG is
    the main line and the 1M-vertex DAG an object of it; with layered1m the 1M DAG is the main line.
    Objects: the host-vertex workload (fixed vertices), the learned path, the batch."""
    # every input is built by spawned workers (or here) before the first CUDA call; the workers are
    # ended before any timed region
    big = args.workload == "layered16m"
    want_batch = world == 1 and not args.no_batch
    bgen = BatchGen(held=not args.no_learned and world == 1, rank=rank, world=world, batch=want_batch) \
        if (want_batch or (not args.no_learned and world == 1)) else None
    big_pool = None
    if big:
        import multiprocessing as mp
        big_pool = mp.get_context("spawn").Pool(1)
        big_async = big_pool.map_async(_build_layered_16m, [0])

    import torch
    import torch.distributed as dist

    import paper_1502_07451_b300 as gp
    from paper_1502_07451_b300 import gen

    g1 = gen.config_layered_1m(0)
    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    W = max(3, args.warmup)
    K = args.steps
    gp.lib()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    g16 = None
    if big:
        g16 = big_async.get()[0]
        big_pool.close()
        big_pool.join()
    if bgen is not None:
        bgen.wait()
    quiet_heap()  # the batch graphs and the held-out graphs make a large heap

    g = g16 if big else g1
    sampler = ClockSampler(physical_index(local_rank)) if rank == 0 else None
    M = measure_plain(g, K, W, stream, flush, world, sampler)
    one_m = measure_plain(g1, K, W, stream, flush, world) if big else M

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    with_oracle = not args.no_cpu_baseline and world == 1
    # ---- CPU baseline (the oracle): the full 1M workload (bit-exact check included), or, for the 16M
    # workload, its first 100 layers; the 16M split is compared with the oracle's recorded result
    cpu = None
    bit_exact = None
    one_m_exact = None
    if with_oracle:
        dt, opart, ores, oms = oracle_step(g1)
        r1 = one_m["res"]
        one_m_exact = bool(np.array_equal(opart, one_m["part"]) and all(r1[k] == v for k, v in ores.items())
                           and oms == one_m["makespan"])
        cpu1 = {"value": g1["m"] / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": "the full 1M workload, one partition + makespan (%.1f s)" % dt}
        if big:
            sample = gen.layered(100, 16000, 12_800_000, 0)
            dts, _, _, _ = oracle_step(sample)
            cpu = {"value": sample["m"] / dts, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": "first 100 layers of the recipe (1.6M vertices, 12.8M edges), one partition + "
                             "makespan (%.1f s)" % dts}
        else:
            cpu = cpu1
            bit_exact = one_m_exact
    if big:
        bit_exact = golden_16m_match(M["part"], M["res"], M["makespan"])

    fixed = bench_fixed(g1, K, W, stream, flush, with_oracle=with_oracle)
    kway = bench_kway(g1, 3, K, W, stream, flush, with_oracle=with_oracle)
    learned = learned16 = None
    if not args.no_learned:
        learned = bench_learned(g1, one_m["part_dev"], one_m["res"], one_m["makespan"], K, W, stream, flush,
                                bgen.held_out() if bgen else [], with_oracle=with_oracle)
        if learned and "ms_per_step" in learned:
            learned["plain_ms_per_step"] = one_m["ms_per_step"]
            learned["speedup_vs_plain"] = one_m["ms_per_step"] / learned["ms_per_step"]
            learned["vcycle"]["speedup_vs_plain"] = one_m["ms_per_step"] / learned["vcycle"]["ms_per_step"]
        if big:
            learned16 = bench_learned(g16, M["part_dev"], M["res"], M["makespan"], K, W, stream, flush, [],
                                      with_oracle=False, workload=WORKLOAD_16M)
            if learned16 and "ms_per_step" in learned16:
                learned16["plain_ms_per_step"] = M["ms_per_step"]
                learned16["speedup_vs_plain"] = M["ms_per_step"] / learned16["ms_per_step"]
                learned16["vcycle"]["speedup_vs_plain"] = M["ms_per_step"] / learned16["vcycle"]["ms_per_step"]
    batch = None
    if bgen is not None and want_batch:
        batch = bench_batch(bgen.graphs(), K, W, stream, flush, with_cpu=not args.no_cpu_baseline)
    if bgen is not None:
        bgen.close()

    res, ms = M["res"], M["makespan"]
    dom = M["roofline"]["kernel"]
    traffic = profiled_traffic(dom, "16m" if big else "1m", M["roofline"]["alg_bytes_per_launch"])
    roof = dict(M["roofline"])
    roof["traffic"] = traffic[0] if traffic else None
    roof["traffic_source"] = traffic[1] if traffic else None
    roof["traffic_how"] = traffic[2] if traffic else None
    line = {
        "metric": METRIC, "value": M["value"], "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": M["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD_16M if big else WORKLOAD, "step": STEP,
                   "graphs_per_sec": world * K / (M["ms_per_step"] * K / 1e3),
                   "l2": "flushed between timed steps (256 MB)" + ("; inputs (5.4 GB) larger than L2" if big else ""),
                   "parallelism": "replicas" if world > 1 else "single", "cut": res["cut"],
                   "feasible": res["feasible"], "levels": res["levels"], "makespan_ns": ms,
                   "bit_exact_vs_oracle": bit_exact,
                   "bit_exact_how": ("split SHA-256, every result field and the makespan against the oracle's "
                                     "record (tests/golden/layered16m_oracle.json)" if big else
                                     "split, every result field and the makespan against the oracle run here"),
                   "e2e_matches_device": M["e2e_ok"],
                   "kernel_time_share": M["share"], "roofline_by_family": M["by_family"],
                   "roofline_pass": "second pass of the same K steps, CUDA events around every launch"},
        "e2e": M["e2e"],
        "gpu_launches": M["launches"],
        "roofline": roof,
        "clocks": M["clocks"],
    }
    if cpu:
        line["cpu_baseline"] = cpu
    if big:
        o = {"workload": WORKLOAD, "step": STEP, "metric": METRIC, "value": one_m["value"], "unit": UNIT,
             "ms_per_step": one_m["ms_per_step"], "cut": one_m["res"]["cut"], "feasible": one_m["res"]["feasible"],
             "levels": one_m["res"]["levels"], "makespan_ns": one_m["makespan"], "bit_exact_vs_oracle": one_m_exact,
             "e2e": one_m["e2e"], "e2e_matches_device": one_m["e2e_ok"], "gpu_launches": one_m["launches"],
             "roofline": one_m["roofline"], "roofline_by_family": one_m["by_family"],
             "kernel_time_share": one_m["share"]}
        t1 = profiled_traffic(one_m["roofline"]["kernel"], "1m", one_m["roofline"]["alg_bytes_per_launch"])
        o["roofline"] = dict(o["roofline"], traffic=t1[0] if t1 else None, traffic_source=t1[1] if t1 else None,
                             traffic_how=t1[2] if t1 else None)
        if with_oracle:
            o["cpu_baseline"] = cpu1
        line["layered1m"] = o
    if batch:
        line["batch"] = batch
    if learned:
        line["learned"] = learned
    if learned16:
        line["learned_16m"] = learned16
    if fixed:
        line["fixed"] = fixed
    if kway:
        line["kway"] = kway
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def bench_fixed(g, K, W, stream, flush, with_oracle):
    """The workload with the paper's host vertex (Sec. III.B: an empty kernel, holding the initial
    data in host memory, feeds every kernel without a predecessor) pinned to the CPU, through
    gp_partition_fixed; the same step as the plain line (deferred create + partition + makespan +
    destroy), K steps after W warm-ups, L2 flushed between steps.  Also: where the plain path puts
    that vertex, and (unless the CPU baseline is off) bit-exactness against the oracle."""
    import numpy as np
    import torch
    import paper_1502_07451_b300 as gp
    from paper_1502_07451_b300 import gen
    hs, src = gen.with_host_source(g, 0)
    n, m = hs["n"], hs["m"]
    keys = ("offsets", "cols", "edge_cost", "cpu_cost", "gpu_cost")
    dg = {k: torch.from_numpy(hs[k]).cuda() for k in keys}
    fx = np.full(n, -1, np.int8)
    fx[src] = 0
    dfx = torch.from_numpy(fx).cuda()
    part = torch.empty(n, dtype=torch.uint8, device="cuda")

    def step():
        h = gp.gp_graph_create_deferred(n, m, dg["offsets"], dg["cols"], dg["edge_cost"], dg["cpu_cost"],
                                        dg["gpu_cost"], stream=stream)
        r = gp.gp_partition_fixed(h, dfx, -1.0, 0.03, 0, part, stream)
        mk = gp.gp_makespan(h, part, None, stream)
        gp.gp_graph_destroy(h)
        return r, mk

    for _ in range(W):
        res, mk = step()
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(K):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        res, mk = step()
        b.record(stream)
        b.synchronize()
        total += a.elapsed_time(b)
    p = part.cpu().numpy()
    # the same graph without the pin
    h = gp.gp_graph_create(n, m, *[dg[k] for k in keys], stream=stream)
    free_part = torch.empty_like(part)
    rfree = gp.gp_partition(h, -1.0, 0.03, 0, free_part, stream)
    gp.gp_graph_destroy(h)
    out = {"workload": "the layered DAG above plus the host vertex feeding its %d kernels without a predecessor "
                       "(%d vertices, %d edges), pinned to the CPU" % (m - g["m"], n, m),
           "entry": "gp_partition_fixed", "metric": METRIC, "value": K * m / (total / 1e3), "unit": UNIT,
           "ms_per_step": total / K, "cut": res["cut"], "feasible": res["feasible"], "makespan_ns": mk,
           "host_vertex_on_cpu": bool(p[src] == 0),
           "without_pin": {"cut": rfree["cut"], "host_vertex_side": int(free_part[src].item())}}
    if with_oracle:  # part of the CPU-baseline leg
        import oracle
        opart, ores = oracle.partition(hs, fixed=fx)
        out["bit_exact_vs_oracle"] = bool(np.array_equal(opart, p) and ores["cut"] == res["cut"]
                                          and ores["load_cpu"] == res["load_cpu"])
    return out


def bench_kway(g, k, K, W, stream, flush, with_oracle):
    """k device classes by recursive bisection (gp_partition_kway) on the workload: CPU, GPU and an
    FPGA-like class (gen.kway_costs), device-resident inputs; K steps after W warm-ups, L2 flushed
    between steps; checked against the oracle in the CPU-baseline leg."""
    import torch
    import paper_1502_07451_b300 as gp
    from paper_1502_07451_b300 import gen
    cs = gen.kway_costs(g, k, 0)
    d = {key: torch.from_numpy(g[key]).cuda() for key in ("offsets", "cols", "edge_cost")}
    d.update(n=g["n"], m=g["m"])
    dcs = torch.from_numpy(cs).cuda()
    cls = torch.empty(g["n"], dtype=torch.uint8, device="cuda")
    for _ in range(W):
        r = gp.gp_partition_kway(d, dcs, cls, stream=stream)
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(K):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = gp.gp_partition_kway(d, dcs, cls, stream=stream)
        b.record(stream)
        b.synchronize()
        tot += a.elapsed_time(b)
    out = {"entry": "gp_partition_kway", "classes": k,
           "class_costs": "CPU, GPU, and an FPGA-like class: CPU time x U(0.1, 0.9) per task (gen.kway_costs)",
           "metric": METRIC, "value": K * g["m"] / (tot / 1e3), "unit": UNIT, "ms_per_step": tot / K,
           "cut": r["cut"], "loads": r["loads"], "feasible": r["feasible"], "bisections": r["bisections"],
           "vertices_per_class": [int(x) for x in np.bincount(cls.cpu().numpy(), minlength=k)]}
    if with_oracle:  # the CPU-baseline leg
        import oracle
        t0 = time.perf_counter()
        ocls, orr = oracle.partition_kway(g, cs)
        out["oracle_s"] = time.perf_counter() - t0
        out["bit_exact_vs_oracle"] = bool(np.array_equal(ocls, cls.cpu().numpy()) and orr == r)
    return out


def bench_learned(g, part_plain, res_plain, ms_plain, K, W, stream, flush, held_out, with_oracle=True,
                  workload=None):
    """The learned path (network proposal + refinement of level 0) on the same workload, with the
    trained checkpoint; plus the cut against the plain path on held-out 1M-vertex layered DAGs."""
    import torch
    import paper_1502_07451_b300 as gp
    if not os.path.exists(MODEL_PATH):
        return {"unavailable": "no trained checkpoint at paper_1502_07451_b300/models/mpnn3_h64.bin"}
    keys = ("offsets", "cols", "edge_cost", "cpu_cost", "gpu_cost")
    n, m = g["n"], g["m"]
    dg = {k: torch.from_numpy(g[k]).cuda() for k in keys}
    model = gp.gp_model_load(MODEL_PATH)
    part = torch.empty(n, dtype=torch.uint8, device="cuda")

    def step():
        h = gp.gp_graph_create(n, m, *[dg[k] for k in keys], stream=stream)
        r = gp.gp_partition_learned(h, model, part, stream=stream)
        mk = gp.gp_makespan(h, part, None, stream)
        gp.gp_graph_destroy(h)
        return r, mk

    for _ in range(W):
        r, mk = step()
    torch.cuda.synchronize()
    tot = 0.0
    launches0 = gp.gp_launch_count()
    for _ in range(K):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r, mk = step()
        b.record(stream)
        b.synchronize()
        tot += a.elapsed_time(b)
    launches = gp.gp_launch_count() - launches0
    # the V-cycle form: the proposal restricts the coarsening to same-side pairs, every level refined
    vpart = torch.empty(n, dtype=torch.uint8, device="cuda")

    def vstep():
        h = gp.gp_graph_create(n, m, *[dg[k] for k in keys], stream=stream)
        rv = gp.gp_partition_learned_vcycle(h, model, vpart, stream=stream)
        mkv = gp.gp_makespan(h, vpart, None, stream)
        gp.gp_graph_destroy(h)
        return rv, mkv

    for _ in range(W):
        rv, mkv = vstep()
    torch.cuda.synchronize()
    vtot = 0.0
    for _ in range(K):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rv, mkv = vstep()
        b.record(stream)
        b.synchronize()
        vtot += a.elapsed_time(b)
    # phase split of one call (events around the network, the proposal, refinement + cut)
    gp.gp_prof_reset()
    gp.gp_prof_enable(True)
    h = gp.gp_graph_create(n, m, *[dg[k] for k in keys], stream=stream)
    rp = gp.gp_partition_learned(h, model, part, stream=stream)
    logits = torch.empty(n, dtype=torch.float32, device="cuda")
    gp.gp_model_forward(model, h, logits, stream)
    gp.gp_graph_destroy(h)
    torch.cuda.synchronize()
    gp.gp_prof_enable(False)
    fams = gp.kernel_families()
    mp = gp.gp_prof_read(fams.index("mpnn"))
    gp.gp_prof_reset()
    # the integer result from these logits, recomputed by the oracle (with the CPU baseline leg only)
    exact = vexact = None
    if with_oracle:
        import oracle
        lh = logits.cpu().numpy()
        opart, ores = oracle.partition_learned(g, lh)
        exact = bool(np.array_equal(opart, part.cpu().numpy()) and ores["cut"] == r["cut"])
        vopart, vores = oracle.partition_vcycle(g, lh)
        vexact = bool(np.array_equal(vopart, vpart.cpu().numpy()) and all(rv[k] == x for k, x in vores.items()))
    held = []
    for seed, hg in zip(HELD_OUT_SEEDS, held_out):
        dh = {k: torch.from_numpy(hg[k]).cuda() for k in keys}
        hh = gp.gp_graph_create(hg["n"], hg["m"], *[dh[k] for k in keys], stream=stream)
        p2 = torch.empty(hg["n"], dtype=torch.uint8, device="cuda")
        rl = gp.gp_partition_learned(hh, model, p2, stream=stream)
        ml = gp.gp_makespan(hh, p2, None, stream)
        rw = gp.gp_partition_learned_vcycle(hh, model, p2, stream=stream)
        mw = gp.gp_makespan(hh, p2, None, stream)
        rq = gp.gp_partition(hh, -1.0, 0.03, 0, p2, stream)
        mq = gp.gp_makespan(hh, p2, None, stream)
        gp.gp_graph_destroy(hh)
        held.append({"seed": seed, "cut_learned": rl["cut"], "cut_vcycle": rw["cut"], "cut_plain": rq["cut"],
                     "feasible_learned": rl["feasible"], "feasible_vcycle": rw["feasible"],
                     "feasible_plain": rq["feasible"],
                     "makespan_learned": ml, "makespan_vcycle": mw, "makespan_plain": mq})
    gp.gp_model_destroy(model)
    summary = None
    if held:
        summary = {"graphs": len(held),
                   "learned_cut_le_plain": sum(h["cut_learned"] <= h["cut_plain"] for h in held),
                   "vcycle_cut_le_plain": sum(h["cut_vcycle"] <= h["cut_plain"] for h in held),
                   "feasible_learned": sum(h["feasible_learned"] for h in held),
                   "feasible_vcycle": sum(h["feasible_vcycle"] for h in held),
                   "feasible_plain": sum(h["feasible_plain"] for h in held),
                   "cut_sum_learned": sum(h["cut_learned"] for h in held),
                   "cut_sum_vcycle": sum(h["cut_vcycle"] for h in held),
                   "cut_sum_plain": sum(h["cut_plain"] for h in held)}
    return {
        "workload": workload or WORKLOAD, "checkpoint": "paper_1502_07451_b300/models/mpnn3_h64.bin",
        "step": "gp_graph_create(device CSR) + gp_partition_learned (network, proposal, level-0 refinement) + "
                "gp_makespan",
        "value": K * m / (tot / 1e3), "unit": UNIT, "graphs_per_sec": K / (tot / 1e3), "ms_per_step": tot / K,
        "plain_ms_per_step": None, "cut": r["cut"], "cut_plain": res_plain["cut"], "feasible": r["feasible"],
        "makespan_ns": mk, "makespan_plain_ns": ms_plain, "rounds": r["rounds"],
        "phase_ms": {"network": rp["ms"][0], "proposal": rp["ms"][1], "refine_and_cut": rp["ms"][2]},
        "mpnn_kernels_ms": mp["total_ms"], "gpu_launches_per_step": int(launches / max(K, 1)),
        "bit_exact_vs_oracle_given_logits": exact, "held_out": held, "held_out_summary": summary,
        "vcycle": {"entry": "gp_partition_learned_vcycle", "step": "gp_graph_create(device CSR) + "
                   "gp_partition_learned_vcycle (network, proposal, coarsening restricted to same-side pairs, "
                   "refinement at every level) + gp_makespan", "value": K * m / (vtot / 1e3), "unit": UNIT,
                   "ms_per_step": vtot / K, "cut": rv["cut"], "feasible": rv["feasible"], "levels": rv["levels"],
                   "makespan_ns": mkv, "bit_exact_vs_oracle_given_logits": vexact},
    }


RES_FIELDS = ("cut", "load_cpu", "load_gpu", "bound_cpu", "bound_gpu", "feasible", "levels", "rounds", "coarsest_n")


def golden_batch_rows():
    """The oracle's per-graph record of the 4,096-graph mix (a table written by a script that runs only
    the oracle), as dicts keyed by its column names; None if absent."""
    path = os.path.join(ROOT, "tests", "golden", "batch4096_oracle.txt")
    try:
        cols, rows = None, []
        with open(path) as f:
            for ln in f:
                if ln.startswith("# columns:"):
                    cols = ln[len("# columns:"):].split()
                elif not ln.startswith("#"):
                    rows.append(dict(zip(cols, ln.split())))
        return rows if cols and "makespan_w31" in cols else None
    except OSError:
        return None


def bench_batch(graphs, K, W, stream, flush, with_cpu=True, golden_ok=True):
    """gp_batch_partition over the batch (graphs resident in HBM) against the plain path in a loop.

    Returns the measurements as a dict (graphs/s, edges/s, the plain loop, e2e with host buffers,
    the batch kernel's achieved bandwidth, the oracle on a bounded sample)."""
    import torch
    import paper_1502_07451_b300 as gp
    keys = ("offsets", "cols", "edge_cost", "cpu_cost", "gpu_cost")
    count = len(graphs)
    m_tot = int(sum(g["m"] for g in graphs))
    n_tot = int(sum(g["n"] for g in graphs))
    dgs = [{k: torch.from_numpy(np.ascontiguousarray(g[k])).cuda() for k in keys} for g in graphs]
    dsrc = [dict(d, n=g["n"], m=g["m"]) for g, d in zip(graphs, dgs)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hs0 = [gp.gp_graph_create(g["n"], g["m"], *[d[k] for k in keys], stream=stream) for g, d in zip(graphs, dgs)]
    torch.cuda.synchronize()
    create_loop_s = time.perf_counter() - t0
    for h in hs0:
        gp.gp_graph_destroy(h)
    gp.gp_graph_create_batch(dsrc[:64], stream=stream)  # warm-up of the create kernel
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hs, sts = gp.gp_graph_create_batch(dsrc, stream=stream)
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t0
    assert all(st == gp.GP_OK for st in sts)
    parts = [torch.zeros(max(g["n"], 1), dtype=torch.uint8, device="cuda") for g in graphs]
    best, sched_ms = gp.gp_batch_autotune(hs, stream=stream)
    for _ in range(W):
        res, mks = gp.gp_batch_partition(hs, parts, makespans=True, stream=stream)
    torch.cuda.synchronize()
    launches0 = gp.gp_launch_count()
    tot_ms = 0.0
    kern_ms = 0.0
    for _ in range(K):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        res, mks = gp.gp_batch_partition(hs, parts, makespans=True, stream=stream)
        b.record(stream)
        b.synchronize()
        tot_ms += a.elapsed_time(b)
        kern_ms += res[0]["ms"][0]
    launches = gp.gp_launch_count() - launches0
    # the learned path for the whole batch (one network forward over the union, then the kernel)
    learned = None
    if os.path.exists(MODEL_PATH):
        model = gp.gp_model_load(MODEL_PATH)
        lparts = [torch.zeros(max(g["n"], 1), dtype=torch.uint8, device="cuda") for g in graphs]
        for _ in range(W):
            lres, _ = gp.gp_batch_partition_learned(hs, model, lparts, makespans=True, stream=stream)
        torch.cuda.synchronize()
        lt = 0.0
        for _ in range(K):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            lres, lms = gp.gp_batch_partition_learned(hs, model, lparts, makespans=True, stream=stream)
            b.record(stream)
            b.synchronize()
            lt += a.elapsed_time(b)
        gp.gp_model_destroy(model)
        learned = {"value": K * count / (lt / 1e3), "unit": BATCH_UNIT, "ms_per_step": lt / K,
                   "step": "gp_batch_partition_learned(4,096 resident handles, makespans on): one network "
                           "forward over the union + the persistent kernel in learned mode",
                   "cut_sum": int(sum(r["cut"] for r in lres)), "cut_sum_plain": int(sum(r["cut"] for r in res)),
                   "feasible": int(sum(r["feasible"] for r in lres)),
                   "makespan_sum": int(sum(lms)), "makespan_sum_plain": int(sum(mks))}
        del lparts
    # achieved bandwidth of the persistent kernel: algorithmic bytes of its steps / its time
    gp.gp_prof_reset()
    gp.gp_prof_enable(True)
    flush.fill_(1)
    gp.gp_batch_partition(hs, parts, makespans=True, stream=stream)
    torch.cuda.synchronize()
    gp.gp_prof_enable(False)
    fams = gp.kernel_families()
    prof = {f: gp.gp_prof_read(i) for i, f in enumerate(fams)}
    gp.gp_prof_reset()
    alg = sum(p["alg_bytes"] for p in prof.values())
    bms = prof["batch"]["total_ms"]
    hbm_peak, peak_kind = peaks()
    # the plain path, one graph after another (same handles, same outputs)
    p2 = [torch.zeros(max(g["n"], 1), dtype=torch.uint8, device="cuda") for g in graphs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = []
    for i, h in enumerate(hs):
        r = gp.gp_partition(h, -1.0, 0.03, 0, p2[i], stream)
        plain.append((r["cut"], gp.gp_makespan(h, p2[i][: graphs[i]["n"]], None, stream) if graphs[i]["n"] else 0))
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    same = all(torch.equal(a, b) for a, b in zip(parts, p2)) and all(
        plain[i] == (res[i]["cut"], mks[i]) for i in range(count))
    del p2
    # the makespan of every split on 3 CPU workers and 1 GPU worker (list schedule, Sec. IV.A's
    # testbed): one launch, a warp per graph
    msw = gp.gp_batch_makespan_workers(hs, parts, 3, 1, stream)
    torch.cuda.synchronize()
    ls_ms = 0.0
    for _ in range(K):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        msw = gp.gp_batch_makespan_workers(hs, parts, 3, 1, stream)
        b.record(stream)
        b.synchronize()
        ls_ms += a.elapsed_time(b)
    rows = golden_batch_rows() if count == BATCH_COUNT and golden_ok else None
    listsched = {"entry": "gp_batch_makespan_workers", "workers_cpu": 3, "workers_gpu": 1,
                 "value": K * count / (ls_ms / 1e3), "unit": BATCH_UNIT, "ms_per_step": ls_ms / K,
                 "tasks_per_sec": K * n_tot / (ls_ms / 1e3), "makespan_sum": int(sum(msw)),
                 "makespan_sum_unbounded": int(sum(mks)),
                 "bit_exact_vs_oracle": (all(int(rw["makespan_w31"]) == msw[i] for i, rw in enumerate(rows))
                                         if rows else None),
                 "bit_exact_how": "every graph's value against the oracle's record (tests/golden/batch4096_oracle.txt)"}
    # end to end: create from pinned host arrays, partition into pinned host buffers, destroy
    hgs = [{k: torch.from_numpy(np.ascontiguousarray(g[k])).pin_memory() for k in keys} for g in graphs]
    hparts = [torch.zeros(max(g["n"], 1), dtype=torch.uint8).pin_memory() for g in graphs]
    h2d = sum(int(t.numel() * t.element_size()) for d in hgs for t in d.values())
    d2h = n_tot + count * 56  # splits + the per-graph result records

    hsrc = [dict(d, n=g["n"], m=g["m"]) for g, d in zip(graphs, hgs)]

    def e2e_step():
        hh, _ = gp.gp_graph_create_batch(hsrc, stream=stream)
        gp.gp_batch_partition(hh, hparts, makespans=True, stream=stream)
        for h in hh:
            gp.gp_graph_destroy(h)

    e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ke = max(1, min(K, 3))
    for _ in range(ke):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / ke
    e2e_ok = all(torch.equal(a.cpu(), b) for a, b in zip(parts, hparts))
    cpu = None
    if with_cpu:
        k, dt = oracle_batch_sample(graphs, 12.0)
        cpu = {"value": k / dt, "unit": BATCH_UNIT, "cores": 1, "kind": "oracle",
               "sample": "the first %d graphs of the batch in order, oracle partition + makespan (%.1f s)" % (k, dt)}
        if count == BATCH_COUNT and golden_ok:
            v, nproc, done, slowest = oracle_batch_all_cores(count, 12.0)
            cpu_all = {"value": v, "unit": BATCH_UNIT, "cores": nproc, "kind": "oracle",
                       "sample": "the batch recipe on %d spawned workers (worker w: graphs w, w+%d, ... in order) "
                                 "until 12 s of oracle time each: %d graphs, slowest worker %.1f s; nproc = %d"
                                 % (nproc, nproc, done, slowest, os.cpu_count() or 0)}
    for h in hs:
        gp.gp_graph_destroy(h)
    out = {
        "metric": BATCH_METRIC, "unit": BATCH_UNIT, "workload": BATCH_WORKLOAD, "graphs": count,
        "vertices": n_tot, "edges": m_tot,
        "value": K * count / (tot_ms / 1e3), "edges_per_sec": K * m_tot / (tot_ms / 1e3),
        "ms_per_step": tot_ms / K, "kernel_ms_per_step": kern_ms / K, "steps": K, "warmup": W,
        "feasible": int(sum(r["feasible"] for r in res)), "cut_sum": int(sum(r["cut"] for r in res)),
        "step": "gp_batch_partition(4,096 resident handles, makespans on), one persistent launch",
        "schedule": gp.gp_batch_schedule_name(best),
        "autotune_ms": {gp.gp_batch_schedule_name(i): round(t, 2) for i, t in enumerate(sched_ms)},
        "plain_graphs_per_sec": count / plain_s, "plain_step": "gp_partition + gp_makespan per graph",
        "speedup_vs_plain": (K * count / (tot_ms / 1e3)) / (count / plain_s),
        "results_equal_plain": bool(same), "gpu_launches": int(launches),
        "create_s": create_s, "create_step": "gp_graph_create_batch over the 4,096 device-resident CSRs "
                                             "(one persistent launch)",
        "create_loop_s": create_loop_s,
        "with_create": {"graphs_per_sec": count / (create_s + tot_ms / K / 1e3),
                        "step": "gp_graph_create_batch + gp_batch_partition"},
        "e2e": {"value": count / e2e_s, "unit": BATCH_UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "step": "gp_graph_create_batch from pinned host CSRs + gp_batch_partition into pinned host "
                        "buffers + destroy", "matches_device": bool(e2e_ok)},
        "roofline": {"bound": "hbm", "kernel": "k_batch (persistent)", "achieved": alg / (bms * 1e-3) / 1e9,
                     "peak": hbm_peak, "unit": "GB/s", "frac": alg / (bms * 1e-3) / 1e9 / hbm_peak,
                     "peak_kind": peak_kind, "traffic": None, "alg_bytes_per_launch": alg, "launch_ms": bms},
    }
    if count == BATCH_COUNT:
        tb = profiled_traffic("batch", "batch4096", alg, gp.gp_batch_schedule_name(best))
        if tb:
            out["roofline"].update(traffic=tb[0], traffic_source=tb[1], traffic_how=tb[2])
    if cpu:
        out["cpu_baseline"] = cpu
        if count == BATCH_COUNT and golden_ok:
            out["cpu_baseline_all_cores"] = cpu_all
    if learned:
        learned["speedup_vs_plain_loop"] = learned["value"] / out["plain_graphs_per_sec"]
        out["learned"] = learned
    out["makespan_workers"] = listsched
    if rows:
        out["bit_exact_vs_oracle"] = all(
            all(int(rw[k]) == res[i][k] for k in RES_FIELDS) and int(rw["makespan"]) == mks[i]
            for i, rw in enumerate(rows))
        out["bit_exact_how"] = ("every graph's result fields and makespan against the oracle's record "
                                "(tests/golden/batch4096_oracle.txt)")
    return out


def run_batch_line(args, rank, world, local_rank, bgen):
    """--workload batch: the batch as the main line (graphs/s)."""
    import torch
    import paper_1502_07451_b300 as gp
    torch.cuda.set_device(local_rank)
    gp.lib()
    W = max(3, args.warmup)
    K = args.steps
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device="cuda")
    graphs = bgen.graphs()
    bgen.wait()
    bgen.close()
    quiet_heap()
    sampler = ClockSampler(physical_index(local_rank)) if rank == 0 else None
    if sampler:
        sampler.start()
    b = bench_batch(graphs, K, W, stream, flush, with_cpu=not args.no_cpu_baseline and world == 1,
                    golden_ok=world == 1)
    clocks = sampler.stop() if sampler else None
    # every rank partitions its own shard; the job's rate is all graphs over the slowest rank's time
    slow_ms = max_over_ranks(b["ms_per_step"], world)
    value = bgen.total / (slow_ms / 1e3)
    e2e = dict(b["e2e"])
    e2e["value"] = bgen.total / max_over_ranks(len(graphs) / b["e2e"]["value"], world)
    if rank != 0:
        return
    line = {"metric": BATCH_METRIC, "value": value, "unit": BATCH_UNIT, "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": slow_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "step": b["step"], "l2": "flushed between timed steps (256 MB)",
                       "edges_per_sec": b["edges_per_sec"], "plain_graphs_per_sec": b["plain_graphs_per_sec"],
                       "speedup_vs_plain": b["speedup_vs_plain"], "schedule": b["schedule"],
                       "autotune_ms": b["autotune_ms"], "results_equal_plain": b["results_equal_plain"],
                       "graphs_total": bgen.total, "graphs_rank0": len(graphs),
                       "parallelism": "lpt shards of %d graphs per GPU, no collective on the data path" % (bgen.total // world)
                       if world > 1 else "single"},
            "e2e": e2e, "gpu_launches": b["gpu_launches"], "roofline": b["roofline"], "clocks": clocks}
    if "cpu_baseline" in b:
        line["cpu_baseline"] = b["cpu_baseline"]
    print(json.dumps(line), flush=True)



PROFILE_BATCH_SCHEDULE = "cta512x2_sixteenth_rows"


def run_profile_case(name):
    """One invocation of the path, for a profiler: layered1m = one plain step (create, partition,
    makespan) on the 1M DAG; layered4m / layered16m = the same on 4M / 16M-vertex layered DAGs of width
    16,000; learned1m = one learned step with the trained checkpoint; batch64 = gp_batch_partition and
    gp_batch_makespan_workers over 64 graphs of the batch recipe (sizes up to 10,000); batch4096 =
    gp_graph_create_batch, gp_batch_partition with makespans (schedule PROFILE_BATCH_SCHEDULE, the one
    the bench's autotuning picks on this mix) and gp_batch_makespan_workers over the whole 4,096-graph
    mix."""
    bgen = BatchGen(held=False) if name == "batch4096" else None
    import torch
    import paper_1502_07451_b300 as gp
    from paper_1502_07451_b300 import gen
    keys = ("offsets", "cols", "edge_cost", "cpu_cost", "gpu_cost")
    if name in ("layered1m", "learned1m", "layered4m", "layered16m"):
        if name == "layered16m":
            g = gen.config_layered_16m(0)
        elif name == "layered4m":
            g = gen.layered(250, 16000, 32_000_000, 0)  # the 16M recipe's layer width, a quarter of its layers
        else:
            g = gen.config_layered_1m(0)
        dg = {k: torch.from_numpy(g[k]).cuda() for k in keys}
        part = torch.empty(g["n"], dtype=torch.uint8, device="cuda")
        create = gp.gp_graph_create if name == "learned1m" else gp.gp_graph_create_deferred
        h = create(g["n"], g["m"], *[dg[k] for k in keys])
        if name != "learned1m":
            res = gp.gp_partition(h, -1.0, 0.03, 0, part)
        else:
            model = gp.gp_model_load(MODEL_PATH)
            res = gp.gp_partition_learned(h, model, part)
            gp.gp_model_destroy(model)
        mk = gp.gp_makespan(h, part)
        gp.gp_graph_destroy(h)
        torch.cuda.synchronize()
        print(json.dumps({"case": name, "cut": res["cut"], "makespan": mk}))
    elif name == "batch4096":
        graphs = bgen.graphs()
        bgen.wait()
        src = [dict({k: torch.from_numpy(np.ascontiguousarray(gg[k])).cuda() for k in keys}, n=gg["n"], m=gg["m"])
               for gg in graphs]
        hs, _ = gp.gp_graph_create_batch(src)
        parts = [torch.zeros(max(gg["n"], 1), dtype=torch.uint8, device="cuda") for gg in graphs]
        names = [gp.gp_batch_schedule_name(i) for i in range(gp.gp_batch_schedule_count())]
        gp.gp_batch_set_schedule(names.index(PROFILE_BATCH_SCHEDULE))
        res, mks = gp.gp_batch_partition(hs, parts, makespans=True)
        msw = gp.gp_batch_makespan_workers(hs, parts, 3, 1)
        for h in hs:
            gp.gp_graph_destroy(h)
        torch.cuda.synchronize()
        print(json.dumps({"case": name, "cut_sum": sum(r["cut"] for r in res), "makespan_w31_sum": sum(msw)}))
    else:
        graphs = [gen.build_from_spec(it) for it in gen.batch_spec(64, nmin=100, nmax=10000, base_seed=0)]
        hs = [gp.gp_graph_create(gg["n"], gg["m"], *[torch.from_numpy(gg[k]).cuda() for k in keys]) for gg in graphs]
        parts = [torch.empty(gg["n"], dtype=torch.uint8, device="cuda") for gg in graphs]
        res, mks = gp.gp_batch_partition(hs, parts, makespans=True)
        msw = gp.gp_batch_makespan_workers(hs, parts, 3, 1)
        for h in hs:
            gp.gp_graph_destroy(h)
        torch.cuda.synchronize()
        print(json.dumps({"case": name, "cut_sum": sum(r["cut"] for r in res), "makespan_w31_sum": sum(msw)}))


def run_cholesky_line(args, rank, world, local_rank):
    """1,024 tiled Cholesky DAGs with T = 64: the learned path batched (the line's value), against the
    plain path batched and one graph after another."""
    import torch
    import paper_1502_07451_b300 as gp
    from paper_1502_07451_b300 import gen
    torch.cuda.set_device(local_rank)
    gp.lib()
    W = max(3, args.warmup)
    K = args.steps
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device="cuda")
    keys = ("offsets", "cols", "edge_cost", "cpu_cost", "gpu_cost")
    g = gen.cholesky(64)
    count = 1024
    n, m = g["n"], g["m"]
    dg = {k: torch.from_numpy(g[k]).cuda() for k in keys}
    t0 = time.perf_counter()
    hs = [gp.gp_graph_create(n, m, *[dg[k] for k in keys], stream=stream) for _ in range(count)]
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t0
    parts = [torch.zeros(n, dtype=torch.uint8, device="cuda") for _ in range(count)]
    seeds = list(range(count))
    model = gp.gp_model_load(MODEL_PATH)

    def timed(fn):
        for _ in range(W):
            r = fn()
        torch.cuda.synchronize()
        quiet_heap()
        tot = 0.0
        for _ in range(K):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r = fn()
            b.record(stream)
            b.synchronize()
            tot += a.elapsed_time(b)
        return tot / K, r

    sampler = ClockSampler(physical_index(local_rank)) if rank == 0 else None
    if sampler:
        sampler.start()
    launches0 = gp.gp_launch_count()
    l_ms, (lres, lmk) = timed(lambda: gp.gp_batch_partition_learned(hs, model, parts, makespans=True, stream=stream))
    launches = (gp.gp_launch_count() - launches0) // max(W + K, 1)
    clocks = sampler.stop() if sampler else None
    p_ms, (pres, pmk) = timed(lambda: gp.gp_batch_partition(hs, parts, seeds=seeds, makespans=True, stream=stream))
    # the plain path, one graph after another
    part1 = torch.zeros(n, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loop_same = True
    for i, h in enumerate(hs):
        r = gp.gp_partition(h, -1.0, 0.03, seeds[i], part1, stream)
        mk = gp.gp_makespan(h, part1, None, stream)
        loop_same = loop_same and r["cut"] == pres[i]["cut"] and mk == pmk[i]
    torch.cuda.synchronize()
    loop_s = time.perf_counter() - t0
    # batch kernel achieved bandwidth (learned mode)
    gp.gp_prof_reset()
    gp.gp_prof_enable(True)
    gp.gp_batch_partition_learned(hs, model, parts, makespans=True, stream=stream)
    torch.cuda.synchronize()
    gp.gp_prof_enable(False)
    fams = gp.kernel_families()
    prof = {f: gp.gp_prof_read(i) for i, f in enumerate(fams)}
    gp.gp_prof_reset()
    hbm_peak, peak_kind = peaks()
    alg = sum(p["alg_bytes"] for p in prof.values())
    tot_ms = sum(p["total_ms"] for p in prof.values())
    dom = max((f for f in fams if prof[f]["launches"]), key=lambda f: prof[f]["total_ms"])
    # end to end: create from pinned host CSR, learned batch into pinned host buffers, destroy
    hg = {k: torch.from_numpy(g[k]).pin_memory() for k in keys}
    hparts = [torch.zeros(n, dtype=torch.uint8).pin_memory() for _ in range(count)]
    h2d = count * sum(int(t.numel() * t.element_size()) for t in hg.values())
    t0 = time.perf_counter()
    hh = [gp.gp_graph_create(n, m, *[hg[k] for k in keys], stream=stream) for _ in range(count)]
    gp.gp_batch_partition_learned(hh, model, hparts, makespans=True, stream=stream)
    for h in hh:
        gp.gp_graph_destroy(h)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_ok = all(torch.equal(a.cpu(), b) for a, b in zip(parts, hparts))
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:  # the CPU-baseline leg
        import oracle
        t0 = time.perf_counter()
        opart, ores = oracle.partition(g, seed=0)
        oracle.makespan(g, opart)
        dt = time.perf_counter() - t0
        cpu = {"value": 1.0 / dt, "unit": BATCH_UNIT, "cores": 1, "kind": "oracle",
               "sample": "one Cholesky T=64 DAG, oracle partition + makespan (%.2f s)" % dt}
    for h in hs:
        gp.gp_graph_destroy(h)
    gp.gp_model_destroy(model)
    if rank != 0:
        return
    line = {"metric": BATCH_METRIC, "value": count / (l_ms / 1e3), "unit": BATCH_UNIT, "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": l_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64", "data": "synthetic",
            "config": {"workload": CHOL_WORKLOAD, "l2": "flushed between timed steps (256 MB)",
                       "step": "gp_batch_partition_learned over 1,024 resident handles, makespans on",
                       "edges_per_sec": count * m / (l_ms / 1e3),
                       "plain_batched_graphs_per_sec": count / (p_ms / 1e3),
                       "plain_loop_graphs_per_sec": count / loop_s, "plain_loop_equals_batched": bool(loop_same),
                       "cut_learned": int(lres[0]["cut"]), "cut_plain_seed0": int(pres[0]["cut"]),
                       "cut_plain_mean": float(np.mean([r["cut"] for r in pres])),
                       "makespan_learned": int(lmk[0]), "makespan_plain_mean": float(np.mean(pmk)),
                       "feasible_learned": int(sum(r["feasible"] for r in lres)),
                       "feasible_plain": int(sum(r["feasible"] for r in pres)),
                       "create_s": create_s, "kernel_time_share": {f: round(prof[f]["total_ms"] / tot_ms, 4)
                                                                   for f in fams if prof[f]["launches"]}},
            "e2e": {"value": count / e2e_s, "unit": BATCH_UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": count * (n + 56), "matches_device": bool(e2e_ok)},
            "gpu_launches": int(launches),
            "roofline": {"bound": "hbm", "kernel": dom + " (all steps of the learned batch)",
                         "achieved": alg / (tot_ms * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                         "frac": alg / (tot_ms * 1e-3) / 1e9 / hbm_peak, "peak_kind": peak_kind, "traffic": None},
            "clocks": clocks}
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
