"""Benchmark: DAG edges partitioned per second on B300.

One step = the whole path on one DAG resident in HBM: gp_graph_create from
device CSR (validation, transpose, symmetrisation, topological levels),
gp_partition (coarsening, initial split, refinement, cut) and gp_makespan.
Workload: layered random DAG, 1,000 layers x 1,000 vertices, 8M edges,
lognormal CPU times, GPU = CPU / U(2, 40), transfer U{1..10,000} ns, seed 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

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


def run_reference(args, rank, world):
    """The oracle on the host cores, timed on a bounded sample of the workload (first 100 layers)."""
    from paper_1502_07451_b300 import gen
    if rank != 0:
        return
    sample = gen.layered(100, 1000, 800_000, 0)
    for _ in range(args.warmup):
        oracle_step(sample)
    tot = 0.0
    for _ in range(args.steps):
        dt, _, _, _ = oracle_step(sample)
        tot += dt
    value = args.steps * sample["m"] / tot
    desc = "first 100 layers of the workload recipe (100,000 vertices, 800,000 edges), oracle partition + makespan"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": desc}, "impl": "reference",
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
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist

    import paper_1502_07451_b300 as gp
    from paper_1502_07451_b300 import gen

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    W = max(3, args.warmup)
    K = args.steps
    gp.lib()
    g = gen.config_layered_1m(0)
    n, m = g["n"], g["m"]
    keys = ("offsets", "cols", "edge_cost", "cpu_cost", "gpu_cost")
    dg = {k: torch.from_numpy(g[k]).cuda() for k in keys}
    part = torch.empty(n, dtype=torch.uint8, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        h = gp.gp_graph_create(n, m, dg["offsets"], dg["cols"], dg["edge_cost"], dg["cpu_cost"], dg["gpu_cost"],
                               stream=stream)
        res = gp.gp_partition(h, -1.0, 0.03, 0, part, stream)
        ms = gp.gp_makespan(h, part, None, stream)
        gp.gp_graph_destroy(h)
        return res, ms

    for _ in range(W):
        res, ms = step()
    torch.cuda.synchronize()

    # ---- timed device pass
    sampler = ClockSampler(physical_index(local_rank)) if rank == 0 else None
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
    if world > 1:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    value = world * K * m / (total_ms / 1e3)

    # ---- end to end through the C-ABI with pinned host buffers (H2D and D2H inside the timed region)
    hg = {k: torch.from_numpy(g[k]).pin_memory() for k in keys}
    hpart = torch.empty(n, dtype=torch.uint8).pin_memory()
    h2d = sum(int(hg[k].numel() * hg[k].element_size()) for k in keys)
    d2h = n + 8 + 8 * 28

    def e2e_step():
        h = gp.gp_graph_create(n, m, hg["offsets"], hg["cols"], hg["edge_cost"], hg["cpu_cost"], hg["gpu_cost"],
                               stream=stream)
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
    if world > 1:
        t = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = world * K * m / e2e_s
    e2e_ok = bool(np.array_equal(hpart.numpy(), part.cpu().numpy()))

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
    dom = max(mem_fams, key=lambda f: prof[f]["total_ms"])
    dp = prof[dom]
    per_launch_bytes = dp["alg_bytes"] / max(dp["launches"], 1)
    per_launch_ms = dp["total_ms"] / max(dp["launches"], 1)
    achieved = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9
    share = {f: round(prof[f]["total_ms"] / max(sum(p["total_ms"] for p in prof.values()), 1e-9), 4)
             for f in fams if prof[f]["launches"]}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- CPU baseline: the oracle on the same full workload, one core, once
    cpu = None
    bit_exact = None
    if not args.no_cpu_baseline and world == 1:
        dt, opart, ores, oms = oracle_step(g)
        cpu = {"value": m / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "the full workload, one partition + makespan (%.1f s)" % dt}
        bit_exact = bool(np.array_equal(opart, part.cpu().numpy()) and ores["cut"] == res["cut"] and oms == ms)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "step": "gp_graph_create(device CSR) + gp_partition + gp_makespan",
                   "graphs_per_sec": world * K / (total_ms / 1e3), "l2": "flushed between timed steps (256 MB)",
                   "parallelism": "replicas" if world > 1 else "single", "cut": res["cut"],
                   "feasible": res["feasible"], "levels": res["levels"], "makespan_ns": ms,
                   "bit_exact_vs_oracle": bit_exact, "e2e_matches_device": e2e_ok,
                   "kernel_time_share": share, "roofline_pass": "second pass of the same K steps, "
                   "CUDA events around every launch"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "peak_kind": peak_kind, "traffic": None,
                     "alg_bytes_per_launch": per_launch_bytes, "launch_ms": per_launch_ms,
                     "launches": dp["launches"]},
        "clocks": clocks,
    }
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
