"""Train the learned proposal's network on generated DAGs labelled by the plain method.

  python -m paper_1502_07451_b300.train --graphs 20000 --out paper_1502_07451_b300/models/mpnn3_h64.bin

Graph i of the training set follows the batch recipe (gen.batch_spec) with base seed 10^6 and
sizes log-uniform in [--nmin, --nmax]: tiled Cholesky and tiled LU (tile counts up to --tmax) and
layered DAGs in turn.  Each
graph is built on the host (spawned worker processes), copied to the GPU, partitioned by the plain
multilevel path (gp_partition), and used for one Adam step of the network (gp_model_train_step),
then released; the network is trained by the library's own forward and backward kernels.  The
learning rate is --lr for the first 80% of the steps and a quarter of it afterwards.
"""
import argparse
import json
import os
import sys
import time

import numpy as np


def _build_one(item):
    from paper_1502_07451_b300 import gen
    g = gen.build_from_spec(item)
    return {k: g[k] for k in ("n", "m", "offsets", "cols", "edge_cost", "cpu_cost", "gpu_cost")}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--graphs", type=int, default=20000)
    ap.add_argument("--nmin", type=int, default=1000)
    ap.add_argument("--nmax", type=int, default=100000)
    ap.add_argument("--epochs", type=int, default=1)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=0, help="network initialisation seed")
    ap.add_argument("--base-seed", type=int, default=1_000_000)
    ap.add_argument("--tmax", type=int, default=80, help="largest tile count of the Cholesky / LU graphs")
    ap.add_argument("--out", required=True)
    ap.add_argument("--log", default=None, help="write the loss curve (JSON) here")
    ap.add_argument("--workers", type=int, default=0)
    args = ap.parse_args(argv)

    import multiprocessing as mp
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    from paper_1502_07451_b300 import gen
    spec = gen.batch_spec(args.graphs, nmin=args.nmin, nmax=args.nmax, base_seed=args.base_seed, tmax=args.tmax)
    nproc = args.workers or max(1, min(32, (os.cpu_count() or 4) - 1))
    pool = mp.get_context("spawn").Pool(nproc)  # before any CUDA call

    import torch
    import paper_1502_07451_b300 as gp
    keys = ("offsets", "cols", "edge_cost", "cpu_cost", "gpu_cost")
    model = gp.gp_model_create(args.seed)
    total = args.graphs * args.epochs
    losses = []
    t0 = time.time()
    step = 0
    try:
        for ep in range(args.epochs):
            for g in pool.imap(_build_one, spec, chunksize=4):
                dg = {k: torch.from_numpy(np.ascontiguousarray(g[k])).cuda() for k in keys}
                h = gp.gp_graph_create(g["n"], g["m"], *[dg[k] for k in keys])
                try:
                    lab = torch.empty(g["n"], dtype=torch.uint8, device="cuda")
                    gp.gp_partition(h, -1.0, 0.03, 0, lab)
                    lr = args.lr if step < 0.8 * total else args.lr * 0.25
                    losses.append(gp.gp_model_train_step(model, h, lab, lr))
                finally:
                    gp.gp_graph_destroy(h)
                step += 1
                if step % 1000 == 0:
                    print("step %d/%d  loss (last 1000) %.4f  %.0f s" % (step, total, float(np.mean(losses[-1000:])),
                                                                        time.time() - t0), flush=True)
        os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
        gp.gp_model_save(model, args.out)
    finally:
        gp.gp_model_destroy(model)
        pool.close()
        pool.join()
    summary = {"graphs": args.graphs, "epochs": args.epochs, "steps": step, "lr": args.lr, "tmax": args.tmax,
               "nmin": args.nmin, "nmax": args.nmax, "base_seed": args.base_seed, "init_seed": args.seed,
               "first_1000_loss": float(np.mean(losses[:1000])), "last_1000_loss": float(np.mean(losses[-1000:])),
               "seconds": time.time() - t0}
    print(json.dumps(summary), flush=True)
    if args.log:
        with open(args.log, "w") as f:
            json.dump({"summary": summary, "loss": [round(x, 5) for x in losses]}, f)


if __name__ == "__main__":
    main()
