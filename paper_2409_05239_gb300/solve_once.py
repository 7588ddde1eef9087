"""Run Hybrid LSLU on a synthetic tomography workload and print one JSON line.

    python -m paper_2409_05239_gb300.solve_once --workload ct512 --K 300
    python -m paper_2409_05239_gb300.solve_once --batch 64 --K 150
    python -m paper_2409_05239_gb300.solve_once --workload ct512 --K 2 --shapes all
    python -m paper_2409_05239_gb300.solve_once --workload ct512 --K 300 --order tiles
    python -m paper_2409_05239_gb300.solve_once --workload ct512 --K 300 --histories

The first form builds one seeded problem of the named size (see tomo.CONFIGS)
and solves it `--repeat` times; the second solves a batch of uneven problems
(tomo.make_uneven_batch) through the batched entry points.  Meant for kernel
profilers: with LSLU_NO_GRAPHS=1 in the environment every kernel is launched
directly instead of from a captured CUDA graph.  `--shapes` repeats the
single-problem solve once per named sparse-product shape (both directions set
to it; "all" = every shape in lslu.Solver.SHAPES order), so that a profiler sees
the products of every shape in one process: each solve launches 2 K products,
A^T d_k then A l_k for k = 0..K-1.  `--order tiles` builds the handle with
tomo.locality_order's renumbering (lslu_create_ordered); `--tune` runs the
sparse-product autotuner first, as the benchmark does; `--loop persistent` or
`--loop cluster` runs the basis loop as one launch (lslu_set_loop);
`--histories` asks for the lambda and residual histories (a projected problem
for every k).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="ct512")
    ap.add_argument("--value-type", default="f32", choices=["f64", "f32", "bf16"])
    ap.add_argument("--K", type=int, default=None)
    ap.add_argument("--rule", default="gcv", choices=["none", "fixed", "gcv", "wgcv"])
    ap.add_argument("--lam", type=float, default=0.0)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--batch", type=int, default=0, help="solve this many uneven problems")
    ap.add_argument("--shapes", default="", help="comma-separated shape names, or 'all'")
    ap.add_argument("--order", default="natural", choices=["natural", "tiles"])
    ap.add_argument("--tune", action="store_true",
                    help="run the sparse-product autotuner before the solves (as bench.py does)")
    ap.add_argument("--loop", default="graph", choices=["graph", "persistent", "cluster"],
                    help="basis-loop execution (lslu_set_loop)")
    ap.add_argument("--histories", action="store_true",
                    help="also solve the projected problem of every k (lambda and residual histories)")
    a = ap.parse_args(argv)

    import torch

    from paper_2409_05239_gb300 import lslu, tomo

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    out = {}
    if a.batch:
        K = a.K or 150
        Ps = tomo.make_uneven_batch(a.batch)
        b = np.concatenate([P.b for P in Ps])
        with lslu.from_problems(Ps, a.value_type, K, stream=stream) as s:
            if a.loop != "graph":
                s.set_loop(a.loop)
            t0 = time.perf_counter()
            for _ in range(a.repeat):
                r = s.solve(b, K, a.rule, a.lam)
            dt = (time.perf_counter() - t0) / a.repeat
        errs = [np.linalg.norm(x - P.x_true) / np.linalg.norm(P.x_true)
                for x, P in zip(r["x"], Ps)]
        out = {"problems": a.batch, "K": K, "k_done_min": int(r["k_done"].min()),
               "seconds_per_solve": dt, "rel_err_x_true_median": float(np.median(errs))}
    else:
        P = tomo.make_config(a.workload)
        K = a.K or tomo.CONFIGS[a.workload]["K"]
        names = list(lslu.Solver.SHAPES) if a.shapes == "all" else \
            [t for t in a.shapes.split(",") if t]
        order = tomo.locality_order(P) if a.order == "tiles" else None
        with lslu.from_problem(P, a.value_type, K, order=order) as s:
            if a.tune:
                s.tune_spmv(reps=3)
            if a.loop != "graph":
                s.set_loop(a.loop)
            runs = []
            for name in names or [None]:
                if name is not None:
                    code = lslu.Solver.SHAPES.index(name)
                    s.set_spmv_shape(code, code)
                t0 = time.perf_counter()
                for _ in range(a.repeat):
                    r = s.solve(P.b, K, a.rule, a.lam, histories=a.histories)
                runs.append({"shape": name, "status": r["status"],
                             "seconds_per_solve": (time.perf_counter() - t0) / a.repeat})
            launches = s.last_launch_count()
            cfg = s.spmv_config()
        out = {"workload": a.workload, "order": a.order, "m": P.m, "n": P.n, "nnz": P.nnz, "K": K,
               "k_done": r["k_done"], "status": r["status"], "launches": launches,
               "spmv_config": cfg,
               "seconds_per_solve": runs[-1]["seconds_per_solve"],
               "rel_err_x_true": float(np.linalg.norm(r["x"] - P.x_true) /
                                       np.linalg.norm(P.x_true))}
        if names:
            out["shapes"] = runs
    print(json.dumps(out))


if __name__ == "__main__":
    main()
