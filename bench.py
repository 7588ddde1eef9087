"""Benchmark: Hybrid LSLU iterations/s on the 512x512 parallel-beam CT workload.

One step = one complete Hybrid LSLU solve (K = 300 iterations of the basis
loop of Algorithm 5, GCV lambda on the projected problem, x_K = L_K y) on a
seeded synthetic problem that stands in for a tomography test problem:
512x512 image (n = 262144), 360 angles x 724 rays (m = 260640), Siddon
ray-pixel lengths (~120M non-zeros), 20-ellipse phantom, 0.5% noise.
A's values are stored in FP32 (default) with FP32 accumulation and FP32 basis
vectors; H, W, the projected solve, lambda and x are FP64.  The handle stores
A renumbered for gather locality (`--order tiles`, the default:
tomo.locality_order through lslu_create_ordered); b, x and the pivots stay in
the natural numbering, and pivot ties are broken by the natural index.

Contract: `python bench.py --gpus N --steps K --warmup W` prints ONE JSON line.
Under torchrun (N > 1) every rank runs an independent replica (the solve of
one problem does not shard); value = all ranks' iterations / max time.
`--impl reference` times the FP64 CPU oracle instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2409_05239_gb300 import tomo  # noqa: E402

METRIC = "Hybrid LSLU iterations/s, 512x512 parallel-beam CT (K=300, GCV)"
WORKLOAD = "ct512"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    p.add_argument("--workload", default=WORKLOAD, choices=sorted(tomo.CONFIGS))
    p.add_argument("--value-type", default="f32", choices=["f32", "bf16", "f64"])
    p.add_argument("--K", type=int, default=None)
    p.add_argument("--order", default="tiles", choices=["tiles", "natural"],
                   help="numbering the handle stores A in (tomo.locality_order)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true", help="skip the precision study")
    p.add_argument("--cpu-sample-s", type=float, default=15.0)
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_seed(seed_base, rank):
    """Each rank solves its own seeded instance of the workload."""
    return seed_base + rank


def replica_rate(local_time, units_per_rank, world, device=None):
    """Whole-job throughput of independent replicas: the units of all ranks
    divided by the slowest rank's time (max over ranks; torch.distributed must
    be initialised when world > 1).  Returns (rate, max_time)."""
    import torch

    t = torch.tensor([float(local_time)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist

        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tmax = float(t.item())
    return units_per_rank * world / tmax, tmax


ORDER_NOTE = {
    "natural": "A as generated (pixels row by row, rays angle by angle)",
    "tiles": "A stored renumbered by lslu_create_ordered (tomo.locality_order: pixels in 2x4 "
             "tiles, rays in tiles of 4 angles x 2 rays); b, x and pivots in the natural "
             "numbering",
}

# DRAM traffic of one k_spmv_pivots launch on the 512x512 FP32 workload per
# numbering and row shape, (A l_k, A^T d_k) in bytes (dram__bytes_read.sum +
# dram__bytes_write.sum, one ncu pass per launch, averaged over the two
# launches of each direction of solve_once --K 2 --shapes all [--order
# tiles]).  It is reported only while the sources that define the sparse
# products and their launches are the ones captured.
SPMV_TRAFFIC = {
    "workload": "ct512", "value_type": "f32",
    "bytes": {
        "natural": {
            "16x2": (972.48e6, 974.17e6), "32x1": (971.89e6, 972.75e6),
            "16x1": (978.13e6, 973.03e6), "8x1": (1004.44e6, 1020.27e6),
            "8x2": (997.67e6, 988.00e6), "4x1": (1011.29e6, 1022.83e6),
            "16x2/16-bit": (800.03e6, 795.78e6), "32x1/16-bit": (791.36e6, 790.76e6),
            "16x1/16-bit": (804.18e6, 809.83e6), "8x1/16-bit": (853.34e6, 904.81e6),
            "8x2/16-bit": (831.13e6, 831.64e6), "4x1/16-bit": (918.39e6, 897.77e6),
            "32x8e": (972.00e6, 972.91e6), "32x8e/16-bit": (791.05e6, 791.10e6),
            "32x4e": (971.93e6, 972.72e6), "32x4e/16-bit": (793.30e6, 791.76e6),
        },
        "tiles": {
            "16x2": (972.37e6, 974.02e6), "32x1": (971.85e6, 972.76e6),
            "16x1": (978.19e6, 972.89e6), "8x1": (1005.26e6, 1020.68e6),
            "8x2": (998.17e6, 993.89e6), "4x1": (1012.00e6, 1022.04e6),
            "16x2/16-bit": (799.68e6, 795.89e6), "32x1/16-bit": (791.28e6, 790.66e6),
            "16x1/16-bit": (804.39e6, 809.88e6), "8x1/16-bit": (854.99e6, 926.65e6),
            "8x2/16-bit": (832.14e6, 837.37e6), "4x1/16-bit": (931.91e6, 894.62e6),
            "32x8e": (972.04e6, 972.82e6), "32x8e/16-bit": (791.14e6, 790.89e6),
            "32x4e": (972.04e6, 972.71e6), "32x4e/16-bit": (793.30e6, 791.71e6),
        },
    },
    "sources": {
        "paper_2409_05239_gb300/csrc/lslu_spmv.cu":
            "6cc9ecd7150c65c3be752d624f2e0cca975c796399ff9f580e1f7746fc9d32e0",
        "paper_2409_05239_gb300/csrc/lslu_spmv_impl.cuh":
            "e618d799b704a719641bc6e6dbf0e35760f17eb2954ef42a4f8cba87f46cebba",
        "paper_2409_05239_gb300/csrc/lslu_spmv_shapes_a.cu":
            "d1fa497a3a9ce3097928ce60e983850dfdd6c9e000f6e80efd0f6e93dd7e0af9",
        "paper_2409_05239_gb300/csrc/lslu_spmv_shapes_b.cu":
            "0e773294834ee47b18af1f88926ceff2d1210b793e4dcb2cf9260028db12f63a",
        "paper_2409_05239_gb300/csrc/lslu_spmv_shapes_c.cu":
            "96910620ae56de115fcdea59e6c10dfb7408ff7c9610c8323ba713ab471e2a0f",
    },
}


def spmv_traffic(workload, value_type, order, shape_A, shape_AT):
    """Measured DRAM bytes of one sparse product (average of the two directions)
    for the numbering and the tuned shapes, or None when no capture matches the
    current build."""
    import hashlib

    if workload != SPMV_TRAFFIC["workload"] or value_type != SPMV_TRAFFIC["value_type"]:
        return None
    tab = SPMV_TRAFFIC["bytes"].get(order, {})
    if shape_A not in tab or shape_AT not in tab:
        return None
    for rel, digest in SPMV_TRAFFIC["sources"].items():
        with open(os.path.join(ROOT, rel), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != digest:
                return None
    return 0.5 * (tab[shape_A][0] + tab[shape_AT][1])


def spmv_bytes(P, value_type, cmp_A=False, cmp_AT=False):
    """Algorithmic bytes of one sparse product (either direction, averaged):
    values + column storage (4 bytes per entry, or 2-byte offsets plus one
    4-byte base per 8 entries) + row pointers + output + input vector."""
    sv = {"f64": 8, "f32": 4, "bf16": 2}[value_type]
    sb = 8 if value_type == "f64" else 4
    a = P.nnz * (sv + (2.5 if cmp_A else 4.0)) + (P.m + 1) * 4 + P.m * sb + P.n * sb
    at = P.nnz * (sv + (2.5 if cmp_AT else 4.0)) + (P.n + 1) * 4 + P.n * sb + P.m * sb
    return 0.5 * (a + at)


def solve_bytes(P, value_type, K, cmp_A=False, cmp_AT=False):
    """Algorithmic HBM bytes of one K-iteration solve (basis loop + recombine)."""
    sb = 8 if value_type == "f64" else 4
    per_iter_spmv = 2 * spmv_bytes(P, value_type, cmp_A, cmp_AT)
    # elimination reads k (resp. k+1) basis columns, plus the new vector read,
    # scaled basis column written, and the scale pass (read v, write b)
    elim = 0
    for k in range(K):
        elim += (P.n * k + P.m * (k + 1)) * sb + 4 * (P.n + P.m) * sb
    recombine = P.n * K * sb + P.n * 8
    return K * per_iter_spmv + elim + recombine


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(P, K, sample_s, oracle_runs=None):
    """The FP64 oracle as it stands: the full K-iteration GCV solve of the
    benchmark instance timed in its own process (one thread) when the
    precision study's oracle runs are available, else the first k_s
    iterations of the same solve, k_s chosen to take ~sample_s."""
    nproc = os.cpu_count()
    if oracle_runs is not None:
        try:
            runs = oracle_runs.get()
            # every run at once, one process (one thread) each: the oracle's
            # aggregate rate on that many host cores
            span = max(r["wall_end"] for r in runs) - min(r["wall_start"] for r in runs)
            together = {"value": sum(r["k_done"] for r in runs) / span, "unit": "iter/s",
                        "cores": len(runs),
                        "sample": f"{len(runs)} full {K}-iteration oracle solves (the precision "
                                  f"study's: FP64/FP32/BF16-rounded A x 2 noise levels of the "
                                  f"same matrix) in {len(runs)} concurrent one-thread "
                                  f"processes, {span:.1f} s wall"}
            for r in runs:
                if r["value_type"] == "f64" and r["eta"] == P.eta:
                    return {"value": r["k_done"] / r["seconds"], "unit": "iter/s", "cores": 1,
                            "kind": "oracle", "host_cores": nproc,
                            "sample": f"the full {r['k_done']}-iteration solve of the same "
                                      f"instance (FP64 numpy/scipy, 1 thread), "
                                      f"{r['seconds']:.1f} s, while the precision study's "
                                      f"other oracle solves ran on other cores",
                            "multi_core": together}
        except Exception as e:  # noqa: BLE001 - fall back to the bounded sample
            print(f"oracle runs failed: {e}", file=sys.stderr)
    import oracle.lslu_oracle as O

    A = P.scipy()
    t0 = time.perf_counter()
    O.hybrid_lslu(A, P.b, None, 2, "gcv", histories=False)
    t_probe = time.perf_counter() - t0
    ks = int(max(2, min(K, 2 * sample_s / max(t_probe, 1e-3))))
    t0 = time.perf_counter()
    O.hybrid_lslu(A, P.b, None, ks, "gcv", histories=False)
    dt = time.perf_counter() - t0
    return {"value": ks / dt, "unit": "iter/s", "cores": 1, "kind": "oracle", "host_cores": nproc,
            "sample": f"first {ks} of {K} iterations of the same solve (FP64 numpy/scipy, "
                      f"1 thread), {dt:.1f} s"}


ORACLE_ETAS = (0.005, 0.02)
VALUE_TYPES_STUDY = ("f64", "f32", "bf16")


def _oracle_job(job):
    """Worker process: the FP64 oracle's K-iteration GCV solve of a workload
    instance with A's values rounded to a value type (one thread)."""
    workload, vt, eta, K = job
    import oracle.lslu_oracle as O

    P = tomo.make_config(workload, eta=eta)
    A = P.scipy(tomo.round_values(P.vals, vt))
    w0 = time.time()
    t0 = time.perf_counter()
    r = O.hybrid_lslu(A, P.b, None, K, "gcv", histories=False)
    dt = time.perf_counter() - t0
    return {"value_type": vt, "eta": eta, "K": K, "x": r.x, "gp": r.gp, "tp": r.tp,
            "k_done": r.k_done, "seconds": dt, "wall_start": w0, "wall_end": time.time()}


def start_oracle_runs(workload, K):
    """The oracle at the full workload, one spawned process per (value type,
    noise level) of the precision study, started with "spawn" (the parent
    already holds a CUDA context) and collected at the end (multiprocessing
    AsyncResult)."""
    import multiprocessing as mp

    jobs = [(workload, vt, eta, K) for eta in ORACLE_ETAS for vt in VALUE_TYPES_STUDY]
    pool = mp.get_context("spawn").Pool(processes=len(jobs))
    return pool, pool.map_async(_oracle_job, jobs), len(jobs)


def precision_study(P, K, dev, order=(None, None), n_phantoms=3, k_step=10, stop_tol=1e-6):
    """Mixed precision against the FP64 GPU path: A's values in FP64 / FP32 /
    BF16 (FP64 or FP32 basis), GCV lambda, on n_phantoms seeded phantoms at
    each noise level of ORACLE_ETAS (instance 0 at the first level is P).
    For every value type: iterations/s of the K-iteration solve; for every
    instance the relative error against x_true at the iterate the stopping
    rule of Eqs. (stop2)/(tol) picks (GCV lambda, tol = stop_tol), at the
    best iterate of a k_step grid and at K.  For the mixed paths: the mean and
    worst difference to the FP64 path's error at each of the three points, and
    on how many instances the error is within 1% of the FP64 path's.  Returns
    the study and what oracle_comparison needs to add x_K of instance 0 at
    each noise level against the FP64 oracle run on the same rounded values."""
    import torch

    from paper_2409_05239_gb300 import lslu

    c = tomo.CONFIGS[WORKLOAD]
    insts = []
    for eta in ORACLE_ETAS:
        for i in range(n_phantoms):
            Q = P if (i == 0 and eta == P.eta) else tomo.same_matrix(
                P, c["seed_base"] + i, eta, c["n_ellipses"])
            insts.append((eta, c["seed_base"] + i, Q))
    stream = torch.cuda.current_stream(dev)
    b_dev = [torch.from_numpy(Q.b).to(dev) for _, _, Q in insts]
    x_dev = torch.empty(P.n, dtype=torch.float64, device=dev)
    ks = list(range(k_step, K + 1, k_step))
    res = {}
    x_K, gp_K = {}, {}
    for vt in VALUE_TYPES_STUDY:
        s = lslu.Solver(P.m, P.n, P.row_ptr, P.col_idx, P.vals, vt, K, stream=stream.cuda_stream,
                        row_order=order[0], col_order=order[1])
        s.tune_spmv(reps=3)
        s.solve_device(b_dev[0], x_dev, K, "gcv")
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = 3
        e0.record(stream)
        for _ in range(reps):
            s.solve_device(b_dev[0], x_dev, K, "gcv")
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        errs = np.zeros((len(insts), len(ks)))
        for j, k in enumerate(ks):  # one captured graph per k, replayed per instance
            for i, (_, _, Q) in enumerate(insts):
                s.solve_device(b_dev[i], x_dev, k, "gcv")
                x = x_dev.cpu().numpy()
                errs[i, j] = np.linalg.norm(x - Q.x_true) / np.linalg.norm(Q.x_true)
                if k == K:
                    x_K[(vt, i)] = x
        for i, (eta, seed, Q) in enumerate(insts):
            if seed == c["seed_base"]:  # the instances the oracle solves: pivots too
                r = s.solve(Q.b, K, "gcv")
                x_K[(vt, i)] = r["x"]
                gp_K[(vt, i)] = r["gp"]
        rows = []
        for i, (eta, seed, Q) in enumerate(insts):
            st = s.solve_stopping(Q.b, K, "gcv", 0.0, stop_tol)
            e_stop = float(np.linalg.norm(st["x"] - Q.x_true) / np.linalg.norm(Q.x_true))
            jb = int(np.argmin(errs[i]))
            rows.append({"eta": eta, "phantom_seed": seed, "k_stop": int(st["k_stop"]),
                         "err_at_stop": e_stop, "k_min": ks[jb], "err_min": float(errs[i, jb]),
                         "err_at_K": float(errs[i, -1])})
        s.close()
        res[vt] = {"iter_per_s": K / (ms / 1e3), "ms_per_solve": ms, "instances": rows}
    for vt in ("f32", "bf16"):
        cmp = {}
        for point in ("err_at_stop", "err_min", "err_at_K"):
            d = np.array([a[point] - b[point] for a, b in
                          zip(res[vt]["instances"], res["f64"]["instances"])])
            within = sum(a[point] <= 1.01 * b[point] for a, b in
                         zip(res[vt]["instances"], res["f64"]["instances"]))
            cmp[point] = {"mean_diff": float(d.mean()), "worst_diff": float(d.max()),
                          "within_1pct_of_f64": f"{within}/{len(insts)}"}
        res[vt]["vs_f64"] = cmp
        res[vt]["speedup_vs_f64"] = res[vt]["iter_per_s"] / res["f64"]["iter_per_s"]
        res[vt]["rel_diff_x_K_vs_f64_gpu"] = [
            float(np.linalg.norm(x_K[(vt, i)] - x_K[("f64", i)]) / np.linalg.norm(x_K[("f64", i)]))
            for i in range(len(insts))]
    res["setup"] = (f"{len(insts)} instances: phantoms seeds {c['seed_base']}.."
                    f"{c['seed_base'] + n_phantoms - 1} x noise {list(ORACLE_ETAS)}; GCV lambda; "
                    f"errors on a {k_step}-iteration grid; stopping rule tol {stop_tol}; "
                    f"differences are mixed minus FP64 (relative error, absolute)")
    return res, (insts, x_K, gp_K, c)


def oracle_comparison(res, data, oracle):
    """res["vs_oracle"]: the GPU's x_K of the precision study's instance 0 at
    each noise level against the oracle runs (the AsyncResult of
    start_oracle_runs; waits for them)."""
    from oracle.perturb import first_difference

    insts, x_K, gp_K, c = data
    try:
        oracle_results = oracle.get()
    except Exception as e:  # noqa: BLE001 - reported, the study stands without it
        res["vs_oracle"] = f"oracle runs failed: {e}"
        return
    out = []
    for r in oracle_results:
        i = next(j for j, (eta, seed, _) in enumerate(insts)
                 if eta == r["eta"] and seed == c["seed_base"])
        Q = insts[i][2]
        xg = x_K[(r["value_type"], i)]
        out.append({"value_type": r["value_type"], "eta": r["eta"], "K": r["K"],
                    "first_pivot_difference": first_difference(gp_K[(r["value_type"], i)],
                                                               r["gp"]),
                    "rel_diff_x_K_vs_oracle": float(np.linalg.norm(xg - r["x"]) /
                                                    np.linalg.norm(r["x"])),
                    "oracle_rel_err_x_true": float(np.linalg.norm(r["x"] - Q.x_true) /
                                                   np.linalg.norm(Q.x_true)),
                    "gpu_rel_err_x_true": float(np.linalg.norm(xg - Q.x_true) /
                                                np.linalg.norm(Q.x_true)),
                    "oracle_seconds": r["seconds"]})
    res["vs_oracle"] = out


def batched_study(dev, K=150, count=64, order="tiles", shape=None):
    """Batched solves: `count` independent problems of uneven size (image side
    64..256, 30..180 angles, 1.41 N rays, own phantom and noise level in
    [0.5%, 3%]) solved together by one launch sequence (FP32, GCV, K
    iterations each), against the same problems solved one after another
    with single-problem handles; every problem renumbered by
    tomo.locality_order when order == "tiles" (the batch in the natural
    numbering is timed beside it).  Every handle runs its sparse products
    with the row shape `shape` where its matrices allow it (None: the
    default), the batch and the single-problem handles alike, so that each
    problem's x can be compared bit for bit."""
    import torch

    from paper_2409_05239_gb300 import lslu

    Ps = tomo.make_uneven_batch(count)
    stream = torch.cuda.current_stream(dev)
    b = np.concatenate([P.b for P in Ps])
    b_dev = torch.from_numpy(b).to(dev)
    x_dev = torch.empty(sum(P.n for P in Ps), dtype=torch.float64, device=dev)
    kd_dev = torch.empty(count, dtype=torch.int32, device=dev)
    orders = [tomo.locality_order(P) for P in Ps] if order == "tiles" else None
    code = None if shape is None else lslu.Solver.SHAPES.index(shape)
    shaped = []

    def use_shape(s):
        cfg = s.spmv_config()
        ok = code is not None and (cfg["compressed_A"] or "16-bit" not in shape) and \
            (cfg["compressed_AT"] or "16-bit" not in shape)
        if ok:
            s.set_spmv_shape(code, code)
        shaped.append(ok)
        return s

    bs = use_shape(lslu.from_problems(Ps, "f32", K, stream=stream.cuda_stream, orders=orders))

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_b = timed(lambda: bs.solve_device(b_dev, x_dev, K, "gcv", k_done=kd_dev), 3)
    launches = bs.last_launch_count()
    x = x_dev.cpu().numpy()
    kd = kd_dev.cpu().numpy()
    bs.close()
    ms_nat = None
    if orders is not None:
        bn = use_shape(lslu.from_problems(Ps, "f32", K, stream=stream.cuda_stream))
        ms_nat = timed(lambda: bn.solve_device(b_dev, x_dev, K, "gcv", k_done=kd_dev), 3)
        bn.close()
    singles = [use_shape(lslu.Solver(P.m, P.n, P.row_ptr, P.col_idx, P.vals, "f32", K,
                                     stream=stream.cuda_stream,
                                     row_order=None if orders is None else orders[p][0],
                                     col_order=None if orders is None else orders[p][1]))
               for p, P in enumerate(Ps)]
    bd = [torch.from_numpy(P.b).to(dev) for P in Ps]
    xd = [torch.empty(P.n, dtype=torch.float64, device=dev) for P in Ps]

    def seq():
        for s, bb, xx in zip(singles, bd, xd):
            s.solve_device(bb, xx, K, "gcv")

    ms_s = timed(seq, 2)
    same = all(np.array_equal(xd[p].cpu().numpy(), x[off:off + P.n])
               for p, (P, off) in enumerate(zip(Ps, np.cumsum([0] + [P.n for P in Ps]))))
    for s in singles:
        s.close()
    iters = int(kd.sum())
    errs = []
    off = 0
    for P in Ps:
        errs.append(np.linalg.norm(x[off:off + P.n] - P.x_true) / np.linalg.norm(P.x_true))
        off += P.n
    nbytes = sum(solve_bytes(P, "f32", K) for P in Ps)
    return {"problems": count, "K": K, "m_total": int(sum(P.m for P in Ps)),
            "n_total": int(sum(P.n for P in Ps)), "nnz_total": int(sum(P.nnz for P in Ps)),
            "numbering": ORDER_NOTE[order],
            "spmv_shape": "default" if shape is None else shape if all(shaped) else
            {"shape": shape, "handles_with_it": int(sum(shaped)), "handles": len(shaped)},
            "ms_per_batch_solve": ms_b,
            "ms_per_batch_solve_natural_numbering": ms_nat,
            "problem_iter_per_s": iters / (ms_b / 1e3),
            "hbm_gbs_solve": nbytes / (ms_b * 1e-3) / 1e9,
            "kernel_launches_per_batch_solve": launches,
            "sequential_single_ms": ms_s, "speedup_vs_sequential": ms_s / ms_b,
            "identical_to_single_solves": bool(same),
            "rel_err_x_true_median": float(np.median(errs)),
            "rel_err_x_true_max": float(np.max(errs))}


def shared_rhs_study(dev, K=150, nrhs=16, order="tiles"):
    """16 right-hand sides for the 256x256 projector (FP32, GCV, K iterations):
    the shared-matrix handle (A read once per product for all of them) against
    the same right-hand sides as a block-diagonal batch of 16 copies of A and
    against 16 single-problem solves one after another; all three renumbered
    by tomo.locality_order when order == "tiles"."""
    import torch

    from paper_2409_05239_gb300 import lslu

    Ps = tomo.make_shared_rhs("ct256", nrhs)
    P0 = Ps[0]
    stream = torch.cuda.current_stream(dev)
    b = np.concatenate([P.b for P in Ps])
    b_dev = torch.from_numpy(b).to(dev)
    x_dev = torch.empty(nrhs * P0.n, dtype=torch.float64, device=dev)

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    o = tomo.locality_order(P0) if order == "tiles" else None
    sh = lslu.shared_rhs(P0, nrhs, "f32", K, stream=stream.cuda_stream, order=o)
    ms_sh = timed(lambda: sh.solve_device(b_dev, x_dev, K, "gcv"))
    x_sh = x_dev.cpu().numpy()
    sh.close()
    bd = lslu.from_problems(Ps, "f32", K, stream=stream.cuda_stream,
                            orders=None if o is None else [o] * nrhs)
    ms_bd = timed(lambda: bd.solve_device(b_dev, x_dev, K, "gcv"))
    same_bd = bool(np.array_equal(x_dev.cpu().numpy(), x_sh))
    bd.close()
    single = lslu.Solver(P0.m, P0.n, P0.row_ptr, P0.col_idx, P0.vals, "f32", K,
                         stream=stream.cuda_stream, row_order=None if o is None else o[0],
                         col_order=None if o is None else o[1])
    bs = [torch.from_numpy(P.b).to(dev) for P in Ps]
    xs = torch.empty(P0.n, dtype=torch.float64, device=dev)
    ms_seq = timed(lambda: [single.solve_device(bb, xs, K, "gcv") for bb in bs], reps=2)
    single.close()
    return {"workload": "ct256 (m=%d, n=%d, nnz=%d) x %d right-hand sides, FP32, K=%d, GCV"
                        % (P0.m, P0.n, P0.nnz, nrhs, K),
            "numbering": ORDER_NOTE[order],
            "ms_per_solve_shared_matrix": ms_sh,
            "ms_per_solve_block_diagonal_copies": ms_bd,
            "ms_sequential_single_solves": ms_seq,
            "rhs_iter_per_s_shared": nrhs * K / (ms_sh / 1e3),
            "speedup_vs_block_diagonal": ms_bd / ms_sh,
            "speedup_vs_sequential": ms_seq / ms_sh,
            "identical_to_block_diagonal": same_bd}


def adjoint_study(dev, K=100, order="tiles"):
    """Differentiable solve on the 256x256 workload (FP32, fixed lambda = the
    GCV choice at K; renumbered by tomo.locality_order when order == "tiles"):
    time of the forward solve and of the reverse-mode derivative
    (lslu_adjoint) on the device, and the log-lambda derivative against
    central differences of solves with the pivots replayed."""
    import torch

    from paper_2409_05239_gb300 import lslu

    P = tomo.make_config("ct256")
    stream = torch.cuda.current_stream(dev)
    ro, co = tomo.locality_order(P) if order == "tiles" else (None, None)
    s = lslu.Solver(P.m, P.n, P.row_ptr, P.col_idx, P.vals, "f32", K, stream=stream.cuda_stream,
                    row_order=ro, col_order=co)
    lam = float(s.solve(P.b, K, "gcv", histories=True)["lam_hist"][-1])
    b_dev = torch.from_numpy(P.b).to(dev)
    x_dev = torch.empty(P.n, dtype=torch.float64, device=dev)
    xt = torch.from_numpy(P.x_true).to(dev)
    bb = torch.empty(P.m, dtype=torch.float64, device=dev)
    lb = torch.empty(1, dtype=torch.float64, device=dev)

    def fwd():
        s.solve_device(b_dev, x_dev, K, "fixed", lam)

    def bwd():
        s.adjoint_device(2.0 * (x_dev - xt), bb, lb)

    fwd()
    bwd()
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    reps = 3
    ms_f = ms_b = 0.0
    for _ in range(reps):
        e[0].record(stream)
        fwd()
        e[1].record(stream)
        bwd()
        e[2].record(stream)
        torch.cuda.synchronize()
        ms_f += e[0].elapsed_time(e[1]) / reps
        ms_b += e[1].elapsed_time(e[2]) / reps
    r = s.solve(P.b, K, "fixed", lam)
    adj = s.adjoint(2.0 * (r["x"] - P.x_true))

    def J(lm):
        o = s.solve_fixed_pivots(P.b, K, r["gp"], r["tp"], "fixed", lm)
        return float(np.sum((o["x"] - P.x_true) ** 2))

    h = 1e-3
    fd = (J(lam * np.exp(h)) - J(lam * np.exp(-h))) / (2 * h)
    g = adj["lambda_bar"] * lam
    # dJ/db along a random direction: the adjoint against central differences
    # of the solve with the pivots replayed, relative steps 1e-3 and 1e-5, at
    # K = 10 (well conditioned) and at K
    db = np.random.default_rng(1).standard_normal(P.m)
    grad_b = {}
    for Kb in (10, K):
        rb = s.solve(P.b, Kb, "fixed", lam)
        gb = float(s.adjoint(2.0 * (rb["x"] - P.x_true))["b_bar"] @ db)

        def Jb(bb):
            o = s.solve_fixed_pivots(bb, Kb, rb["gp"], rb["tp"], "fixed", lam)
            return float(np.sum((o["x"] - P.x_true) ** 2))

        fds = {}
        for step in (1e-3, 1e-5):
            hb = step * np.linalg.norm(P.b) / np.linalg.norm(db)
            fds[step] = (Jb(P.b + hb * db) - Jb(P.b - hb * db)) / (2 * hb)
        grad_b[f"K={Kb}"] = {"adjoint": gb, "fd_step_1e-3": fds[1e-3], "fd_step_1e-5": fds[1e-5],
                             "rel_err_vs_fd_1e-5": abs(gb - fds[1e-5]) / abs(fds[1e-5]),
                             "fd_steps_disagree_by": abs(fds[1e-3] - fds[1e-5]) / abs(fds[1e-5])}
    s.close()
    return {"workload": "ct256 (m=%d, n=%d), FP32, K=%d, lambda=%.4g (GCV at K)" % (P.m, P.n, K, lam),
            "numbering": ORDER_NOTE[order],
            "forward_ms": ms_f, "backward_ms": ms_b, "backward_over_forward": ms_b / ms_f,
            "dJ_dloglam_adjoint": g, "dJ_dloglam_fd": fd,
            "dJ_dloglam_rel_err_vs_fd": abs(g - fd) / abs(fd),
            "dJ_db_direction": grad_b,
            "dJ_db_note": "with the pivots fixed, the b-derivative at K=100 is not determined in "
                          "floating point: differences at two step sizes disagree, and two FP64 "
                          "evaluations of the oracle's tangent in different summation orders "
                          "differ by several per cent (tests/test_gpu_adjoint.py)"}


def persistent_study(dev, batch_count=64, K_batch=150, order="tiles"):
    """Launch-bound workloads with the basis loop as six kernels per iteration
    replayed from a CUDA graph against one persistent cooperative launch and
    (single problems) one thread-block cluster (lslu_set_loop): the 32x32
    workload in FP64 and FP32 (K = 50, GCV), and the 64-problem uneven batch
    (FP32, K = 150, GCV; renumbered like batched_study)."""
    import torch

    from paper_2409_05239_gb300 import lslu

    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {}
    P = tomo.make_config("ct32")
    K = tomo.CONFIGS["ct32"]["K"]
    b = torch.from_numpy(P.b).to(dev)
    x = torch.empty(P.n, dtype=torch.float64, device=dev)
    xs = {}
    for vt in ("f64", "f32"):
        s = lslu.Solver(P.m, P.n, P.row_ptr, P.col_idx, P.vals, vt, K, stream=stream.cuda_stream)
        ms_g = timed(lambda: s.solve_device(b, x, K, "gcv"), 200)
        launches_g = s.last_launch_count()
        xg = x.cpu().numpy()
        s.set_loop("persistent")
        blocks = s.loop_config()["blocks"]
        ms_p = timed(lambda: s.solve_device(b, x, K, "gcv"), 200)
        launches_p = s.last_launch_count()
        xs[vt] = x.cpu().numpy()
        s.set_loop("cluster")
        ctas = s.loop_config()["blocks"]
        ms_c = timed(lambda: s.solve_device(b, x, K, "gcv"), 200)
        xc = x.cpu().numpy()
        s.close()
        out[f"ct32_{vt}"] = {
            "workload": f"ct32 (m={P.m}, n={P.n}, nnz={P.nnz}), {vt.upper()}, K={K}, GCV",
            "graph_ms_per_solve": ms_g, "graph_iter_per_s": K / (ms_g / 1e3),
            "graph_launches_per_solve": launches_g,
            "persistent_ms_per_solve": ms_p, "persistent_iter_per_s": K / (ms_p / 1e3),
            "persistent_launches_per_solve": launches_p, "persistent_blocks": blocks,
            "speedup": ms_g / ms_p,
            "rel_diff_x_persistent_vs_graph": float(np.linalg.norm(xs[vt] - xg) /
                                                    np.linalg.norm(xg)),
            "cluster_ms_per_solve": ms_c, "cluster_iter_per_s": K / (ms_c / 1e3),
            "cluster_ctas": ctas, "cluster_speedup_vs_graph": ms_g / ms_c,
            "rel_diff_x_cluster_vs_graph": float(np.linalg.norm(xc - xg) / np.linalg.norm(xg))}
    Ps = tomo.make_uneven_batch(batch_count)
    bb = torch.from_numpy(np.concatenate([Q.b for Q in Ps])).to(dev)
    xb = torch.empty(sum(Q.n for Q in Ps), dtype=torch.float64, device=dev)
    kd = torch.empty(batch_count, dtype=torch.int32, device=dev)
    orders = [tomo.locality_order(Q) for Q in Ps] if order == "tiles" else None
    bs = lslu.from_problems(Ps, "f32", K_batch, stream=stream.cuda_stream, orders=orders)
    ms_g = timed(lambda: bs.solve_device(bb, xb, K_batch, "gcv", k_done=kd), 3)
    xg = xb.cpu().numpy()
    bs.set_loop("persistent")
    ms_p = timed(lambda: bs.solve_device(bb, xb, K_batch, "gcv", k_done=kd), 3)
    iters = int(kd.sum().item())
    out["batch64_f32"] = {
        "workload": f"{batch_count} uneven problems, FP32, K={K_batch}, GCV",
        "numbering": ORDER_NOTE[order],
        "graph_ms_per_batch_solve": ms_g, "persistent_ms_per_batch_solve": ms_p,
        "persistent_blocks": bs.loop_config()["blocks"],
        "graph_problem_iter_per_s": iters / (ms_g / 1e3),
        "persistent_problem_iter_per_s": iters / (ms_p / 1e3), "speedup": ms_g / ms_p,
        "rel_diff_x_persistent_vs_graph": float(np.linalg.norm(xb.cpu().numpy() - xg) /
                                                np.linalg.norm(xg))}
    bs.close()
    return out


def ct256_study(dev, K=200, order="tiles", reps=20):
    """The 256x256 workload as its configuration states it: Hybrid LSLU, FP32
    values and accumulation, K = 200, GCV lambda (renumbered like the
    benchmark when order == "tiles", products autotuned): iterations/s of the
    device-resident solve (CUDA events on the launch stream over `reps`
    replays) and the error against x_true; parity against the oracle at this
    size is tests/test_gpu_parity_large.py::test_ct256_f32_k200_against_oracle."""
    import torch

    from paper_2409_05239_gb300 import lslu

    P = tomo.make_config("ct256")
    stream = torch.cuda.current_stream(dev)
    ro, co = tomo.locality_order(P) if order == "tiles" else (None, None)
    s = lslu.Solver(P.m, P.n, P.row_ptr, P.col_idx, P.vals, "f32", K, stream=stream.cuda_stream,
                    row_order=ro, col_order=co)
    try:
        s.tune_spmv(reps=5)
        tuned = {k: v for k, v in s.spmv_config().items() if k.startswith("shape")}
        b = torch.from_numpy(P.b).to(dev)
        x = torch.empty(P.n, dtype=torch.float64, device=dev)
        for _ in range(3):
            s.solve_device(b, x, K, "gcv")
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            s.solve_device(b, x, K, "gcv")
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        xh = x.cpu().numpy()
        return {"workload": f"ct256 (m={P.m}, n={P.n}, nnz={P.nnz}), FP32, K={K}, GCV",
                "numbering": ORDER_NOTE[order], "spmv_shape": tuned, "ms_per_solve": ms,
                "iter_per_s": K / (ms / 1e3),
                "rel_err_x_true": float(np.linalg.norm(xh - P.x_true) / np.linalg.norm(P.x_true))}
    finally:
        s.close()


def variants_study(solver, P, K, reps=3):
    """The method's variants on the benchmark handle (same workload, numbering
    and tuned products), each through the public host API (b in, x out):
    the plain GCV solve for reference; the stopping rule of Eqs. (stop2)/(tol)
    (the basis to K, the projected solve of every k, the stopping k, x there);
    sampled pivots (Section 2.2) with 25, 50 and 100 samples per step; the
    optimal-lambda reference rule; the low-rank posterior variances of Section
    4.2 after a solve.  Times are per call (the host copies included)."""
    from paper_2409_05239_gb300 import lslu

    def timed(fn):
        out = fn()
        t0 = time.perf_counter()
        for _ in range(reps):
            out = fn()
        return (time.perf_counter() - t0) / reps * 1e3, out

    def err(x):
        return float(np.linalg.norm(x - P.x_true) / np.linalg.norm(P.x_true))

    res = {"workload": f"ct512, K={K}, FP32 values, GCV, the benchmark's handle", "reps": reps}
    ms, r = timed(lambda: solver.solve(P.b, K, "gcv"))
    res["plain_solve"] = {"ms": ms, "iter_per_s": K / (ms / 1e3), "rel_err_x_true": err(r["x"])}
    ms, r = timed(lambda: solver.solve(P.b, K, "gcv", histories=True))
    lam = float(r["lam_hist"][r["k_done"] - 1])
    res["solve_with_histories"] = {
        "ms": ms, "lambda": lam,
        "note": "lambda_k and the projected residual of every k: a projected solve per k"}
    ms, r = timed(lambda: solver.solve_stopping(P.b, K, "gcv", 0.0, 1e-6))
    ne = int(np.count_nonzero(r["G"]))
    res["stopping_rule"] = {"ms": ms, "tol": 1e-6, "k_stop": int(r["k_stop"]),
                            "iterations_evaluated": ne,
                            "rel_err_x_true_at_k_stop": err(r["x"]),
                            "over_plain_solve": ms / res["plain_solve"]["ms"],
                            "note": "online: the basis in chunks of 8 iterations, the criterion "
                                    "after each chunk"}
    res["sampled_pivots"] = {}
    for ns in (25, 50, 100):
        table = lslu.sample_table(K, ns, P.m, P.n, seed=5000 + ns)
        ms, r = timed(lambda: solver.solve_sampled(P.b, K, table, "gcv"))
        res["sampled_pivots"][str(ns)] = {"ms": ms, "iter_per_s": r["k_done"] / (ms / 1e3),
                                          "k_done": int(r["k_done"]),
                                          "rel_err_x_true": err(r["x"])}
    ms, r = timed(lambda: solver.solve_optimal(P.b, K, P.x_true))
    res["optimal_lambda"] = {"ms": ms, "lambda": r["lam"], "rel_err_x_true": err(r["x"])}
    solver.solve(P.b, K, "gcv")
    sigma2 = float((P.eta * np.linalg.norm(P.b)) ** 2 / P.m)
    ms, u = timed(lambda: solver.uq(sigma2, lam, want_diag=True))
    res["uq_after_solve"] = {"ms": ms, "k": K, "sigma2": sigma2, "var_sum": u["var_sum"],
                             "note": "diag(Gamma_K) (n entries) and 1^T Gamma_K 1 from the "
                                     "solve's bases"}
    return res


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cfg = tomo.CONFIGS[args.workload]
    K = args.K or cfg["K"]
    P = tomo.make_config(args.workload)
    import oracle.lslu_oracle as O

    A = P.scipy()

    def solve_seconds(k):
        t0 = time.perf_counter()
        O.hybrid_lslu(A, P.b, None, k, "gcv", histories=False)
        return time.perf_counter() - t0

    # each step: a bounded sample of the same solve (its first ks iterations),
    # sized so the whole run stays within a few minutes.  Iteration j
    # eliminates against j earlier basis vectors, so k iterations cost about
    # a k + b k^2; two probes fix a and b.
    t2, t10 = solve_seconds(2), solve_seconds(10)
    b = max((t10 - 5.0 * t2) / 80.0, 0.0)
    a = max((t2 - 4.0 * b) / 2.0, 1e-4)
    per_solve = 120.0 / max(1, args.steps + args.warmup)
    ks = 2
    while ks < K and a * (ks + 1) + b * (ks + 1) ** 2 <= per_solve:
        ks += 1
    for _ in range(args.warmup):
        O.hybrid_lslu(A, P.b, None, ks, "gcv", histories=False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.hybrid_lslu(A, P.b, None, ks, "gcv", histories=False)
    dt = time.perf_counter() - t0
    v = ks * args.steps / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "iter/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload} (m={P.m}, n={P.n}, nnz={P.nnz})",
                   "iterations_per_step": ks},
        "cpu_baseline": {"value": v, "unit": "iter/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {ks} of {K} iterations per step"},
        "e2e": {"value": v, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2409_05239_gb300 import build, lslu

    rank, world, local = dist_env()
    cfg = tomo.CONFIGS[args.workload]
    K = args.K or cfg["K"]
    oracle_pool = oracle_runs = None
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    P = tomo.make_problem(cfg["N"], cfg["n_ang"], cfg["p"], cfg["n_ellipses"], cfg["etas"][0],
                          seed=replica_seed(cfg["seed_base"], rank))
    stream = torch.cuda.current_stream(dev)
    ro, co = tomo.locality_order(P) if args.order == "tiles" else (None, None)
    solver = lslu.Solver(P.m, P.n, P.row_ptr, P.col_idx, P.vals, args.value_type, K,
                         stream=stream.cuda_stream, row_order=ro, col_order=co)
    # autotuner: the fastest row shape of the sparse products for this A and A^T
    tuned = solver.tune_spmv(reps=5)
    b_dev = torch.from_numpy(P.b).to(dev)
    x_dev = torch.empty(P.n, dtype=torch.float64, device=dev)
    rule = "gcv"

    def step():
        solver.solve_device(b_dev, x_dev, K, rule)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    launches = 0
    for _ in range(args.steps):
        step()
        launches += solver.last_launch_count()
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    # kernel timing: the same steps again with CUDA-event nodes around every
    # sparse product inside the replayed graph (kept out of the timed region
    # above, whose throughput they would lower by a few per cent)
    solver.profile(True)
    solver.timing()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    n_spmv, spmv_ms = solver.timing()
    solver.profile(False)
    total_iters = K * args.steps * world
    value, s_max = replica_rate(ms / 1e3, K * args.steps, world, dev)
    ms_max = s_max * 1e3

    # end to end through the C ABI with host buffers (H2D of b, D2H of x)
    b_host = torch.from_numpy(P.b).pin_memory()
    x_host = torch.empty(P.n, dtype=torch.float64).pin_memory()

    def step_host():
        st = solver.lib.lslu_solve(solver.h, b_host.data_ptr(), None, K, lslu.RULES[rule], 0.0,
                                   lslu.HOST, x_host.data_ptr(), None, None, None, None, None)
        solver._check(st, allow_breakdown=True)

    step_host()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_host()
    e2e_s = time.perf_counter() - t0
    e2e_value, _ = replica_rate(e2e_s, K * args.steps, world, dev)

    out = None
    if rank == 0:
        x = x_dev.cpu().numpy()
        rel_true = float(np.linalg.norm(x - P.x_true) / np.linalg.norm(P.x_true))
        cfg_sp = solver.spmv_config()
        cmp_A, cmp_AT = "16-bit" in cfg_sp["shape_A"], "16-bit" in cfg_sp["shape_AT"]
        sbytes = spmv_bytes(P, args.value_type, cmp_A, cmp_AT)
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except (OSError, ValueError):
            pass
        hbm = peaks.get("hbm_gbs", 6800.0)
        avg_ms = spmv_ms / max(n_spmv, 1)
        achieved = sbytes / (avg_ms * 1e-3) / 1e9 if n_spmv else None
        total_bytes = solve_bytes(P, args.value_type, K, cmp_A, cmp_AT)
        out = {
            "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.value_type != "f64" else "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {cfg['N']}x{cfg['N']} image, "
                                   f"{cfg['n_ang']} angles x {cfg['p']} rays",
                       "m": P.m, "n": P.n, "nnz": P.nnz, "K": K, "lambda_rule": rule,
                       "numbering": ORDER_NOTE[args.order],
                       "A_values": args.value_type, "basis": "f64" if args.value_type == "f64"
                       else "f32", "projected_solve": "f64",
                       "l2": "inputs larger than L2 (CSR of A and A^T ~%.1f GB)" % (
                           2 * P.nnz * 8 / 1e9),
                       "spmv_shape": {"A": lslu.Solver.SHAPES[tuned["shape_A"]],
                                      "AT": lslu.Solver.SHAPES[tuned["shape_AT"]],
                                      "tuning_us_A": tuned["us_A"],
                                      "tuning_us_AT": tuned["us_AT"]}},
            "roofline": {"bound": "hbm", "kernel": "csr_spmv (A l_k and A^T d_k)",
                         "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm if achieved else None,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)",
                         "timing": "CUDA events around each product, second pass of the timed steps",
                         "algorithmic_bytes_per_launch": sbytes,
                         "bytes_model": "the stored format's bytes: values, column storage "
                                        "(2.5 B per entry with 16-bit offsets), row pointers, "
                                        "output and input vector",
                         "frac_value_plus_int32_column_model": (
                             P.nnz * ({"f64": 8, "f32": 4, "bf16": 2}[args.value_type] + 4) /
                             (avg_ms * 1e-3) / 1e9 / hbm if n_spmv else None),
                         "launches": n_spmv,
                         "avg_launch_ms": avg_ms,
                         "traffic": spmv_traffic(args.workload, args.value_type, args.order,
                                                 cfg_sp["shape_A"], cfg_sp["shape_AT"]),
                         "traffic_source": "profiles/spmv_traffic_by_shape_ct512.md (ncu dram "
                                           "bytes per launch for the tuned shapes)"},
            "hbm_gbs_solve": total_bytes * args.steps * world / (ms_max / 1e3) / 1e9,
            "rel_err_x_true": rel_true,
            "e2e": {"value": e2e_value, "unit": "iter/s", "h2d_bytes_per_step": P.m * 8,
                    "d2h_bytes_per_step": P.n * 8},
            "gpu_launches": launches,
            "clocks": clocks,
        }
    def study(name, fn):
        # a study that fails reports its error in its own field; the line stands
        try:
            out[name] = fn()
        except Exception as e:  # noqa: BLE001
            out[name] = {"error": f"{type(e).__name__}: {e}"}
            print(f"{name} failed: {e}", file=sys.stderr)

    extras = rank == 0 and not args.no_extras and world == 1
    if extras:
        study("variants_study", lambda: variants_study(solver, P, K))
    solver.close()
    # the FP64 oracle at the full workload for the precision study and the CPU
    # baseline, in spawned processes that run beside the studies (after the
    # host-timed measurements above, which they would disturb)
    if extras and args.workload == WORKLOAD:
        oracle_pool, oracle_runs, _ = start_oracle_runs(args.workload, K)
    prec_data = None
    if extras:
        def prec():
            nonlocal prec_data
            res, prec_data = precision_study(P, K, dev, (ro, co))
            return res

        study("precision_study", prec)
        study("batched_study", lambda: batched_study(dev, order=args.order))
        study("shared_rhs_study", lambda: shared_rhs_study(dev, order=args.order))
        study("adjoint_study", lambda: adjoint_study(dev, order=args.order))
        study("persistent_study", lambda: persistent_study(dev, order=args.order))
        study("ct256_study", lambda: ct256_study(dev, order=args.order))
        if oracle_runs is not None and prec_data is not None:
            try:
                oracle_comparison(out["precision_study"], prec_data, oracle_runs)
            except Exception as e:  # noqa: BLE001
                out["precision_study"]["vs_oracle"] = f"{type(e).__name__}: {e}"
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(P, K, args.cpu_sample_s, oracle_runs)
    if oracle_pool is not None:
        oracle_pool.close()
        oracle_pool.join()
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
