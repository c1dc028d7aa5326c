"""Benchmark of the HCA-DBSCAN hot path on one GB300 (or N independent replicas).

One step = one full clustering (every stage: origin shift, binning, sort, cells, pencil
hash, core counts, representative points, merge, labels) of the 3-D mixed workload
(n = 2,000,000 float32 points on the 2^-16 lattice, 40 Gaussian blobs + 8 noisy arcs + 5%
uniform noise in [0,1000]^3, eps = 2, minPts = 10), with the points already resident in
device memory.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload mixed3d|blobs2d] [--no-cpu-baseline]

--impl reference times the CPU oracle (the plain C implementation the CUDA path is checked
against) on the host cores, on a bounded sample of the same workload each step.

With N > 1 (torchrun) every rank clusters its own copy of the workload drawn with its own
seed: the method has no exchange step, so the ranks are independent replicas and `value`
is the points of all ranks divided by the slowest rank's time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "points clustered/sec at 1 GB300 (labels == oracle)"

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one k_reps launch on the
# mixed3d workload at n = 2,000,000, from an ncu full capture of that launch; reported for that
# workload and size only
REPS_TRAFFIC_MIXED3D_2M = 44.760832e6 + 1.304576e6
L2_FLUSH_BYTES = 256 << 20

# Algorithmic bytes per stage, per point (n) and per cell (C) / pencil (P): the data each
# stage must move at least once (reads + writes), with 4-byte keys for <= 32 key bits.
#   bin:   read the point (4 d), write key + index (8)
#   sort:  per 8-bit pass read and write key + value (16)
#   cells: read index (4) + the point (4 d), write the padded point (16 for d = 3) + cell id (4);
#          per cell write start (4) + key (8)
#   reps:  see below (the stage is the k_reps kernel alone)
def stage_bytes(stage, n, d, C, P, passes, key_bytes, core_cells=0, esz=4):
    # esz: bytes per coordinate; sorted points are padded to 4 coordinates at d = 3
    pt = esz * d
    pad = 4 * esz if d == 3 else pt
    if stage == "minmax":
        return n * pt
    if stage == "bin":
        return n * (pt + key_bytes + 4)
    if stage == "sort":
        return passes * n * 2 * (key_bytes + 4)
    if stage == "cells":
        return n * (4 + pt + pad + 4) + C * 12
    if stage == "hash":
        return C * 8 + P * 16
    if stage == "reps":
        # k_reps: read every point, its core flag and its cell id; per cell holding a core
        # point read its key and write, for every representative direction, the 64-bit
        # (distance, index) word and the representative's coordinates
        ndir = {1: 2, 2: 8, 3: 26, 4: 8}.get(d, 0)
        return n * (pad + 1 + 4) + core_cells * (8 + ndir * (8 + pad))
    return None


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mixed3d",
                    choices=["mixed3d", "blobs2d", "aniso16d", "batched", "serving"])
    ap.add_argument("--sets", type=int, default=4096, help="batched: number of point sets")
    ap.add_argument("--seconds", type=float, default=20.0, help="serving: arrival window")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: Poisson arrivals per second")
    ap.add_argument("--workers", type=int, default=4, help="serving: server worker threads (streams)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def workload(name, rank):
    from paper_1912_00323_gb300 import workloads
    seed = workloads.SEED_BASE + {"blobs2d": 0, "mixed3d": 1, "aniso16d": 2}[name] + 1000 * rank
    X, eps, min_pts = workloads.WORKLOADS[name](seed=seed)
    desc = {
        "mixed3d": "d=3, n=2,000,000 float32 on the 2^-16 lattice: 40 Gaussian blobs (sigma 0.5-3) "
                   "+ 8 noisy arcs/rings + 5% uniform noise in [0,1000]^3; eps=2.0, minPts=10",
        "blobs2d": "d=2, n=10,000 float64 on the 2^-12 lattice: 5 Gaussian blobs (sigma 2) + 10% "
                   "uniform noise in [0,100]^2; eps=1.5, minPts=5",
        "aniso16d": "d=16, n=1,000,000 float32 on the 2^-12 lattice: 100 anisotropic Gaussian clusters "
                    "in [0,100]^16 + 10% uniform noise; eps=4.0, minPts=20",
    }[name]
    return X, eps, min_pts, desc


def max_over_ranks(x, dist, device):
    """The largest value of x over all ranks (x itself without a process group): every rank's
    step time is reduced this way, so the reported time is the slowest rank's."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(points_per_rank, world_size, ms):
    """Whole-job throughput of independent replicas: every rank's points over the slowest time."""
    return points_per_rank * world_size / (ms / 1e3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9 and f[1].replace(".", "").isdigit():
                    rows.append(f)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_baseline_oracle(X, eps, min_pts, budget_s=20.0):
    """Time the oracle (as it stands, one host thread) on a bounded sample of the workload."""
    import oracle
    oracle.build()
    n = len(X)
    # first estimate on 10% of the points, then size the sample to about budget_s seconds
    m = max(1000, n // 10)
    t0 = time.perf_counter()
    oracle.grid(X[:m].astype(np.float64), eps, min_pts)
    t1 = time.perf_counter() - t0
    m2 = int(min(n, m * max(1.0, budget_s / max(t1, 1e-3)) * 0.8))
    if m2 > m:
        t0 = time.perf_counter()
        oracle.grid(X[:m2].astype(np.float64), eps, min_pts)
        t1 = time.perf_counter() - t0
        m = m2
    return {"value": m / t1, "unit": "points/s", "cores": 1, "kind": "oracle",
            "sample": f"first {m:,} of the {n:,} workload points (oracle hca_oracle_grid, 1 thread), "
                      f"{t1:.1f} s"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    X, eps, min_pts, desc = workload(args.workload, 0)
    import oracle
    oracle.build()
    n = len(X)
    m = min(n, 200_000)
    sample = X[:m].astype(np.float64)
    for _ in range(args.warmup):
        oracle.grid(sample[: min(m, 20_000)], eps, min_pts)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.grid(sample, eps, min_pts)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = m / (ms / 1e3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload + ": " + desc, "sample_points_per_step": m},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {m:,} of the {n:,} workload points per step"},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import paper_1912_00323_gb300 as pkg
    from paper_1912_00323_gb300 import build as pkg_build

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    if rank == 0 or ws == 1:
        pkg_build.build()
    if dist:
        dist.barrier()
    pkg.load()

    X, eps, min_pts, desc = workload(args.workload, rank)
    n, d = X.shape
    pts = torch.from_numpy(X).to(dev)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(timing):
        return pkg.hca_dbscan_device(pts, eps, min_pts, labels=labels, stream=stream, stats=True,
                                     timing=timing)

    for _ in range(max(args.warmup, 0)):
        step(False)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, stage_ms, stats = [], {}, None
    with ClockSampler(dev.index) as clocks:
        wall0 = time.perf_counter()
        for _ in range(args.steps):
            flush.zero_()                     # evict the previous step's data from L2
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, stats = step(True)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            for k, v in stats["stage_ms"].items():
                stage_ms.setdefault(k, []).append(v)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms = max_over_ranks(sum(step_ms) / len(step_ms), dist, dev)
    value = replica_value(n, ws, ms)

    # end to end through the host entry point: pinned host points in, host labels out
    host_pts = torch.from_numpy(X).pin_memory()
    host_lab = torch.empty(n, dtype=torch.int32).pin_memory()
    pkg.hca_dbscan(host_pts, eps, min_pts, labels=host_lab)
    e2e_t = []
    for _ in range(max(3, min(args.steps, 10))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pkg.hca_dbscan(host_pts, eps, min_pts, labels=host_lab)
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(statistics.median(e2e_t), dist, dev)
    if not np.array_equal(host_lab.numpy(), labels.cpu().numpy()):
        raise RuntimeError("host and device entry points disagree")

    # the plain per-instance path on the same GPU: every distance decided in FP64, no FP32
    # filter and no tensor cores (labels must be identical)
    plain_lab = torch.empty_like(labels)
    def plain_step():
        pkg.hca_dbscan_device(pts, eps, min_pts, labels=plain_lab, stream=stream, fp64_only=True,
                              tensor_cores=False)
    for _ in range(2):
        plain_step()
    plain_ms = []
    for _ in range(max(3, min(args.steps, 20))):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plain_step()
        e1.record(stream)
        e1.synchronize()
        plain_ms.append(e0.elapsed_time(e1))
    if not torch.equal(plain_lab, labels):
        raise RuntimeError("plain FP64 path and tuned path disagree")
    plain = statistics.median(plain_ms)

    # the autotuner on this workload (hca_autotune: neighbour search and tensor-core split),
    # then the same timed steps with its choice; the table is reset afterwards
    t0 = time.perf_counter()
    tune, _ = pkg.hca_autotune(pts, eps, min_pts, stream=stream, repeats=3)
    tune_s = time.perf_counter() - t0
    auto_lab = torch.empty_like(labels)
    for _ in range(2):
        pkg.hca_dbscan_device(pts, eps, min_pts, labels=auto_lab, stream=stream)
    auto_ms = []
    for _ in range(max(3, min(args.steps, 20))):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pkg.hca_dbscan_device(pts, eps, min_pts, labels=auto_lab, stream=stream)
        e1.record(stream)
        e1.synchronize()
        auto_ms.append(e0.elapsed_time(e1))
    pkg.hca_tuning_set(d, None)
    if not torch.equal(auto_lab, labels):
        raise RuntimeError("autotuned and default tuning disagree")

    # d <= 4: the same clustering as a plan (declared extents = the data's, captured once as a
    # CUDA graph, one graph launch per step, no host round trip inside the call)
    graph = None
    if d <= 4:
        with pkg.Plan(pts, eps, min_pts, X.min(axis=0), X.max(axis=0)) as plan:
            for _ in range(2):
                plan.launch(stream)
                plan.wait(stream)
            g_ms = []
            for _ in range(max(3, min(args.steps, 20))):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                plan.launch(stream)
                e1.record(stream)
                e1.synchronize()
                plan.wait(stream)
                g_ms.append(e0.elapsed_time(e1))
            if not torch.equal(plan.labels, labels):
                raise RuntimeError("plan and call disagree")
        gm = statistics.median(g_ms)
        graph = {"ms_per_step": gm, "value": replica_value(n, ws, gm),
                 "path": "hca_plan_create with the data's extents; hca_plan_launch = one CUDA graph launch",
                 "labels": "identical to the call"}
    auto = max_over_ranks(statistics.median(auto_ms), dist, dev)
    plain = max_over_ranks(plain, dist, dev)
    if graph is not None:
        graph["ms_per_step"] = max_over_ranks(graph["ms_per_step"], dist, dev)
        graph["value"] = replica_value(n, ws, graph["ms_per_step"])

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    # roofline of the dominant memory-bound stage (stage times are CUDA events on `stream`)
    peak, peak_kind = measured_peaks()
    C, P = stats["n_cells"], stats["n_pencils"]
    key_bytes = 4 if stats["key_bits"] <= 32 else 8
    med = {k: statistics.median(v) for k, v in stage_ms.items()}
    dominant = max(med, key=med.get)
    roof_rows = {}
    for k, t in med.items():
        b = stage_bytes(k, n, d, C, P, stats["sort_passes"], key_bytes, stats["n_core_cells"],
                        X.dtype.itemsize)
        if b is not None and t > 0:
            roof_rows[k] = {"ms": t, "bytes": b, "gbs": b / (t / 1e3) / 1e9}
    # the roofline object describes k_reps (the representative stage is that one launch) when
    # the path has it, else the slowest stage with a byte model
    if "reps" in roof_rows and roof_rows["reps"]["bytes"] > 0 and d <= 4:
        mem_stage = "reps"
    else:
        mem_stage = max(roof_rows, key=lambda k: roof_rows[k]["ms"]) if roof_rows else None
    roofline = None
    if mem_stage:
        r = roof_rows[mem_stage]
        traffic = None
        if mem_stage == "reps" and args.workload == "mixed3d" and n == 2_000_000:
            traffic = REPS_TRAFFIC_MIXED3D_2M
        roofline = {"bound": "hbm", "kernel": "k_reps" if mem_stage == "reps" else mem_stage,
                    "achieved": r["gbs"], "peak": peak, "unit": "GB/s", "frac": r["gbs"] / peak,
                    "traffic": traffic, "algorithmic_bytes": r["bytes"], "peak_source": peak_kind}

    line = {
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload + ": " + desc, "n": n, "d": d, "eps": eps,
                   "min_pts": min_pts, "l2": "flushed between steps (256 MiB write)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "e2e": {"value": replica_value(n, ws, 1e3 * e2e_s), "unit": "points/s", "h2d_bytes_per_step": int(X.nbytes),
                "d2h_bytes_per_step": 4 * n},
        "gpu_launches": int(stats["kernel_launches"]) * args.steps,
        "roofline": roofline,
        "stage_ms": med, "dominant_stage": dominant,
        "stage_gbs": {k: round(v["gbs"], 1) for k, v in roof_rows.items()},
        "clocks": clocks.summary(),
        "result": {"cells": C, "pencils": P, "dense_cells": stats["n_dense_cells"],
                   "core_points": stats["n_core_points"], "clusters": stats["n_clusters"],
                   "noise": stats["n_noise"]},
        "work": {k: stats[k] for k in ("n_count_chunks", "n_rep_tests", "n_rep_hits",
                                       "n_exhaustive_pairs", "n_exhaustive_chunks", "n_border_chunks",
                                       "n_tc_tiles", "n_tc_rechecks")},
        "autotuned": {"ms_per_step": auto, "value": n * ws / (auto / 1e3), "tuning": tune,
                      "tuning_seconds": tune_s, "labels": "identical to the default tuning"},
        "graph_plan": graph,
        "plain_fp64_gpu": {"ms_per_step": plain, "value": n * ws / (plain / 1e3), "unit": "points/s",
                           "speedup_of_tuned": plain / ms,
                           "path": "same library, HCA_FLAG_FP64_ONLY | HCA_FLAG_NO_TENSOR_CORES, "
                                   "labels identical"},
        "wall_s": wall,
    }
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline_oracle(X, eps, min_pts)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_batched(args):
    """Config B: many independent sets (n log-uniform [1e3, 2e5], d in {2, 3, 8}, own eps and
    MINPTS), one hca_dbscan_batched call per d per step, each d group autotuned on its sets
    first; value = points of all sets / step."""
    import torch
    import paper_1912_00323_gb300 as pkg
    from paper_1912_00323_gb300 import build as pkg_build, workloads
    pkg_build.build()
    pkg.load()
    sets = workloads.batched_sets(n_sets=args.sets)
    groups = {}
    for X, e, m in sets:
        groups.setdefault(X.shape[1], []).append((X, e, m))
    dev_groups, group_arrays = [], []
    for d, g in sorted(groups.items()):
        X = np.concatenate([x for x, _, _ in g], axis=0)
        off = np.zeros(len(g) + 1, np.int64)
        off[1:] = np.cumsum([len(x) for x, _, _ in g])
        dev_groups.append((d, torch.from_numpy(X).cuda(), off, [e for _, e, _ in g], [m for _, _, m in g]))
        group_arrays.append((X, None, None))
    n_total = sum(len(x) for x, _, _ in sets)
    per_d, stages, work = {}, {}, {}
    def step():
        for d, t, off, e, m in dev_groups:
            t0 = time.perf_counter()
            _, st = pkg.hca_dbscan_batched(t, off, e, m, timing=True)
            per_d[d] = time.perf_counter() - t0
            stages[int(d)] = {k: round(v, 3) for k, v in st["stage_ms"].items()}
            work[int(d)] = {k: st[k] for k in ("n_cells", "n_core_points", "n_count_chunks", "n_rep_tests",
                                               "n_rep_hits", "n_exhaustive_pairs", "n_exhaustive_chunks",
                                               "n_border_chunks", "n_tc_tiles", "n_tc_rechecks")}
    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()
    # one step with the default tuning, then the autotuner picks each group's neighbour search
    # and tensor-core split on these sets (hca_autotune_batched), and the timed steps use it
    t0 = time.perf_counter()
    step()
    torch.cuda.synchronize()
    default_ms = 1e3 * (time.perf_counter() - t0)
    tunings = {}
    t0 = time.perf_counter()
    for d, t, off, e, m in dev_groups:
        tune, tms = pkg.hca_autotune_batched(t, off, e, m, repeats=1)
        tunings[int(d)] = dict(tune, best_ms=round(tms, 3))
    tune_s = time.perf_counter() - t0
    step()
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.median(times)

    # the same step as one CUDA graph per d group (plans with the sets' extents, captured with
    # the autotuned tuning): three graph launches on one stream, one wait
    plans = []
    for (d, t, off, e, m), (X_g, _, _) in zip(dev_groups, group_arrays):
        lo = np.stack([X_g[off[s]:off[s + 1]].min(axis=0) for s in range(len(e))])
        hi = np.stack([X_g[off[s]:off[s + 1]].max(axis=0) for s in range(len(e))])
        plans.append(pkg.Plan(t, e, m, lo, hi, offsets=off))
    def plan_step():
        for pl in plans:
            pl.launch()
        for pl in plans:
            pl.wait()
    plan_step()
    g_times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        plan_step()
        g_times.append(time.perf_counter() - t0)
    graph_ms = 1e3 * statistics.median(g_times)
    for pl, (d, t, off, e, m) in zip(plans, dev_groups):
        if not torch.equal(pl.labels, pkg.hca_dbscan_batched(t, off, e, m)):
            raise RuntimeError("batched plan and batched call disagree")
        pl.close()
    for d, *_ in dev_groups:
        pkg.hca_tuning_set(int(d), None)   # the comparisons below run the default tuning
    # the same batched calls on the CUDA cores only, and the plain per-instance path: one
    # hca_dbscan_device call per set, every distance in FP64 (labels must be identical)
    def cuda_core_step():
        for d, t, off, e, m in dev_groups:
            pkg.hca_dbscan_batched(t, off, e, m, tensor_cores=False)
    cuda_core_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cuda_core_step()
    torch.cuda.synchronize()
    cc_ms = 1e3 * (time.perf_counter() - t0)
    ref_labels = [pkg.hca_dbscan_batched(t, off, e, m) for d, t, off, e, m in dev_groups]
    singles = []
    for (d, t, off, e, m), lab in zip(dev_groups, ref_labels):
        for s in range(len(e)):
            singles.append((t[off[s]:off[s + 1]], e[s], m[s], lab[off[s]:off[s + 1]]))
    for x, e, m, _ in singles[:8]:
        pkg.hca_dbscan_device(x, e, m, fp64_only=True, tensor_cores=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    outs = [pkg.hca_dbscan_device(x, e, m, fp64_only=True, tensor_cores=False) for x, e, m, _ in singles]
    torch.cuda.synchronize()
    plain_ms = 1e3 * (time.perf_counter() - t0)
    if not all(torch.equal(o, lab) for o, (_, _, _, lab) in zip(outs, singles)):
        raise RuntimeError("per-set plain FP64 calls and the batched call disagree")

    line = {"metric": "points clustered/sec, batched sets (labels == oracle per set)",
            "value": n_total / (ms / 1e3), "unit": "points/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batched: {args.sets} sets, n log-uniform [1e3, 2e5], d in {{2,3,8}}, "
                                   "blobs + 10% noise, eps U[0.5,3], minPts U{4..16}",
                       "points": n_total, "sets_per_d": {int(d): len(g) for d, g in groups.items()}},
            "ms_per_d": {int(d): 1e3 * t for d, t in per_d.items()}, "stage_ms_per_d": stages,
            "work_per_d": work,
            "cuda_cores_only": {"ms_per_step": cc_ms, "value": n_total / (cc_ms / 1e3),
                                "speedup_of_tuned": cc_ms / ms},
            "autotune": {"tuning_per_d": tunings, "tuning_seconds": tune_s,
                         "default_tuning_ms_per_step": default_ms},
            "graph_plans": {"ms_per_step": graph_ms, "value": n_total / (graph_ms / 1e3),
                            "path": "one hca_plan per d group (declared per-set extents, autotuned), "
                                    "captured as a CUDA graph: three graph launches and one wait per step",
                            "labels": "identical to the batched calls"},
            "plain_fp64_per_set": {"ms_per_step": plain_ms, "value": n_total / (plain_ms / 1e3),
                                   "speedup_of_tuned": plain_ms / ms,
                                   "path": "one hca_dbscan_device call per set, HCA_FLAG_FP64_ONLY | "
                                           "HCA_FLAG_NO_TENSOR_CORES, labels identical"}}
    print(json.dumps(line), flush=True)
    return 0


def run_serving(args):
    """Config S: Poisson arrivals of clustering jobs (n log-uniform [1e3, 2e6], d uniform in
    2..16, blob + noise data, float32 lattice) to the request server; p50 / p99 latency from
    submit to labels, and points/s.  Jobs draw their data from a pool of pre-generated sets."""
    import threading
    import torch
    import paper_1912_00323_gb300 as pkg
    from paper_1912_00323_gb300 import build as pkg_build, workloads
    pkg_build.build()
    pkg.load()
    r = np.random.Generator(np.random.PCG64(workloads.SEED_BASE + 4))
    pool = []
    for k in range(48):
        d = int(r.integers(2, 17))
        (X, e, m), = workloads.batched_sets(n_sets=1, seed=workloads.SEED_BASE + 100 + k, n_min=1_000,
                                            n_max=2_000_000, dims=(d,))
        e = float(np.round(1.5 * np.sqrt(d / 2.0) * 4096) / 4096)
        pool.append((np.ascontiguousarray(X), e, int(r.integers(4, 21))))
    arrivals = np.cumsum(r.exponential(1.0 / args.rate, size=int(args.rate * args.seconds * 1.2) + 10))
    arrivals = arrivals[arrivals < args.seconds]
    picks = r.integers(0, len(pool), size=len(arrivals))
    lat, pts = [], 0
    with pkg.Server(hbm_budget_bytes=64 << 30, workers=args.workers) as sv:
        sv.wait(sv.submit(*pool[0]))          # warm-up
        tickets = []
        t0 = time.perf_counter()
        def collect():
            nonlocal pts
            i = 0
            while i < len(arrivals):
                if i >= len(tickets):
                    time.sleep(0.0005)
                    continue
                _, l = sv.wait(tickets[i])
                lat.append(l)
                pts += len(pool[picks[i]][0])
                i += 1
        th = threading.Thread(target=collect)
        th.start()
        for a, k in zip(arrivals, picks):
            delay = a - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets.append(sv.submit(*pool[k]))
        th.join()
        wall = time.perf_counter() - t0
    lat = np.array(lat)
    line = {"metric": "serving: p50/p99 submit-to-labels latency and points/s",
            "value": pts / wall, "unit": "points/s", "n_gpus": 1, "higher_is_better": True,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "requests": int(len(lat)), "offered_rate_per_s": args.rate, "window_s": args.seconds,
            "wall_s": wall, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serving: Poisson arrivals, n log-uniform [1e3, 2e6], d uniform 2..16, "
                                   "blobs + noise, eps = 1.5 sqrt(d/2), minPts U{4..20}; jobs drawn from 48 "
                                   "pre-generated sets", "workers": args.workers}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
