"""Benchmark of the HCA-DBSCAN hot path on one GB300 (or N independent replicas).

One step = one full clustering (every stage: origin shift, binning, sort, cells, pencil
hash, core counts, representative points, merge, labels) of the 3-D mixed workload
(n = 2,000,000 float32 points on the 2^-16 lattice, 40 Gaussian blobs + 8 noisy arcs + 5%
uniform noise in [0,1000]^3, eps = 2, minPts = 10), with the points already resident in
device memory.  Prints one JSON line whose headline `value` is that workload; on one GPU the
line also carries, under "configs", the other workloads measured in the same run:
  c1_blobs2d    d=2, n=10,000 float64 (labels checked against the CPU oracle)
  c3_aniso16d   d=16, n=1,000,000 float32, tensor-core distance tiles, with the contraction's
                roofline (candidate pairs x 2*16 flops per launch of the tile kernel)
  batched       4096 sets, d in {2,3,8}, one hca_dbscan_batched call per step, and the same
                step as one graph launch
  serving       Poisson arrivals to the request server (short window), p50/p99, beside a plain
                sequential per-request path
Every result is checked against the tuned default call (and C1 against the oracle).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload mixed3d|blobs2d|aniso16d|batched|serving] [--no-cpu-baseline]
                  [--no-extras]

--impl reference times the CPU oracle (the plain C implementation the CUDA path is checked
against) on the host cores, on a bounded sample of the same workload each step.

With N > 1 (torchrun) every rank clusters its own copy of the workload drawn with its own
seed: the method has no exchange step, so the ranks are independent replicas and `value`
is the points of all ranks divided by the slowest rank's time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "points clustered/sec at 1 GB300 (labels == oracle)"
L2_FLUSH_BYTES = 256 << 20

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one radix sort pass
# (k_os_pass) on the mixed3d workload at n = 2,000,000, from an ncu capture of that kernel;
# None until a capture of the current kernel exists
SORT_PASS_TRAFFIC_MIXED3D_2M = 16_050_000  # dram read + write per k_os_pass launch (ncu, mean of 4)

# Nominal dense tensor-core rates of a GB300 (TFLOP/s): the TF32 peak of the tile kernel is the
# measured bf16 GEMM rate scaled by their ratio
NOMINAL_BF16_TFLOPS, NOMINAL_TF32_TFLOPS = 2250.0, 1100.0
# FP32 lanes per SM of the GB300 (CUDA cores), for the ALU peak of the pair tests
FP32_LANES_PER_SM, SMS = 128, 152


# Algorithmic bytes per stage, per point (n) and per cell (C) / pencil (P): the data each
# stage must move at least once (reads + writes), with 4-byte keys for <= 32 key bits.
#   bin:   read the point (esz d), write key + index (key_bytes + 4)
#   sort:  per radix pass read and write key + value (2 (key_bytes + 4))
#   cells: read index (4) + the point (esz d), write the padded point + cell id (4);
#          per cell write start (4) + key (8)
#   reps:  read every point, its core flag and its cell id; per cell holding a core point read
#          its key and write, per representative direction, the (distance, index) word and the
#          representative's coordinates
def stage_bytes(stage, n, d, C, P, passes, key_bytes, core_cells=0, esz=4):
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
        ndir = {1: 2, 2: 8, 3: 26, 4: 8}.get(d, 0)
        return n * (pad + 1 + 4) + core_cells * (8 + ndir * (8 + pad))
    return None


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mixed3d",
                    choices=["mixed3d", "blobs2d", "aniso16d", "batched", "serving"])
    ap.add_argument("--sets", type=int, default=4096, help="batched: number of point sets")
    ap.add_argument("--seconds", type=float, default=60.0, help="serving: arrival window after the warm-up")
    ap.add_argument("--warmup-seconds", type=float, default=5.0, help="serving: arrivals before the window")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: Poisson arrivals per second")
    ap.add_argument("--exact-rate", action="store_true",
                    help="serving: keep --rate even above the measured capacity (the queue then grows)")
    ap.add_argument("--workers", type=int, default=4, help="serving: server worker threads (streams)")
    ap.add_argument("--pool", type=int, default=256, help="serving: distinct generated job sets")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="headline workload only")
    return ap.parse_args(argv)


DESC = {
    "mixed3d": "d=3, n=2,000,000 float32 on the 2^-16 lattice: 40 Gaussian blobs (sigma 0.5-3) "
               "+ 8 noisy arcs/rings + 5% uniform noise in [0,1000]^3; eps=2.0, minPts=10",
    "blobs2d": "d=2, n=10,000 float64 on the 2^-12 lattice: 5 Gaussian blobs (sigma 2) + 10% "
               "uniform noise in [0,100]^2; eps=1.5, minPts=5",
    "aniso16d": "d=16, n=1,000,000 float32 on the 2^-12 lattice: 100 anisotropic Gaussian clusters "
                "in [0,100]^16 + 10% uniform noise; eps=4.0, minPts=20",
}


def workload(name, rank):
    from paper_1912_00323_gb300 import workloads
    seed = workloads.SEED_BASE + {"blobs2d": 0, "mixed3d": 1, "aniso16d": 2}[name] + 1000 * rank
    X, eps, min_pts = workloads.WORKLOADS[name](seed=seed)
    return X, eps, min_pts, DESC[name]


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
    """(HBM GB/s, bf16 TFLOP/s burst, bf16 TFLOP/s sustained, source) from MEASURED_PEAKS.json,
    else the fallback figures."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return (float(p["hbm_gbs"]), float(p["bf16_tflops"]),
                float(p.get("bf16_tflops_sustained", p["bf16_tflops"])), "measured")
    except (OSError, KeyError, ValueError):
        return 6800.0, 1900.0, 1700.0, "fallback"


# ------------------------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, on a bounded sample, one thread and all host cores
# ------------------------------------------------------------------------------------------

def _time_oracle(X, eps, min_pts, threads, budget_s):
    import oracle
    n = len(X)
    m = max(1000, n // 20)
    t0 = time.perf_counter()
    oracle.grid(X[:m].astype(np.float64), eps, min_pts, threads=threads)
    t1 = time.perf_counter() - t0
    m2 = int(min(n, m * max(1.0, budget_s / max(t1, 1e-3)) * 0.8))
    if m2 > m:
        t0 = time.perf_counter()
        oracle.grid(X[:m2].astype(np.float64), eps, min_pts, threads=threads)
        t1 = time.perf_counter() - t0
        m = m2
    return m, t1


def cpu_baseline_oracle(X, eps, min_pts, budget_s=10.0):
    """Time the oracle (hca_oracle_grid as it stands) on the host cores: on all of them (the
    reported value) and on one thread, each on a prefix of the workload sized to about
    budget_s seconds."""
    import oracle
    oracle.build()
    n = len(X)
    cores = os.cpu_count() or 1
    m1, t1 = _time_oracle(X, eps, min_pts, 1, budget_s)
    ma, ta = _time_oracle(X, eps, min_pts, cores, budget_s)
    return {"value": ma / ta, "unit": "points/s", "cores": cores, "kind": "oracle",
            "sample": f"first {ma:,} of the {n:,} workload points (hca_oracle_grid_mt, {cores} threads = "
                      f"nproc), {ta:.1f} s",
            "single_thread": {"value": m1 / t1, "unit": "points/s", "cores": 1,
                              "sample": f"first {m1:,} points (hca_oracle_grid, 1 thread), {t1:.1f} s"},
            "nproc": cores}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    name = args.workload if args.workload in DESC else "mixed3d"
    X, eps, min_pts, desc = workload(name, 0)
    import oracle
    oracle.build()
    n = len(X)
    cores = os.cpu_count() or 1
    m = min(n, 200_000)
    sample = X[:m].astype(np.float64)
    for _ in range(args.warmup):
        oracle.grid(sample[: min(m, 20_000)], eps, min_pts, threads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.grid(sample, eps, min_pts, threads=cores)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = m / (ms / 1e3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name + ": " + desc, "sample_points_per_step": m},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores, "kind": "oracle",
                         "sample": f"first {m:,} of the {n:,} workload points per step, "
                                   f"hca_oracle_grid_mt on {cores} threads"},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------
# Timing helpers (CUDA events on the launching stream; L2 flushed outside the events)
# ------------------------------------------------------------------------------------------

def time_steps(torch, stream, flush, fn, steps):
    """Run fn() `steps` times, each bracketed by CUDA events on `stream` after an L2 flush;
    returns (list of ms, list of fn's return values)."""
    ms, outs = [], []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        outs.append(fn())
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return ms, outs


def single_config(pkg, torch, X, eps, min_pts, steps, warmup, flush, stream, plain_steps, plan=True):
    """One workload on the single-set entry points: the tuned default call (timed, stage times
    from the library's events), the plain FP64 GPU path and, for d <= 4, a plan (one graph
    launch per step).  Every label vector is checked against the tuned call's."""
    n, d = X.shape
    pts = torch.from_numpy(X).to("cuda")
    labels = torch.empty(n, dtype=torch.int32, device="cuda")

    def step(timing=False):
        return pkg.hca_dbscan_device(pts, eps, min_pts, labels=labels, stream=stream, stats=True,
                                     timing=timing)[1]

    for _ in range(max(warmup, 2)):
        step()
    torch.cuda.synchronize()
    ms, _ = time_steps(torch, stream, flush, step, steps)
    med = statistics.median(ms)
    # stage times from the library's events (those calls launch directly, without the graph)
    _, stats = time_steps(torch, stream, flush, lambda: step(True), max(3, min(steps, 10)))
    stage = {k: statistics.median([s["stage_ms"][k] for s in stats]) for k in stats[0]["stage_ms"]}
    tc = {k: statistics.median([s["tc_ms"][k] for s in stats]) for k in stats[0]["tc_ms"]}
    out = {"ms_per_step": med, "value": n / (med / 1e3), "unit": "points/s", "steps": steps,
           "stage_ms": stage, "tc_ms": tc, "stats": stats[-1], "labels": labels}
    direct_lab = torch.empty_like(labels)

    def direct():
        pkg.hca_dbscan_device(pts, eps, min_pts, labels=direct_lab, stream=stream, graph_cache=False)
    direct()
    dms, _ = time_steps(torch, stream, flush, direct, max(3, min(steps, 20)))
    if not torch.equal(direct_lab, labels):
        raise RuntimeError("direct launches and the repeated-call graph disagree")
    out["direct_launches"] = {"ms_per_step": statistics.median(dms),
                              "path": "HCA_FLAG_NO_GRAPH_CACHE: each kernel launched by the host in turn"}

    plain_lab = torch.empty_like(labels)

    def plain():
        pkg.hca_dbscan_device(pts, eps, min_pts, labels=plain_lab, stream=stream, fp64_only=True,
                              tensor_cores=False)
    plain()
    if plain_steps > 1:
        plain()  # the second identical call captures its graph: keep that out of the timing
    pms, _ = time_steps(torch, stream, flush, plain, plain_steps)
    if not torch.equal(plain_lab, labels):
        raise RuntimeError("plain FP64 path and tuned path disagree")
    pm = statistics.median(pms)
    out["plain_fp64_gpu"] = {"ms_per_step": pm, "value": n / (pm / 1e3), "unit": "points/s",
                             "speedup_of_tuned": pm / med, "steps": plain_steps,
                             "path": "same library, HCA_FLAG_FP64_ONLY | HCA_FLAG_NO_TENSOR_CORES, "
                                     "labels identical"}
    if plan and d <= 4:
        with pkg.Plan(pts, eps, min_pts, X.min(axis=0), X.max(axis=0)) as pl:
            for _ in range(2):
                pl.launch(stream)
                pl.wait(stream)
            gms, _ = time_steps(torch, stream, flush, lambda: pl.launch(stream), max(3, min(steps, 20)))
            pl.wait(stream)
            if not torch.equal(pl.labels, labels):
                raise RuntimeError("plan and call disagree")
        gm = statistics.median(gms)
        out["graph_plan"] = {"ms_per_step": gm, "value": n / (gm / 1e3),
                             "path": "hca_plan_create with the data's extents; hca_plan_launch = one CUDA "
                                     "graph launch", "labels": "identical to the call"}
    return out


def sort_roofline(stats, stage, n, peak, peak_kind, traffic):
    """The radix sort pass (k_os_pass, the largest kernel of the 3-D call): algorithmic bytes
    per launch = n (key_bytes + 4) read + written; duration = the sort stage's CUDA-event time
    over its passes (the stage holds only the passes and the clearing of their look-back words)."""
    key_bytes = 4 if stats["key_bits"] <= 32 else 8
    passes = max(1, stats["sort_passes"])
    per_launch_ms = stage["sort"] / passes
    bytes_per_launch = n * 2 * (key_bytes + 4)
    achieved = bytes_per_launch / (per_launch_ms / 1e3) / 1e9
    return {"bound": "hbm", "kernel": "k_os_pass (one radix pass of the cell-key sort)", "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
            "algorithmic_bytes": bytes_per_launch, "launches_per_step": passes,
            "launch_ms": per_launch_ms, "peak_source": f"hbm_gbs of {peak_kind}"}


def pair_rates(stats, stage, d):
    """Pair tests per second of the count and merge stages (32 pair slots per warp chunk; the
    merge adds one test per representative pair), against the FP32 ALU rate of the pair test
    (d subtractions and d FMAs per pair)."""
    alu_pairs = SMS * FP32_LANES_PER_SM * 2.07e9 / (2 * d)
    count_pairs = 32 * stats["n_count_chunks"]
    merge_pairs = stats["n_rep_tests"] + 32 * stats["n_exhaustive_chunks"]
    out = {}
    for name, pairs in (("core", count_pairs), ("merge", merge_pairs)):
        t = stage.get(name, 0.0)
        rate = pairs / (t / 1e3) if t > 0 else None
        out[name] = {"bound": "alu", "pairs": int(pairs), "stage_ms": t, "pairs_per_s": rate,
                     "peak_pairs_per_s": alu_pairs, "frac": (rate / alu_pairs) if rate else None}
    out["peak_note"] = (f"{SMS} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2.07 GHz / {2 * d} instructions per "
                        "pair (d subtractions + d FMAs); the stages are bound by dependent loads, not ALU")
    return out


def tensor_roofline(stats, tc_ms, d, bf16_burst, peak_kind):
    """The tensor-core tile kernel (k_tc_hd): algorithmic flops = candidate pairs x 2 d;
    duration = the CUDA-event time of its four launches (counts, the recount of the rows the
    counts hand over with the few kernels that list them, unions, labels); peak = the measured
    bf16 GEMM rate x (nominal TF32 / nominal bf16)."""
    t = sum(tc_ms.values())
    pairs = stats["n_tc_pairs"]
    if t <= 0 or pairs <= 0:
        return None
    flops = pairs * 2.0 * d
    peak = bf16_burst * NOMINAL_TF32_TFLOPS / NOMINAL_BF16_TFLOPS
    achieved = flops / (t / 1e3) / 1e12
    dp = max(8, 1 << (d - 1).bit_length())
    kp = dp + 8
    mmas = kp // 8 + 2 * (dp // 8)   # hi.hi per K step, hi.lo and lo.hi on the coordinate steps
    issued = stats["n_tc_tiles"] * mmas * 2.0 * 128 * 128 * 8
    return {"bound": "tensor", "kernel": "k_tc_hd (counts + recount, unions, labels: four launches)",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
            "algorithmic_flops": flops, "candidate_pairs": int(pairs), "launch_ms": tc_ms,
            "issued_mma_flops": issued, "issued_tflops": issued / (t / 1e3) / 1e12,
            "peak_source": f"bf16_tflops of {peak_kind} x {NOMINAL_TF32_TFLOPS:g}/{NOMINAL_BF16_TFLOPS:g} "
                           "(nominal TF32/bf16 dense)"}


# ------------------------------------------------------------------------------------------
# Configs beside the headline workload
# ------------------------------------------------------------------------------------------

def config_c1(pkg, torch, stream, flush, steps, warmup):
    import oracle
    X, eps, mp, desc = workload("blobs2d", 0)
    r = single_config(pkg, torch, X, eps, mp, steps, warmup, flush, stream, plain_steps=max(3, min(steps, 20)))
    want, _ = oracle.grid(X, eps, mp)
    if not np.array_equal(r["labels"].cpu().numpy(), want):
        raise RuntimeError("blobs2d labels differ from the oracle")
    st = r.pop("stats")
    r.pop("labels")
    r.update({"workload": "blobs2d: " + desc, "dtype": "f64", "labels": "identical to the CPU oracle",
              "result": {"core_points": st["n_core_points"], "clusters": st["n_clusters"], "noise": st["n_noise"]}})
    return r


def config_c3(pkg, torch, stream, flush, steps, warmup, bf16_burst, peak_kind):
    X, eps, mp, desc = workload("aniso16d", 0)
    r = single_config(pkg, torch, X, eps, mp, steps, warmup, flush, stream, plain_steps=3)
    st = r.pop("stats")
    r.pop("labels")
    r["roofline"] = tensor_roofline(st, r["tc_ms"], X.shape[1], bf16_burst, peak_kind)
    r.update({"workload": "aniso16d: " + desc, "dtype": "f32",
              "labels": "plain FP64 path identical to the tuned call (full-size oracle parity is a GPU test)",
              "tensor_cores": {"n_tc_tiles": st["n_tc_tiles"], "n_tc_rechecks": st["n_tc_rechecks"],
                               "n_tc_pairs": st["n_tc_pairs"]},
              "result": {"core_points": st["n_core_points"], "clusters": st["n_clusters"], "noise": st["n_noise"]}})
    return r


def literal_divergence(db, core, lit):
    """Where the printed algorithm's labels (lit) depart from DBSCAN's (db, with core flags):
    noise_clustered = DBSCAN noise points the printed algorithm puts in a cluster; split =
    DBSCAN clusters whose core points fall into several printed clusters; merged = printed
    clusters holding core points of several DBSCAN clusters; points_moved = clustered points
    whose printed cluster is not the one holding most of their DBSCAN cluster's core points."""
    core = core.astype(bool)
    split, merged, majority = 0, 0, {}
    for cid in np.unique(db[core]):
        vals, cnt = np.unique(lit[core & (db == cid)], return_counts=True)
        split += int(len(vals) > 1)
        majority[int(cid)] = int(vals[np.argmax(cnt)])
    for lid in np.unique(lit[core]):
        merged += int(len(np.unique(db[core & (lit == lid)])) > 1)
    clustered = db >= 0
    maj = np.array([majority[int(c)] for c in db[clustered]], dtype=np.int64)
    return {"n": int(len(db)), "dbscan_clusters": len(majority), "printed_clusters": int(len(np.unique(lit))),
            "dbscan_noise": int((~clustered).sum()), "noise_clustered": int(((~clustered) & (lit >= 0)).sum()),
            "split": split, "merged": merged, "points_moved": int((lit[clustered] != maj).sum())}


def config_literal(pkg, torch, stream):
    """The paper's Algorithms 2-4 as printed (hca_dbscan_literal_device: representatives only,
    strict "<", no MINPTS) beside DBSCAN (hca_dbscan_device) on blobs2d, mixed3d and six small
    batched sets: how far the printed algorithm departs, and its time on mixed3d."""
    from paper_1912_00323_gb300 import workloads
    out = {}
    cases = [("blobs2d",) + workloads.blobs2d(), ("mixed3d",) + workloads.mixed3d()]
    for k, (X, e, m) in enumerate(workloads.batched_sets(n_sets=6, n_min=1_000, n_max=20_000, dims=(2, 3))):
        cases.append((f"batched set {k}", X, e, m))
    for name, X, e, m in cases:
        pts = torch.from_numpy(X).cuda()
        core = torch.empty(len(X), dtype=torch.uint8, device="cuda")
        db = pkg.hca_dbscan_device(pts, e, m, core=core, graph_cache=False).cpu().numpy()
        lit = pkg.hca_dbscan_literal_device(pts, e).cpu().numpy()
        row = literal_divergence(db, core.cpu().numpy(), lit)
        if name == "mixed3d":
            ms = []
            for _ in range(5):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pkg.hca_dbscan_literal_device(pts, e, stream=stream)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            row["ms_per_call"] = statistics.median(ms)
        out[name] = row
    return out


def config_batched(pkg, torch, stream, flush, steps, warmup, n_sets, plain_sample=16):
    """4096 sets (n log-uniform [1e3, 2e5], d in {2, 3, 8}, own eps and MINPTS) in their
    generated order: one hca_dbscan_batched call per step, each d autotuned first; the same
    step as one graph launch (a batched plan); CUDA cores only; and the plain per-instance FP64
    path on every plain_sample-th set against the batched call on those same sets."""
    from paper_1912_00323_gb300 import workloads
    t0 = time.perf_counter()
    sets = workloads.batched_sets(n_sets=n_sets)
    gen_s = time.perf_counter() - t0
    flat, off, dims = pkg.pack_sets([s[0] for s in sets])
    eps = [s[1] for s in sets]
    mps = [s[2] for s in sets]
    n_total = int(off[-1])
    labels = torch.empty(n_total, dtype=torch.int32, device="cuda")

    def call(**kw):
        return pkg.hca_dbscan_batched(flat, off, eps, mps, dims=dims, labels=labels, stream=stream, **kw)

    call()
    torch.cuda.synchronize()
    dms, _ = time_steps(torch, stream, flush, call, 1)
    t0 = time.perf_counter()
    tunings, tune_ms = pkg.hca_autotune_batched(flat, off, eps, mps, dims=dims, stream=stream, repeats=1)
    tune_s = time.perf_counter() - t0
    for _ in range(max(warmup, 1)):
        call()
    ms, outs = time_steps(torch, stream, flush, lambda: call(stats=True, timing=True)[1], steps)
    ref = labels.clone()
    med = statistics.median(ms)
    st = outs[-1]
    lo = np.concatenate([s[0].min(0) for s in sets])
    hi = np.concatenate([s[0].max(0) for s in sets])
    with pkg.Plan(flat, eps, mps, lo, hi, offsets=off, dims=dims) as pl:
        for _ in range(2):
            pl.launch(stream)
            pl.wait(stream)
        gms, _ = time_steps(torch, stream, flush, lambda: pl.launch(stream), steps)
        pl.wait(stream)
        if not torch.equal(pl.labels, ref):
            raise RuntimeError("batched plan and batched call disagree")
    gm = statistics.median(gms)
    cms, _ = time_steps(torch, stream, flush, lambda: call(tensor_cores=False), 1)
    if not torch.equal(labels, ref):
        raise RuntimeError("CUDA-core batched call disagrees")
    for d in tunings:
        pkg.hca_tuning_set(d, None)
    # plain per-instance FP64 path on a sample of the sets, and the batched call on the same sets
    sample = list(range(0, len(sets), plain_sample))
    s_flat, s_off, s_dims = pkg.pack_sets([sets[i][0] for i in sample])
    s_eps = [eps[i] for i in sample]
    s_mp = [mps[i] for i in sample]
    singles = [(torch.from_numpy(sets[i][0]).cuda(), eps[i], mps[i]) for i in sample]
    for x, e, m in singles[:4]:
        pkg.hca_dbscan_device(x, e, m, fp64_only=True, tensor_cores=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    outs_plain = [pkg.hca_dbscan_device(x, e, m, fp64_only=True, tensor_cores=False, stream=stream)
                  for x, e, m in singles]
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    pkg.hca_dbscan_batched(s_flat, s_off, s_eps, s_mp, dims=s_dims, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s_lab = pkg.hca_dbscan_batched(s_flat, s_off, s_eps, s_mp, dims=s_dims, stream=stream)
    torch.cuda.synchronize()
    s_batched_s = time.perf_counter() - t0
    ref_h = ref.cpu().numpy()
    s_lab_h = s_lab.cpu().numpy()
    for k, i in enumerate(sample):
        want = ref_h[off[i]:off[i + 1]]
        if not (np.array_equal(outs_plain[k].cpu().numpy(), want)
                and np.array_equal(s_lab_h[s_off[k]:s_off[k + 1]], want)):
            raise RuntimeError(f"set {i}: per-set plain path or sampled batch disagrees with the batched call")
    s_points = int(s_off[-1])
    per_d = {int(d): int(np.sum(dims == d)) for d in np.unique(dims)}
    return {"workload": f"batched: {n_sets} sets in generated order, n log-uniform [1e3, 2e5], d in {{2,3,8}}, "
                        "5 blobs + 10% noise in [0,100]^d, eps U[0.5,3], minPts U{4..16}, float32 on 2^-12",
            "points": n_total, "sets_per_d": per_d, "generation_s": gen_s,
            "ms_per_step": med, "value": n_total / (med / 1e3), "unit": "points/s", "steps": steps,
            "path": "one hca_dbscan_batched call per step (one segmented pipeline per d, d groups gathered "
                    "from the interleaved sets), each d autotuned",
            "stage_ms": {k: round(v, 3) for k, v in st["stage_ms"].items()}, "tc_ms": st["tc_ms"],
            "work": {k: st[k] for k in ("n_cells", "n_core_points", "n_tc_tiles", "n_tc_rechecks", "n_tc_pairs")},
            "default_tuning_ms": dms[0], "autotune": {"tuning_per_d": tunings, "seconds": tune_s,
                                                     "best_ms_sum": tune_ms},
            "graph_plan": {"ms_per_step": gm, "value": n_total / (gm / 1e3),
                           "path": "one batched plan: the d groups captured one after another into one CUDA "
                                   "graph, one graph launch per step", "labels": "identical to the batched call"},
            "cuda_cores_only": {"ms_per_step": cms[0], "value": n_total / (cms[0] / 1e3),
                                "speedup_of_tuned": cms[0] / med},
            "plain_fp64_per_set": {"sets": len(sample), "points": s_points, "seconds": plain_s,
                                   "value": s_points / plain_s,
                                   "batched_same_sets_value": s_points / s_batched_s,
                                   "speedup_of_batched": plain_s / s_batched_s,
                                   "path": f"every {plain_sample}th set: one hca_dbscan_device call per set, "
                                           "HCA_FLAG_FP64_ONLY | HCA_FLAG_NO_TENSOR_CORES, against one batched "
                                           "call on the same sets; labels identical"}}


def serving_pool(torch, count, seed):
    """Job data for the serving run, drawn on the GPU (torch's Philox generator) and kept in
    pinned host memory: n log-uniform [1e3, 2e6], d uniform in 2..16, eps = 1.5 sqrt(d/2) on the
    2^-12 lattice, MINPTS uniform in 4..20, 5 Gaussian blobs (centres U[10,90]^d) + 10% uniform
    noise in [0,100]^d, float32 coordinates on the 2^-12 lattice.

    Blob sigma: the batched sets' 2 eps / sqrt(d), capped where a blob of m = 0.18 n points
    would leave a typical point fewer than K = 40 neighbours.  A point of an isotropic Gaussian
    typically lies where the density is m (2 pi sigma^2)^(-d/2) e^(-d/2); times the volume V_d
    eps^d of the eps-ball that is K for sigma = eps (m V_d / K)^(1/d) e^(-1/2) / sqrt(2 pi).
    Without the cap almost no point of a d >= 12 set is core (the sets are noise)."""
    r = np.random.Generator(np.random.PCG64(seed))
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    pool = []
    for _ in range(count):
        n = int(round(math.exp(r.uniform(math.log(1e3), math.log(2e6)))))
        d = int(r.integers(2, 17))
        eps = float(np.round(1.5 * math.sqrt(d / 2.0) * 4096) / 4096)
        mp = int(r.integers(4, 21))
        n_noise = n // 10
        sizes = [(n - n_noise) // 5 + (1 if k < (n - n_noise) % 5 else 0) for k in range(5)]
        m_blob = (n - n_noise) / 5.0
        v_d = math.pi ** (d / 2.0) / math.gamma(d / 2.0 + 1.0)
        sigma = min(2.0 * eps / math.sqrt(d),
                    eps * (m_blob * v_d / 40.0) ** (1.0 / d) * math.exp(-0.5) / math.sqrt(2.0 * math.pi))
        parts = []
        for m in sizes:
            c = torch.rand(d, generator=g, device="cuda", dtype=torch.float64) * 80.0 + 10.0
            parts.append(c + sigma * torch.randn((m, d), generator=g, device="cuda", dtype=torch.float64))
        parts.append(torch.rand((n_noise, d), generator=g, device="cuda", dtype=torch.float64) * 100.0)
        X = torch.cat(parts)[torch.randperm(n, generator=g, device="cuda")]
        X = (torch.round(X * 4096.0) / 4096.0).to(torch.float32)
        pool.append((X.cpu().pin_memory(), eps, mp))
    return pool


def config_serving(pkg, torch, seconds, warmup_s, rate, workers, pool_size, seed=1912_00323 + 4,
                   plain_jobs=200, plain_seconds=30.0, burst_jobs=128, exact_rate=False):
    """Poisson arrivals of jobs drawn from a pool of generated sets, submitted to the request
    server with host buffers: the jobs arriving in the first warmup_s seconds are left out of
    the statistics, p50 / p99 submit-to-labels latency and points/s over the window.

    Before the window: every pool set is clustered once alone on the tuned path (device
    resident; its realised core fraction and its service time), and a burst of burst_jobs
    arrivals is submitted to the server at once, whose drain time gives the server's capacity
    in points/s, and in jobs/s of the arrival mix (that rate / the pool's mean job size).  The
    window runs at `rate` jobs/s, or at 0.8 of that capacity when `rate` is above it (unless
    exact_rate), and the line says which.

    Beside it, the plain sequential per-request path: the first plain_jobs jobs of the same
    arrival list (fewer once their service times pass plain_seconds), each copied in, clustered
    with every distance in FP64 and no tensor cores, and copied out alone; their latencies
    follow from the measured service times in arrival order (one request at a time, first come
    first served)."""
    t0 = time.perf_counter()
    pool = serving_pool(torch, pool_size, seed)
    gen_s = time.perf_counter() - t0
    # realised data and the tuned per-request service time of every pool set
    core_d, noise_d, pts_d = {}, {}, {}
    service_tuned = []
    for X, eps, mp in pool:
        xd = X.to("cuda")
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        _, st = pkg.hca_dbscan_device(xd, eps, mp, stats=True)
        torch.cuda.synchronize()
        service_tuned.append(time.perf_counter() - t1)
        dd = int(X.shape[1])
        core_d[dd] = core_d.get(dd, 0) + st["n_core_points"]
        noise_d[dd] = noise_d.get(dd, 0) + st["n_noise"]
        pts_d[dd] = pts_d.get(dd, 0) + int(X.shape[0])
        del xd
    pool_pts = np.array([len(X) for X, _, _ in pool], dtype=np.float64)
    realised = {"core_fraction": sum(core_d.values()) / sum(pts_d.values()),
                "noise_fraction": sum(noise_d.values()) / sum(pts_d.values()),
                "core_fraction_by_d": {dd: round(core_d[dd] / pts_d[dd], 3) for dd in sorted(pts_d)}}
    by_d = {}
    for (X, _, _), t in zip(pool, service_tuned):
        by_d[int(X.shape[1])] = by_d.get(int(X.shape[1]), 0.0) + t
    tuned_seq = {"mean_service_ms": 1e3 * float(np.mean(service_tuned)),
                 "service_share_by_d": {dd: round(by_d[dd] / sum(service_tuned), 3) for dd in sorted(by_d)},
                 "capacity_points_per_s": float(pool_pts.sum() / sum(service_tuned)),
                 "capacity_jobs_per_s": len(pool) / sum(service_tuned),
                 "path": "every pool set alone, device resident, hca_dbscan_device on the tuned path"}
    r = np.random.Generator(np.random.PCG64(seed + 1))
    lat = done_t = None
    with pkg.Server(hbm_budget_bytes=96 << 30, workers=workers) as sv:
        sv.wait(sv.submit(*pool[0]))          # warm-up of the server's streams and pools
        # capacity: a burst submitted at once, drained by the server
        bpicks = r.integers(0, len(pool), size=burst_jobs)
        t1 = time.perf_counter()
        btk = [sv.submit(*pool[k]) for k in bpicks]
        for tk in btk:
            sv.wait(tk)
        burst_s = time.perf_counter() - t1
        cap_pts = float(pool_pts[bpicks].sum()) / burst_s
        # jobs per second at that point rate for the arrival mix (uniform over the pool)
        max_rate = cap_pts / float(pool_pts.mean())
        capacity = {"jobs": int(burst_jobs), "seconds": burst_s, "points_per_s": cap_pts,
                    "jobs_per_s_of_the_mix": max_rate,
                    "path": "a burst of jobs submitted at once; the time until the last one completes"}
        rate_used = rate if (exact_rate or rate <= 0.8 * max_rate) else 0.8 * max_rate
        total = warmup_s + seconds
        arrivals = np.cumsum(r.exponential(1.0 / rate_used, size=int(rate_used * total * 1.3) + 16))
        arrivals = arrivals[arrivals < total]
        picks = r.integers(0, len(pool), size=len(arrivals))
        lat = np.zeros(len(arrivals))
        done_t = np.zeros(len(arrivals))
        tickets = []
        start = time.perf_counter()

        def collect():
            i = 0
            while i < len(arrivals):
                if i >= len(tickets):
                    time.sleep(0.0005)
                    continue
                _, lat[i] = sv.wait(tickets[i])
                done_t[i] = time.perf_counter() - start
                i += 1
        th = threading.Thread(target=collect)
        th.start()
        for a, k in zip(arrivals, picks):
            delay = a - (time.perf_counter() - start)
            if delay > 0:
                time.sleep(delay)
            tickets.append(sv.submit(*pool[k]))
        th.join()
        wall = time.perf_counter() - start
    keep = arrivals >= warmup_s
    pts = np.array([len(pool[k][0]) for k in picks])
    window_end = max(float(done_t[keep].max()), total) if keep.any() else total
    served = float(pts[keep].sum()) / (window_end - warmup_s)
    offered = float(pts[keep].sum()) / seconds
    # plain sequential per-request path on the first plain_jobs arrivals
    m = min(plain_jobs, len(arrivals))
    service = []
    for i in range(m):
        if sum(service) > plain_seconds:
            m = i
            break
        X, eps, mp = pool[picks[i]]
        lab = torch.empty(len(X), dtype=torch.int32).pin_memory()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        xd = X.to("cuda", non_blocking=True)
        ld = pkg.hca_dbscan_device(xd, eps, mp, fp64_only=True, tensor_cores=False)
        lab.copy_(ld, non_blocking=True)
        torch.cuda.synchronize()
        service.append(time.perf_counter() - t1)
    finish, plain_lat = 0.0, []
    for i in range(m):
        finish = max(finish, arrivals[i]) + service[i]
        plain_lat.append(1e3 * (finish - arrivals[i]))
    plain_pts = float(pts[:m].sum())
    return {"workload": f"serving: Poisson arrivals at {rate_used:.4g}/s, {warmup_s:g} s warm-up + {seconds:g} s "
                        "window; n log-uniform [1e3, 2e6], d uniform 2..16, blobs + 10% noise, eps = 1.5 sqrt(d/2), "
                        f"minPts U{{4..20}}; jobs drawn from {len(pool)} generated sets, host buffers",
            "requested_rate_per_s": rate, "rate_per_s": rate_used,
            "saturated_at_requested_rate": bool(rate > max_rate),
            "max_sustainable_rate_per_s": max_rate, "capacity": capacity,
            "tuned_sequential": tuned_seq,
            "pool_generation_s": gen_s, "pool_data": realised, "workers": workers, "requests": int(keep.sum()),
            "p50_ms": float(np.percentile(lat[keep], 50)), "p99_ms": float(np.percentile(lat[keep], 99)),
            "value": served, "unit": "points/s", "offered_points_per_s": offered,
            "keeps_up": bool(window_end - total < 1.0), "wall_s": wall,
            "plain_sequential": {"jobs": m, "p50_ms": float(np.percentile(plain_lat, 50)),
                                 "p99_ms": float(np.percentile(plain_lat, 99)),
                                 "capacity_points_per_s": plain_pts / sum(service),
                                 "offered_points_per_s_same_jobs": plain_pts / float(arrivals[m - 1]),
                                 "path": "one request at a time: H2D copy, hca_dbscan_device with "
                                         "HCA_FLAG_FP64_ONLY | HCA_FLAG_NO_TENSOR_CORES, D2H copy; latency "
                                         "from the measured service times, first come first served"}}


# ------------------------------------------------------------------------------------------
# The headline run
# ------------------------------------------------------------------------------------------

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
    hbm_peak, bf16_burst, _, peak_kind = measured_peaks()

    name = args.workload
    X, eps, min_pts, desc = workload(name, rank)
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
    step_ms, stage_ms, tc_ms, stats = [], {}, {}, None
    with ClockSampler(dev.index) as clocks:
        wall0 = time.perf_counter()
        for _ in range(args.steps):
            flush.zero_()                     # evict the previous step's data from L2
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, call_stats = step(False)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms = max_over_ranks(sum(step_ms) / len(step_ms), dist, dev)
    value = replica_value(n, ws, ms)

    # stage times: the same call with the library's stage events (HCA_FLAG_TIMING runs the
    # launches directly, not the graph of repeated calls)
    for _ in range(max(3, min(args.steps, 10))):
        flush.zero_()
        _, stats = step(True)
        for k, v in stats["stage_ms"].items():
            stage_ms.setdefault(k, []).append(v)
        for k, v in stats["tc_ms"].items():
            tc_ms.setdefault(k, []).append(v)
    torch.cuda.synchronize()

    # the call without the graph of repeated calls: every kernel launched by the host in turn
    direct_lab = torch.empty_like(labels)

    def direct_step():
        pkg.hca_dbscan_device(pts, eps, min_pts, labels=direct_lab, stream=stream, graph_cache=False)
    direct_step()
    direct_ms, _ = time_steps(torch, stream, flush, direct_step, max(3, min(args.steps, 20)))
    if not torch.equal(direct_lab, labels):
        raise RuntimeError("direct launches and the repeated-call graph disagree")
    direct = max_over_ranks(statistics.median(direct_ms), dist, dev)

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
    plain_step()
    plain_step()  # the second identical call captures its graph: keep that out of the timing
    plain_ms, _ = time_steps(torch, stream, flush, plain_step, max(3, min(args.steps, 20)))
    if not torch.equal(plain_lab, labels):
        raise RuntimeError("plain FP64 path and tuned path disagree")
    plain = max_over_ranks(statistics.median(plain_ms), dist, dev)

    # the autotuner on this workload, then the same timed steps with its choice; the table is
    # reset afterwards
    t0 = time.perf_counter()
    tune, _ = pkg.hca_autotune(pts, eps, min_pts, stream=stream, repeats=3)
    tune_s = time.perf_counter() - t0
    auto_lab = torch.empty_like(labels)

    def auto_step():
        pkg.hca_dbscan_device(pts, eps, min_pts, labels=auto_lab, stream=stream)
    auto_step()
    auto_step()
    auto_ms, _ = time_steps(torch, stream, flush, auto_step, max(3, min(args.steps, 20)))
    pkg.hca_tuning_set(d, None)
    if not torch.equal(auto_lab, labels):
        raise RuntimeError("autotuned and default tuning disagree")
    auto = max_over_ranks(statistics.median(auto_ms), dist, dev)

    # d <= 4: the same clustering as a plan (declared extents = the data's, captured once as a
    # CUDA graph, one graph launch per step, no host round trip inside the call)
    graph = None
    if d <= 4:
        with pkg.Plan(pts, eps, min_pts, X.min(axis=0), X.max(axis=0)) as plan:
            for _ in range(2):
                plan.launch(stream)
                plan.wait(stream)
            g_ms, _ = time_steps(torch, stream, flush, lambda: plan.launch(stream), max(3, min(args.steps, 20)))
            plan.wait(stream)
            if not torch.equal(plan.labels, labels):
                raise RuntimeError("plan and call disagree")
        gm = max_over_ranks(statistics.median(g_ms), dist, dev)
        graph = {"ms_per_step": gm, "value": replica_value(n, ws, gm),
                 "path": "hca_plan_create with the data's extents; hca_plan_launch = one CUDA graph launch",
                 "labels": "identical to the call"}

    configs = None
    if ws == 1 and not args.no_extras and name == "mixed3d":
        k_small = max(3, min(args.steps, 20))
        configs = {
            "c1_blobs2d": config_c1(pkg, torch, stream, flush, k_small, args.warmup),
            "c3_aniso16d": config_c3(pkg, torch, stream, flush, max(3, min(args.steps, 10)), args.warmup,
                                     bf16_burst, peak_kind),
            "batched": config_batched(pkg, torch, stream, flush, max(2, min(args.steps, 4)), 1, args.sets),
            "serving": config_serving(pkg, torch, 10.0, 2.0, args.rate, args.workers, 64, plain_jobs=150,
                                      plain_seconds=15.0, burst_jobs=64),
            "literal_ablation": config_literal(pkg, torch, stream),
        }

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    C, P = stats["n_cells"], stats["n_pencils"]
    key_bytes = 4 if stats["key_bits"] <= 32 else 8
    med = {k: statistics.median(v) for k, v in stage_ms.items()}
    med_tc = {k: statistics.median(v) for k, v in tc_ms.items()}
    dominant = max(med, key=med.get)
    roof_rows = {}
    for k, t in med.items():
        b = stage_bytes(k, n, d, C, P, stats["sort_passes"], key_bytes, stats["n_core_cells"], X.dtype.itemsize)
        if b is not None and t > 0:
            roof_rows[k] = {"ms": t, "bytes": b, "gbs": b / (t / 1e3) / 1e9}
    if d <= 4:
        traffic = SORT_PASS_TRAFFIC_MIXED3D_2M if (name == "mixed3d" and n == 2_000_000) else None
        roofline = sort_roofline(stats, med, n, hbm_peak, peak_kind, traffic)
    else:
        roofline = tensor_roofline(stats, med_tc, d, bf16_burst, peak_kind)

    line = {
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if X.dtype == np.float32 else "f64", "data": "synthetic",
        "config": {"workload": name + ": " + desc, "n": n, "d": d, "eps": eps,
                   "min_pts": min_pts, "l2": "flushed between steps (256 MiB write)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "e2e": {"value": replica_value(n, ws, 1e3 * e2e_s), "unit": "points/s", "h2d_bytes_per_step": int(X.nbytes),
                "d2h_bytes_per_step": 4 * n},
        "gpu_launches": int(call_stats["kernel_launches"]) * args.steps,
        "path": ("hca_dbscan_device, the default call: the extents measured on the device and read "
                 "back, then the repeated call's CUDA graph replayed (captured by the library on the "
                 "second identical call; every kernel runs every step)"),
        "direct_launches": {"ms_per_step": direct, "value": n * ws / (direct / 1e3),
                            "path": "the same call with HCA_FLAG_NO_GRAPH_CACHE: each kernel launched "
                                    "by the host in turn", "labels": "identical"},
        "roofline": roofline,
        "stage_ms": med, "dominant_stage": dominant,
        "stage_gbs": {k: round(v["gbs"], 1) for k, v in roof_rows.items()},
        "stage_frac_of_hbm": {k: round(v["gbs"] / hbm_peak, 3) for k, v in roof_rows.items()},
        "pair_tests": pair_rates(stats, med, d) if d <= 4 else None,
        "clocks": clocks.summary(),
        "result": {"cells": C, "pencils": P, "dense_cells": stats["n_dense_cells"],
                   "core_points": stats["n_core_points"], "clusters": stats["n_clusters"],
                   "noise": stats["n_noise"]},
        "work": {k: stats[k] for k in ("n_count_chunks", "n_rep_tests", "n_rep_hits",
                                       "n_exhaustive_pairs", "n_exhaustive_chunks", "n_border_chunks",
                                       "n_tc_tiles", "n_tc_rechecks", "n_tc_pairs")},
        "autotuned": {"ms_per_step": auto, "value": n * ws / (auto / 1e3), "tuning": tune,
                      "tuning_seconds": tune_s, "labels": "identical to the default tuning"},
        "graph_plan": graph,
        "plain_fp64_gpu": {"ms_per_step": plain, "value": n * ws / (plain / 1e3), "unit": "points/s",
                           "speedup_of_tuned": plain / ms,
                           "path": "same library, HCA_FLAG_FP64_ONLY | HCA_FLAG_NO_TENSOR_CORES, "
                                   "labels identical"},
        "wall_s": wall,
    }
    if configs is not None:
        line["configs"] = configs
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline_oracle(X, eps, min_pts)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_batched(args):
    import torch
    import paper_1912_00323_gb300 as pkg
    from paper_1912_00323_gb300 import build as pkg_build
    pkg_build.build()
    pkg.load()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    r = config_batched(pkg, torch, torch.cuda.current_stream(), flush, args.steps, args.warmup, args.sets)
    line = {"metric": "points clustered/sec, batched sets (labels equal to separate calls)",
            "n_gpus": 1, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", **r}
    print(json.dumps(line), flush=True)
    return 0


def run_serving(args):
    import torch
    import paper_1912_00323_gb300 as pkg
    from paper_1912_00323_gb300 import build as pkg_build
    pkg_build.build()
    pkg.load()
    r = config_serving(pkg, torch, args.seconds, args.warmup_seconds, args.rate, args.workers, args.pool,
                       exact_rate=args.exact_rate)
    line = {"metric": "serving: p50/p99 submit-to-labels latency and points/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic", **r}
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
