"""How far the paper's algorithms as printed drift from DBSCAN on the synthetic workloads.

Test infrastructure, CPU only: it runs `hca_oracle_literal` (Algorithms 2-4 as printed:
representative points only, strict "<", no MINPTS, Sec. 2) beside `hca_oracle_grid` (exact
DBSCAN, Definitions 1-5) on seeded inputs and reports, per workload:

  noise_clustered  points DBSCAN labels noise (-1) that the printed algorithm puts in a cluster
                   (it has no MINPTS, so every non-empty hypercube belongs to some cluster);
  split            DBSCAN clusters whose core points fall into more than one printed cluster
                   (representative points miss a pair of neighbouring cubes that has a core
                   pair within eps);
  merged           printed clusters that hold core points of more than one DBSCAN cluster
                   (cubes joined through non-core points);
  points_moved     points whose printed cluster is not the one holding most of their DBSCAN
                   cluster's core points (noise points excluded).

usage: python -m oracle.literal_report [--max-n N]
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
from paper_1912_00323_gb300 import workloads  # noqa: E402


def compare(X, eps, min_pts):
    X = np.ascontiguousarray(X, dtype=np.float64)
    db, core = oracle.grid(X, eps, min_pts)
    lit = oracle.literal(X, eps)
    core = core.astype(bool)
    noise_clustered = int(np.sum((db < 0) & (lit >= 0)))
    split = 0
    majority = {}
    for cid in np.unique(db[core]):
        members = lit[core & (db == cid)]
        vals, cnt = np.unique(members, return_counts=True)
        split += int(len(vals) > 1)
        majority[int(cid)] = int(vals[np.argmax(cnt)])
    merged = 0
    for lid in np.unique(lit[core]):
        merged += int(len(np.unique(db[core & (lit == lid)])) > 1)
    clustered = db >= 0
    moved = sum(int(lit[i] != majority[int(db[i])]) for i in np.flatnonzero(clustered))
    return {"n": int(len(X)), "d": int(X.shape[1]), "eps": float(eps), "min_pts": int(min_pts),
            "dbscan_clusters": int(len(majority)), "printed_clusters": int(len(np.unique(lit))),
            "dbscan_noise": int(np.sum(db < 0)), "noise_clustered": noise_clustered,
            "split": split, "merged": merged, "points_moved": int(moved)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--max-n", type=int, default=200_000,
                    help="largest prefix of a workload that is compared (the printed algorithm "
                         "has no MINPTS, so a prefix is a sparser but valid input)")
    args = ap.parse_args()
    oracle.build()
    rows = {}
    X, e, m = workloads.blobs2d()
    rows["blobs2d"] = compare(X, e, m)
    X, e, m = workloads.mixed3d()
    rows[f"mixed3d (first {args.max_n:,} points)"] = compare(X[:args.max_n], e, m)
    for k, (X, e, m) in enumerate(workloads.batched_sets(n_sets=6, n_min=1_000, n_max=20_000, dims=(2, 3))):
        rows[f"batched set {k}"] = compare(X, e, m)
    for name, r in rows.items():
        print(json.dumps({"workload": name, **r}))


if __name__ == "__main__":
    main()
