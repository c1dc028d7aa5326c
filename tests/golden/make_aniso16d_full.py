"""Write aniso16d_full.npz: the oracle's labels and core flags for the full 16-D workload
(workloads.aniso16d(): n = 1,000,000 float32 points on the 2^-12 lattice, 100 anisotropic
Gaussian clusters + 10% noise, eps = 4, MINPTS = 20), with the SHA-256 of the coordinates they
belong to.  The labels follow Definitions 1-5 of the paper's DBSCAN supplement with the canonical
ids of the oracle.  This script calls only the oracle (hca_oracle_grid_mt on every host core) and
the input generator.

    python tests/golden/make_aniso16d_full.py
"""
import hashlib
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1912_00323_gb300 import workloads  # noqa: E402

OUT = os.path.join(HERE, "aniso16d_full.npz")


def encode(labels, core):
    """Labels as uint8 codes into their sorted distinct values (at most 256), core flags as bits."""
    values = np.unique(labels)
    if len(values) > 256:
        raise ValueError("more than 256 distinct labels")
    codes = np.searchsorted(values, labels).astype(np.uint8)
    return values.astype(np.int32), codes, np.packbits(core.astype(np.uint8))


def decode(npz):
    n = int(npz["n"])
    labels = npz["label_values"][npz["label_codes"]].astype(np.int32)
    core = np.unpackbits(npz["core_bits"])[:n].astype(np.uint8)
    return labels, core


def input_sha256(X):
    return hashlib.sha256(np.ascontiguousarray(X).tobytes()).hexdigest()


def main():
    X, eps, min_pts = workloads.aniso16d()
    t0 = time.time()
    labels, core = oracle.grid(X.astype(np.float64), eps, min_pts, threads=0)
    secs = time.time() - t0
    values, codes, bits = encode(labels, core)
    np.savez_compressed(OUT, sha256=input_sha256(X), n=len(X), eps=eps, min_pts=min_pts,
                        label_values=values, label_codes=codes, core_bits=bits)
    print(f"wrote {OUT}: {len(values) - (values[0] < 0)} clusters, {int(core.sum())} core points, "
          f"{int((labels < 0).sum())} noise points; oracle {secs:.0f} s on {os.cpu_count()} threads")


if __name__ == "__main__":
    main()
