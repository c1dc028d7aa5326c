"""Reader for the hand-derived fixtures in tests/golden/ (no clustering arithmetic here)."""
import glob
import os

import numpy as np

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(path):
    rows = [l.split() for l in open(path) if l.strip() and not l.lstrip().startswith("#")]
    d, n = int(rows[0][0]), int(rows[0][1])
    eps, min_pts = float(rows[0][2]), int(rows[0][3])
    X = np.array([[float(v) for v in r] for r in rows[1:1 + n]], dtype=np.float64).reshape(n, d)
    expected = {r[0]: np.array([int(v) for v in r[1:]], dtype=np.int64) for r in rows[1 + n:]}
    return X, eps, min_pts, expected


def all_cases():
    return sorted(glob.glob(os.path.join(GOLDEN_DIR, "*.txt")))
