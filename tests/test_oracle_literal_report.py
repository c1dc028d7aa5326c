"""The divergence report of the printed algorithm (Algorithms 2-4 as printed) against DBSCAN:
its measures are checked on the hand-derived counterexample, where representative-only
merging splits one DBSCAN cluster, and on a case where both agree."""
import os

import numpy as np
import pytest

from golden_io import GOLDEN_DIR, load


@pytest.fixture(scope="module")
def report():
    import oracle
    oracle.build()
    from oracle import literal_report
    return literal_report


def test_counterexample_is_a_split(report):
    X, eps, min_pts, exp = load(os.path.join(GOLDEN_DIR, "rep_counterexample_2d.txt"))
    r = report.compare(X, eps, min_pts)
    assert r["dbscan_clusters"] == 1 and r["printed_clusters"] == 2
    assert r["split"] == 1 and r["merged"] == 0
    assert r["points_moved"] == 2          # the two points of the second cube
    assert r["noise_clustered"] == 0


def test_noise_is_clustered_without_minpts(report):
    # two far-apart singletons are noise for MINPTS = 2, each its own printed cluster
    X = np.array([[0.0, 0.0], [10.0, 10.0]])
    r = report.compare(X, 1.0, 2)
    assert r["dbscan_clusters"] == 0 and r["dbscan_noise"] == 2
    assert r["noise_clustered"] == 2 and r["printed_clusters"] == 2
    assert r["split"] == 0 and r["merged"] == 0 and r["points_moved"] == 0
