"""Oracle against hand-derived fixtures (tests/golden/*.txt, each citing the definitions it
follows).  Both oracle algorithms must give the fixture's labels and core flags."""
import os

import numpy as np
import pytest

from golden_io import all_cases, load


@pytest.mark.parametrize("path", all_cases(), ids=lambda p: os.path.basename(p)[:-4])
def test_bruteforce_matches_fixture(oracle_mod, path):
    X, eps, min_pts, exp = load(path)
    labels, core = oracle_mod.bruteforce(X, eps, min_pts, threads=1)
    np.testing.assert_array_equal(labels, exp["labels"])
    np.testing.assert_array_equal(core, exp["core"])


@pytest.mark.parametrize("path", all_cases(), ids=lambda p: os.path.basename(p)[:-4])
def test_grid_matches_fixture(oracle_mod, path):
    X, eps, min_pts, exp = load(path)
    labels, core = oracle_mod.grid(X, eps, min_pts)
    np.testing.assert_array_equal(labels, exp["labels"])
    np.testing.assert_array_equal(core, exp["core"])


def test_literal_misses_the_counterexample_merge(oracle_mod):
    """Algorithm 3 with representative points only keeps the two cubes apart (the fixture's
    'literal' row), while DBSCAN joins them."""
    from golden_io import GOLDEN_DIR
    X, eps, _, exp = load(os.path.join(GOLDEN_DIR, "rep_counterexample_2d.txt"))
    np.testing.assert_array_equal(oracle_mod.literal(X, eps), exp["literal"])
