"""The hypercube oracle (Sec. 2, Algorithms 1-4 with MINPTS) against the brute-force
definitions, plus the structural facts the paper states about the hypercube grid."""
import math

import numpy as np
import pytest

from paper_1912_00323_gb300 import workloads


CASES = [(d, seed, mp) for d in (1, 2, 3, 4, 5, 6) for seed in (0, 1) for mp in (1, 3, 6)]


@pytest.mark.parametrize("d,seed,min_pts", CASES)
def test_grid_equals_bruteforce_on_lattice_ties(oracle_mod, d, seed, min_pts):
    X, eps, _ = workloads.lattice(600, d, seed=100 * d + seed, spread=2.0 + d, box=8.0 + 4 * d)
    a = oracle_mod.bruteforce(X, eps, min_pts)
    for threads in (1, 4):
        b = oracle_mod.grid(X, eps, min_pts, threads=threads)
        np.testing.assert_array_equal(b[1], a[1])
        np.testing.assert_array_equal(b[0], a[0])


@pytest.mark.parametrize("name,n", [("blobs2d", 3000), ("mixed3d", 6000), ("aniso16d", 3000)])
def test_grid_equals_bruteforce_on_workload_recipes(oracle_mod, name, n):
    X, eps, min_pts = workloads.WORKLOADS[name](n=n)
    if name == "aniso16d":
        X, eps, min_pts = workloads.aniso16d(n=n, n_clusters=5)
    a = oracle_mod.bruteforce(X.astype(np.float64), eps, min_pts)
    assert a[1].any() and (a[0] < 0).any()       # not degenerate: core and noise present
    for threads in (1, 3, 8):
        b = oracle_mod.grid(X.astype(np.float64), eps, min_pts, threads=threads)
        np.testing.assert_array_equal(b[1], a[1])
        np.testing.assert_array_equal(b[0], a[0])


@pytest.mark.parametrize("name,n", [("mixed3d", 40_000), ("aniso16d", 20_000)])
def test_threaded_grid_equals_one_thread(oracle_mod, name, n):
    """Larger than the brute-force cases: the threaded counts, merging and border points
    give the one-thread result (each thread's merges are joined into one union-find)."""
    X, eps, min_pts = workloads.WORKLOADS[name](n=n)
    if name == "aniso16d":
        X, eps, min_pts = workloads.aniso16d(n=n, n_clusters=10)
    X = X.astype(np.float64)
    a = oracle_mod.grid(X, eps, min_pts, threads=1)
    b = oracle_mod.grid(X, eps, min_pts, threads=6)
    assert len(np.unique(a[0][a[0] >= 0])) > 2
    np.testing.assert_array_equal(b[1], a[1])
    np.testing.assert_array_equal(b[0], a[0])


def test_paper_neighbour_count_2d(oracle_mod):
    """Sec. 2 ('Depth First Search'): 20 neighbour hypercubes in 2-D.  Both the printed
    formula (2*ceil(sqrt(d))+1)^d - (C+1) and the exact geometric rule with strict '<' give 20."""
    assert oracle_mod.stencil_count(2, 0) == 20
    assert oracle_mod.stencil_count(2, 1) == 20


def test_exact_rule_extends_the_formula(oracle_mod):
    # d=1: offsets +-1, +-2 minus nothing (the corner of a 1-cube block is its end) -> strict rule
    assert oracle_mod.stencil_count(1, 1) == 2
    assert oracle_mod.stencil_count(3, 1) == 5 ** 3 - 8 - 1
    assert oracle_mod.stencil_count(4, 1) == 608


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_conservative_stencil_is_a_superset(oracle_mod, d):
    """The oracle's stencil (<= with the shrunk side) includes every strict-rule offset."""
    eps = 1.5
    side = eps / math.sqrt(d) * (1 - 2 ** -20)
    assert oracle_mod.stencil_count(d, 2, side, eps) >= oracle_mod.stencil_count(d, 1)
    if d == 2:
        assert oracle_mod.stencil_count(d, 2, side, eps) == 24   # 5x5 block minus the cube itself


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_representative_directions(oracle_mod, d):
    """Sec. 2: 3^d - 1 representative points per hypercube (8 in 2-D: Top, TopRight, ...)."""
    dirs = oracle_mod.rep_dirs(d)
    assert len(dirs) == 3 ** d - 1
    assert len({tuple(r) for r in dirs}) == len(dirs)
    assert not (dirs == 0).all(axis=1).any()
    # complementary direction of row k is row (3^d - 2 - k)
    np.testing.assert_array_equal(dirs[::-1], -dirs)


@pytest.mark.parametrize("name,n", [("blobs2d", 4000), ("mixed3d", 4000)])
def test_hypercube_diameter_at_most_eps(oracle_mod, name, n):
    """Sec. 2 / Conclusion: all points of one hypercube lie within eps of each other."""
    X, eps, _ = workloads.WORKLOADS[name](n=n)
    X = X.astype(np.float64)
    cells = oracle_mod.grid_cells(X, eps)
    _, inv = np.unique(cells, axis=0, return_inverse=True)
    inv = inv.ravel()
    order = np.argsort(inv, kind="stable")
    bounds = np.flatnonzero(np.diff(inv[order])) + 1
    worst = 0.0
    for grp in np.split(order, bounds):
        if len(grp) < 2:
            continue
        P = X[grp]
        worst = max(worst, ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1).max())
    assert worst <= eps * eps


def test_literal_is_not_dbscan_in_general(oracle_mod):
    """The printed algorithm has no MINPTS, so on data with noise it labels noise points as
    clusters of their own: it differs from the DBSCAN definitions."""
    X, eps, min_pts = workloads.blobs2d(n=2000)
    lit = oracle_mod.literal(X, eps)
    ref, _ = oracle_mod.bruteforce(X, eps, min_pts)
    assert (lit >= 0).all() and (ref < 0).any()
