"""Pins of the brute-force oracle to things other than itself: library routines (scikit-learn
DBSCAN, scipy connected components), closed forms, and exact invariances of the definitions."""
import numpy as np
import pytest

from paper_1912_00323_gb300 import workloads


def canonical_from_partition(groups, n):
    """Canonical ids from a partition given as an array of group ids (-1 = none)."""
    out = np.full(n, -1, np.int64)
    for g in np.unique(groups[groups >= 0]):
        idx = np.flatnonzero(groups == g)
        out[idx] = idx.min()
    return out


@pytest.mark.parametrize("d,seed", [(2, 1), (3, 2), (5, 3)])
def test_bruteforce_vs_sklearn(oracle_mod, d, seed):
    skl = pytest.importorskip("sklearn.cluster")
    r = np.random.Generator(np.random.PCG64(seed))
    X = np.concatenate([r.normal(r.uniform(0, 20, d), 1.0, size=(300, d)) for _ in range(4)]
                       + [r.uniform(0, 20, size=(300, d))])
    eps, min_pts = 0.9 + 0.2 * d, 6
    labels, core = oracle_mod.bruteforce(X, eps, min_pts)
    db = skl.DBSCAN(eps=eps, min_samples=min_pts, algorithm="kd_tree").fit(X)
    core_ref = np.zeros(len(X), np.uint8)
    core_ref[db.core_sample_indices_] = 1
    np.testing.assert_array_equal(core, core_ref)
    ref = db.labels_.copy()
    ref[core_ref == 0] = -1                   # compare the core partition exactly
    ours = labels.copy()
    ours[core == 0] = -1
    np.testing.assert_array_equal(ours, canonical_from_partition(ref, len(X)))
    # noise is the same set; a border point's id is the smallest of its candidate clusters,
    # so it can only be <= the canonical id of the cluster scikit-learn picked
    np.testing.assert_array_equal(labels < 0, db.labels_ < 0)
    canon_of_skl = {}
    for g in np.unique(db.labels_[db.labels_ >= 0]):
        canon_of_skl[g] = np.flatnonzero((db.labels_ == g) & (core_ref == 1)).min()
    border = np.flatnonzero((core == 0) & (labels >= 0))
    assert len(border) > 0
    for p in border:
        assert labels[p] <= canon_of_skl[db.labels_[p]]


@pytest.mark.parametrize("d", [1, 2, 4])
def test_minpts_one_is_eps_graph_components(oracle_mod, d):
    """MINPTS = 1: every point is core, clusters = connected components of the eps-graph."""
    sp = pytest.importorskip("scipy.spatial")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    import scipy.sparse as sparse
    r = np.random.Generator(np.random.PCG64(10 + d))
    X = r.uniform(0, 10, size=(800, d))
    eps = 0.35 * d
    labels, core = oracle_mod.bruteforce(X, eps, 1)
    pairs = np.array(sorted(sp.cKDTree(X).query_pairs(eps)), dtype=np.int64).reshape(-1, 2)
    g = sparse.coo_matrix((np.ones(len(pairs)), (pairs[:, 0], pairs[:, 1])), shape=(800, 800))
    _, comp = csg.connected_components(g, directed=False)
    assert core.all()
    np.testing.assert_array_equal(labels, canonical_from_partition(comp, 800))


@pytest.mark.parametrize("n,min_pts", [(7, 3), (7, 8), (1, 1), (1, 2)])
def test_identical_points_closed_form(oracle_mod, n, min_pts):
    X = np.full((n, 3), 2.5)
    for f in (oracle_mod.bruteforce, oracle_mod.grid):
        labels, core = f(X, 0.1, min_pts)
        if n >= min_pts:
            assert core.all() and (labels == 0).all()
        else:
            assert not core.any() and (labels == -1).all()


@pytest.mark.parametrize("npts", [5, 6, 12])
def test_evenly_spaced_line_closed_form(oracle_mod, npts):
    """Points k*h on a line, eps = 2h: interior points have 5 neighbours, the two ends 3 and
    the next ones 4.  With MINPTS = 5, points 2..n-3 are core (one cluster, id 2) and the four
    outer points are its border."""
    h = 0.25
    X = (np.arange(npts) * h)[:, None]
    for f in (oracle_mod.bruteforce, oracle_mod.grid):
        labels, core = f(X, 2 * h, 5)
        exp_core = np.zeros(npts, np.uint8)
        exp_core[2:npts - 2] = 1
        np.testing.assert_array_equal(core, exp_core)
        exp = np.full(npts, 2 if npts > 4 else -1)
        if exp_core.sum() == 0:
            exp[:] = -1
        np.testing.assert_array_equal(labels, exp)


def _canon_under_perm(labels, core, perm, X, eps):
    """Expected labels after reordering the points by perm (new i = old perm[i])."""
    n = len(perm)
    inv = np.empty(n, np.int64)
    inv[perm] = np.arange(n)
    old_core = core.astype(bool)
    # clusters of core points: old canonical id -> min new index among its core points
    new_id = {}
    for lab in np.unique(labels[old_core]):
        members = np.flatnonzero((labels == lab) & old_core)
        new_id[lab] = inv[members].min()
    out = np.full(n, -1, np.int64)
    for i in range(n):
        p = perm[i]
        if old_core[p]:
            out[i] = new_id[labels[p]]
    d2 = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    for i in range(n):
        p = perm[i]
        if old_core[p]:
            continue
        nb = np.flatnonzero((d2[p] <= eps * eps) & old_core)
        if len(nb):
            out[i] = min(new_id[labels[q]] for q in nb)
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_permutation_invariance(oracle_mod, seed):
    X, eps, min_pts = workloads.lattice(400, 2, seed=seed, spread=3.0, box=20.0)
    labels, core = oracle_mod.bruteforce(X, eps, min_pts)
    perm = np.random.Generator(np.random.PCG64(99 + seed)).permutation(len(X))
    l2, c2 = oracle_mod.bruteforce(X[perm], eps, min_pts)
    np.testing.assert_array_equal(c2, core[perm])
    np.testing.assert_array_equal(l2, _canon_under_perm(labels, core, perm, X, eps))


@pytest.mark.parametrize("seed", [0, 1])
def test_translation_and_power_of_two_scaling(oracle_mod, seed):
    """Lattice coordinates: translating by a lattice multiple and scaling coordinates and eps
    by 2^k leave every squared distance exact, so labels must be identical."""
    X, eps, min_pts = workloads.lattice(500, 3, seed=seed, spread=3.0, box=20.0)
    base = oracle_mod.bruteforce(X, eps, min_pts)
    for Y, e in ((X + 37.25, eps), (X - 1024.5, eps), (X * 8.0, eps * 8.0), (X / 4.0, eps / 4.0)):
        out = oracle_mod.bruteforce(Y, e, min_pts)
        np.testing.assert_array_equal(out[0], base[0])
        np.testing.assert_array_equal(out[1], base[1])
