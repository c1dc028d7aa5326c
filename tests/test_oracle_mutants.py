"""Plant one mistake at a time in a copy of the oracle (on the CPU) and check that the pins
catch it: the golden fixtures, the scikit-learn / scipy cross-checks and the agreement of
the two oracle algorithms.  A pin set that let one of these through would be too weak."""
import os

import numpy as np
import pytest

from golden_io import all_cases, load
from paper_1912_00323_gb300 import workloads

MUTANTS = {
    # Definition 1 reads "<= eps"; strict "<" is the paper's Sec. 2 wording
    "strict_less": ("return s <= eps2;", "return s < eps2;"),
    # a dropped index: every coordinate compared against coordinate 0 of q
    "wrong_index": ("double t = p[i] - q[i];", "double t = p[i] - q[0];"),
    # a dropped term: the last coordinate left out of the sum
    "dropped_term": ("for (int i = 0; i < d; ++i) {\n        double t = p[i] - q[i];",
                     "for (int i = 0; i < d - 1; ++i) {\n        double t = p[i] - q[i];"),
    # |N_eps(p)| without p itself
    "no_self": ("c += le_eps(j->X + p * j->d, j->X + q * j->d, j->d, j->eps2);",
                "c += (q != p) && le_eps(j->X + p * j->d, j->X + q * j->d, j->d, j->eps2);"),
    # border point takes the largest instead of the smallest cluster id
    "border_max": ("if (best < 0 || l < best) best = l;", "if (best < 0 || l > best) best = l;"),
    # cluster id = index of the point that reached it, not the component's smallest index
    "bfs_label": ("labels[q] = (int32_t)p;", "labels[q] = (int32_t)u;"),
    # grid: neighbour stencil too small
    "small_stencil": ("keep = gap2 <= eps * eps * (1.0 + 1e-6);", "keep = gap2 <= eps * eps * 0.25;"),
    # grid: hypercube side eps instead of eps/sqrt(d) (diagonal above eps)
    "wide_cube": ("return eps / sqrt((double)d) * (1.0 - 1.0 / 1048576.0);",
                  "return eps * (1.0 - 1.0 / 1048576.0);"),
    # grid: a border point ignores the core points of its own hypercube
    "border_own_cube": ("int64_t best = c->cell_label[own];", "int64_t best = INT64_MAX;"),
    # grid, threaded merging: the pairs joined by the calling thread are not carried over
    "lost_thread_merges": ("for (int t = 0; t < threads; ++t) {\n        if (jobs[t].rc) goto done;",
                           "for (int t = 1; t < threads; ++t) {\n        if (jobs[t].rc) goto done;"),
    # grid, counts: the early stop one short of MINPTS
    "count_stops_early": ("c->core[p] = cnt >= c->min_pts;", "c->core[p] = cnt >= c->min_pts - 1;"),
}


def _pins_hold(o):
    grid3 = lambda X, eps, mp: o.grid(X, eps, mp, threads=3)   # noqa: E731
    for path in all_cases():
        X, eps, min_pts, exp = load(path)
        for f in (o.bruteforce, o.grid, grid3):
            lab, core = f(X, eps, min_pts)
            if not (np.array_equal(lab, exp["labels"]) and np.array_equal(core, exp["core"])):
                return False
    for d, seed in ((2, 5), (3, 6), (1, 7), (5, 8)):
        X, eps, mp = workloads.lattice(300, d, seed=seed, spread=2.0 + d, box=6.0 + 3 * d)
        a = o.bruteforce(X, eps, mp)
        for b in (o.grid(X, eps, mp), grid3(X, eps, mp)):
            if not (np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])):
                return False
    skl = pytest.importorskip("sklearn.cluster")
    r = np.random.Generator(np.random.PCG64(3))
    X = np.concatenate([r.normal(r.uniform(0, 10, 2), 0.7, size=(150, 2)) for _ in range(3)]
                       + [r.uniform(0, 10, size=(100, 2))])
    lab, core = o.bruteforce(X, 0.5, 5)
    db = skl.DBSCAN(eps=0.5, min_samples=5, algorithm="kd_tree").fit(X)
    ref_core = np.zeros(len(X), np.uint8)
    ref_core[db.core_sample_indices_] = 1
    return np.array_equal(core, ref_core) and np.array_equal(lab < 0, db.labels_ < 0)


def test_unmodified_copy_passes(oracle_mod, tmp_path):
    assert _pins_hold(oracle_mod.compile_variant(oracle_mod.source_text(), str(tmp_path)))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(oracle_mod, tmp_path, name):
    old, new = MUTANTS[name]
    src = oracle_mod.source_text()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    o = oracle_mod.compile_variant(src.replace(old, new), str(tmp_path))
    assert not _pins_hold(o), f"planted mistake '{name}' passed every pin"
