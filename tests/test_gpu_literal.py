"""The GPU form of the paper's Algorithms 2-4 as printed (hca_dbscan_literal_device, an
ablation): labels equal to the oracle's literal variant element by element, on the hand-derived
4-point case where representative points split a DBSCAN cluster, on lattice data with pairs at
exactly eps (the printed "<" decides them), on blobs2d, on a 200,000-point prefix of mixed3d and
on batched sets; and where it departs from DBSCAN on those inputs."""
import os

import numpy as np
import pytest

from golden_io import GOLDEN_DIR, load
from paper_1912_00323_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_00323_gb300 import build
    build.build()
    import oracle
    oracle.build()
    import paper_1912_00323_gb300 as pkg
    pkg.load()
    return torch, pkg, oracle


def gpu_literal(env, X, eps, dtype=None):
    torch, pkg, _ = env
    t = torch.from_numpy(np.ascontiguousarray(X if dtype is None else X.astype(dtype))).cuda()
    return pkg.hca_dbscan_literal_device(t, eps).cpu().numpy()


def test_rep_counterexample_splits_a_cluster(env):
    X, eps, mp, exp = load(os.path.join(GOLDEN_DIR, "rep_counterexample_2d.txt"))
    got = gpu_literal(env, X, eps)
    np.testing.assert_array_equal(got, exp["literal"])
    assert len(np.unique(got)) == 2


@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_lattice_ties(env, d, dtype):
    _, _, oracle = env
    X, eps, _ = workloads.lattice(4000, d, seed=800 + d, step=0.25, eps_steps=4, spread=3.0, box=12.0)
    np.testing.assert_array_equal(gpu_literal(env, X, eps, dtype), oracle.literal(X, eps))


def test_blobs2d_and_mixed3d_prefix(env):
    _, _, oracle = env
    X, eps, _ = workloads.blobs2d()
    np.testing.assert_array_equal(gpu_literal(env, X, eps), oracle.literal(X, eps))
    X, eps, _ = workloads.mixed3d()
    X = X[:200_000]
    np.testing.assert_array_equal(gpu_literal(env, X, eps), oracle.literal(X.astype(np.float64), eps))


def test_batched_sets(env):
    _, _, oracle = env
    for X, eps, _ in workloads.batched_sets(n_sets=6, n_min=1_000, n_max=20_000, dims=(2, 3)):
        np.testing.assert_array_equal(gpu_literal(env, X, eps), oracle.literal(X.astype(np.float64), eps))


def test_departs_from_dbscan_by_clustering_noise(env):
    """No MINPTS in the printed algorithm: DBSCAN's noise points all land in clusters."""
    torch, pkg, _ = env
    X, eps, mp = workloads.blobs2d()
    lit = gpu_literal(env, X, eps)
    db = pkg.hca_dbscan_device(torch.from_numpy(X).cuda(), eps, mp).cpu().numpy()
    assert (lit >= 0).all()
    assert (db < 0).sum() > 0
    assert len(np.unique(lit)) > len(np.unique(db[db >= 0]))
