"""Tunings change how the exact result is computed, never the result: the coarse-grid
neighbour search forced at d = 3 and 4, extreme tensor-core splits, and the autotuners, each
checked element by element against the CPU oracle."""
import math

import numpy as np
import pytest

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
    yield torch, pkg, oracle
    for d in range(1, 65):
        pkg.hca_tuning_set(d, None)


@pytest.fixture(autouse=True)
def reset(env):
    yield
    for d in range(1, 65):
        env[1].hca_tuning_set(d, None)


def run(env, X, eps, mp):
    torch, pkg, _ = env
    t = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    core = torch.empty(len(X), dtype=torch.uint8, device="cuda")
    lab = pkg.hca_dbscan_device(t, eps, mp, core=core)
    return lab.cpu().numpy(), core.cpu().numpy()


def check(got, want):
    np.testing.assert_array_equal(got[0], want[0])
    np.testing.assert_array_equal(got[1], want[1])


@pytest.mark.parametrize("d", [3, 4])
@pytest.mark.parametrize("min_pts", [1, 4, 12])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_coarse_grid_at_low_d(env, d, min_pts, dtype):
    _, pkg, oracle = env
    X, eps, _ = workloads.lattice(3000, d, seed=40 + d, step=0.25, eps_steps=4, spread=3.0, box=12.0)
    want = oracle.grid(X, eps, min_pts)
    pkg.hca_tuning_set(d, {"path": 2})
    check(run(env, X.astype(dtype), eps, min_pts), want)
    pkg.hca_tuning_set(d, {"path": 1})
    check(run(env, X.astype(dtype), eps, min_pts), want)


def test_coarse_grid_mixed3d_reduced(env):
    _, pkg, oracle = env
    X, eps, mp = workloads.mixed3d(n=60_000)
    want = oracle.grid(X.astype(np.float64), eps, mp)
    pkg.hca_tuning_set(3, {"path": 2})
    check(run(env, X, eps, mp), want)


@pytest.mark.parametrize("tune", [
    {"tc_min_count": 1, "tc_min_merge": 1, "tc_min_labels": 1, "tc_handoff": 0, "first_links": 0},
    {"tc_min_count": 1, "tc_min_merge": 1, "tc_min_labels": 1, "tc_handoff": 127, "first_links": 1},
    {"tc_min_count": 1 << 30, "tc_min_merge": 1 << 30, "tc_min_labels": 1 << 30},
    {"tc_min_count": 200, "tc_min_merge": 3, "tc_min_labels": 50, "tc_handoff": 30, "first_links": 0},
    {"cta_warps": 2, "first_links": 0},
    {"cta_warps": 8, "tc_min_count": 1 << 30, "tc_min_merge": 1 << 30, "tc_min_labels": 1 << 30}])
@pytest.mark.parametrize("d", [8, 16, 40])
def test_extreme_splits(env, tune, d):
    _, pkg, oracle = env
    X, eps, _ = workloads.lattice(3000, d, seed=700 + d, step=0.25,
                                  eps_steps=int(round(math.sqrt(2 * d) * 1.8)), spread=2.0, box=2.0 * d,
                                  n_blobs=3)
    want = oracle.grid(X, eps, 5)
    pkg.hca_tuning_set(d, tune)
    check(run(env, X.astype(np.float32), eps, 5), want)


@pytest.mark.parametrize("warps", [2, 8])
@pytest.mark.parametrize("d", [6, 40])
def test_cta_warps_double_input(env, warps, d):
    """Double input keeps every phase on the CUDA-core chunk kernels: each CTA size gives the
    oracle's labels (d = 40 pads rows to 64 doubles: 128 KiB of rows per 8-warp CTA)."""
    _, pkg, oracle = env
    X, eps, _ = workloads.lattice(2500, d, seed=900 + d, step=0.25,
                                  eps_steps=int(round(math.sqrt(2 * d) * 1.8)), spread=2.0, box=2.0 * d,
                                  n_blobs=3)
    want = oracle.grid(X, eps, 5)
    pkg.hca_tuning_set(d, {"cta_warps": warps})
    check(run(env, X, eps, 5), want)


def test_autotune_keeps_labels(env):
    torch, pkg, oracle = env
    X, eps, mp = workloads.aniso16d(n=20_000, n_clusters=20)
    want = oracle.grid(X.astype(np.float64), eps, mp)
    t = torch.from_numpy(X).cuda()
    tune, ms = pkg.hca_autotune(t, eps, mp, repeats=1)
    assert ms > 0 and tune["path"] == 2
    assert tune["cta_warps"] in (2, 4, 8) and tune["tc_handoff"] in (8, 16, 32, 64)
    assert pkg.hca_tuning_get(16) == tune
    check(run(env, X, eps, mp), want)


def test_autotune_batched_low_d(env):
    torch, pkg, oracle = env
    sets = workloads.batched_sets(n_sets=40, n_min=200, n_max=8000, dims=(3,), seed=33)
    X = np.concatenate([s[0] for s in sets], axis=0)
    off = np.zeros(len(sets) + 1, np.int64)
    off[1:] = np.cumsum([len(s[0]) for s in sets])
    eps = [s[1] for s in sets]
    mp = [s[2] for s in sets]
    t = torch.from_numpy(X).cuda()
    tune, ms = pkg.hca_autotune_batched(t, off, eps, mp, repeats=1)
    assert set(tune) == {3} and tune[3]["path"] in (1, 2) and ms > 0
    for path in (1, 2):
        pkg.hca_tuning_set(3, {"path": path})
        lab = pkg.hca_dbscan_batched(t, off, eps, mp).cpu().numpy()
        for s in range(0, len(sets), 5):
            want = oracle.grid(sets[s][0].astype(np.float64), eps[s], mp[s])
            np.testing.assert_array_equal(lab[off[s]:off[s + 1]], want[0], err_msg=f"path {path} set {s}")
