"""The tensor-core distance tiles of the d >= 5 float path (tcgen05 kind::tf32 with a guard
band and exact rechecks): element-by-element parity with the CPU oracle, equality with the
CUDA-core path, and the cases where the host keeps them off."""
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
    return torch, pkg, oracle


def run(env, X, eps, min_pts, **kw):
    torch, pkg, _ = env
    t = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    core = torch.empty(len(X), dtype=torch.uint8, device="cuda")
    lab, st = pkg.hca_dbscan_device(t, eps, min_pts, core=core, stats=True, **kw)
    return lab.cpu().numpy(), core.cpu().numpy(), st


def check(got, want):
    bad = np.flatnonzero(got[0] != want[0])
    assert len(bad) == 0, f"{len(bad)} labels differ, first at {bad[:5]}"
    np.testing.assert_array_equal(got[1], want[1])


@pytest.mark.parametrize("d", [5, 8, 12, 16, 24, 32, 40, 64])
def test_lattice_ties_on_tensor_cores(env, d):
    """Lattice sets (many pairs at exactly eps, coarse cells with several hundred points, so
    several 128-row chunks per cell and ragged last tiles), MINPTS 1, 5 and 30, with the default
    split and with every cell on the tensor cores: the tensor-core path is used, some pairs fall
    in its guard band (the first links, root links and pointer jumping can leave every union tile
    skipped, so the band is met in the labels phase), and the labels equal the oracle's."""
    _, pkg, oracle = env
    X, eps, _ = workloads.lattice(3000, d, seed=900 + d, step=0.25,
                                  eps_steps=int(round(math.sqrt(2 * d) * 1.8)), spread=2.0,
                                  box=2.0 * d, n_blobs=3)
    rechecks = 0
    for tiles_from in (None, 1):   # the default split, then every cell on the tensor cores
        if tiles_from:
            pkg.hca_tuning_set(d, {"tc_min_count": 1, "tc_min_merge": 1, "tc_min_labels": 1})
        try:
            for min_pts in (1, 5, 30):
                want = oracle.grid(X, eps, min_pts)
                got = run(env, X.astype(np.float32), eps, min_pts)
                assert got[2]["n_tc_tiles"] > 0
                rechecks += got[2]["n_tc_rechecks"]
                check(got, want)
        finally:
            pkg.hca_tuning_set(d, None)
    assert rechecks > 0


@pytest.mark.parametrize("n", [1, 2, 127, 128, 129, 255, 257, 1000])
def test_tile_edges(env, n):
    """Sizes around the 128-row tile: one dense cell, empty tails, single rows."""
    _, _, oracle = env
    r = np.random.Generator(np.random.PCG64(n))
    X = np.round(r.normal(0.0, 0.6, size=(n, 16)) * 64) / 64
    want = oracle.grid(X, 2.0, 4)
    check(run(env, X.astype(np.float32), 2.0, 4), want)


def test_far_from_origin(env):
    """Coordinates near 2^12 with a 2^-10 lattice: the centring on the chunk's first row keeps
    the filter's error relative to the spread of the chunk, not to the coordinates."""
    _, _, oracle = env
    X, eps, mp = workloads.lattice(4000, 16, seed=31, step=2.0 ** -6, eps_steps=24, spread=6.0,
                                   box=1.0, n_blobs=4)
    X = X + 4096.0
    assert np.array_equal(X.astype(np.float32).astype(np.float64), X)
    want = oracle.grid(X, eps, mp)
    got = run(env, X.astype(np.float32), eps, mp)
    assert got[2]["n_tc_tiles"] > 0
    check(got, want)


def test_huge_extent_keeps_cuda_cores(env):
    """An extent with d * extent^2 > 2^100 turns the tensor-core filter off (its FP32 norms
    could overflow); the labels stay exact."""
    _, _, oracle = env
    X, eps, mp = workloads.lattice(1500, 16, seed=5, step=2.0 ** 26, eps_steps=4, spread=2.0,
                                   box=2.0 ** 34, n_blobs=3)
    X[0, 0] = 2.0 ** 49
    want = oracle.grid(X, eps, mp)
    got = run(env, X.astype(np.float32), eps, mp)
    assert got[2]["n_tc_tiles"] == 0
    check(got, want)


@pytest.mark.parametrize("kw", [dict(tensor_cores=False), dict(fp64_only=True)])
def test_switches_off(env, kw):
    X, eps, mp = workloads.aniso16d(n=20000, n_clusters=20)
    got = run(env, X, eps, mp, **kw)
    assert got[2]["n_tc_tiles"] == 0
    ref = run(env, X, eps, mp)
    assert ref[2]["n_tc_tiles"] > 0
    check(got, ref[:2])


def test_float64_input_never_uses_tensor_cores(env):
    X, eps, mp = workloads.aniso16d(n=5000, n_clusters=5)
    got = run(env, X.astype(np.float64), eps, mp)
    assert got[2]["n_tc_tiles"] == 0


def test_aniso16d_full_equals_cuda_core_path(env):
    """Full 16-D workload (n = 1,000,000): the tensor-core path and the CUDA-core path (both
    checked against the oracle on the reduced sizes and on sampled properties at full size)
    give identical labels and core flags, also when repeated."""
    X, eps, mp = workloads.aniso16d()
    ref = run(env, X, eps, mp, tensor_cores=False)
    for _ in range(3):
        got = run(env, X, eps, mp)
        assert got[2]["n_tc_tiles"] > 0
        check(got, ref[:2])


@pytest.mark.parametrize("n,clusters", [(5000, 5), (36000, 40)])
def test_aniso16d_reduced_on_tensor_cores(env, n, clusters):
    _, _, oracle = env
    X, eps, mp = workloads.aniso16d(n=n, n_clusters=clusters)
    want = oracle.grid(X.astype(np.float64), eps, mp)
    got = run(env, X, eps, mp)
    assert got[2]["n_tc_tiles"] > 0
    check(got, want)


@pytest.mark.parametrize("n,clusters", [(20000, 1), (40000, 2)])
def test_dense_clusters_split_union_streams(env, n, clusters):
    """One or two clusters of 18,000 points: the unions' candidate streams hold more core
    points than one window (2,048), so every 128-row chunk runs as several work items; the
    labels and core flags equal the oracle's."""
    _, _, oracle = env
    X, eps, mp = workloads.aniso16d(n=n, n_clusters=clusters)
    want = oracle.grid(X.astype(np.float64), eps, mp)
    got = run(env, X, eps, mp)
    assert got[2]["n_tc_tiles"] > 0
    check(got, want)


def test_recount_windows_from_early_handoff(env):
    """Two dense clusters with the handoff at 127 open rows: nearly every row leaves its first
    tensor-core count after one block and is counted again in windows of 2,048 candidates, the
    tallies summed over the windows; labels and core flags equal the oracle's."""
    _, pkg, oracle = env
    X, eps, mp = workloads.aniso16d(n=40000, n_clusters=2)
    want = oracle.grid(X.astype(np.float64), eps, mp)
    base = pkg.hca_tuning_get(16)
    try:
        pkg.hca_tuning_set(16, dict(base, tc_handoff=127))
        got = run(env, X, eps, mp)
    finally:
        pkg.hca_tuning_set(16, None)
    assert got[2]["n_tc_tiles"] > 0
    check(got, want)


def test_batched_many_chunks_whole_union_streams(env):
    """About eight million d = 8 points in 140 sets: more than 32 core-row chunks per resident
    CTA, so every unions chunk runs whole (no windows); tensor-core labels equal the CUDA-core
    labels of the same call and, on the two smallest sets, the oracle's."""
    torch, pkg, oracle = env
    sets = workloads.batched_sets(n_sets=140, n_min=30000, n_max=100000, dims=(8,), seed=81)
    X = np.concatenate([s[0] for s in sets], axis=0)
    off = np.zeros(len(sets) + 1, np.int64)
    off[1:] = np.cumsum([len(s[0]) for s in sets])
    t = torch.from_numpy(X).cuda()
    eps = [s[1] for s in sets]
    mp = [s[2] for s in sets]
    lab, st = pkg.hca_dbscan_batched(t, off, eps, mp, stats=True)
    assert st["n_tc_tiles"] > 0 and st["n_core_points"] > 32 * 128 * 4 * 152
    ref = pkg.hca_dbscan_batched(t, off, eps, mp, tensor_cores=False).cpu().numpy()
    lab = lab.cpu().numpy()
    np.testing.assert_array_equal(lab, ref)
    for s in np.argsort([len(x[0]) for x in sets])[:2]:
        want = oracle.grid(sets[s][0].astype(np.float64), eps[s], mp[s])
        np.testing.assert_array_equal(lab[off[s]:off[s + 1]], want[0], err_msg=f"set {s}")


def test_batched_sets_on_tensor_cores(env):
    """The batched recipe at d = 8 (per-set eps and MINPTS): tensor-core labels equal the
    CUDA-core labels of the same call and, on every tenth set, the oracle's."""
    torch, pkg, oracle = env
    sets = workloads.batched_sets(n_sets=120, n_min=100, n_max=20000, dims=(8,), seed=8)
    X = np.concatenate([s[0] for s in sets], axis=0)
    off = np.zeros(len(sets) + 1, np.int64)
    off[1:] = np.cumsum([len(s[0]) for s in sets])
    t = torch.from_numpy(X).cuda()
    eps = [s[1] for s in sets]
    mp = [s[2] for s in sets]
    lab, st = pkg.hca_dbscan_batched(t, off, eps, mp, stats=True)
    ref = pkg.hca_dbscan_batched(t, off, eps, mp, tensor_cores=False)
    assert st["n_tc_tiles"] > 0
    lab, ref = lab.cpu().numpy(), ref.cpu().numpy()
    np.testing.assert_array_equal(lab, ref)
    for s in range(0, len(sets), 10):
        want = oracle.grid(sets[s][0].astype(np.float64), eps[s], mp[s])
        np.testing.assert_array_equal(lab[off[s]:off[s + 1]], want[0], err_msg=f"set {s}")
