"""Plans (one clustering captured as a CUDA graph, replayed): labels equal the oracle's on
every launch, also after the points are rewritten, for declared boxes equal to and larger than
the data; a point outside the box and a NaN are reported by hca_plan_wait."""
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


@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("pad", [0.0, 7.5])
def test_plan_matches_oracle_and_relaunches(env, d, dtype, pad):
    torch, pkg, oracle = env
    X1, eps, mp = workloads.lattice(3000, d, seed=60 + d, step=0.25, eps_steps=4, spread=3.0, box=12.0)
    X2, _, _ = workloads.lattice(3000, d, seed=90 + d, step=0.25, eps_steps=4, spread=3.0, box=12.0)
    lo = np.minimum(X1.min(0), X2.min(0)) - pad
    hi = np.maximum(X1.max(0), X2.max(0)) + pad
    pts = torch.from_numpy(X1.astype(dtype)).cuda()
    core = torch.empty(len(X1), dtype=torch.uint8, device="cuda")
    with pkg.Plan(pts, eps, mp, lo, hi, core=core) as plan:
        for X in (X1, X2, X1):
            pts.copy_(torch.from_numpy(X.astype(dtype)))
            plan.launch()
            st = plan.wait()
            want = oracle.grid(X, eps, mp)
            np.testing.assert_array_equal(plan.labels.cpu().numpy(), want[0])
            np.testing.assert_array_equal(core.cpu().numpy(), want[1])
            assert st["n_core_points"] == int(want[1].sum())


def test_plan_mixed3d_reduced(env):
    torch, pkg, oracle = env
    X, eps, mp = workloads.mixed3d(n=100_000)
    pts = torch.from_numpy(X).cuda()
    with pkg.Plan(pts, eps, mp, X.min(0), X.max(0)) as plan:
        plan.launch()
        plan.wait()
        want = oracle.grid(X.astype(np.float64), eps, mp)
        np.testing.assert_array_equal(plan.labels.cpu().numpy(), want[0])
        # equal to the regular entry point on the same device
        np.testing.assert_array_equal(plan.labels.cpu().numpy(),
                                      pkg.hca_dbscan_device(pts, eps, mp).cpu().numpy())


def test_plan_reports_points_outside_the_box_and_nan(env):
    torch, pkg, _ = env
    X, eps, mp = workloads.lattice(2000, 2, seed=5, step=0.25, eps_steps=4, spread=3.0, box=12.0)
    pts = torch.from_numpy(X).cuda()
    with pkg.Plan(pts, eps, mp, X.min(0), X.max(0)) as plan:
        plan.launch()
        plan.wait()
        Y = X.copy()
        Y[17, 1] = X[:, 1].max() + 1.0
        pts.copy_(torch.from_numpy(Y))
        plan.launch()
        with pytest.raises(pkg.HcaError) as e:
            plan.wait()
        assert e.value.code == pkg.HCA_ERANGE
        Y = X.copy()
        Y[3, 0] = np.nan
        pts.copy_(torch.from_numpy(Y))
        plan.launch()
        with pytest.raises(pkg.HcaError) as e:
            plan.wait()
        assert e.value.code == pkg.HCA_EINVAL
        pts.copy_(torch.from_numpy(X))           # back inside: the plan is still usable
        plan.launch()
        plan.wait()


@pytest.mark.parametrize("d", [2, 3])
def test_batched_plan(env, d):
    torch, pkg, oracle = env
    sets = workloads.batched_sets(n_sets=30, n_min=100, n_max=6000, dims=(d,), seed=d + 40)
    X = np.concatenate([s[0] for s in sets], axis=0)
    off = np.zeros(len(sets) + 1, np.int64)
    off[1:] = np.cumsum([len(s[0]) for s in sets])
    lo = np.stack([s[0].min(0) for s in sets])
    hi = np.stack([s[0].max(0) for s in sets])
    eps = [s[1] for s in sets]
    mp = [s[2] for s in sets]
    pts = torch.from_numpy(X).cuda()
    with pkg.Plan(pts, eps, mp, lo, hi, offsets=off) as plan:
        for _ in range(2):
            plan.launch()
            plan.wait()
            lab = plan.labels.cpu().numpy()
            np.testing.assert_array_equal(lab, pkg.hca_dbscan_batched(pts, off, eps, mp).cpu().numpy())
        for s in range(0, len(sets), 6):
            want = oracle.grid(sets[s][0].astype(np.float64), eps[s], mp[s])
            np.testing.assert_array_equal(lab[off[s]:off[s + 1]], want[0], err_msg=f"set {s}")


def test_batched_plan_mixed_dimensions_one_graph(env):
    """A batched plan over interleaved sets of d = 2, 3 and 8: the d groups are captured into
    one graph (one launch); every relaunch equals the batched call and the oracle."""
    torch, pkg, oracle = env
    sets = []
    for k in range(27):
        d = (2, 3, 8)[k % 3]
        (X, e, m), = workloads.batched_sets(n_sets=1, seed=5000 + k, n_min=100, n_max=5000, dims=(d,))
        sets.append((X, e, m))
    flat, off, dims = pkg.pack_sets([s[0] for s in sets])
    lo = np.concatenate([s[0].min(0) for s in sets])
    hi = np.concatenate([s[0].max(0) for s in sets])
    eps = [s[1] for s in sets]
    mp = [s[2] for s in sets]
    core = torch.empty(int(off[-1]), dtype=torch.uint8, device="cuda")
    with pkg.Plan(flat, eps, mp, lo, hi, offsets=off, dims=dims, core=core) as plan:
        for _ in range(3):
            plan.labels.fill_(-7)
            plan.launch()
            st = plan.wait()
            lab = plan.labels.cpu().numpy()
            np.testing.assert_array_equal(
                lab, pkg.hca_dbscan_batched(flat, off, eps, mp, dims=dims).cpu().numpy())
        assert st["n_core_points"] == int(core.sum().item())
        for s in range(len(sets)):
            want = oracle.grid(sets[s][0].astype(np.float64), eps[s], mp[s])
            np.testing.assert_array_equal(lab[off[s]:off[s + 1]], want[0], err_msg=f"set {s}")


@pytest.mark.parametrize("d", [5, 8, 16])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_plan_coarse_grid(env, d, dtype):
    """d >= 5 (coarse grid, tensor-core tiles for float input) as a plan, relaunched on new points."""
    torch, pkg, oracle = env
    import math
    mk = lambda seed: workloads.lattice(2500, d, seed=seed, step=0.25,
                                        eps_steps=int(round(math.sqrt(2 * d) * 1.8)), spread=2.0,
                                        box=2.0 * d, n_blobs=3)
    X1, eps, _ = mk(300 + d)
    X2, _, _ = mk(400 + d)
    lo = np.minimum(X1.min(0), X2.min(0))
    hi = np.maximum(X1.max(0), X2.max(0))
    pts = torch.from_numpy(X1.astype(dtype)).cuda()
    core = torch.empty(len(X1), dtype=torch.uint8, device="cuda")
    with pkg.Plan(pts, eps, 5, lo, hi, core=core) as plan:
        for X in (X1, X2):
            pts.copy_(torch.from_numpy(X.astype(dtype)))
            plan.launch()
            plan.wait()
            want = oracle.grid(X, eps, 5)
            np.testing.assert_array_equal(plan.labels.cpu().numpy(), want[0])
            np.testing.assert_array_equal(core.cpu().numpy(), want[1])


def test_batched_plan_d8_and_outside(env):
    torch, pkg, oracle = env
    sets = workloads.batched_sets(n_sets=24, n_min=200, n_max=6000, dims=(8,), seed=48)
    X = np.concatenate([s[0] for s in sets], axis=0)
    off = np.zeros(len(sets) + 1, np.int64)
    off[1:] = np.cumsum([len(s[0]) for s in sets])
    lo = np.stack([s[0].min(0) for s in sets])
    hi = np.stack([s[0].max(0) for s in sets])
    eps = [s[1] for s in sets]
    mp = [s[2] for s in sets]
    pts = torch.from_numpy(X).cuda()
    with pkg.Plan(pts, eps, mp, lo, hi, offsets=off) as plan:
        plan.launch()
        plan.wait()
        lab = plan.labels.cpu().numpy()
        np.testing.assert_array_equal(lab, pkg.hca_dbscan_batched(pts, off, eps, mp).cpu().numpy())
        for s in range(0, len(sets), 6):
            want = oracle.grid(sets[s][0].astype(np.float64), eps[s], mp[s])
            np.testing.assert_array_equal(lab[off[s]:off[s + 1]], want[0], err_msg=f"set {s}")
        Y = X.copy()
        Y[off[5] + 1, 3] = hi[5, 3] + 0.5          # one point of set 5 leaves its box
        pts.copy_(torch.from_numpy(Y))
        plan.launch()
        with pytest.raises(pkg.HcaError) as e:
            plan.wait()
        assert e.value.code == pkg.HCA_ERANGE
