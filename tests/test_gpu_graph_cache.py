"""The graph a thread keeps for repeated identical hca_dbscan_device calls: every call of a
repeated sequence gives the oracle's labels and core flags, also after the points in the same
buffers are rewritten inside the captured extents, outside them (the call runs again without
the graph), with a NaN (HCA_EINVAL), after a change of tuning, and after
hca_graph_cache_release; the counts of a replayed call equal those of a direct call."""
import threading

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
    pkg.hca_graph_cache_release()
    for d in range(1, 65):
        pkg.hca_tuning_set(d, None)


def call(env, pts, lab, core, eps, mp, **kw):
    torch, pkg, _ = env
    _, st = pkg.hca_dbscan_device(pts, eps, mp, labels=lab, core=core, stats=True, **kw)
    return lab.cpu().numpy(), core.cpu().numpy(), st


def check(got, want):
    np.testing.assert_array_equal(got[0], want[0])
    np.testing.assert_array_equal(got[1], want[1])


@pytest.mark.parametrize("d,dtype", [(2, np.float64), (3, np.float32), (4, np.float32),
                                     (8, np.float32), (16, np.float32), (8, np.float64)])
def test_repeated_calls_and_rewritten_points(env, d, dtype):
    torch, pkg, oracle = env
    pkg.hca_graph_cache_release()
    kw = dict(step=0.25, eps_steps=4 if d <= 4 else int(round(np.sqrt(2 * d) * 1.8)), spread=3.0,
              box=12.0 if d <= 4 else 2.0 * d)
    X1, eps, mp = workloads.lattice(4000, d, seed=300 + d, **kw)
    # same extents (X1's bounding points kept), other interior points
    X2, _, _ = workloads.lattice(4000, d, seed=500 + d, **kw)
    X2 = np.clip(X2, X1.min(0), X1.max(0))
    X2[:2] = X1[[X1[:, 0].argmin(), X1[:, 0].argmax()]]
    # beyond the first extents
    X3 = X1.copy()
    X3[7] = X1.max(0) + 3.0
    pts = torch.from_numpy(X1.astype(dtype)).cuda()
    lab = torch.empty(len(X1), dtype=torch.int32, device="cuda")
    core = torch.empty(len(X1), dtype=torch.uint8, device="cuda")
    direct = None
    for i, X in enumerate((X1, X1, X1, X1, X2, X2, X3, X3, X3, X1)):
        pts.copy_(torch.from_numpy(X.astype(dtype)))
        got = call(env, pts, lab, core, eps, mp)
        check(got, oracle.grid(X, eps, mp))
        if i == 0:
            direct = got[2]
        if i == 3:  # replayed from the graph: the same counts as the direct call
            for key in ("n_points", "n_cells", "n_core_points", "n_clusters", "n_noise", "key_bits"):
                assert got[2][key] == direct[key], key
            assert got[2]["kernel_launches"] > 0


def test_nan_and_bypass_flag(env):
    torch, pkg, oracle = env
    pkg.hca_graph_cache_release()
    X, eps, mp = workloads.mixed3d(n=50_000)
    want = oracle.grid(X.astype(np.float64), eps, mp)
    pts = torch.from_numpy(X).cuda()
    lab = torch.empty(len(X), dtype=torch.int32, device="cuda")
    core = torch.empty(len(X), dtype=torch.uint8, device="cuda")
    for _ in range(3):
        check(call(env, pts, lab, core, eps, mp), want)
    bad = X.copy()
    bad[123, 1] = np.nan
    pts.copy_(torch.from_numpy(bad))
    with pytest.raises(pkg.HcaError) as e:
        pkg.hca_dbscan_device(pts, eps, mp, labels=lab)
    assert e.value.code == pkg.HCA_EINVAL
    pts.copy_(torch.from_numpy(X))
    check(call(env, pts, lab, core, eps, mp), want)
    check(call(env, pts, lab, core, eps, mp, graph_cache=False), want)
    pkg.hca_graph_cache_release()
    check(call(env, pts, lab, core, eps, mp), want)


def test_tuning_change_and_other_thread(env):
    torch, pkg, oracle = env
    pkg.hca_graph_cache_release()
    X, eps, mp = workloads.aniso16d(n=20_000, n_clusters=20)
    want = oracle.grid(X.astype(np.float64), eps, mp)
    pts = torch.from_numpy(X).cuda()
    lab = torch.empty(len(X), dtype=torch.int32, device="cuda")
    core = torch.empty(len(X), dtype=torch.uint8, device="cuda")
    for _ in range(3):
        check(call(env, pts, lab, core, eps, mp), want)
    pkg.hca_tuning_set(16, {"tc_min_count": 1 << 30, "tc_min_merge": 1 << 30, "tc_min_labels": 1 << 30})
    for _ in range(3):
        check(call(env, pts, lab, core, eps, mp), want)
    pkg.hca_tuning_set(16, None)
    # another host thread with its own buffers keeps a graph of its own
    out = {}

    def worker():
        lab2 = torch.empty(len(X), dtype=torch.int32, device="cuda")
        core2 = torch.empty(len(X), dtype=torch.uint8, device="cuda")
        res = [call(env, pts, lab2, core2, eps, mp) for _ in range(3)]
        pkg.hca_graph_cache_release()
        out["res"] = res
    th = threading.Thread(target=worker)
    th.start()
    th.join()
    for got in out["res"]:
        check(got, want)
    check(call(env, pts, lab, core, eps, mp), want)
