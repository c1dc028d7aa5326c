"""The workspace bound of hca_workspace_bytes (used by the request server's admission) holds
for the workspace each call actually takes (hca_stats.workspace_bytes), on both neighbour
searches, both coordinate types and batched calls."""
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
    import paper_1912_00323_gb300 as pkg
    pkg.load()
    return torch, pkg


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 8, 16, 33])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_call_workspace_within_bound(env, d, dtype):
    torch, pkg = env
    X, eps, mp = workloads.lattice(20_000, d, seed=70 + d, spread=2.0 + d, box=8.0 + 4 * d)
    t = torch.from_numpy(X.astype(dtype)).cuda()
    _, st = pkg.hca_dbscan_device(t, eps, mp, stats=True)
    bound = pkg.hca_workspace_bytes(len(X), d, np.dtype(dtype).name)
    assert 0 < st["workspace_bytes"] <= bound


def test_batched_workspace_within_bound(env):
    torch, pkg = env
    sets = workloads.batched_sets(n_sets=60, n_min=100, n_max=20_000, dims=(2, 3, 8), seed=12)
    sets = sorted(sets, key=lambda s: s[0].shape[1])      # each d group in place
    flat, off, dims = pkg.pack_sets([s[0] for s in sets])
    _, st = pkg.hca_dbscan_batched(flat, off, [s[1] for s in sets], [s[2] for s in sets], dims=dims, stats=True)
    bound = 0
    for d in np.unique(dims):
        m = dims == d
        n_d = int(np.sum(np.diff(off)[m]))
        bound += pkg.hca_workspace_bytes(n_d, int(d)) + 16 * n_d + 1024 * int(m.sum())
    assert 0 < st["workspace_bytes"] <= bound
