"""The request server: jobs of different n, d and memory kinds submitted concurrently are
batched together on the device; each job's labels must equal a separate call's (and the
oracle's); cancellation and deadlines behave as documented."""
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
    return torch, pkg, oracle


def _jobs(count, seed):
    sets = workloads.batched_sets(n_sets=count, n_min=50, n_max=30000, dims=(2, 3, 8), seed=seed)
    return sets


def test_each_result_same_alone_and_in_the_mix(env):
    torch, pkg, oracle = env
    jobs = _jobs(60, 5)
    alone = [pkg.hca_dbscan(X, e, m) for X, e, m in jobs]
    results = [None] * len(jobs)
    with pkg.Server(hbm_budget_bytes=1 << 30, workers=2) as sv:
        tickets = [None] * len(jobs)

        def submit_range(lo, hi):
            for i in range(lo, hi):
                X, e, m = jobs[i]
                pts = torch.from_numpy(X).cuda() if i % 3 == 0 else X   # device and host jobs
                tickets[i] = sv.submit(pts, e, m)

        threads = [threading.Thread(target=submit_range, args=(k * 15, (k + 1) * 15)) for k in range(4)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        for i, t in enumerate(tickets):
            lab, lat = sv.wait(t)
            results[i] = lab.cpu().numpy() if hasattr(lab, "cpu") else lab
            assert lat >= 0.0
    for i, (X, e, m) in enumerate(jobs):
        np.testing.assert_array_equal(results[i], alone[i], err_msg=f"job {i}")
        if i % 10 == 0:
            np.testing.assert_array_equal(results[i], oracle.grid(X.astype(np.float64), e, m)[0])


def test_cancel_and_deadline(env):
    torch, pkg, _ = env
    X, e, m = workloads.mixed3d(n=300_000)
    with pkg.Server(hbm_budget_bytes=1 << 20, workers=1) as sv:   # one job at a time
        tickets = [sv.submit(X, e, m) for _ in range(6)]
        # the last ones are still queued behind the first: they can be cancelled
        rc = sv.cancel(tickets[-1])
        assert rc in (pkg.HCA_OK, pkg.HCA_EBUSY)
        if sv.poll(tickets[-2]) == 0:   # still queued or running: a zero deadline times out
            with pytest.raises(pkg.HcaError) as err:
                sv.wait(tickets[-2], timeout_ms=0)
            assert err.value.code == pkg.HCA_ETIMEDOUT
        first, _ = sv.wait(tickets[0])
        for t in tickets[1:-1]:
            lab, _ = sv.wait(t)
            np.testing.assert_array_equal(lab, first)
        if rc == pkg.HCA_OK:
            with pytest.raises(pkg.HcaError) as err:
                sv.wait(tickets[-1])
            assert err.value.code == pkg.HCA_ECANCELED
