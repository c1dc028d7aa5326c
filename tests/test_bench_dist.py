"""The N > 1 path of bench.py on the CPU: two gloo ranks (one process each, as torchrun starts
them).  Ranks are independent replicas with their own seeds; the reported step time is the
slowest rank's and the value counts every rank's points; the reference arm runs on rank 0
only."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # every rank reports its own step time; all see the slowest
    mine = 1.5 + 2.0 * rank
    slowest = bench.max_over_ranks(mine, dist, "cpu")
    X, eps, mp, _ = bench.workload("blobs2d", rank)
    value = bench.replica_value(len(X), world, slowest)
    dist.barrier()
    dist.destroy_process_group()
    np.save(os.path.join(out_dir, f"rank{rank}.npy"),
            np.array([slowest, value, float(X[:, 0].sum()), eps, mp], dtype=np.float64))


@pytest.mark.timeout(300)
def test_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(240)
        assert p.exitcode == 0
    r0 = np.load(tmp_path / "rank0.npy")
    r1 = np.load(tmp_path / "rank1.npy")
    assert r0[0] == r1[0] == 3.5                       # the slowest rank's time, on both
    assert r0[1] == r1[1] == 2 * 10_000 / 3.5e-3       # both ranks' points over that time
    assert r0[2] != r1[2]                              # own seeds: different replicas
    assert r0[3] == r1[3] and r0[4] == r1[4]           # same recipe parameters


def test_reference_arm_runs_on_rank_zero_only():
    base = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
            "--workload", "blobs2d", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run(base, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env.update(RANK="0", LOCAL_RANK="0")
    r = subprocess.run(base, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
