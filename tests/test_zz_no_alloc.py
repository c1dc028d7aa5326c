"""hca_radix_sort_pairs_noalloc: the sort for callers that cannot allocate device memory
while they run (it uses a fixed scratch array inside the library instead).  Called through
the C ABI and compared with hca_radix_sort_pairs on two calls in a row; both are exact
integer sorts, so the outputs must be identical.  This file is collected last."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MAX_PAIRS = 1 << 18   # HCA_SORT_NOALLOC_MAX_PAIRS in include/hca_dbscan.h
HCA_ETOOLARGE = -7


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_00323_gb300 import build
    build.build()
    import paper_1912_00323_gb300 as pkg
    lib = pkg.load()
    f = lib.hca_radix_sort_pairs_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                  ctypes.c_int32, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return torch, pkg, f


def _inputs(torch, n, kbytes, seed):
    r = np.random.Generator(np.random.PCG64(seed))
    dt = np.uint32 if kbytes == 4 else np.uint64
    keys = r.integers(0, np.iinfo(dt).max, size=n, dtype=dt, endpoint=True)
    keys[: n // 4] = keys[n // 2]
    vals = np.arange(n, dtype=np.uint32)[::-1].copy()
    ik = np.int32 if kbytes == 4 else np.int64
    return (torch.from_numpy(keys.view(ik)).cuda(), torch.from_numpy(vals.view(np.int32)).cuda())


@pytest.mark.parametrize("kbytes,bits", [(4, (0, 32)), (8, (3, 50))])
def test_noalloc_sort_matches_allocating_sort_twice(env, kbytes, bits):
    torch, pkg, noalloc = env
    stream = torch.cuda.current_stream().cuda_stream
    for call, (n, seed) in enumerate([(MAX_PAIRS, 1), (100_003, 2)]):
        k1, v1 = _inputs(torch, n, kbytes, seed + kbytes)
        k2, v2 = k1.clone(), v1.clone()
        pkg.hca_radix_sort_pairs(k1, v1, bits[0], bits[1])
        rc = noalloc(k2.data_ptr(), v2.data_ptr(), n, kbytes, bits[0], bits[1], stream)
        assert rc == 0, f"call {call}: {pkg.hca_strerror(rc)}"
        torch.cuda.synchronize()
        assert torch.equal(k1, k2), f"keys differ on call {call}"
        assert torch.equal(v1, v2), f"values differ on call {call}"


@pytest.mark.parametrize("kbytes,bits", [(4, (0, 32)), (8, (3, 50))])
def test_noalloc_sort_matches_numpy_stable_argsort(env, kbytes, bits):
    """Independent of the allocating sort: numpy's stable argsort of the keys masked to bits
    [begin, end) fixes the permutation, so keys and values must match it exactly."""
    torch, pkg, noalloc = env
    stream = torch.cuda.current_stream().cuda_stream
    n = 200_003
    k, v = _inputs(torch, n, kbytes, 7 + kbytes)
    kh = k.cpu().numpy().view(np.uint32 if kbytes == 4 else np.uint64)
    vh = v.cpu().numpy().view(np.uint32)
    lo, hi = bits
    mask = (1 << (hi - lo)) - 1
    digit = (kh.astype(np.uint64) >> np.uint64(lo)) & np.uint64(mask)
    order = np.argsort(digit, kind="stable")
    rc = noalloc(k.data_ptr(), v.data_ptr(), n, kbytes, lo, hi, stream)
    assert rc == 0, pkg.hca_strerror(rc)
    torch.cuda.synchronize()
    got_k = k.cpu().numpy().view(kh.dtype)
    got_v = v.cpu().numpy().view(np.uint32)
    assert np.array_equal(got_k, kh[order])
    assert np.array_equal(got_v, vh[order])


def test_noalloc_sort_rejects_more_than_its_scratch(env):
    torch, pkg, noalloc = env
    k = torch.zeros(MAX_PAIRS + 1, dtype=torch.int32, device="cuda")
    v = torch.zeros(MAX_PAIRS + 1, dtype=torch.int32, device="cuda")
    rc = noalloc(k.data_ptr(), v.data_ptr(), MAX_PAIRS + 1, 4, 0, 32, None)
    assert rc == HCA_ETOOLARGE
    assert "no-allocation" in pkg.hca_strerror(rc)
