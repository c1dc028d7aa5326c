"""The C-ABI library builds, loads and exports every function include/*.h declares; argument
checks answer without touching a GPU."""
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        names += re.findall(r"^HCA_API\s+[\w\s\*]+?\b(\w+)\s*\(", open(h).read(), re.M)
    return names


@pytest.fixture(scope="module")
def pkg():
    from paper_1912_00323_gb300 import build
    build.build()
    import paper_1912_00323_gb300 as p
    p.load()
    return p


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("hca_dbscan", "hca_dbscan_device", "hca_dbscan_device_ex", "hca_radix_sort_pairs",
              "hca_strerror", "hca_version"):
        assert f in names


def test_library_exports_every_declared_symbol(pkg):
    lib = pkg.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(pkg.ABI_FUNCTIONS) <= set(declared_functions())


def test_strerror_and_version(pkg):
    assert pkg.hca_version() >= 100
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert pkg.hca_strerror(code)
    assert pkg.hca_strerror(-999) == "unknown error"


@pytest.mark.parametrize("kw,code", [
    (dict(eps=0.0), -1), (dict(eps=float("nan")), -1), (dict(eps=float("inf")), -1),
    (dict(min_pts=0), -1), (dict(d=0), -1), (dict(dtype=7), -1), (dict(n=-1), -1),
])
def test_invalid_arguments_rejected_on_the_host(pkg, kw, code):
    lib = pkg.load()
    X = np.zeros((4, 2))
    labels = np.zeros(4, np.int32)
    a = dict(n=4, d=2, eps=1.0, min_pts=2, dtype=pkg.HCA_F64)
    a.update(kw)
    rc = lib.hca_dbscan(X.ctypes.data, a["dtype"], a["n"], a["d"], a["eps"], a["min_pts"], labels.ctypes.data)
    assert rc == code


def test_empty_input_is_ok_without_device(pkg):
    lib = pkg.load()
    assert lib.hca_dbscan(None, pkg.HCA_F32, 0, 3, 1.0, 2, None) == 0


def test_sort_argument_checks(pkg):
    lib = pkg.load()
    assert lib.hca_radix_sort_pairs(None, None, 10, 3, 0, 8, None) == -1
    assert lib.hca_radix_sort_pairs(None, None, 10, 4, 0, 40, None) == -1
    assert lib.hca_radix_sort_pairs(None, None, 0, 8, 0, 64, None) == 0


def test_oracle_and_library_share_no_code():
    """The oracle and the CUDA path are independent: neither includes or imports the other."""
    csrc = os.path.join(ROOT, "paper_1912_00323_gb300")
    for path in glob.glob(os.path.join(csrc, "**", "*"), recursive=True):
        if os.path.isfile(path) and path.endswith((".py", ".cu", ".cuh", ".h", ".c")):
            assert "oracle" not in re.sub(r"#.*|//.*", "", open(path).read()).lower() or \
                path.endswith("workloads.py"), path
    src = open(os.path.join(ROOT, "oracle", "hca_oracle.c")).read()
    assert "hca_dbscan.h" not in src and "csrc" not in src


def test_server_argument_checks(pkg):
    import ctypes
    lib = pkg.load()
    h = ctypes.c_void_p()
    assert lib.hca_server_create(ctypes.byref(h), 0, 0, 2) == pkg.HCA_EINVAL
    assert lib.hca_server_create(ctypes.byref(h), 0, 1 << 30, 0) == pkg.HCA_EINVAL
    assert lib.hca_submit(None, None, None) == pkg.HCA_EINVAL
    assert lib.hca_poll(None, 1) == pkg.HCA_EINVAL
    assert lib.hca_cancel(None, 1) == pkg.HCA_EINVAL


def test_batched_call_checks_per_set_dimensions_on_the_host(pkg):
    """hca_dbscan_batched takes one d per set: a d outside 1..64, a NULL d array, decreasing
    offsets or a bad eps are refused before any device work."""
    import ctypes
    lib = pkg.load()
    off = (ctypes.c_int64 * 3)(0, 4, 9)
    eps = (ctypes.c_double * 2)(1.0, 1.0)
    mp = (ctypes.c_int32 * 2)(3, 3)
    for dims in ((2, 0), (2, 65)):
        dd = (ctypes.c_int32 * 2)(*dims)
        assert lib.hca_dbscan_batched(None, 0, 2, off, dd, eps, mp, None, None, None, None, 0) == pkg.HCA_EINVAL
    assert lib.hca_dbscan_batched(None, 0, 2, off, None, eps, mp, None, None, None, None, 0) == pkg.HCA_EINVAL
    dd = (ctypes.c_int32 * 2)(2, 3)
    bad_eps = (ctypes.c_double * 2)(1.0, float("nan"))
    assert lib.hca_dbscan_batched(None, 0, 2, off, dd, bad_eps, mp, None, None, None, None, 0) == pkg.HCA_EINVAL
    dec = (ctypes.c_int64 * 3)(0, 4, 2)
    assert lib.hca_dbscan_batched(None, 0, 2, dec, dd, eps, mp, None, None, None, None, 0) == pkg.HCA_EINVAL


def test_pack_sets_layout():
    """pack_sets lays the sets' row-major blocks one after another (argument marshalling only)."""
    torch = pytest.importorskip("torch")
    import paper_1912_00323_gb300 as p
    a = np.arange(6, dtype=np.float32).reshape(3, 2)
    b = np.arange(100, 108, dtype=np.float32).reshape(2, 4)
    c = np.zeros((0, 3), np.float32)
    flat, off, dims = p.pack_sets([a, c, b], device="cpu")
    assert off.tolist() == [0, 3, 3, 5] and dims.tolist() == [2, 3, 4]
    assert flat.numpy().tolist() == a.ravel().tolist() + b.ravel().tolist()
    o, dd, e, m = p._set_args(flat, off, [1.0, 1.0, 1.0], [2, 2, 2], dims)
    assert dd.dtype == np.int32 and o.dtype == np.int64
    with pytest.raises(ValueError):
        p._set_args(flat, off, [1.0, 1.0, 1.0], [2, 2, 2], [2, 3, 5])   # 3*2 + 2*5 != 14 values


def test_workspace_bound_on_the_host(pkg):
    """hca_workspace_bytes needs no device: positive for n > 0, zero for n = 0, non-decreasing
    in n, and arguments checked."""
    lib = pkg.load()
    for d in (1, 2, 3, 4, 5, 16, 64):
        prev = 0
        for n in (1, 1000, 100_000, 2_000_000):
            b = pkg.hca_workspace_bytes(n, d)
            assert b > 0 and b >= prev
            prev = b
        assert pkg.hca_workspace_bytes(0, d) == 0
    import ctypes
    out = ctypes.c_int64()
    assert lib.hca_workspace_bytes(10, 0, 0, 0, ctypes.byref(out)) == pkg.HCA_EINVAL
    assert lib.hca_workspace_bytes(10, 3, 9, 0, ctypes.byref(out)) == pkg.HCA_EINVAL
    assert lib.hca_workspace_bytes(-1, 3, 0, 0, ctypes.byref(out)) == pkg.HCA_EINVAL
    assert lib.hca_workspace_bytes(10, 3, 0, 0, None) == pkg.HCA_EINVAL


def test_graph_cache_release_without_a_graph(pkg):
    """A thread that holds no graph of repeated calls releases nothing (no device needed)."""
    assert pkg.load().hca_graph_cache_release() == pkg.HCA_OK
    pkg.hca_graph_cache_release()


def test_literal_entry_point_rejects_high_d_on_the_host(pkg):
    """The printed algorithm's neighbour block is enumerated for d <= 4 only."""
    lib = pkg.load()
    assert lib.hca_dbscan_literal_device(None, pkg.HCA_F32, 0, 5, 1.0, None, None) == pkg.HCA_EINVAL
    assert lib.hca_dbscan_literal_device(None, pkg.HCA_F32, 0, 2, 1.0, None, None) == pkg.HCA_OK
