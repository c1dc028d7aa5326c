"""Plan entry points: argument checks on the host (no GPU needed)."""
import ctypes

import pytest


@pytest.fixture
def lib():
    import paper_1912_00323_gb300 as pkg
    try:
        return pkg, pkg.load()
    except OSError as e:
        pytest.skip(f"library not built: {e}")


def test_create_refuses_bad_arguments(lib):
    pkg, L = lib
    h = ctypes.c_void_p()
    box = (ctypes.c_double * 4)(0, 0, 1, 1)
    E = pkg.HCA_EINVAL
    assert L.hca_plan_create(None, None, 0, 10, 2, 1.0, 4, box, box, None, None) == E          # no out
    assert L.hca_plan_create(ctypes.byref(h), None, 0, 0, 2, 1.0, 4, box, box, None, None) == E  # n = 0
    assert L.hca_plan_create(ctypes.byref(h), None, 0, 10, 2, 1.0, 4, None, box, None, None) == E
    assert L.hca_plan_create(ctypes.byref(h), None, 0, 10, 65, 1.0, 4, box, box, None, None) == E  # d > 64
    assert L.hca_plan_create(ctypes.byref(h), None, 0, 10, 2, -1.0, 4, box, box, None, None) == E
    assert L.hca_plan_create(ctypes.byref(h), None, 0, 10, 2, 1.0, 0, box, box, None, None) == E
    assert h.value is None
    off = (ctypes.c_int64 * 3)(0, 5, 3)                 # decreasing offsets
    eps = (ctypes.c_double * 2)(1.0, 1.0)
    mp = (ctypes.c_int32 * 2)(4, 4)
    dims = (ctypes.c_int32 * 2)(2, 2)
    assert L.hca_plan_create_batched(ctypes.byref(h), None, 0, 2, off, dims, eps, mp, box, box, None, None) == E
    off = (ctypes.c_int64 * 3)(0, 5, 8)
    bad_dims = (ctypes.c_int32 * 2)(2, 65)              # d above 64
    assert L.hca_plan_create_batched(ctypes.byref(h), None, 0, 2, off, bad_dims, eps, mp, box, box, None,
                                     None) == E
    inverted = (ctypes.c_double * 4)(1, 1, 0, 0)        # box_min above box_max
    assert L.hca_plan_create_batched(ctypes.byref(h), None, 0, 2, off, dims, eps, mp, inverted, box, None,
                                     None) == E
    assert L.hca_plan_launch(None, None) == E
    assert L.hca_plan_wait(None, None, None) == E
    assert L.hca_plan_destroy(None) == E
