"""The tuning table (hca_tuning_get / hca_tuning_set) and the autotuners' argument checks, on
the host: no GPU needed."""
import ctypes

import pytest


@pytest.fixture
def pkg():
    import paper_1912_00323_gb300 as pkg
    try:
        pkg.load()
    except OSError as e:
        pytest.skip(f"library not built: {e}")
    yield pkg
    for d in range(1, 65):
        pkg.hca_tuning_set(d, None)


LOW_D = {"path": 0, "tc_min_count": 16, "tc_min_merge": 1, "tc_min_labels": 4, "tc_handoff": 32,
         "first_links": 1, "cta_warps": 4}
HIGH_D = {"path": 0, "tc_min_count": 8, "tc_min_merge": 1, "tc_min_labels": 1, "tc_handoff": 32,
          "first_links": 1, "cta_warps": 4}


def default(d):
    return LOW_D if d <= 8 else HIGH_D


def test_defaults_and_roundtrip(pkg):
    for d in (1, 3, 5, 8, 9, 16, 64):
        assert pkg.hca_tuning_get(d) == default(d)
    DEFAULT = default(16)
    pkg.hca_tuning_set(16, {"tc_min_count": 40, "tc_handoff": 0, "first_links": 0, "cta_warps": 8})
    assert pkg.hca_tuning_get(16) == dict(DEFAULT, tc_min_count=40, tc_handoff=0, first_links=0, cta_warps=8)
    assert pkg.hca_tuning_get(15) == default(15)        # per dimension
    pkg.hca_tuning_set(16, None)
    assert pkg.hca_tuning_get(16) == DEFAULT


@pytest.mark.parametrize("d,field,value", [
    (5, "path", 1), (2, "path", 2), (3, "path", 3), (3, "path", -1),
    (8, "tc_min_count", 0), (8, "tc_min_merge", 0), (8, "tc_min_labels", 0),
    (8, "tc_handoff", -1), (8, "tc_handoff", 128), (8, "first_links", 2),
    (8, "cta_warps", 0), (8, "cta_warps", 3), (8, "cta_warps", 16)])
def test_rejects_out_of_range(pkg, d, field, value):
    with pytest.raises(pkg.HcaError) as e:
        pkg.hca_tuning_set(d, {field: value})
    assert e.value.code == pkg.HCA_EINVAL
    assert pkg.hca_tuning_get(d) == default(d)          # nothing changed


def test_bad_dimension(pkg):
    lib = pkg.load()
    t = pkg.HcaTuning()
    for d in (0, 65, -3):
        assert lib.hca_tuning_get(d, ctypes.byref(t)) == pkg.HCA_EINVAL
        assert lib.hca_tuning_set(d, None) == pkg.HCA_EINVAL
    assert lib.hca_tuning_get(3, None) == pkg.HCA_EINVAL


def test_autotune_argument_checks(pkg):
    lib = pkg.load()
    t, ms = pkg.HcaTuning(), ctypes.c_double()
    # empty input, bad d, bad eps, bad dtype: refused before touching a device
    assert lib.hca_autotune(None, 0, 0, 3, 1.0, 4, None, 2, ctypes.byref(t), ctypes.byref(ms)) == pkg.HCA_EINVAL
    assert lib.hca_autotune(None, 0, 10, 3, 1.0, 4, None, 2, None, None) == pkg.HCA_EINVAL
    assert lib.hca_autotune(None, 0, 10, 65, 1.0, 4, None, 2, None, None) == pkg.HCA_EINVAL
    assert lib.hca_autotune(None, 7, 10, 3, 1.0, 4, None, 2, None, None) == pkg.HCA_EINVAL
    off = (ctypes.c_int64 * 2)(1, 5)
    dims = (ctypes.c_int32 * 1)(3)
    assert lib.hca_autotune_batched(None, 0, 1, off, dims, None, None, None, 2, None, None) == pkg.HCA_EINVAL
