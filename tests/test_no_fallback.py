"""The product path has no CPU fallback: with the CUDA library missing, every entry point of the
binding raises before computing anything (the oracle is never consulted)."""
import numpy as np
import pytest

import paper_1912_00323_gb300 as pkg


@pytest.fixture
def no_library(monkeypatch, tmp_path):
    monkeypatch.setattr(pkg, "LIB_PATH", str(tmp_path / "libhca_dbscan.so"))
    monkeypatch.setattr(pkg, "_lib", None)


@pytest.mark.parametrize("call", [
    lambda: pkg.hca_dbscan(np.zeros((16, 2)), 1.0, 3),
    lambda: pkg.hca_tuning_get(3),
    lambda: pkg.hca_tuning_set(3, None),
    lambda: pkg.load(),
])
def test_every_entry_point_raises_without_the_library(no_library, call):
    with pytest.raises(RuntimeError, match="missing"):
        call()
