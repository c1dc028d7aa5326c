"""CPU oracle for HCA-DBSCAN (arXiv 1912.00323) -- test infrastructure only.

The plain C implementation in ``hca_oracle.c`` is the reference the CUDA path is checked
against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the library under ``paper_1912_00323_gb300`` never
does.  Everything here computes in IEEE double precision.

Functions (numpy in, numpy out):
  bruteforce(X, eps, min_pts, threads)  DBSCAN from Definitions 1-5 of the supplement, O(n^2)
  grid(X, eps, min_pts, threads)        HCA-DBSCAN with DBSCAN semantics (Sec. 2, Alg. 1-4);
                                        threads > 1 shares the counts, merging and border
                                        points among host threads (same result)
  literal(X, eps)                       Alg. 2-4 as printed (representative points only)
  stencil_count(d, rule, side, eps)     neighbour hypercube counts (Sec. 2)
  rep_dirs(d)                           the 3^d - 1 representative directions (Sec. 2)
  grid_cells(X, eps)                    hypercube coordinates of each point (Alg. 1)
Each returns (labels int32[n], core uint8[n]) where both apply.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hca_oracle.c")
_LIB = os.path.join(_HERE, "libhca_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable C, no fused multiply-add)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-Wall", "-o", _LIB, _SRC, "-lpthread", "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


def _bind(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    i32p = ctypes.POINTER(ctypes.c_int32)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.hca_oracle_bruteforce.argtypes = [dp, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                          ctypes.c_int32, ctypes.c_int32, i32p, u8p]
    lib.hca_oracle_grid.argtypes = [dp, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                    ctypes.c_int32, i32p, u8p]
    lib.hca_oracle_grid_mt.argtypes = [dp, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                       ctypes.c_int32, ctypes.c_int32, i32p, u8p]
    lib.hca_oracle_literal.argtypes = [dp, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, i32p]
    lib.hca_oracle_stencil_count.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                             ctypes.c_double]
    lib.hca_oracle_stencil_count.restype = ctypes.c_int64
    lib.hca_oracle_rep_dirs.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_int8)]
    lib.hca_oracle_rep_dirs.restype = ctypes.c_int64
    lib.hca_oracle_grid_cells.argtypes = [dp, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, i64p]
    for f in (lib.hca_oracle_bruteforce, lib.hca_oracle_grid, lib.hca_oracle_grid_mt, lib.hca_oracle_literal,
              lib.hca_oracle_grid_cells):
        f.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


def compile_variant(source_text: str, out_dir: str):
    """Compile a modified copy of the oracle source into out_dir and return an object with
    the same functions as this module, bound to that copy.  Used by the tests that plant a
    mistake in the oracle to show that the pins catch it."""
    src = os.path.join(out_dir, "hca_oracle_variant.c")
    so = os.path.join(out_dir, "libhca_oracle_variant.so")
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                    "-shared", "-w", "-o", so, src, "-lpthread", "-lm"], check=True)
    return _Bound(_bind(ctypes.CDLL(so)))


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _prep(X):
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
    if X.ndim == 1:
        X = X[:, None]
    if X.ndim != 2:
        raise ValueError("points must be an (n, d) array")
    return X


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"{what} failed with code {rc}")


def bruteforce(X, eps: float, min_pts: int, threads: int = 0, lib=None):
    lib = lib or _load()
    X = _prep(X)
    n, d = X.shape
    labels = np.empty(n, np.int32)
    core = np.empty(n, np.uint8)
    threads = threads or os.cpu_count() or 1
    rc = lib.hca_oracle_bruteforce(_ptr(X, ctypes.c_double), n, d, float(eps), int(min_pts),
                                   int(threads), _ptr(labels, ctypes.c_int32),
                                   _ptr(core, ctypes.c_uint8))
    _check(rc, "hca_oracle_bruteforce")
    return labels, core


def grid(X, eps: float, min_pts: int, threads: int = 1, lib=None):
    """threads: host threads (0 = every core); 1 runs hca_oracle_grid itself."""
    lib = lib or _load()
    X = _prep(X)
    n, d = X.shape
    labels = np.empty(n, np.int32)
    core = np.empty(n, np.uint8)
    threads = threads or os.cpu_count() or 1
    if threads == 1:
        rc = lib.hca_oracle_grid(_ptr(X, ctypes.c_double), n, d, float(eps), int(min_pts),
                                 _ptr(labels, ctypes.c_int32), _ptr(core, ctypes.c_uint8))
    else:
        rc = lib.hca_oracle_grid_mt(_ptr(X, ctypes.c_double), n, d, float(eps), int(min_pts),
                                    int(threads), _ptr(labels, ctypes.c_int32), _ptr(core, ctypes.c_uint8))
    _check(rc, "hca_oracle_grid")
    return labels, core


def literal(X, eps: float, lib=None):
    lib = lib or _load()
    X = _prep(X)
    n, d = X.shape
    labels = np.empty(n, np.int32)
    rc = lib.hca_oracle_literal(_ptr(X, ctypes.c_double), n, d, float(eps),
                                _ptr(labels, ctypes.c_int32))
    _check(rc, "hca_oracle_literal")
    return labels


def stencil_count(d: int, rule: int, side: float = 1.0, eps: float = 1.0) -> int:
    return int(_load().hca_oracle_stencil_count(int(d), int(rule), float(side), float(eps)))


def rep_dirs(d: int) -> np.ndarray:
    lib = _load()
    k = lib.hca_oracle_rep_dirs(int(d), None)
    out = np.empty((k, d), np.int8)
    lib.hca_oracle_rep_dirs(int(d), _ptr(out, ctypes.c_int8))
    return out


def grid_cells(X, eps: float) -> np.ndarray:
    lib = _load()
    X = _prep(X)
    n, d = X.shape
    out = np.empty((n, d), np.int64)
    rc = lib.hca_oracle_grid_cells(_ptr(X, ctypes.c_double), n, d, float(eps),
                                   _ptr(out, ctypes.c_int64))
    _check(rc, "hca_oracle_grid_cells")
    return out


class _Bound:
    """The module's functions bound to another compiled copy of the oracle."""

    def __init__(self, lib):
        self._lib = lib

    def bruteforce(self, X, eps, min_pts, threads=0):
        return bruteforce(X, eps, min_pts, threads, lib=self._lib)

    def grid(self, X, eps, min_pts, threads=1):
        return grid(X, eps, min_pts, threads, lib=self._lib)

    def literal(self, X, eps):
        return literal(X, eps, lib=self._lib)
