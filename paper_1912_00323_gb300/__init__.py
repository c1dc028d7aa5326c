"""GB300-native HCA-DBSCAN (arXiv 1912.00323): Python binding of the C ABI.

This module only marshals arguments for the CUDA library ``libhca_dbscan.so`` (built from
``csrc/`` by ``build.py``); every step of the clustering runs in its kernels.  There is no
CPU fallback: if the library is missing or cannot be loaded, every call raises.

Names follow include/hca_dbscan.h:
  hca_dbscan(points, eps, min_pts)               host numpy array in, int32 labels out
  hca_dbscan_device(points, eps, min_pts, ...)   CUDA torch tensor in, CUDA labels out
  hca_dbscan_batched(points, offsets, eps, min_pts, dims)  many sets (each its own d), one call
  pack_sets(sets)                                 concatenate sets of any d for the batched calls
  hca_radix_sort_pairs(keys, vals, begin, end)   in-place device sort (the Sec. 2 pre-sort)
  hca_strerror(code), hca_version()
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhca_dbscan.so")

HCA_F32, HCA_F64 = 0, 1
HCA_OK, HCA_EINVAL, HCA_ENOMEM, HCA_ECUDA, HCA_ERANGE, HCA_ENOTIMPL, HCA_EDEVICE = 0, -1, -2, -3, -4, -5, -6
HCA_ETOOLARGE, HCA_ETIMEDOUT, HCA_ECANCELED, HCA_EBUSY = -7, -8, -9, -10
HCA_FLAG_TIMING, HCA_FLAG_FP64_ONLY, HCA_FLAG_NO_TENSOR_CORES, HCA_FLAG_NO_GRAPH_CACHE = 1, 2, 4, 8
STAGES = ("minmax", "bin", "sort", "cells", "hash", "core", "reps", "merge", "labels")

ABI_FUNCTIONS = ("hca_dbscan", "hca_dbscan_device", "hca_dbscan_device_ex", "hca_dbscan_batched",
                 "hca_radix_sort_pairs", "hca_tuning_get", "hca_tuning_set", "hca_autotune",
                 "hca_autotune_batched", "hca_plan_create", "hca_plan_create_batched", "hca_plan_launch",
                 "hca_plan_wait", "hca_plan_destroy", "hca_workspace_bytes", "hca_graph_cache_release",
                 "hca_dbscan_literal_device",
                 "hca_strerror", "hca_version")


class HcaStats(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("n_cells", ctypes.c_int64),
                ("n_pencils", ctypes.c_int64), ("n_dense_cells", ctypes.c_int64),
                ("n_core_points", ctypes.c_int64), ("n_clusters", ctypes.c_int64),
                ("n_noise", ctypes.c_int64), ("key_bits", ctypes.c_int32),
                ("sort_passes", ctypes.c_int32), ("kernel_launches", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("stage_ms", ctypes.c_float * len(STAGES)),
                ("n_count_chunks", ctypes.c_int64), ("n_rep_tests", ctypes.c_int64),
                ("n_rep_hits", ctypes.c_int64), ("n_exhaustive_pairs", ctypes.c_int64),
                ("n_exhaustive_chunks", ctypes.c_int64), ("n_border_chunks", ctypes.c_int64),
                ("n_tc_tiles", ctypes.c_int64), ("n_tc_rechecks", ctypes.c_int64),
                ("n_core_cells", ctypes.c_int64), ("n_tc_pairs", ctypes.c_int64),
                ("tc_ms", ctypes.c_float * 3), ("reserved2", ctypes.c_int32),
                ("workspace_bytes", ctypes.c_int64)]

    def as_dict(self):
        skip = ("stage_ms", "reserved", "tc_ms", "reserved2")
        d = {name: getattr(self, name) for name, _ in self._fields_ if name not in skip}
        d["stage_ms"] = {s: float(self.stage_ms[i]) for i, s in enumerate(STAGES)}
        d["tc_ms"] = {s: float(self.tc_ms[i]) for i, s in enumerate(("counts", "unions", "labels"))}
        return d


class HcaTuning(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("tc_min_count", ctypes.c_int32),
                ("tc_min_merge", ctypes.c_int32), ("tc_min_labels", ctypes.c_int32),
                ("tc_handoff", ctypes.c_int32), ("first_links", ctypes.c_int32),
                ("cta_warps", ctypes.c_int32)]

    def as_dict(self):
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


class HcaRequest(ctypes.Structure):
    _fields_ = [("points", ctypes.c_void_p), ("labels", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("d", ctypes.c_int32), ("dtype", ctypes.c_int32), ("eps", ctypes.c_double),
                ("min_pts", ctypes.c_int32), ("on_device", ctypes.c_int32)]


class HcaError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {hca_strerror(code)} (code {code})")


_lib = None


def load():
    """Load libhca_dbscan.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_1912_00323_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    lib.hca_dbscan.argtypes = [vp, i32, i64, i32, dbl, i32, vp]
    lib.hca_dbscan_device.argtypes = [vp, i32, i64, i32, dbl, i32, vp, vp]
    lib.hca_dbscan_device_ex.argtypes = [vp, i32, i64, i32, dbl, i32, vp, vp, vp,
                                         ctypes.POINTER(HcaStats), i32]
    lib.hca_radix_sort_pairs.argtypes = [vp, vp, i64, i32, i32, i32, vp]
    lib.hca_dbscan_batched.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, vp, vp,
                                       ctypes.POINTER(HcaStats), i32]
    lib.hca_dbscan_batched.restype = ctypes.c_int
    lib.hca_server_create.argtypes = [ctypes.POINTER(vp), i32, i64, i32]
    lib.hca_server_destroy.argtypes = [vp]
    lib.hca_submit.argtypes = [vp, ctypes.POINTER(HcaRequest), ctypes.POINTER(i64)]
    lib.hca_poll.argtypes = [vp, i64]
    lib.hca_wait.argtypes = [vp, i64, i64, ctypes.POINTER(ctypes.c_double)]
    lib.hca_cancel.argtypes = [vp, i64]
    for f in ("hca_server_create", "hca_server_destroy", "hca_submit", "hca_poll", "hca_wait", "hca_cancel"):
        getattr(lib, f).restype = ctypes.c_int
    lib.hca_tuning_get.argtypes = [i32, ctypes.POINTER(HcaTuning)]
    lib.hca_tuning_set.argtypes = [i32, ctypes.POINTER(HcaTuning)]
    lib.hca_autotune.argtypes = [vp, i32, i64, i32, dbl, i32, vp, i32, ctypes.POINTER(HcaTuning),
                                 ctypes.POINTER(ctypes.c_double)]
    lib.hca_autotune_batched.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, i32, ctypes.POINTER(HcaTuning),
                                         ctypes.POINTER(ctypes.c_double)]
    for f in ("hca_tuning_get", "hca_tuning_set", "hca_autotune", "hca_autotune_batched"):
        getattr(lib, f).restype = ctypes.c_int
    lib.hca_plan_create.argtypes = [ctypes.POINTER(vp), vp, i32, i64, i32, dbl, i32, vp, vp, vp, vp]
    lib.hca_plan_create_batched.argtypes = [ctypes.POINTER(vp), vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.hca_plan_launch.argtypes = [vp, vp]
    lib.hca_plan_wait.argtypes = [vp, vp, ctypes.POINTER(HcaStats)]
    lib.hca_plan_destroy.argtypes = [vp]
    for f in ("hca_plan_create", "hca_plan_create_batched", "hca_plan_launch", "hca_plan_wait", "hca_plan_destroy"):
        getattr(lib, f).restype = ctypes.c_int
    lib.hca_workspace_bytes.argtypes = [i64, i32, i32, i32, ctypes.POINTER(i64)]
    lib.hca_graph_cache_release.argtypes = []
    lib.hca_dbscan_literal_device.argtypes = [vp, i32, i64, i32, dbl, vp, vp]
    lib.hca_dbscan_literal_device.restype = ctypes.c_int
    lib.hca_graph_cache_release.restype = ctypes.c_int
    lib.hca_workspace_bytes.restype = ctypes.c_int
    lib.hca_strerror.argtypes = [ctypes.c_int]
    lib.hca_strerror.restype = ctypes.c_char_p
    lib.hca_version.restype = i32
    for f in ("hca_dbscan", "hca_dbscan_device", "hca_dbscan_device_ex", "hca_radix_sort_pairs"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def hca_strerror(code: int) -> str:
    return load().hca_strerror(int(code)).decode()


def hca_version() -> int:
    return int(load().hca_version())


def _dtype_code(dt):
    name = str(dt)
    if name.endswith("float32"):
        return HCA_F32
    if name.endswith("float64"):
        return HCA_F64
    raise TypeError(f"points must be float32 or float64, got {dt}")


def hca_dbscan(points, eps: float, min_pts: int, labels=None):
    """Cluster host points (numpy (n, d) float32/float64, or a CPU torch tensor, possibly
    pinned).  Returns int32 labels of length n (a numpy array unless `labels` is given)."""
    lib = load()
    if hasattr(points, "data_ptr"):  # torch CPU tensor
        if points.is_cuda:
            raise ValueError("hca_dbscan takes host points; use hca_dbscan_device for CUDA tensors")
        pts = points.contiguous()
        n, d = (pts.shape[0], pts.shape[1]) if pts.dim() == 2 else (pts.shape[0], 1)
        code = _dtype_code(pts.dtype)
        ptr = pts.data_ptr()
    else:
        pts = np.ascontiguousarray(points)
        if pts.ndim == 1:
            pts = pts[:, None]
        n, d = pts.shape
        code = _dtype_code(pts.dtype)
        ptr = pts.ctypes.data
    if labels is None:
        labels = np.empty(n, np.int32)
        lptr = labels.ctypes.data
    else:
        lptr = labels.data_ptr() if hasattr(labels, "data_ptr") else labels.ctypes.data
    rc = lib.hca_dbscan(ptr, code, n, d, float(eps), int(min_pts), lptr)
    if rc != HCA_OK:
        raise HcaError(rc, "hca_dbscan")
    return labels


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def hca_dbscan_device(points, eps: float, min_pts: int, labels=None, core=None, stream=None,
                      stats: bool = False, timing: bool = False, fp64_only: bool = False,
                      tensor_cores: bool = True, graph_cache: bool = True):
    """Cluster a CUDA tensor of shape (n, d).  Returns the int32 label tensor, or
    (labels, stats_dict) when stats or timing is requested.  `core`, if given, is a uint8
    CUDA tensor of length n that receives the core flags.  tensor_cores=False keeps the d >= 5
    float path on the CUDA cores (same labels).  graph_cache=False runs the call's launches
    directly even when the same call repeats (the library otherwise replays a CUDA graph of
    it; same labels)."""
    import torch
    lib = load()
    if not points.is_cuda:
        raise ValueError("hca_dbscan_device takes a CUDA tensor")
    pts = points.contiguous()
    n = pts.shape[0]
    d = pts.shape[1] if pts.dim() == 2 else 1
    code = _dtype_code(pts.dtype)
    if labels is None:
        labels = torch.empty(n, dtype=torch.int32, device=pts.device)
    flags = ((HCA_FLAG_TIMING if timing else 0) | (HCA_FLAG_FP64_ONLY if fp64_only else 0)
             | (0 if tensor_cores else HCA_FLAG_NO_TENSOR_CORES)
             | (0 if graph_cache else HCA_FLAG_NO_GRAPH_CACHE))
    st = HcaStats()
    rc = lib.hca_dbscan_device_ex(pts.data_ptr(), code, n, d, float(eps), int(min_pts),
                                  labels.data_ptr(), core.data_ptr() if core is not None else None,
                                  _stream_ptr(stream), ctypes.byref(st), flags)
    if rc != HCA_OK:
        raise HcaError(rc, "hca_dbscan_device")
    if stats or timing:
        return labels, st.as_dict()
    return labels


def _set_args(points, offsets, eps, min_pts, dims):
    """Host arrays of a batched call: int64 offsets, int32 dims, float64 eps, int32 min_pts,
    checked against the length of the flat point buffer."""
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    e = np.ascontiguousarray(np.asarray(eps, dtype=np.float64))
    m = np.ascontiguousarray(np.asarray(min_pts, dtype=np.int32))
    if off.ndim != 1 or len(off) != len(e) + 1 or len(e) != len(m):
        raise ValueError("offsets must have n_sets + 1 entries; eps and min_pts n_sets")
    if dims is None:
        if points.dim() != 2:
            raise ValueError("dims is required when points is not an (N, d) tensor")
        dims = [points.shape[1]] * len(e)
    dd = np.ascontiguousarray(np.asarray(dims, dtype=np.int32))
    if dd.shape != e.shape:
        raise ValueError("dims must have n_sets entries")
    if int(np.sum(np.diff(off) * dd.astype(np.int64))) != points.numel():
        raise ValueError("the sets' n_s * d_s must add up to the number of point values")
    return off, dd, e, m


def pack_sets(sets, device="cuda"):
    """Concatenate point sets of any dimension for the batched calls: `sets` is a sequence of
    (n_s, d_s) arrays or tensors of one float dtype.  Returns (flat CUDA tensor, offsets, dims)."""
    import torch
    parts, offs, dims = [], [0], []
    for x in sets:
        t = x if hasattr(x, "data_ptr") else torch.from_numpy(np.ascontiguousarray(x))
        if t.dim() == 1:
            t = t[:, None]
        parts.append(t.reshape(-1))
        offs.append(offs[-1] + t.shape[0])
        dims.append(t.shape[1])
    flat = torch.cat(parts).to(device) if parts else torch.empty(0, device=device)
    return flat.contiguous(), np.asarray(offs, np.int64), np.asarray(dims, np.int32)


def hca_dbscan_batched(points, offsets, eps, min_pts, dims=None, labels=None, core=None, stream=None,
                       stats: bool = False, timing: bool = False, fp64_only: bool = False,
                       tensor_cores: bool = True):
    """Cluster many sets in one call, each with its own dimension dims[s], eps[s] and
    min_pts[s] (host sequences).  `points` is a CUDA tensor holding the sets' row-major blocks
    one after another (an (N, d) tensor when every set has d = points.shape[1] and dims is
    None; any flat layout from pack_sets otherwise).  Labels are per set (ids are indices within
    the set), laid out by offsets.  Returns the label tensor, or (labels, stats_dict) when stats
    or timing is requested."""
    import torch
    lib = load()
    if not points.is_cuda:
        raise ValueError("hca_dbscan_batched takes a CUDA tensor")
    pts = points.contiguous()
    off, dd, e, m = _set_args(pts, offsets, eps, min_pts, dims)
    n = int(off[-1])
    if labels is None:
        labels = torch.empty(n, dtype=torch.int32, device=pts.device)
    flags = ((HCA_FLAG_TIMING if timing else 0) | (HCA_FLAG_FP64_ONLY if fp64_only else 0)
             | (0 if tensor_cores else HCA_FLAG_NO_TENSOR_CORES))
    st = HcaStats()
    rc = lib.hca_dbscan_batched(pts.data_ptr(), _dtype_code(pts.dtype), len(e), off.ctypes.data, dd.ctypes.data,
                                e.ctypes.data, m.ctypes.data, labels.data_ptr(),
                                core.data_ptr() if core is not None else None, _stream_ptr(stream),
                                ctypes.byref(st), flags)
    if rc != HCA_OK:
        raise HcaError(rc, "hca_dbscan_batched")
    if stats or timing:
        return labels, st.as_dict()
    return labels


def hca_dbscan_literal_device(points, eps: float, labels=None, stream=None):
    """The paper's Algorithms 2-4 as printed (representative points only, strict "<", no
    MINPTS; an ablation, not DBSCAN) on a CUDA tensor of shape (n, d), d <= 4.  Returns the
    int32 labels (every point in a cluster)."""
    import torch
    lib = load()
    if not points.is_cuda:
        raise ValueError("hca_dbscan_literal_device takes a CUDA tensor")
    pts = points.contiguous()
    n = pts.shape[0]
    d = pts.shape[1] if pts.dim() == 2 else 1
    if labels is None:
        labels = torch.empty(n, dtype=torch.int32, device=pts.device)
    rc = lib.hca_dbscan_literal_device(pts.data_ptr(), _dtype_code(pts.dtype), n, d, float(eps),
                                       labels.data_ptr(), _stream_ptr(stream))
    if rc != HCA_OK:
        raise HcaError(rc, "hca_dbscan_literal_device")
    return labels


def hca_graph_cache_release():
    """Free the calling thread's graph of repeated hca_dbscan_device calls and its workspace."""
    rc = load().hca_graph_cache_release()
    if rc != HCA_OK:
        raise HcaError(rc, "hca_graph_cache_release")


def hca_workspace_bytes(n: int, d: int, dtype="float32", fp64_only: bool = False, tensor_cores: bool = True) -> int:
    """Upper bound on the device workspace of one clustering call on n points of dimension d
    (no device needed)."""
    flags = (HCA_FLAG_FP64_ONLY if fp64_only else 0) | (0 if tensor_cores else HCA_FLAG_NO_TENSOR_CORES)
    out = ctypes.c_int64()
    rc = load().hca_workspace_bytes(int(n), int(d), _dtype_code(dtype), flags, ctypes.byref(out))
    if rc != HCA_OK:
        raise HcaError(rc, "hca_workspace_bytes")
    return int(out.value)


def hca_radix_sort_pairs(keys, vals, begin_bit: int = 0, end_bit: int | None = None, stream=None):
    """Stable in-place sort of CUDA tensors keys (int32/int64 viewed as unsigned) and vals
    (int32 viewed as uint32) by key bits [begin_bit, end_bit)."""
    lib = load()
    kb = keys.element_size()
    if end_bit is None:
        end_bit = 8 * kb
    rc = lib.hca_radix_sort_pairs(keys.data_ptr(), vals.data_ptr(), keys.numel(), kb,
                                  int(begin_bit), int(end_bit), _stream_ptr(stream))
    if rc != HCA_OK:
        raise HcaError(rc, "hca_radix_sort_pairs")
    return keys, vals


def hca_tuning_get(d: int) -> dict:
    """The tuning used for dimension d (neighbour search, tensor-core split)."""
    t = HcaTuning()
    rc = load().hca_tuning_get(int(d), ctypes.byref(t))
    if rc != HCA_OK:
        raise HcaError(rc, "hca_tuning_get")
    return t.as_dict()


def hca_tuning_set(d: int, tuning: dict | None = None):
    """Set the tuning of dimension d from a dict with the fields of hca_tuning (missing fields
    keep their current values); None restores the defaults."""
    lib = load()
    if tuning is None:
        rc = lib.hca_tuning_set(int(d), None)
    else:
        cur = hca_tuning_get(d)
        cur.update(tuning)
        t = HcaTuning(**{k: int(v) for k, v in cur.items()})
        rc = lib.hca_tuning_set(int(d), ctypes.byref(t))
    if rc != HCA_OK:
        raise HcaError(rc, "hca_tuning_set")


def hca_autotune(points, eps: float, min_pts: int, stream=None, repeats: int = 2):
    """Time candidate tunings for points.shape[1] on a CUDA tensor of points and keep the fastest;
    returns (tuning dict, best ms)."""
    lib = load()
    pts = points.contiguous()
    d = pts.shape[1] if pts.dim() == 2 else 1
    t, ms = HcaTuning(), ctypes.c_double()
    rc = lib.hca_autotune(pts.data_ptr(), _dtype_code(pts.dtype), pts.shape[0], d, float(eps), int(min_pts),
                          _stream_ptr(stream), int(repeats), ctypes.byref(t), ctypes.byref(ms))
    if rc != HCA_OK:
        raise HcaError(rc, "hca_autotune")
    return t.as_dict(), ms.value


def hca_autotune_batched(points, offsets, eps, min_pts, dims=None, stream=None, repeats: int = 2):
    """hca_autotune for the sets of a batched call (arguments as hca_dbscan_batched): every d
    present is tuned on its own sets.  Returns ({d: tuning dict}, sum of the best ms)."""
    lib = load()
    pts = points.contiguous()
    off, dd, e, m = _set_args(pts, offsets, eps, min_pts, dims)
    table = (HcaTuning * 64)()
    ms = ctypes.c_double()
    rc = lib.hca_autotune_batched(pts.data_ptr(), _dtype_code(pts.dtype), len(e), off.ctypes.data, dd.ctypes.data,
                                  e.ctypes.data, m.ctypes.data, _stream_ptr(stream), int(repeats),
                                  table, ctypes.byref(ms))
    if rc != HCA_OK:
        raise HcaError(rc, "hca_autotune_batched")
    present = sorted({int(x) for x, a, b in zip(dd, off[:-1], off[1:]) if b > a})
    return {d: table[d - 1].as_dict() for d in present}, ms.value


class Plan:
    """One clustering call captured as a CUDA graph (hca_plan_*), with the tuning of d at creation.
    Bound to the CUDA tensors `points` (n, d) and `labels` (n,) (and `core`, optional); the
    points may be rewritten between launches as long as they stay inside the declared box
    (box_min, box_max: d values; for a batched plan, d_s values per set, set after set).  A
    batched plan (offsets given) takes the sets of hca_dbscan_batched, each with its own d
    (dims), and runs them all in one graph launch."""

    def __init__(self, points, eps, min_pts, box_min, box_max, labels=None, core=None, offsets=None,
                 dims=None):
        import torch
        lib = load()
        if not points.is_cuda or not points.is_contiguous():
            raise ValueError("Plan takes a contiguous CUDA tensor")
        self.points = points
        n = points.shape[0] if offsets is None else int(np.asarray(offsets)[-1])
        d = points.shape[1] if points.dim() == 2 else 1
        self.labels = labels if labels is not None else torch.empty(n, dtype=torch.int32, device=points.device)
        self.core = core
        self._bmn = np.ascontiguousarray(np.asarray(box_min, dtype=np.float64).ravel())
        self._bmx = np.ascontiguousarray(np.asarray(box_max, dtype=np.float64).ravel())
        h = ctypes.c_void_p()
        cp = core.data_ptr() if core is not None else None
        if offsets is None:
            rc = lib.hca_plan_create(ctypes.byref(h), points.data_ptr(), _dtype_code(points.dtype), n, d,
                                     float(eps), int(min_pts), self._bmn.ctypes.data, self._bmx.ctypes.data,
                                     self.labels.data_ptr(), cp)
        else:
            self._off, self._dims, self._eps, self._mp = _set_args(points, offsets, eps, min_pts, dims)
            rc = lib.hca_plan_create_batched(ctypes.byref(h), points.data_ptr(), _dtype_code(points.dtype),
                                             len(self._eps), self._off.ctypes.data, self._dims.ctypes.data,
                                             self._eps.ctypes.data, self._mp.ctypes.data, self._bmn.ctypes.data,
                                             self._bmx.ctypes.data, self.labels.data_ptr(), cp)
        if rc != HCA_OK:
            raise HcaError(rc, "hca_plan_create")
        self._h = h

    def launch(self, stream=None):
        rc = load().hca_plan_launch(self._h, _stream_ptr(stream))
        if rc != HCA_OK:
            raise HcaError(rc, "hca_plan_launch")

    def wait(self, stream=None):
        st = HcaStats()
        rc = load().hca_plan_wait(self._h, _stream_ptr(stream), ctypes.byref(st))
        if rc != HCA_OK:
            raise HcaError(rc, "hca_plan_wait")
        return {k: st.as_dict()[k] for k in ("n_cells", "n_pencils", "n_dense_cells", "n_core_points",
                                              "n_clusters", "n_noise")}

    def close(self):
        if getattr(self, "_h", None):
            load().hca_plan_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Asynchronous clustering jobs with continuous batching (hca_server_* / hca_submit /
    hca_poll / hca_wait / hca_cancel).  submit() takes host numpy arrays or CUDA tensors and
    keeps them alive until the job is waited for."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 32 << 30, workers: int = 4):
        lib = load()
        self._lib = lib
        h = ctypes.c_void_p()
        rc = lib.hca_server_create(ctypes.byref(h), int(device), int(hbm_budget_bytes), int(workers))
        if rc != HCA_OK:
            raise HcaError(rc, "hca_server_create")
        self._h = h
        self._keep = {}

    def submit(self, points, eps: float, min_pts: int, labels=None) -> int:
        on_device = hasattr(points, "is_cuda") and points.is_cuda
        if hasattr(points, "data_ptr"):
            pts = points.contiguous()
            ptr = pts.data_ptr()
            n, d = pts.shape[0], (pts.shape[1] if pts.dim() == 2 else 1)
            if labels is None:
                import torch
                labels = torch.empty(n, dtype=torch.int32, device=pts.device)
            lptr = labels.data_ptr()
        else:
            pts = np.ascontiguousarray(points)
            if pts.ndim == 1:
                pts = pts[:, None]
            n, d = pts.shape
            ptr = pts.ctypes.data
            if labels is None:
                labels = np.empty(n, np.int32)
            lptr = labels.ctypes.data
        req = HcaRequest(ptr, lptr, n, d, _dtype_code(pts.dtype), float(eps), int(min_pts), int(on_device))
        t = ctypes.c_int64()
        rc = self._lib.hca_submit(self._h, ctypes.byref(req), ctypes.byref(t))
        if rc != HCA_OK:
            raise HcaError(rc, "hca_submit")
        self._keep[t.value] = (pts, labels)
        return t.value

    def poll(self, ticket: int) -> int:
        return int(self._lib.hca_poll(self._h, int(ticket)))

    def wait(self, ticket: int, timeout_ms: int = 600_000):
        """Returns (labels, latency_ms); raises HcaError on a job error or a timeout."""
        lat = ctypes.c_double()
        rc = self._lib.hca_wait(self._h, int(ticket), int(timeout_ms), ctypes.byref(lat))
        if rc == HCA_ETIMEDOUT:
            raise HcaError(rc, "hca_wait")
        _, labels = self._keep.pop(int(ticket))
        if rc != HCA_OK:
            raise HcaError(rc, "hca_wait")
        return labels, lat.value

    def cancel(self, ticket: int) -> int:
        return int(self._lib.hca_cancel(self._h, int(ticket)))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.hca_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
