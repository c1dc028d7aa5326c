"""Host logic of the hypercube grid (Algorithm 1): make_grid chooses the cell side so that a
cell holds only points within eps of each other, which is what lets a cell of at least MINPTS
points be core as a whole (Sec. 2).  A host-only program compiled against csrc/lowd_run.cuh
dumps the grids built for 96 seeded random cases (d = 1..4, float and double input, eps over
six decades, extents up to 10^5 eps); the checks below hold them against exact rational
arithmetic:

* the side inequality  d ((1 + 2 tau) side)^2 <= (eps (1 - 2^-20))^2,  side = 1 / inv_side;
* the binning error bound: the band coordinate the device computes (float input: two FP32
  roundings, fl32(fl32(x - o) * inv); double: the same in FP64) lies within tau of the exact
  (x - o) * inv for random points and the extremes of every extent, and the last cell index
  is inside the grid;
* the FP32 filter thresholds bracket fl64(eps^2) by at least the relative guard band 2^-16.

The cell-box test (box_class) on the same grids: a neighbour cell classified wholly within eps
of a point (or wholly beyond) holds only points that the exact predicate puts within (beyond).

For the coarse grid of the d >= 5 path (make_coarse_grid, 64 seeded cases): a side of at least
eps (1 + 2^-50) beyond the binning error, so two points within eps (whose coordinates differ
by at most eps (1 + 2^-50)) always fall in the same or adjacent coarse cells; checked exactly
and on sampled pairs at up to that distance per coordinate.

Needs nvcc (host code only, no GPU)."""
import math
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    exe = shutil.which("nvcc")
    if exe:
        return exe
    cand = "/usr/local/cuda/bin/nvcc"
    return cand if os.path.exists(cand) else None


def _f32(text):
    """A float printed with 9 significant digits, read back as that float (round trip)."""
    return float(np.float32(float(text)))


@pytest.fixture(scope="module")
def grids(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = tmp_path_factory.mktemp("grid") / "grid_dump"
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_1912_00323_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host", "grid_dump.cu"), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines()
    cases = []
    for line in out:
        head, tail = line.split("|")
        h, t = head.split(), tail.split()
        D, f32, eps = int(h[1]), h[2] == "1", float(h[3])
        ext = [float(x) for x in h[4:4 + 2 * D]]
        rc, bin64 = int(t[0]), t[1] == "1"
        cases.append({"D": D, "f32": f32, "eps": eps, "mn": ext[0::2], "mx": ext[1::2], "rc": rc,
                      "bin64": bin64, "inv": float(t[2]), "inv_f": _f32(t[3]), "tau": float(t[4]),
                      "ncell": [int(x) for x in t[5:5 + D]], "key_bits": int(t[5 + D]),
                      "lo32": _f32(t[6 + D]), "hi32": _f32(t[7 + D]), "box_ok": t[8 + D] == "1",
                      "tau_box": _f32(t[9 + D]), "box_full": _f32(t[10 + D]), "box_none": _f32(t[11 + D])})
    assert len(cases) == 96
    assert all(c["rc"] == 0 for c in cases)
    return cases


def test_cell_diagonal_stays_within_eps(grids):
    shrink = 1 - Fraction(1, 2 ** 20)
    for c in grids:
        side = 1 / Fraction(c["inv"])
        w = side * (1 + 2 * Fraction(c["tau"]))
        assert c["D"] * w * w <= (Fraction(c["eps"]) * shrink) ** 2, c


def test_band_coordinates_within_tau(grids):
    rng = np.random.default_rng(1912)
    for c in grids:
        tau = Fraction(c["tau"])
        inv = Fraction(c["inv"])
        for i in range(c["D"]):
            lo, hi = c["mn"][i], c["mx"][i]
            xs = np.concatenate([[lo, hi], lo + (hi - lo) * rng.random(300)])
            if c["f32"]:
                xs = np.clip(xs.astype(np.float32), np.float32(lo), np.float32(hi))
            if c["f32"] and not c["bin64"]:
                assert c["inv"] == c["inv_f"]  # FP32 binning uses the float factor exactly
                o = np.float32(lo)
                t = (xs - o).astype(np.float32) * np.float32(c["inv_f"])
                t = t.astype(np.float32)
            else:
                o = np.float64(lo)
                t = (xs.astype(np.float64) - o) * np.float64(c["inv"])
            for x, tv in zip(xs.tolist(), t.tolist()):
                exact = (Fraction(x) - Fraction(float(o))) * inv
                assert abs(Fraction(tv) - exact) <= tau, (c, x)
            assert math.floor(max(t.tolist())) <= c["ncell"][i] - 1
        assert c["key_bits"] == sum(max(1, math.ceil(math.log2(n))) for n in c["ncell"])
        assert c["key_bits"] <= 63


def test_fp32_filter_thresholds_bracket_eps2(grids):
    for c in grids:
        eps2 = Fraction(c["eps"] * c["eps"])  # fl64(eps * eps), the exact predicate's threshold
        if c["f32"]:
            assert Fraction(c["lo32"]) <= eps2 * (1 - Fraction(1, 2 ** 16))
            assert Fraction(c["hi32"]) >= eps2 * (1 + Fraction(1, 2 ** 16))
        else:
            assert c["lo32"] == -1.0 and c["hi32"] == math.inf


@pytest.fixture(scope="module")
def coarse(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = tmp_path_factory.mktemp("coarse") / "coarse_grid_dump"
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_1912_00323_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host", "coarse_grid_dump.cu"), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines()
    cases = []
    for line in out:
        head, tail = line.split("|")
        h, t = head.split(), tail.split()
        ext = [float(x) for x in h[3:9]]
        cases.append({"f32": h[1] == "1", "eps": float(h[2]), "mn": ext[0::2], "mx": ext[1::2],
                      "rc": int(t[0]), "inv": float(t[1]), "tau": float(t[2]), "ncell": [int(x) for x in t[3:6]]})
    assert len(cases) == 64 and all(c["rc"] == 0 for c in cases)
    return cases


def test_coarse_side_covers_eps(coarse):
    for c in coarse:
        side = 1 / Fraction(c["inv"])
        reach = Fraction(c["eps"]) * (1 + Fraction(1, 2 ** 50))
        assert Fraction(c["tau"]) <= Fraction(1, 2 ** 14)
        # the band coordinates of two points at most `reach` apart differ by < 1 - 2 tau
        assert reach / side < 1 - 2 * Fraction(c["tau"]), c


def test_points_within_eps_land_in_adjacent_coarse_cells(coarse):
    rng = np.random.default_rng(5)
    for c in coarse:
        mn, mx = np.array(c["mn"]), np.array(c["mx"])
        reach = c["eps"] * (1 + 2.0 ** -50)
        p = mn + (mx - mn) * rng.random((400, 3))
        step = reach * rng.choice([-1.0, 1.0], size=(400, 3)) * np.where(rng.random((400, 3)) < 0.2, 1.0,
                                                                          rng.random((400, 3)))
        q = np.clip(p + step, mn, mx)
        if c["f32"]:
            p, q = p.astype(np.float32).astype(np.float64), q.astype(np.float32).astype(np.float64)
        keep = np.all(np.abs(q - p) <= reach, axis=1)
        inv = np.float64(c["inv"])
        top = np.array(c["ncell"]) - 1

        def cells(x):
            return np.minimum(np.floor((x - mn) * inv), top)
        assert keep.sum() > 100
        assert np.all(np.abs(cells(p[keep]) - cells(q[keep])) <= 1), c


def _band32(x, c, i):
    """The band coordinate as the device's box tests see it (FP32)."""
    if c["f32"] and not c["bin64"]:
        return ((x.astype(np.float32) - np.float32(c["mn"][i])).astype(np.float32)
                * np.float32(c["inv_f"])).astype(np.float32)
    return ((x.astype(np.float64) - np.float64(c["mn"][i])) * np.float64(c["inv"])).astype(np.float32)


def _cell(x, c, i):
    """The device's cell index of coordinate i (binning in FP32 or FP64, clamped)."""
    if c["f32"] and not c["bin64"]:
        t = _band32(x, c, i).astype(np.float64)
    else:
        t = (x.astype(np.float64) - np.float64(c["mn"][i])) * np.float64(c["inv"])
    return np.minimum(np.floor(t), c["ncell"][i] - 1).astype(np.int64)


def _box_class(tp, cb, c):
    """0: the cell is wholly beyond eps of the point, 2: wholly within, 1: undecided."""
    f = np.float32
    mn = np.zeros(len(tp), f)
    mx = np.zeros(len(tp), f)
    for i in range(tp.shape[1]):
        lo = (cb[:, i].astype(f) - f(c["tau_box"])).astype(f)
        hi = ((cb[:, i].astype(f) + f(1.0)).astype(f) + f(c["tau_box"])).astype(f)
        t = tp[:, i]
        gap = np.maximum(np.maximum((lo - t).astype(f), (t - hi).astype(f)), f(0))
        far = np.maximum(np.abs((t - lo).astype(f)), np.abs((t - hi).astype(f)))
        mn = (gap.astype(np.float64) * gap + mn).astype(f)
        mx = (far.astype(np.float64) * far + mx).astype(f)
    return np.where(mn > f(c["box_none"]), 0, np.where(mx < f(c["box_full"]), 2, 1))


def test_cell_box_classes_agree_with_exact_predicate(grids):
    """The cell-box test (a neighbour cell wholly within eps of a point counts whole, one wholly
    beyond is dropped): for random points and neighbour cells, every point binned into the cell
    obeys the class the box test gives."""
    rng = np.random.default_rng(11)
    dtype_of = {True: np.float32, False: np.float64}
    n_full = n_none = 0
    for c in grids:
        if not c["box_ok"]:
            continue
        D, dt = c["D"], dtype_of[c["f32"]]
        mn, mx = np.array(c["mn"]), np.array(c["mx"])
        P = 200
        p = (mn + (mx - mn) * rng.random((P, D))).astype(dt)
        tp = np.stack([_band32(p[:, i], c, i) for i in range(D)], axis=1)
        cp = np.stack([_cell(p[:, i], c, i) for i in range(D)], axis=1)
        cb = cp + rng.integers(-2, 3, (P, D))
        inside = np.all((cb >= 0) & (cb <= np.array(c["ncell"]) - 1), axis=1)
        cls = _box_class(tp, cb, c)
        for k in np.nonzero(inside & (cls != 1))[0]:
            M = 64
            frac = rng.random((M, D))
            frac[:8] = np.where(rng.random((8, D)) < 0.5, 0.0, 1.0 - 1e-9)  # cell faces
            q = (mn + (cb[k] + frac) / c["inv"]).astype(dt)
            qc = np.stack([_cell(q[:, i], c, i) for i in range(D)], axis=1)
            q = q[np.all(qc == cb[k], axis=1)]
            if len(q) == 0:
                continue
            s = np.zeros(len(q))
            for i in range(D):
                t = p[k, i].astype(np.float64) - q[:, i].astype(np.float64)
                s = s + t * t
            within = s <= c["eps"] * c["eps"]
            if cls[k] == 2:
                assert np.all(within), (c, k)
                n_full += 1
            else:
                assert not np.any(within), (c, k)
                n_none += 1
    assert n_full > 50 and n_none > 50  # both decisions are exercised
