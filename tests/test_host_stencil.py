"""Host logic of the hypercube path: the neighbour stencil (Sec. 2's neighbouring hypercubes,
taken as pencils of cells along the last dimension).  A host-only program compiled against
csrc/lowd_run.cuh dumps the stencils that make_stencil builds for d = 1..4 and several binning
error bounds tau; the checks below hold them against brute force over cell offsets:

* coverage: every offset whose cells can hold two points within eps (per dimension a gap of
  max(|delta_i| - 1 - 2 tau, 0) cells) lies in a pencil of the stencil, within its reach;
* pencil 0 is the zero offset, the offsets are distinct and symmetric (delta and -delta, same
  reach), and pencils [0, n_half) are the zero offset and the offsets whose first non-zero
  coordinate is positive (the half the merge pass walks);
* the counting order is a permutation that starts with pencil 0 and never moves away from the
  cell: the gap of its offsets is non-decreasing.

Needs nvcc (host code only, no GPU)."""
import itertools
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    exe = shutil.which("nvcc")
    if exe:
        return exe
    cand = "/usr/local/cuda/bin/nvcc"
    return cand if os.path.exists(cand) else None


@pytest.fixture(scope="module")
def stencils(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = tmp_path_factory.mktemp("stencil") / "stencil_dump"
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_1912_00323_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host", "stencil_dump.cu"), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines()
    cases, cur = [], None
    for line in out:
        f = line.split()
        if f[0] == "case":
            cur = {"D": int(f[1]), "tau": float(f[2]), "side": float(f[3]), "eps": float(f[4]),
                   "n_all": int(f[5]), "n_half": int(f[6]), "off": [], "reach": [], "near": []}
            cases.append(cur)
        elif f[0] == "pencil":
            cur["off"].append(tuple(int(x) for x in f[2:-1]))
            cur["reach"].append(int(f[-1]))
        elif f[0] == "near":
            cur["near"].append(int(f[2]))
    assert len(cases) == 16
    return cases


def _gap2(delta, tau, side):
    return sum((max(abs(x) - 1 - 2 * tau, 0.0) * side) ** 2 for x in delta)


def test_stencil_covers_every_reachable_cell(stencils):
    for c in stencils:
        D, eps = c["D"], c["eps"]
        reach = dict(zip(c["off"], c["reach"]))
        R = max(c["reach"]) + 2
        for delta in itertools.product(range(-R - 2, R + 3), repeat=D):
            if _gap2(delta, c["tau"], c["side"]) <= eps * eps:
                head, last = delta[:-1], delta[-1]
                assert head in reach, (D, c["tau"], delta)
                assert abs(last) <= reach[head], (D, c["tau"], delta, reach[head])


def test_stencil_offsets_and_halves(stencils):
    for c in stencils:
        off = c["off"]
        assert len(off) == c["n_all"] == len(set(off))
        assert off[0] == tuple([0] * (c["D"] - 1))
        reach = dict(zip(off, c["reach"]))
        for o, r in reach.items():
            neg = tuple(-x for x in o)
            assert neg in reach and reach[neg] == r

        def upper(o):
            nz = [x for x in o if x != 0]
            return not nz or nz[0] > 0
        assert all(upper(o) for o in off[:c["n_half"]])
        assert not any(upper(o) for o in off[c["n_half"]:])


def test_counting_order_is_nearest_first(stencils):
    for c in stencils:
        near = c["near"]
        assert sorted(near) == list(range(c["n_all"]))
        assert near[0] == 0
        gaps = [sum(max(abs(x) - 1, 0) ** 2 for x in c["off"][k]) for k in near]
        assert gaps == sorted(gaps)


def test_stencil_sizes_in_two_and_three_dimensions(stencils):
    # the pencil counts the design relies on: 5 pencils in 2-D and 25 in 3-D at tau = 0
    # (side eps / sqrt(d) shrunk by 2^-20: two cells apart along one axis can still hold points
    # within eps, three cannot)
    by = {(c["D"], c["tau"]): c for c in stencils}
    assert by[(2, 0.0)]["n_all"] == 5
    assert by[(3, 0.0)]["n_all"] == 25
