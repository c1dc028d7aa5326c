"""The FP32 filters of the GPU path against the exact predicate, emulated on the CPU: the
tensor-core filter of the coarse-grid path and the scalar FP32 pair test with its guard band.

The coarse-grid path (d >= 5, float input) classifies pairs from D = x.y - colA, accumulated by
the tensor cores from TF32 hi/lo splits of the centred rows x and candidates y (three products
per coordinate, hi.hi + hi.lo + lo.hi, plus two threshold columns carrying colA).  It accepts a
pair when D > rowA and rejects it when D < thr_near (row quantities only); the pairs between go
to the exact predicate.  This test repeats those steps in numpy -- FP32 centring and norms,
the TF32 truncation, exact products, FP32 accumulation both rounded to nearest and truncated
towards zero, in two orders -- on adversarial pairs whose distance lies within 2^-6 .. 2^-20
of eps, and checks that no accepted pair is outside eps and no rejected pair is inside by the
exact FP64 predicate fl64(sum (a_i - b_i)^2) <= fl64(eps^2) (Definition 1).  It pins the
filter's error-bound arithmetic, not the hardware (the GPU parity tests do that)."""
import numpy as np
import pytest

F32 = np.float32


def _tf32(x):
    return (x.view(np.uint32) & np.uint32(0xFFFFE000)).view(F32)


def _round32(v64, truncate):
    """float64 -> float32, to nearest or towards zero."""
    r = v64.astype(F32)
    if truncate:
        over = np.abs(r.astype(np.float64)) > np.abs(v64)
        r = np.where(over, np.nextafter(r, F32(0)), r)
    return r


def _fma32(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(F32)


def _terms(p, c):
    """Centred FP32 row, its FP32 squared norm (fused multiply-add chain) and TF32 split."""
    x = (p - c).astype(F32)
    n = np.zeros(len(p), F32)
    for i in range(p.shape[1]):
        n = _fma32(x[:, i], x[:, i], n)
    hi = _tf32(x)
    lo = (x - hi).astype(F32)
    return n, hi, lo


def _classify(a, b, c, eps2, truncate, reverse):
    DP = a.shape[1]
    na, ahi, alo = _terms(a, c)
    nb, bhi, blo = _terms(b, c)
    colA = (F32(0.5) * (nb * F32(1.000244140625)).astype(F32)).astype(F32)
    chi = _tf32(colA)
    clo = (colA - chi).astype(F32)
    # the MMAs in issue order: per K step of 8 columns hi.hi, hi.lo, lo.hi; then the threshold step
    groups = []
    for ks in range(DP // 8):
        cols = range(8 * ks, 8 * ks + 8)
        groups.append([ahi[:, i].astype(np.float64) * bhi[:, i] for i in cols])
        groups.append([ahi[:, i].astype(np.float64) * blo[:, i] for i in cols])
        groups.append([alo[:, i].astype(np.float64) * bhi[:, i] for i in cols])
    groups.append([-chi.astype(np.float64), -clo.astype(np.float64)])
    terms = [t for g in groups for t in (reversed(g) if reverse else g)]
    D = np.zeros(len(a), F32)
    for t in terms:
        D = _round32(D.astype(np.float64) + t, truncate)
    lo_e = F32(eps2 * (1.0 - 2.0 ** -20))
    hi_e = F32(eps2 * (1.0 + 2.0 ** -20))
    rowA = (F32(0.5) * ((na * F32(1.000244140625)).astype(F32) - lo_e).astype(F32)).astype(F32)
    thr_near = ((F32(0.5) * (na - hi_e).astype(F32)).astype(F32)
                - (F32(2.0 ** -11) * (na + hi_e).astype(F32)).astype(F32)).astype(F32)
    return D > rowA, D < thr_near


def _exact_within(a, b, eps2):
    s = np.zeros(len(a))
    for i in range(a.shape[1]):
        t = a[:, i].astype(np.float64) - b[:, i].astype(np.float64)
        s = s + t * t
    return s <= eps2


def _pairs(rng, d, DP, eps, n):
    """Rows a inside one coarse cell around the centre c, candidates b at eps (1 + delta) from
    a with |delta| in 2^-20 .. 2^-6 and either sign, all on the 2^-12 lattice in FP32."""
    lat = 2.0 ** -12
    c = np.zeros(DP)
    c[:d] = np.round(rng.uniform(10, 90, d) / lat) * lat
    a = np.zeros((n, DP))
    a[:, :d] = c[:d] + rng.uniform(-1.0, 1.0, (n, d)) * eps
    u = rng.normal(size=(n, d))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    delta = rng.choice([-1.0, 1.0], n) * 2.0 ** rng.uniform(-20, -6, n)
    b = np.zeros((n, DP))
    b[:, :d] = a[:, :d] + u * (eps * (1 + delta))[:, None]
    a, b = np.round(a / lat) * lat, np.round(b / lat) * lat
    return a.astype(F32), b.astype(F32), c.astype(F32)


@pytest.mark.parametrize("d,DP", [(5, 8), (8, 8), (16, 16), (24, 32), (64, 64)])
def test_filter_never_contradicts_the_exact_predicate(d, DP):
    rng = np.random.default_rng(1000 + d)
    eps = 4.0
    eps2 = eps * eps
    a, b, c = _pairs(rng, d, DP, eps, 20000)
    exact = _exact_within(a, b, eps2)
    assert 0.2 < exact.mean() < 0.8  # both sides of eps are exercised
    for truncate in (False, True):
        for reverse in (False, True):
            acc, rej = _classify(a, b, c, eps2, truncate, reverse)
            assert not np.any(acc & ~exact), "accepted a pair outside eps"
            assert not np.any(rej & exact), "rejected a pair within eps"


def test_filter_decides_pairs_away_from_eps():
    """Pairs at 0.8 eps and 1.25 eps are decided by the filter alone (no exact recheck)."""
    rng = np.random.default_rng(7)
    d, DP, eps = 16, 16, 4.0
    a, b, c = _pairs(rng, d, DP, eps, 4000)
    near = b.astype(np.float64) - a
    for scale, want_acc in ((0.8, True), (1.25, False)):
        bb = (a + near * scale).astype(F32)
        acc, rej = _classify(a, bb, c, eps * eps, False, False)
        assert np.all(acc if want_acc else rej)


@pytest.mark.parametrize("d", [1, 2, 3, 4, 8, 16, 64])
def test_fp32_pair_filter_outside_the_guard_band(d):
    """The CUDA-core pair test for float input: the FP32 sum of squared differences (fused
    multiply-add, dimension order) decides a pair when it lies below fl32(eps^2 (1 - 2^-16))
    (rounded down) or above fl32(eps^2 (1 + 2^-16)) (rounded up); inside that band the FP64
    sum decides.  Outside the band the FP32 decision must equal the exact predicate."""
    rng = np.random.default_rng(50 + d)
    eps = 1.5 * np.sqrt(d / 2.0)
    eps2 = eps * eps
    lo32 = F32(eps2 * (1 - 2.0 ** -16))
    if float(lo32) > eps2 * (1 - 2.0 ** -16):
        lo32 = np.nextafter(lo32, F32(0))
    hi32 = F32(eps2 * (1 + 2.0 ** -16))
    if float(hi32) < eps2 * (1 + 2.0 ** -16):
        hi32 = np.nextafter(hi32, F32(np.inf))
    n = 50000
    a = rng.uniform(-1000, 1000, (n, d))
    u = rng.normal(size=(n, d))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    delta = rng.choice([-1.0, 1.0], n) * 2.0 ** rng.uniform(-24, -10, n)
    b = a + u * (eps * (1 + delta))[:, None]
    a, b = a.astype(F32), b.astype(F32)
    s = np.zeros(n, F32)
    for i in range(d):
        t = (a[:, i] - b[:, i]).astype(F32)
        s = _fma32(t, t, s)
    exact = _exact_within(a, b, eps2)
    assert not np.any((s < lo32) & ~exact)
    assert not np.any((s > hi32) & exact)
    assert np.mean((s >= lo32) & (s <= hi32)) < 0.9  # most pairs are decided in FP32
