"""Seeded synthetic point sets for HCA-DBSCAN.

This module only draws random numbers (numpy PCG64) and rounds them to binary lattices; it
holds none of the clustering arithmetic, so both the CUDA path and the CPU oracle can take
their inputs from it.  The paper's own data sets (UCI Vicon, PAMAP2, Household, Leaf; Sec. 3,
Table 1) are not available; these recipes stand in for them with the same roles (low d and
large n, high d and moderate n).

Every generator returns (X, eps, min_pts) where X is an (n, d) C-contiguous array.  The
points are shuffled so that input order carries no cluster structure.

Recipes (sizes are parameters so the same recipe can be run small):
  blobs2d   d=2, float64: 5 isotropic Gaussian blobs (sigma 2, centres U[0,100]^2), 90% of
            the points, plus 10% uniform noise over [0,100]^2; coordinates rounded to
            multiples of 2^-12; eps 1.5, minPts 5.  Default n = 10,000.
  mixed3d   d=3, float32: 40 Gaussian blobs (sigma U[0.5,3], centres U[50,950]^3) holding
            80% of the points, 8 noisy arcs or rings (radius U[20,100], random plane, angular
            span U[pi/2, 2 pi], Gaussian jitter sigma 0.75) holding 15%, and 5% uniform noise
            over [0,1000]^3; coordinates rounded to multiples of 2^-16, then to float32 (every
            float32 at or above 128 is a multiple of 2^-16, so the lattice survives); eps 2,
            minPts 10.  Default n = 2,000,000.
  aniso16d  d=16, float32: 100 anisotropic Gaussian clusters (diagonal sigma_i U[0.2,1],
            random rotation, centres U[10,90]^16) holding 90% of the points and 10% uniform
            noise over [0,100]^16; coordinates on multiples of 2^-12; eps 4, minPts 20.
            Default n = 1,000,000.
  batched   4096 independent sets: n log-uniform in [1,000, 200,000], d from {2, 3, 8}, 5 blobs
            (sigma 2 eps / sqrt(d)) + 10% noise in [0,100]^d, eps U[0.5, 3] on 2^-12, MINPTS
            U{4..16}, float32 on the 2^-12 lattice (sizes are parameters).
  lattice   any d: points on the integer lattice times `step` (default 0.25) drawn from a few
            small blobs plus noise, so that many pairs sit at exactly eps; for tie tests.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1912_00323


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _round_lattice(x, bits):
    scale = float(2 ** bits)
    return np.round(x * scale) / scale


def _split(n, fracs):
    counts = [int(round(n * f)) for f in fracs[:-1]]
    counts.append(n - sum(counts))
    return counts


def _even(total, parts):
    base = total // parts
    out = [base] * parts
    for i in range(total - base * parts):
        out[i] += 1
    return out


def blobs2d(n: int = 10_000, seed: int = SEED_BASE + 0):
    r = _rng(seed)
    n_blob, n_noise = _split(n, [0.9, 0.1])
    centres = r.uniform(0.0, 100.0, size=(5, 2))
    parts = [r.normal(c, 2.0, size=(m, 2)) for c, m in zip(centres, _even(n_blob, 5))]
    parts.append(r.uniform(0.0, 100.0, size=(n_noise, 2)))
    X = np.concatenate(parts, axis=0)
    X = X[r.permutation(n)]
    X = _round_lattice(X, 12)
    return np.ascontiguousarray(X, dtype=np.float64), 1.5, 5


def _random_rotation(r, d):
    q, rr = np.linalg.qr(r.normal(size=(d, d)))
    return q * np.sign(np.diag(rr))


def mixed3d(n: int = 2_000_000, seed: int = SEED_BASE + 1):
    r = _rng(seed)
    n_blob, n_arc, n_noise = _split(n, [0.80, 0.15, 0.05])
    parts = []
    for m in _even(n_blob, 40):
        c = r.uniform(50.0, 950.0, size=3)
        sigma = r.uniform(0.5, 3.0)
        parts.append(r.normal(c, sigma, size=(m, 3)))
    for m in _even(n_arc, 8):
        c = r.uniform(100.0, 900.0, size=3)
        radius = r.uniform(20.0, 100.0)
        rot = _random_rotation(r, 3)
        u, v = rot[:, 0], rot[:, 1]
        start = r.uniform(0.0, 2.0 * np.pi)
        span = r.uniform(0.5 * np.pi, 2.0 * np.pi)
        theta = start + span * r.uniform(0.0, 1.0, size=m)
        pts = c + radius * (np.cos(theta)[:, None] * u + np.sin(theta)[:, None] * v)
        parts.append(pts + r.normal(0.0, 0.75, size=(m, 3)))
    parts.append(r.uniform(0.0, 1000.0, size=(n_noise, 3)))
    X = np.concatenate(parts, axis=0)
    X = X[r.permutation(n)]
    X = _round_lattice(X, 16).astype(np.float32)
    return np.ascontiguousarray(X), 2.0, 10


def aniso16d(n: int = 1_000_000, seed: int = SEED_BASE + 2, n_clusters: int = 100):
    r = _rng(seed)
    d = 16
    n_cl, n_noise = _split(n, [0.9, 0.1])
    parts = []
    for m in _even(n_cl, n_clusters):
        c = r.uniform(10.0, 90.0, size=d)
        sig = r.uniform(0.2, 1.0, size=d)
        rot = _random_rotation(r, d)
        z = r.normal(size=(m, d)) * sig
        parts.append(c + z @ rot.T)
    parts.append(r.uniform(0.0, 100.0, size=(n_noise, d)))
    X = np.concatenate(parts, axis=0)
    X = X[r.permutation(n)]
    X = _round_lattice(X, 12).astype(np.float32)
    return np.ascontiguousarray(X), 4.0, 20


def lattice(n: int, d: int, seed: int, step: float = 0.25, eps_steps: int = 4,
            min_pts: int = 4, n_blobs: int = 3, spread: float = 6.0, box: float = 40.0,
            noise_frac: float = 0.2, dtype=np.float64):
    """Points on the lattice step*Z^d; eps = eps_steps*step, so exact-eps pairs are common."""
    r = _rng(seed)
    n_noise = int(round(n * noise_frac))
    n_bl = n - n_noise
    parts = []
    for m in _even(n_bl, max(n_blobs, 1)):
        c = r.uniform(0.0, box, size=d)
        parts.append(r.normal(c, spread * step, size=(m, d)))
    parts.append(r.uniform(0.0, box, size=(n_noise, d)))
    X = np.concatenate(parts, axis=0)[:n]
    X = X[r.permutation(len(X))]
    X = np.round(X / step) * step
    return np.ascontiguousarray(X, dtype=dtype), eps_steps * step, min_pts


def batched_sets(n_sets: int = 4096, seed: int = SEED_BASE + 3, n_min: int = 1_000,
                 n_max: int = 200_000, dims=(2, 3, 8)):
    """Many independent point sets: n log-uniform in [n_min, n_max], d drawn from `dims`, 5
    Gaussian blobs (sigma = c_d * eps) plus 10% uniform noise in [0,100]^d, eps uniform in
    [0.5, 3] and rounded to 2^-12, MINPTS uniform in {4..16}, float32 coordinates on the 2^-12
    lattice.  c_d = 2 / sqrt(d) keeps roughly half of the points core at every d.
    Returns a list of (X, eps, min_pts)."""
    r = _rng(seed)
    out = []
    for _ in range(n_sets):
        n = int(round(np.exp(r.uniform(np.log(n_min), np.log(n_max)))))
        d = int(r.choice(dims))
        eps = float(np.round(r.uniform(0.5, 3.0) * 4096) / 4096)
        min_pts = int(r.integers(4, 17))
        sigma = 2.0 / np.sqrt(d) * eps
        n_noise = n // 10
        parts = [r.normal(r.uniform(10.0, 90.0, size=d), sigma, size=(m, d)) for m in _even(n - n_noise, 5)]
        parts.append(r.uniform(0.0, 100.0, size=(n_noise, d)))
        X = np.concatenate(parts, axis=0)
        X = X[r.permutation(n)]
        out.append((np.ascontiguousarray(_round_lattice(X, 12).astype(np.float32)), eps, min_pts))
    return out


WORKLOADS = {
    "blobs2d": blobs2d,
    "mixed3d": mixed3d,
    "aniso16d": aniso16d,
}
