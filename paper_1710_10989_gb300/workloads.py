"""Seeded synthetic inputs shaped like the paper's experiments (Section 4).

This module holds input generation only -- none of the exponential's
arithmetic -- and is the one piece that both the CUDA path's tests/benchmark
and the CPU oracle's tests use. Every generator is numpy ``default_rng(seed)``
(PCG64) in float64 on the host. The 1-norm rescaling uses numpy's own
column sums; it only places the input at the intended norm.

Stand-ins: the paper measures on 46 MATLAB gallery matrices and a set of
random matrices (Section 4, Fig. 2); neither set is available, so these
seeded Gaussian / non-normal / diagonalisable families stand in for them.
"""
from __future__ import annotations

import numpy as np

# Dense single-matrix workloads: one run per (norm, seed).
SMALL_N = 64
SMALL_SEED = 0
SMALL_NORM = 1.0
DENSE_N = 4096
DENSE_NORMS = (0.01, 0.1, 1.0, 5.0, 20.0, 100.0)
DENSE_SEEDS = (1, 2, 3, 4, 5, 6)
NONNORMAL_SEEDS = (101, 102, 103, 104, 105, 106)
LARGE_N = 8192
LARGE_NORMS = (0.5, 5.0, 50.0)
LARGE_SEEDS = (1, 2, 3)
# Batched workload.
BATCH_COUNT = 20000
BATCH_SEED = 7
BATCH_SIZES = tuple(range(8, 257, 8))
BATCH_NORM_RANGE = (1e-3, 1e2)


def rescale_norm1(A: np.ndarray, target: float) -> np.ndarray:
    """Scale A so that its maximum absolute column sum is `target`."""
    cur = np.abs(A).sum(axis=0).max()
    if cur == 0:
        return A
    return A * (target / cur)


def gaussian(n: int, seed: int, norm1: float | None = None, scale_sqrt_n: bool = True) -> np.ndarray:
    """iid N(0,1) entries (divided by sqrt(n) when asked), rescaled to 1-norm `norm1`."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    if scale_sqrt_n:
        A /= np.sqrt(n)
    return rescale_norm1(A, norm1) if norm1 is not None else A


def nonnormal_upper(n: int, seed: int, norm1: float | None = None) -> np.ndarray:
    """Upper triangular: diagonal N(0,1), strict upper part N(0,1) * 10."""
    rng = np.random.default_rng(seed)
    A = np.triu(rng.standard_normal((n, n)) * 10.0, 1)
    A[np.diag_indices(n)] = rng.standard_normal(n)
    return rescale_norm1(A, norm1) if norm1 is not None else A


def conditioned_basis(n: int, rng: np.random.Generator, cond: float = 1e3) -> np.ndarray:
    """V = U diag(logspace(0, -log10(cond), n)) W^T with U, W orthogonal (QR of
    Gaussians, signs fixed), so the 2-norm condition number of V is `cond`."""
    def orth():
        Q, R = np.linalg.qr(rng.standard_normal((n, n)))
        return Q * np.sign(np.diag(R))
    U, W = orth(), orth()
    sv = np.logspace(0.0, -np.log10(cond), n)
    return (U * sv) @ W.T


def diagonalisable(n: int, seed: int, norm1: float | None = None) -> np.ndarray:
    """A = V diag(lambda) V^-1 with lambda ~ N(0, 4) and cond_2(V) = 1e3."""
    rng = np.random.default_rng(seed)
    lam = rng.standard_normal(n) * 2.0
    V = conditioned_basis(n, rng)
    A = (V * lam) @ np.linalg.inv(V)
    return rescale_norm1(A, norm1) if norm1 is not None else A


def dense_case(index: int, n: int = DENSE_N, nonnormal: bool = False) -> np.ndarray:
    """One of the six dense runs (index 0..5 -> norms 0.01 .. 100)."""
    if nonnormal:
        return nonnormal_upper(n, NONNORMAL_SEEDS[index], DENSE_NORMS[index])
    return gaussian(n, DENSE_SEEDS[index], DENSE_NORMS[index])


def large_case(index: int, n: int = LARGE_N) -> np.ndarray:
    return gaussian(n, LARGE_SEEDS[index], LARGE_NORMS[index])


def small_case() -> np.ndarray:
    """64 x 64, N(0,1) entries from seed 0, 1-norm 1.0."""
    return gaussian(SMALL_N, SMALL_SEED, SMALL_NORM, scale_sqrt_n=False)


def batch_spec(count: int = BATCH_COUNT, seed: int = BATCH_SEED,
               sizes=BATCH_SIZES, norm_range=BATCH_NORM_RANGE):
    """Sizes and target norms of the batched workload (no matrices yet)."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(sizes), size=count)
    lo, hi = np.log(norm_range[0]), np.log(norm_range[1])
    norms = np.exp(rng.uniform(lo, hi, size=count))
    return ns.astype(np.int64), norms


def batch_matrix(i: int, n: int, norm1: float, seed: int = BATCH_SEED) -> np.ndarray:
    """Matrix i of the batch: even i Gaussian, odd i diagonalisable; float64."""
    s = seed * 1_000_003 + i
    if i % 2 == 0:
        return gaussian(int(n), s, norm1)
    return diagonalisable(int(n), s, norm1)
