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
    """A = V diag(lambda) V^-1 with lambda ~ N(0, 4) and cond_2(V) = 1e3, where
    V = U S W^T, so V^-1 = W S^-1 U^T exactly (U, W orthogonal)."""
    rng = np.random.default_rng(seed)
    lam = rng.standard_normal(n) * 2.0

    def orth():
        Q, R = np.linalg.qr(rng.standard_normal((n, n)))
        return Q * np.sign(np.diag(R))
    U, Wm = orth(), orth()
    sv = np.logspace(0.0, -3.0, n)
    V = (U * sv) @ Wm.T
    Vinv = (Wm / sv) @ U.T
    A = (V * lam) @ Vinv
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


def _batch_chunk(args):
    lo, hi, ns, norms, seed = args
    return [batch_matrix(i, int(ns[i - lo]), float(norms[i - lo]), seed).astype(np.float32)
            for i in range(lo, hi)]


def _batch_pick(args):
    idx, ns, norms, seed = args
    return [batch_matrix(int(i), int(n), float(v), seed).astype(np.float32) for i, n, v in zip(idx, ns, norms)]


def batch_matrices(count: int = BATCH_COUNT, seed: int = BATCH_SEED, workers: int = 0):
    """All matrices of the batched workload as binary32 arrays (their storage type).

    Canonical generation: LAPACK's QR gives last-bit differences with the BLAS
    thread count, so the matrices are always built in worker processes started
    with 'spawn' and single-threaded BLAS (safe before or after CUDA starts);
    the result does not depend on `workers` (0 = one per core, at most 16)."""
    import multiprocessing as mp
    import os
    ns, norms = batch_spec(count, seed)
    workers = workers or min(16, os.cpu_count() or 1)
    step = max(1, (count + workers * 4 - 1) // (workers * 4))
    jobs = [(lo, min(count, lo + step), ns[lo:lo + step], norms[lo:lo + step], seed)
            for lo in range(0, count, step)]
    keys = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(workers) as pool:
            parts = pool.map(_batch_chunk, jobs)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return [m for part in parts for m in part]


def batch_matrices_subset(indices, count: int = BATCH_COUNT, seed: int = BATCH_SEED, workers: int = 0):
    """Matrices `indices` of the batch of `count` (a rank's shard), generated as
    canonically as batch_matrices (spawned single-threaded-BLAS workers)."""
    import multiprocessing as mp
    import os
    ns, norms = batch_spec(count, seed)
    idx = np.asarray(list(indices), dtype=np.int64)
    workers = workers or min(16, os.cpu_count() or 1)
    parts = np.array_split(np.arange(len(idx)), max(1, workers * 4))
    jobs = [(idx[p], ns[idx[p]], norms[idx[p]], seed) for p in parts if len(p)]
    keys = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(workers) as pool:
            out = pool.map(_batch_pick, jobs)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return [m for part in out for m in part]
