"""Seeded synthetic inputs shaped like the paper's workloads.

This module is the one piece shared by the FP64 oracle (under ``oracle/``) and
the CUDA path (``paper_1007_3753_gb300``): it draws problem data and nothing
else.  It contains none of the solvers' arithmetic.  Every array is FP64,
column-major (Fortran order) so that the oracle reads it without a copy; the
CUDA path receives an FP32 cast.

Workload recipes (the paper's Multi-PIE face database is not available, so
the cross-and-bouquet generator stands in for it, following the shapes of
§VI-B: 40x30-pixel images give m = 1200-class row counts, a fraction p of the
pixels is replaced by uniform noise):

* ``p1_instance`` -- §VI-A: i.i.d. Gaussian A with unit-norm columns, a
  d-sparse x0 with random support, b = A x0.  Entries of x0 are Rademacher
  (+-1) by default, or uniform in [-10, 10] as in §VI-A.
* ``cab_problem`` -- §II-A (Eq. 5, the cross-and-bouquet model): C classes,
  each class a rank-r nonnegative subspace; training columns are random
  nonnegative combinations of the class basis plus 1 % Gaussian noise,
  normalised to unit l2 norm; a test vector is a combination of one class's
  basis, rescaled to peak 1, with a fraction of its entries replaced by
  uniform [0, 1] gross errors.
* ``qp_group_sizes`` / ``qp_instance`` -- many (QP_lambda) instances (Eq. 3)
  of uneven size: m log-uniform in [256, 4096], n/m log-uniform in [2, 4]
  (n rounded to a multiple of 8), Gaussian unit-column A, k = m/10 sparse
  N(0,1) x0, b = A x0 + N(0, 0.01^2).
* ``unrolled_instance`` -- unrolled PALM differentiation: Gaussian
  unit-column A, k-sparse N(0,1) targets, b = A x_target + N(0, 0.01^2).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng",
    "gaussian_dictionary",
    "p1_instance",
    "cab_problem",
    "qp_group_sizes",
    "qp_instance",
    "unrolled_instance",
]


def rng(seed: int) -> np.random.Generator:
    """Counter-stable PCG64 stream for ``seed``."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def _unit_columns(A: np.ndarray) -> np.ndarray:
    nrm = np.sqrt(np.sum(A * A, axis=0, keepdims=True))
    nrm[nrm == 0] = 1.0
    return np.asfortranarray(A / nrm)


def gaussian_dictionary(m: int, n: int, g: np.random.Generator) -> np.ndarray:
    """i.i.d. N(0,1) entries, each column scaled to unit l2 norm (§VI-A)."""
    return _unit_columns(g.standard_normal((m, n)))


def p1_instance(m: int = 200, n: int = 400, k: int = 20, seed: int = 0,
                entries: str = "pm1") -> dict:
    """Noise-free basis-pursuit instance b = A x0 with a k-sparse x0.

    ``entries`` is ``"pm1"`` (Rademacher) or ``"uniform10"`` (U[-10, 10],
    the distribution §VI-A states).
    """
    g = rng(seed)
    A = gaussian_dictionary(m, n, g)
    support = g.choice(n, size=k, replace=False)
    x0 = np.zeros(n)
    if entries == "pm1":
        x0[support] = g.choice(np.array([-1.0, 1.0]), size=k)
    elif entries == "uniform10":
        x0[support] = g.uniform(-10.0, 10.0, size=k)
    else:
        raise ValueError(entries)
    b = A @ x0
    return {"A": A, "x0": x0, "b": b, "support": np.sort(support)}


def p1_batch(m: int, n: int, k: int, N: int, seed: int = 0, entries: str = "uniform10") -> dict:
    """N noise-free basis-pursuit right-hand sides b_j = A x0_j on one
    Gaussian unit-column dictionary, each x0_j k-sparse on its own random
    support (entries as in ``p1_instance``)."""
    g = rng(seed)
    A = gaussian_dictionary(m, n, g)
    X0 = np.zeros((n, N), order="F")
    for j in range(N):
        s = g.choice(n, size=k, replace=False)
        if entries == "pm1":
            X0[s, j] = g.choice(np.array([-1.0, 1.0]), size=k)
        elif entries == "uniform10":
            X0[s, j] = g.uniform(-10.0, 10.0, size=k)
        else:
            raise ValueError(entries)
    B = np.asfortranarray(A @ X0)
    return {"A": A, "X0": X0, "B": B}


def cab_problem(m: int, classes: int, per_class: int, n_test: int,
                corrupt: float = 0.3, rank: int = 9, noise: float = 0.01,
                seed: int = 1000) -> dict:
    """Cross-and-bouquet dictionary A (m x classes*per_class) and test set.

    Returns ``A`` (unit columns), ``offsets`` (class c owns columns
    offsets[c]:offsets[c+1]), ``B`` (m x n_test test vectors, column-major),
    ``labels`` (true class of each test vector) and ``corrupted`` (boolean
    mask of the replaced entries).
    """
    g = rng(seed)
    n = classes * per_class
    A = np.empty((m, n), order="F")
    bases = []
    for c in range(classes):
        U = g.uniform(0.0, 1.0, size=(m, rank))
        bases.append(U)
        alpha = g.uniform(0.0, 1.0, size=(rank, per_class))
        cols = U @ alpha
        z = g.standard_normal((m, per_class))
        z *= noise * np.linalg.norm(cols, axis=0) / np.linalg.norm(z, axis=0)
        A[:, c * per_class:(c + 1) * per_class] = cols + z
    A = _unit_columns(A)
    offsets = np.arange(classes + 1, dtype=np.int32) * per_class
    labels = g.integers(0, classes, size=n_test).astype(np.int32)
    B = np.empty((m, n_test), order="F")
    corrupted = np.zeros((m, n_test), dtype=bool, order="F")
    n_bad = int(np.floor(corrupt * m))
    for j in range(n_test):
        alpha = g.uniform(0.0, 1.0, size=rank)
        b0 = bases[labels[j]] @ alpha
        b0 /= np.max(b0)
        idx = g.choice(m, size=n_bad, replace=False)
        b0[idx] = g.uniform(0.0, 1.0, size=n_bad)
        corrupted[idx, j] = True
        B[:, j] = b0
    return {"A": A, "offsets": offsets, "B": B, "labels": labels,
            "corrupted": corrupted}


def qp_group_sizes(count: int = 8192, seed: int = 4000, m_lo: int = 256,
                   m_hi: int = 4096, r_lo: float = 2.0, r_hi: float = 4.0):
    """Sizes (m_i, n_i) of an uneven QP_lambda batch (log-uniform m, n/m)."""
    g = rng(seed)
    m = np.exp(g.uniform(np.log(m_lo), np.log(m_hi), size=count))
    m = np.clip(np.rint(m), m_lo, m_hi).astype(np.int64)
    r = np.exp(g.uniform(np.log(r_lo), np.log(r_hi), size=count))
    n = (np.rint(r * m / 8.0) * 8).astype(np.int64)
    n = np.maximum(n, 8)
    return m, n


def qp_instance(m: int, n: int, seed: int, noise: float = 0.01,
                sparsity: float = 0.1) -> dict:
    """One (QP_lambda) instance: Gaussian unit-column A, k = m/10 sparse x0."""
    g = rng(seed)
    A = gaussian_dictionary(m, n, g)
    k = max(1, int(m * sparsity))
    support = g.choice(n, size=k, replace=False)
    x0 = np.zeros(n)
    x0[support] = g.standard_normal(k)
    b = A @ x0 + noise * g.standard_normal(m)
    return {"A": A, "x0": x0, "b": b}


def unrolled_instance(m: int = 1024, n: int = 2048, N: int = 256, k: int = 50,
                      noise: float = 0.01, seed: int = 5000) -> dict:
    """Batch of N targets for unrolled-PALM differentiation."""
    g = rng(seed)
    A = gaussian_dictionary(m, n, g)
    X = np.zeros((n, N), order="F")
    for j in range(N):
        s = g.choice(n, size=k, replace=False)
        X[s, j] = g.standard_normal(k)
    B = np.asfortranarray(A @ X + noise * g.standard_normal((m, N)))
    return {"A": A, "X_target": X, "B": B}
