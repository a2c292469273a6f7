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
* ``p1_batch`` -- N noise-free P1 right-hand sides on one Gaussian dictionary.
* ``alignment_images`` -- the alignment experiment of §VI-C on synthetic
  faces (Multi-PIE is not available): per task a smooth "face" (a sum of
  Gaussian blobs on the 40 x 30 canonical frame), n = 7 training images under
  different smooth illuminations, and an 80 x 60 query image showing the
  face under a random mix of those illuminations at a known similarity
  transformation, with a block of 10 % of the face area replaced by noise
  (the paper's occluding baboon block); the starting transformation is the
  true one moved by 4 pixels along x (translation) or rotated by 15 degrees
  about the frame centre (rotation).
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
    "p1_batch",
    "alignment_images",
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


def _similarity_inverse(tau, x, y):
    """Canonical coordinates (u, v) that the similarity tau = (a, b, tx, ty)
    maps to image coordinates (x, y) = (a u - b v + tx, b u + a v + ty)."""
    a, b, tx, ty = tau
    d = a * a + b * b
    xx, yy = x - tx, y - ty
    return (a * xx + b * yy) / d, (-b * xx + a * yy) / d


def alignment_images(count: int, kind: str = "translation", rows: int = 40, cols: int = 30, n_train: int = 7,
                     H: int = 80, W: int = 60, occlusion: float = 0.1, seed: int = 7000) -> dict:
    """``count`` alignment tasks (§II-B, §VI-C), each with its own subject.

    Returns A (count, rows*cols, n_train; pixel (v, u) of the canonical frame
    at index v*cols + u), img (count, H, W; row-major, pixel (y, x) at
    [y, x]), tau_true and tau_init (count, 4) as (a, b, tx, ty): canonical
    pixel (u, v) lies at (a u - b v + tx, b u + a v + ty) in the query image.
    The true transformation is the identity similarity centring the frame
    in the query image.  ``kind``: "translation" (4 pixels along x) or
    "rotation" (15 degrees about the frame centre)."""
    g = rng(seed)
    m = rows * cols
    vv, uu = np.mgrid[0:rows, 0:cols].astype(np.float64)
    u, v = uu.ravel(), vv.ravel()
    yq, xq = np.mgrid[0:H, 0:W].astype(np.float64)
    A = np.zeros((count, m, n_train))
    img = np.zeros((count, H, W))
    t_true = np.array([1.0, 0.0, (W - cols) / 2.0, (H - rows) / 2.0])
    tau_true = np.tile(t_true, (count, 1))
    tau_init = np.zeros((count, 4))
    side = int(round(np.sqrt(occlusion * m)))
    for k in range(count):
        nb = 24
        bu, bv = g.uniform(2, cols - 2, nb), g.uniform(2, rows - 2, nb)
        bs, ba = g.uniform(1.8, 4.0, nb), g.uniform(0.3, 1.0, nb)
        lin = g.uniform(-0.6, 0.6, (n_train, 2))
        lu, lv = g.uniform(0, cols, n_train), g.uniform(0, rows, n_train)
        ls, la = g.uniform(10, 20, n_train), g.uniform(0.3, 1.0, n_train)

        def face(pu, pv):
            out = 0.2 + np.zeros(np.broadcast(pu, pv).shape)
            for j in range(nb):
                out = out + ba[j] * np.exp(-((pu - bu[j]) ** 2 + (pv - bv[j]) ** 2) / (2 * bs[j] ** 2))
            return out

        def light(l, pu, pv):
            return (1 + lin[l, 0] * (pu - cols / 2) / cols + lin[l, 1] * (pv - rows / 2) / rows
                    + la[l] * np.exp(-((pu - lu[l]) ** 2 + (pv - lv[l]) ** 2) / (2 * ls[l] ** 2)))

        fa = face(u, v)
        for l in range(n_train):
            A[k, :, l] = fa * light(l, u, v)
        c = g.dirichlet(np.ones(n_train))
        pu, pv = _similarity_inverse(t_true, xq, yq)
        img[k] = face(pu, pv) * sum(c[l] * light(l, pu, pv) for l in range(n_train))
        oy = int(g.integers(int(t_true[3]), int(t_true[3]) + rows - side))
        ox = int(g.integers(int(t_true[2]), int(t_true[2]) + cols - side))
        img[k, oy:oy + side, ox:ox + side] = g.uniform(0.0, 1.0, (side, side))
        if kind == "translation":
            tau_init[k] = t_true + np.array([0.0, 0.0, 4.0, 0.0])
        elif kind == "rotation":
            th = np.deg2rad(15.0)
            a, b = np.cos(th), np.sin(th)
            cu, cv = (cols - 1) / 2.0, (rows - 1) / 2.0
            tau_init[k] = [a, b, t_true[2] + cu - (a * cu - b * cv), t_true[3] + cv - (b * cu + a * cv)]
        else:
            raise ValueError(kind)
    return {"A": A, "img": img, "tau_true": tau_true, "tau_init": tau_init, "rows": rows, "cols": cols}
