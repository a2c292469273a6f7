"""FP64 CPU oracle of the PALM / DALM l1 solvers (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``l1_oracle.c`` (plain C, IEEE
double, no BLAS) through ctypes.  It shares no code with the CUDA library in
``paper_1007_3753_gb300``; the two meet only at the seeded input generators in
``synthetic``.

Every entry point cites the passage of the paper it restates; the readings of
ambiguous passages (R1-R18) are listed at the top of ``l1_oracle.c``.

Parity pins (tests/test_oracle_pins.py) tie each function to something other
than itself: brute-force LP vertex enumeration and HiGHS on the LP of Eq. 10,
brute-force lasso enumeration, KKT / subgradient certificates (Eq. 11),
exact recovery (§VI-A), closed forms, invariances (including the independence
of the limits from beta and xi), FISTA's O(1/k^2) rate and the potential
function of its proof (§IV-A), hand-computed classification fixtures, and
central finite differences plus the adjoint identity for the unrolled
gradient.  tests/test_oracle_mutants.py plants one mistake at a time in
l1_oracle.c and checks that some pin fails on each.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "l1_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

MODE_P1, MODE_P12, MODE_QP, MODE_CAB = 0, 1, 2, 3
ERR_ARG, ERR_NOT_SPD, ERR_NOMEM = -1, -2, -3

_lock = threading.Lock()
_lib = None


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("inner_total", C.c_int), ("converged", C.c_int),
                ("rel_change", C.c_double), ("param", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class PalmOpts(C.Structure):
    _fields_ = [("mode", C.c_int), ("tol", C.c_double), ("max_outer", C.c_int),
                ("inner_max", C.c_int), ("inner_tol", C.c_double), ("xi0", C.c_double),
                ("xi_growth", C.c_double), ("xi_max", C.c_double), ("L", C.c_double),
                ("epsilon", C.c_double)]


def compile_source(src: str, out: str) -> str:
    """Compile one C source of the oracle into the shared library ``out``
    (gcc, IEEE double: no contraction into FMA, no fast-math)."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile ``l1_oracle.c`` into ``_build/liboracle.so`` with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    return compile_source(_SRC, _LIB_PATH)


def lib() -> C.CDLL:
    """The oracle library.  ``L1_ORACLE_LIB`` names another build of it (the
    planted-mistake tests load deliberately broken copies that way)."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("L1_ORACLE_LIB") or build()
            L = C.CDLL(path)
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int)
            L.orc_lipschitz.restype = C.c_double
            L.orc_lipschitz.argtypes = [dp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, ip]
            L.orc_fista_qp.restype = C.c_int
            L.orc_fista_qp.argtypes = [dp, C.c_int, C.c_int, dp, C.c_double, C.c_double,
                                       C.c_double, C.c_int, dp, C.POINTER(Stats)]
            L.orc_fista_cont.restype = C.c_int
            L.orc_fista_cont.argtypes = [dp, C.c_int, C.c_int, dp, C.c_double, C.c_double, C.c_double,
                                         C.c_double, C.c_double, C.c_int, dp, C.POINTER(Stats)]
            L.orc_amp.restype = C.c_int
            L.orc_amp.argtypes = [dp, C.c_int, C.c_int, dp, C.c_double, C.c_double, C.c_int,
                                  dp, dp, dp, C.POINTER(Stats)]
            L.orc_palm.restype = C.c_int
            L.orc_palm.argtypes = [dp, C.c_int, C.c_int, dp, C.POINTER(PalmOpts), dp, dp, dp,
                                   C.POINTER(Stats)]
            L.orc_dalm.restype = C.c_int
            L.orc_dalm.argtypes = [dp, C.c_int, C.c_int, C.c_int, dp, C.c_double, C.c_double,
                                   C.c_int, C.c_int, dp, dp, C.POINTER(Stats)]
            L.orc_palm_align.restype = C.c_int
            L.orc_palm_align.argtypes = [dp, C.c_int, C.c_int, dp, C.c_double, C.c_int, C.c_double,
                                         dp, dp, dp, C.POINTER(Stats)]
            L.orc_classify.restype = C.c_int
            L.orc_classify.argtypes = [dp, C.c_int, C.c_int, ip, C.c_int, dp, dp, dp, dp, dp,
                                       ip, ip]
            L.orc_unrolled_palm.restype = C.c_int
            L.orc_unrolled_palm.argtypes = [dp, C.c_int, C.c_int, dp, C.c_double, C.c_double,
                                            C.c_int, C.c_int, dp, dp, dp, dp, dp]
            _lib = L
    return _lib


def _f64(a, fortran: bool = False) -> np.ndarray:
    return np.asfortranarray(a, dtype=np.float64) if fortran else np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _check(rc: int, what: str):
    if rc == ERR_NOT_SPD:
        raise np.linalg.LinAlgError(f"{what}: B B^T is not positive definite")
    if rc != 0:
        raise RuntimeError(f"{what}: oracle error {rc}")


def lipschitz(A, max_iter: int = 1000, rtol: float = 1e-10, safety: float = 1.01) -> float:
    """Power-iteration bound of ||A||_2^2 (reading R4 of §IV-A / Algorithm 1)."""
    A = _f64(A, True)
    it = C.c_int(0)
    return float(lib().orc_lipschitz(_p(A), A.shape[0], A.shape[1], max_iter, rtol, safety,
                                     C.byref(it)))


def fista_qp(A, b, lam: float, L: float | None = None, tol: float = 1e-10,
             max_iter: int = 100000):
    """FISTA, Eq. 18 (§IV-A), on (QP_lambda) of Eq. 3.  Returns (x, stats)."""
    A = _f64(A, True)
    b = _f64(b)
    m, n = A.shape
    if L is None:
        L = lipschitz(A)
    x = np.zeros(n)
    st = Stats()
    _check(lib().orc_fista_qp(_p(A), m, n, _p(b), lam, L, tol, max_iter, _p(x), C.byref(st)),
           "fista_qp")
    return x, st.as_dict()


def fista_cont(A, b, lam: float, lam0: float, rho: float = 0.95, L: float | None = None,
               tol: float = 1e-10, max_iter: int = 100000):
    """FISTA with fixed-point continuation (reading R17): Eq. 18 with lambda_k
    decreasing geometrically (factor rho per iteration) from lam0 to lam.
    Returns (x, stats)."""
    A = _f64(A, True)
    b = _f64(b)
    m, n = A.shape
    if L is None:
        L = lipschitz(A)
    x = np.zeros(n)
    st = Stats()
    _check(lib().orc_fista_cont(_p(A), m, n, _p(b), lam0, lam, rho, L, tol, max_iter, _p(x), C.byref(st)),
           "fista_cont")
    return x, st.as_dict()


def amp(A, b, tau0: float = 0.0, tol: float = 1e-10, max_iter: int = 10000):
    """Approximate message passing for P1 (§IV, reading R18): x_0 = 0, z_0 = b,
    tau_0 = 1.5 ||b||_2 / sqrt(m) unless tau0 > 0.  Returns (x, z, tau, stats):
    z and tau are those of the last x-step; stats["converged"] is 1 (R6 met),
    0 (max_iter) or -1 (an iterate stopped being finite)."""
    A = _f64(A, True)
    b = _f64(b)
    m, n = A.shape
    x = np.zeros(n)
    z = np.zeros(m)
    tau = C.c_double(0.0)
    st = Stats()
    _check(lib().orc_amp(_p(A), m, n, _p(b), tau0, tol, max_iter, _p(x), _p(z), C.byref(tau), C.byref(st)),
           "amp")
    return x, z, tau.value, st.as_dict()


def palm(A, b, mode: int = MODE_CAB, tol: float = 1e-10, max_outer: int = 10000,
         inner_max: int = 50, inner_tol: float | None = None, xi0: float = 0.0,
         xi_growth: float = 1.2, xi_max: float = 1e4, L: float | None = None,
         epsilon: float = 0.0):
    """Primal ALM: Algorithm 1 (CAB), Eq. 33 + FISTA (P1), reading R10 (P1,2).

    Returns (x, e, theta, stats); e is None in P1 mode."""
    A = _f64(A, True)
    b = _f64(b)
    m, n = A.shape
    if L is None:
        L = lipschitz(A)
    o = PalmOpts(mode=mode, tol=tol, max_outer=max_outer, inner_max=inner_max,
                 inner_tol=(0.1 * tol if inner_tol is None else inner_tol), xi0=xi0,
                 xi_growth=xi_growth, xi_max=xi_max, L=L, epsilon=epsilon)
    x = np.zeros(n)
    e = np.zeros(m) if mode != MODE_P1 else None
    th = np.zeros(m)
    st = Stats()
    _check(lib().orc_palm(_p(A), m, n, _p(b), C.byref(o), _p(x), _p(e), _p(th), C.byref(st)),
           "palm")
    return x, e, th, st.as_dict()


def dalm(A, b, cab: bool = True, beta: float = 0.0, tol: float = 1e-10,
         max_iter: int = 100000, cg_steps: int = 0):
    """Dual ALM, Algorithm 2 (§V-B) with reading R1.  cg_steps > 0 replaces
    the exact y-step by that many conjugate-gradient steps from the previous
    y (the inexact variant §V-B mentions).

    Returns (w, y, stats); w = [x; e] for CAB, w = x for P1."""
    A = _f64(A, True)
    b = _f64(b)
    m, n = A.shape
    w = np.zeros(n + m if cab else n)
    y = np.zeros(m)
    st = Stats()
    _check(lib().orc_dalm(_p(A), m, n, int(bool(cab)), _p(b), beta, tol, max_iter, int(cg_steps), _p(w),
                          _p(y), C.byref(st)), "dalm")
    return w, y, st.as_dict()


def palm_align(B, b, tol: float = 1e-10, max_outer: int = 100000, xi0: float = 0.0):
    """The alignment step of §II-B, min ||e||_1 s.t. b = B w + e with w not
    penalised, by PALM with an exact least-squares w-step (reading R16).

    Returns (w, e, theta, stats)."""
    B = _f64(B, True)
    b = _f64(b)
    m, p = B.shape
    w = np.zeros(p)
    e = np.zeros(m)
    th = np.zeros(m)
    st = Stats()
    _check(lib().orc_palm_align(_p(B), m, p, _p(b), tol, max_outer, xi0, _p(w), _p(e), _p(th),
                                C.byref(st)), "palm_align")
    return w, e, th, st.as_dict()


def warp_jacobian(img, tau, rows: int, cols: int):
    """b = y o tau and its Jacobian J = d(y o tau)/d tau (§II-B), reading R19.

    tau = (a, b, tx, ty) is a similarity: canonical pixel (u, v) (column u <
    cols, row v < rows, index v*cols + u) lies at x = a u - b v + tx,
    y = b u + a v + ty of the query image img (H x W, img[y, x]).  y o tau is
    the bilinear interpolant of img there, the point first clamped to
    [0, W-1] x [0, H-1]; the cell is the one whose lower corner is
    (min(floor(x), W-2), min(floor(y), H-2)).  Its derivative in x (in y)
    is the interpolant's slope in that cell, and 0 where x (y) was clamped.
    Returns (b (m,), J (m, 4)) in FP64."""
    img = np.asarray(img, dtype=np.float64)
    H, W = img.shape
    a, bb, tx, ty = (float(t) for t in tau)
    vv, uu = np.mgrid[0:rows, 0:cols].astype(np.float64)
    u, v = uu.ravel(), vv.ravel()
    x = a * u - bb * v + tx
    y = bb * u + a * v + ty
    xc = np.clip(x, 0.0, W - 1.0)
    yc = np.clip(y, 0.0, H - 1.0)
    x0 = np.minimum(np.floor(xc), W - 2).astype(np.int64)
    y0 = np.minimum(np.floor(yc), H - 2).astype(np.int64)
    fx, fy = xc - x0, yc - y0
    p00, p01 = img[y0, x0], img[y0, x0 + 1]
    p10, p11 = img[y0 + 1, x0], img[y0 + 1, x0 + 1]
    val = (1.0 - fy) * ((1.0 - fx) * p00 + fx * p01) + fy * ((1.0 - fx) * p10 + fx * p11)
    gx = np.where((x >= 0.0) & (x <= W - 1.0), (1.0 - fy) * (p01 - p00) + fy * (p11 - p10), 0.0)
    gy = np.where((y >= 0.0) & (y <= H - 1.0), (1.0 - fx) * (p10 - p00) + fx * (p11 - p01), 0.0)
    # dx/dtau = (u, -v, 1, 0), dy/dtau = (v, u, 0, 1)
    J = np.stack([gx * u + gy * v, -gx * v + gy * u, gx, gy], axis=1)
    return val, J


def corner_shift(dtau, rows: int, cols: int) -> float:
    """Largest displacement of the four corners of the canonical frame under
    the linear change dtau of the similarity parameters (reading R19's step
    size): max over corners (u, v) of |(da u - db v + dtx, db u + da v + dty)|."""
    da, db, dtx, dty = (float(t) for t in dtau)
    best = 0.0
    for u, v in ((0, 0), (cols - 1, 0), (0, rows - 1), (cols - 1, rows - 1)):
        best = max(best, float(np.hypot(da * u - db * v + dtx, db * u + da * v + dty)))
    return best


def align_images(A, img, tau, rows: int, cols: int, tol: float = 1e-3, max_outer: int = 5000,
                 tau_tol: float = 0.05, max_align: int = 30):
    """The face-alignment loop of §II-B for one query (reading R19): from
    tau, repeat b = y o tau, J = d(y o tau)/d tau, w = [x; dtau] from the
    convex step min ||e||_1 s.t. b = [A, -J] w + e (``palm_align``, R16, to
    the relative change tol), tau <- tau + dtau, until the step moves no
    corner of the canonical frame by tau_tol pixels or more (converged) or
    max_align steps were taken.  Returns (tau, steps, converged)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[1]
    tau = np.array(tau, dtype=np.float64)
    for k in range(1, max_align + 1):
        b, J = warp_jacobian(img, tau, rows, cols)
        w, _, _, st = palm_align(np.hstack([A, -J]), b, tol=tol, max_outer=max_outer)
        dtau = w[n:n + 4]
        if not np.all(np.isfinite(dtau)):
            return tau, k, False
        tau = tau + dtau
        if corner_shift(dtau, rows, cols) < tau_tol:
            return tau, k, True
    return tau, max_align, False


def classify(A, offsets, b, x, e=None):
    """Per-class residual argmin and SCI argmax (§II-A, Eq. 40).

    Returns (label, sci_label, residuals, sci)."""
    A = _f64(A, True)
    m, n = A.shape
    off = np.ascontiguousarray(offsets, dtype=np.int32)
    Cn = len(off) - 1
    b = _f64(b)
    x = _f64(x)
    e = None if e is None else _f64(e)
    resid = np.zeros(Cn)
    sci = np.zeros(Cn)
    lab = C.c_int(-1)
    slab = C.c_int(-1)
    _check(lib().orc_classify(_p(A), m, n, off.ctypes.data_as(C.POINTER(C.c_int)), Cn, _p(b),
                              _p(x), _p(e), _p(resid), _p(sci), C.byref(lab), C.byref(slab)),
           "classify")
    return lab.value, slab.value, resid, sci


def unrolled_palm(A, b, xi: float, L: float, K: int, J: int, x_target, grad: bool = True):
    """Unrolled PALM (reading R11) for one right-hand side and its reverse sweep.

    Returns (x_K, loss, grad_A, grad_b); the gradients are None if grad=False."""
    A = _f64(A, True)
    b = _f64(b)
    xt = _f64(x_target)
    m, n = A.shape
    x = np.zeros(n)
    loss = C.c_double(0.0)
    gA = np.zeros((m, n), order="F") if grad else None
    gb = np.zeros(m) if grad else None
    _check(lib().orc_unrolled_palm(_p(A), m, n, _p(b), xi, L, K, J, _p(xt), _p(x),
                                   C.byref(loss), _p(gA), _p(gb)), "unrolled_palm")
    return x, loss.value, gA, gb
