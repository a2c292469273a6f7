"""Python binding of libl1alm: GB300 (sm_103a) PALM / DALM l1 solvers.

Thin ctypes layer over the C ABI declared in ``include/l1alm.h``: argument
marshalling only.  Every step of a solve runs in the library's CUDA kernels;
PyTorch supplies device memory and the current stream.  There is no CPU
fallback: if the compiled library is missing, importing the solver raises.

Method: Yang, Zhou, Ganesh, Sastry, Ma, "Fast l1-Minimization Algorithms for
Robust Face Recognition" -- Algorithm 1 (PALM), Algorithm 2 (DALM), FISTA
(Eq. 18) and the per-class residual / SCI classifiers (§II-A, Eq. 40).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libl1alm.so")

P1, P1_2, QP_LAMBDA, CAB = 0, 1, 2, 3
PALM, DALM, AMP = 0, 1, 2
A_FP32, A_BF16, A_FP8E4M3 = 0, 1, 2
ENGINE_AUTO, ENGINE_SIMT, ENGINE_TC = 0, 1, 2
OK, ERR_INVALID_ARG, ERR_NOT_SPD, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_NO_TAPE, ERR_UNSUPPORTED = \
    0, -1, -2, -3, -4, -5, -6, -7
CONVERGED, MAX_ITER, NONFINITE = 0, 1, 2

# every symbol include/l1alm.h declares
EXPORTS = ("l1_options_init", "l1_setup", "l1_setup_group", "l1_group_load", "l1_solve_batch",
           "l1_backward", "l1_set_stream", "l1_get_info", "l1_destroy", "l1_status_string",
           "l1_last_error", "l1_lipschitz_static", "l1_solve_plain", "l1_tuning", "l1_align_batch",
           "l1_align_warp", "l1_align_images")


class Options(C.Structure):
    _fields_ = [("solver", C.c_int32), ("precision", C.c_int32), ("engine", C.c_int32),
                ("inner_max", C.c_int32), ("lambda_", C.c_double), ("epsilon", C.c_double),
                ("xi0", C.c_double), ("xi_growth", C.c_double), ("xi_max", C.c_double),
                ("beta", C.c_double), ("lipschitz", C.c_double), ("inner_tol", C.c_double),
                ("check_every", C.c_int32), ("class_count", C.c_int32),
                ("class_offsets", C.POINTER(C.c_int32)), ("stream", C.c_void_p),
                ("unroll_K", C.c_int32), ("unroll_J", C.c_int32), ("ckpt_every", C.c_int32),
                ("profile", C.c_int32), ("tc_pieces", C.c_int32), ("refine", C.c_int32),
                ("tc_pieces_y", C.c_int32), ("tc_min_cols", C.c_int32), ("tune", C.c_int32),
                ("cg_steps", C.c_int32), ("lambda0", C.c_double), ("cont_rho", C.c_double),
                ("tau0", C.c_double)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("inner_iters", C.c_int32),
                ("label", C.c_int32), ("sci_label", C.c_int32), ("reserved", C.c_int32),
                ("rel_change", C.c_double), ("primal_obj", C.c_double), ("dual_obj", C.c_double),
                ("gap", C.c_double), ("resid", C.c_double), ("param", C.c_double)]


class Info(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("mode", C.c_int32), ("solver", C.c_int32),
                ("precision", C.c_int32), ("engine", C.c_int32), ("lipschitz", C.c_double),
                ("setup_ms", C.c_double), ("device_bytes", C.c_int64), ("gpu_launches", C.c_int64),
                ("sweep_launches", C.c_int64 * 4), ("sweep_ms", C.c_double * 4),
                ("sweep_flop", C.c_double * 4)]


RESULT_FIELDS = [f for f, _ in Result._fields_ if f != "reserved"]

_lib = None


class L1Error(RuntimeError):
    def __init__(self, code: int, what: str):
        lib = load()
        msg = lib.l1_status_string(code).decode()
        extra = lib.l1_last_error().decode() if code == ERR_CUDA else ""
        super().__init__(f"{what}: {msg} ({code}) {extra}".strip())
        self.code = code


def load() -> C.CDLL:
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libl1alm.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    L.l1_options_init.argtypes = [C.POINTER(Options)]
    L.l1_options_init.restype = None
    L.l1_setup.argtypes = [vp, i64, i64, i64, i32, C.POINTER(Options), C.POINTER(vp)]
    L.l1_setup.restype = C.c_int
    L.l1_setup_group.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), i64, i32, C.POINTER(Options),
                                 C.POINTER(vp)]
    L.l1_setup_group.restype = C.c_int
    L.l1_group_load.argtypes = [vp, i64, i64, vp]
    L.l1_group_load.restype = C.c_int
    L.l1_solve_batch.argtypes = [vp, vp, i64, i64, dbl, i32, vp, i64, vp, i64, C.POINTER(Result), vp, i64,
                                 vp, i64]
    L.l1_solve_batch.restype = C.c_int
    L.l1_backward.argtypes = [vp, vp, i64, vp, vp]
    L.l1_backward.restype = C.c_int
    L.l1_set_stream.argtypes = [vp, vp]
    L.l1_set_stream.restype = C.c_int
    L.l1_get_info.argtypes = [vp, C.POINTER(Info)]
    L.l1_get_info.restype = C.c_int
    L.l1_destroy.argtypes = [vp]
    L.l1_destroy.restype = C.c_int
    L.l1_status_string.argtypes = [C.c_int]
    L.l1_status_string.restype = C.c_char_p
    L.l1_last_error.argtypes = []
    L.l1_last_error.restype = C.c_char_p
    L.l1_lipschitz_static.argtypes = [vp, i64, i64, i64, i32, dbl, vp, C.POINTER(dbl), C.POINTER(i32),
                                      C.POINTER(i32)]
    L.l1_lipschitz_static.restype = C.c_int
    L.l1_solve_plain.argtypes = [vp, vp, dbl, i32, vp, C.POINTER(Result)]
    L.l1_solve_plain.restype = C.c_int
    L.l1_tuning.argtypes = [vp, C.POINTER(i32), i32]
    L.l1_tuning.restype = C.c_int
    L.l1_align_batch.argtypes = [vp, i64, i64, i64, i64, vp, i64, i64, dbl, i32, dbl, vp, vp, vp,
                                 C.POINTER(Result)]
    L.l1_align_batch.restype = C.c_int
    L.l1_align_warp.argtypes = [vp, i64, i64, i64, vp, i64, i32, i32, i32, vp, vp, i64, i64, vp, i64, vp]
    L.l1_align_warp.restype = C.c_int
    L.l1_align_images.argtypes = [vp, i64, i64, i64, vp, i32, i64, i32, i32, i64, vp, dbl, i32, dbl, i32, vp,
                                  C.POINTER(i32), C.POINTER(i32)]
    L.l1_align_images.restype = C.c_int
    _lib = L
    return L


def _ptr(a):
    """Address of a float32 torch tensor (device or host) or numpy array.

    Every buffer of the C ABI holds FP32 values: another dtype would make the
    library read or write past the end of the buffer, and a CUDA tensor on a
    device other than the current one would be dereferenced as a peer
    pointer, so both are refused here, before any call."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float32:
            raise TypeError(f"expected a float32 tensor, got {a.dtype}")
        if a.is_cuda and a.device.index is not None and a.device.index != torch.cuda.current_device():
            raise ValueError(f"tensor on cuda:{a.device.index} but cuda:{torch.cuda.current_device()} is current")
        return C.c_void_p(a.data_ptr())
    if a.dtype != np.float32:
        raise TypeError(f"expected a float32 array, got {a.dtype}")
    return C.c_void_p(a.ctypes.data)


def _check(rc: int, what: str):
    if rc != OK:
        raise L1Error(rc, what)


def _ld(a) -> int:
    """Leading dimension of a column-major 2-D array / tensor (or a vector)."""
    if a.ndim == 1:
        return a.shape[0]
    st = a.stride() if hasattr(a, "stride") and callable(a.stride) else tuple(s // a.itemsize for s in a.strides)
    if st[0] != 1:
        raise ValueError("expected a column-major (Fortran-order) 2-D array")
    return max(st[1], a.shape[0])


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:  # pragma: no cover - torch without CUDA
        pass
    return C.c_void_p(None)


class Solver:
    """A handle of the C ABI: one dictionary A, many right-hand sides.

    ``A`` is m x n FP32 column-major, host (numpy, Fortran order) or device
    (a torch CUDA tensor whose transpose is contiguous, e.g. ``A.t().contiguous().t()``).
    """

    def __init__(self, A, mode: int = CAB, solver: int = DALM, *, lam: float = 0.0,
                 epsilon: float = 0.0, beta: float = 0.0, xi0: float = 0.0,
                 xi_growth: float = 0.0, xi_max: float = 0.0, lipschitz: float = 0.0,
                 inner_max: int = 0, inner_tol: float = 0.0, check_every: int = 0,
                 class_offsets=None, precision: int = A_FP32, engine: int = ENGINE_AUTO,
                 profile: bool = False, tc_pieces: int = 0, tc_pieces_y: int = 0, tc_min_cols: int = 0,
                 unroll_K: int = 0, unroll_J: int = 0, ckpt_every: int = 0, refine: bool = True,
                 tune: bool = True, cg_steps: int = 0, lam0: float = 0.0, cont_rho: float = 0.0,
                 tau0: float = 0.0, stream=None):
        L = load()
        o = Options()
        L.l1_options_init(C.byref(o))
        o.solver, o.precision, o.engine = solver, precision, engine
        if inner_max:
            o.inner_max = inner_max
        o.lambda_, o.epsilon, o.beta, o.xi0 = lam, epsilon, beta, xi0
        if xi_growth:
            o.xi_growth = xi_growth
        if xi_max:
            o.xi_max = xi_max
        o.lipschitz, o.inner_tol = lipschitz, inner_tol
        o.profile = 1 if profile else 0
        o.tc_pieces, o.tc_pieces_y, o.tc_min_cols = tc_pieces, tc_pieces_y, tc_min_cols
        o.unroll_K = unroll_K
        o.refine = 0 if refine else -1
        o.tune = 0 if tune else -1
        o.cg_steps = cg_steps
        o.lambda0, o.cont_rho = lam0, cont_rho
        o.tau0 = tau0
        if unroll_J:
            o.unroll_J = unroll_J
        if ckpt_every:
            o.ckpt_every = ckpt_every
        if check_every:
            o.check_every = check_every
        self._offsets = None
        if class_offsets is not None:
            self._offsets = np.ascontiguousarray(class_offsets, dtype=np.int32)
            o.class_count = len(self._offsets) - 1
            o.class_offsets = self._offsets.ctypes.data_as(C.POINTER(C.c_int32))
        o.stream = stream if stream is not None else _current_stream()
        if isinstance(A, np.ndarray):
            A = np.asfortranarray(A, dtype=np.float32)
        m, n = A.shape
        h = C.c_void_p()
        _check(L.l1_setup(_ptr(A), m, n, _ld(A), mode, C.byref(o), C.byref(h)), "l1_setup")
        self._h = h
        self.m, self.n, self.mode, self.solver = m, n, mode, solver

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = Info()
        _check(load().l1_get_info(self._h, C.byref(inf)), "l1_get_info")
        out = {}
        for k, _ in Info._fields_:
            v = getattr(inf, k)
            out[k] = list(v) if k.startswith("sweep_") else v
        return out

    def solve(self, b, tol: float, max_iter: int, x=None, y=None, want_y: bool = False, x_init=None,
              y_init=None):
        """Solve one problem per column of b (m x N).

        b may be a host numpy array or a torch tensor (device or host,
        column-major).  Outputs are allocated like b when not given: x is
        (n + m) x N for CAB ([x; e] per column), n x N otherwise; y (the dual
        iterate) only if ``want_y`` or given.  ``x_init`` / ``y_init`` (laid
        out like x / y) warm-start the iteration.  Returns (x, y, results).
        """
        L = load()
        is_np = isinstance(b, np.ndarray)
        if is_np:
            b = np.asfortranarray(b, dtype=np.float32)
            if b.ndim == 1:
                b = b.reshape(-1, 1, order="F")
        elif b.dim() == 1:
            b = b.reshape(-1, 1)
        N = b.shape[1]
        nx = self.n + self.m if self.mode == CAB else self.n
        if x is None:
            if is_np:
                x = np.zeros((nx, N), dtype=np.float32, order="F")
            else:
                import torch
                x = torch.empty((N, nx), dtype=torch.float32, device=b.device).t()
        if y is None and want_y:
            if is_np:
                y = np.zeros((self.m, N), dtype=np.float32, order="F")
            else:
                import torch
                y = torch.empty((N, self.m), dtype=torch.float32, device=b.device).t()
        res = (Result * N)()
        if isinstance(x_init, np.ndarray):
            x_init = np.asfortranarray(x_init, dtype=np.float32)
        if isinstance(y_init, np.ndarray):
            y_init = np.asfortranarray(y_init, dtype=np.float32)
        _check(L.l1_solve_batch(self._h, _ptr(b), _ld(b), N, float(tol), int(max_iter), _ptr(x), _ld(x),
                                _ptr(y), _ld(y) if y is not None else 0, res,
                                _ptr(x_init), _ld(x_init) if x_init is not None else 0,
                                _ptr(y_init), _ld(y_init) if y_init is not None else 0), "l1_solve_batch")
        return x, y, results_to_dict(res)

    def tuning(self) -> list:
        """l1_tuning: the autotuner's tile strategies, one dict per (sweep
        shape, tile count)."""
        cap = 256
        buf = (C.c_int32 * (7 * cap))()
        k = load().l1_tuning(self._h, buf, cap)
        _check(k if k < 0 else 0, "l1_tuning")
        return [dict(zip(("M", "K", "tiles", "ksplit", "deferred", "bn", "us"), buf[7 * e:7 * e + 7]))
                for e in range(k)]

    def solve_plain(self, b, tol: float, max_iter: int, x=None):
        """l1_solve_plain: DALM for one right-hand side b (m) with plain,
        unfused FP32 kernels (the baseline of the batched solve).  Returns
        (x, result dict)."""
        L = load()
        is_np = isinstance(b, np.ndarray)
        if is_np:
            b = np.ascontiguousarray(b, dtype=np.float32).reshape(-1)
        nx = self.n + self.m if self.mode == CAB else self.n
        if x is None:
            if is_np:
                x = np.zeros(nx, dtype=np.float32)
            else:
                import torch
                x = torch.empty(nx, dtype=torch.float32, device=b.device)
        res = (Result * 1)()
        _check(L.l1_solve_plain(self._h, _ptr(b), float(tol), int(max_iter), _ptr(x), res), "l1_solve_plain")
        return x, {k: v[0] for k, v in results_to_dict(res).items()}

    def backward(self, grad_x, grad_b=None, grad_A=None, want_b: bool = True, want_A: bool = True):
        """l1_backward after an unrolled forward: grad_x is n x N (column-major,
        like x); returns (grad_b m x N, grad_A m x n), allocated like grad_x
        when not given (None where not wanted)."""
        L = load()
        is_np = isinstance(grad_x, np.ndarray)
        if is_np:
            grad_x = np.asfortranarray(grad_x, dtype=np.float32)
        if _ld(grad_x) != self.n:
            raise ValueError("grad_x must be n x N with leading dimension n")
        N = grad_x.shape[1]

        def alloc(rows, cols):
            if is_np:
                return np.zeros((rows, cols), dtype=np.float32, order="F")
            import torch
            return torch.empty((cols, rows), dtype=torch.float32, device=grad_x.device).t()
        if grad_b is None and want_b:
            grad_b = alloc(self.m, N)
        if grad_A is None and want_A:
            grad_A = alloc(self.m, self.n)
        for t in (grad_b, grad_A):
            if t is not None and _ld(t) != self.m:
                raise ValueError("grad_b and grad_A must have leading dimension m")
        _check(L.l1_backward(self._h, _ptr(grad_x), N, _ptr(grad_b), _ptr(grad_A)), "l1_backward")
        return grad_b, grad_A

    def set_stream(self, stream):
        _check(load().l1_set_stream(self._h, stream), "l1_set_stream")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().l1_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Group:
    """A handle over an uneven batch of (QP_lambda) problems (l1_setup_group).

    ``As`` is a list of m_i x n_i FP32 arrays (numpy Fortran order, or CUDA
    tensors in column-major layout), or None to load later with ``load``.
    """

    def __init__(self, As, ms, ns, lam: float, precision: int = A_FP32, lipschitz: float = 0.0,
                 stream=None):
        L = load()
        o = Options()
        L.l1_options_init(C.byref(o))
        o.lambda_ = lam
        o.precision = precision
        o.lipschitz = lipschitz
        o.stream = stream if stream is not None else _current_stream()
        self.ms = np.ascontiguousarray(ms, dtype=np.int64)
        self.ns = np.ascontiguousarray(ns, dtype=np.int64)
        self.count = len(self.ms)
        self.boff = np.concatenate([[0], np.cumsum(self.ms)])
        self.xoff = np.concatenate([[0], np.cumsum(self.ns)])
        h = C.c_void_p()
        ptrs = None
        keep = None
        if As is not None:
            keep = [np.asfortranarray(a, dtype=np.float32) if isinstance(a, np.ndarray) else a for a in As]
            ptrs = (C.c_void_p * self.count)(*[_ptr(a).value for a in keep])
        _check(L.l1_setup_group(ptrs, self.ms.ctypes.data_as(C.POINTER(C.c_int64)),
                                self.ns.ctypes.data_as(C.POINTER(C.c_int64)), self.count, QP_LAMBDA,
                                C.byref(o), C.byref(h)), "l1_setup_group")
        self._h = h

    def load(self, first: int, As):
        keep = [np.asfortranarray(a, dtype=np.float32) if isinstance(a, np.ndarray) else a for a in As]
        ptrs = (C.c_void_p * len(keep))(*[_ptr(a).value for a in keep])
        _check(load().l1_group_load(self._h, first, len(keep), ptrs), "l1_group_load")

    def solve(self, b_packed, tol: float, max_iter: int, x_packed=None):
        """b_packed: sum(m_i) FP32 (numpy or torch); returns (x_packed, results)."""
        if isinstance(b_packed, np.ndarray):
            b_packed = np.ascontiguousarray(b_packed, dtype=np.float32)
            if x_packed is None:
                x_packed = np.zeros(int(self.xoff[-1]), dtype=np.float32)
        elif x_packed is None:
            import torch
            x_packed = torch.empty(int(self.xoff[-1]), dtype=torch.float32, device=b_packed.device)
        res = (Result * self.count)()
        _check(load().l1_solve_batch(self._h, _ptr(b_packed), 0, self.count, float(tol), int(max_iter),
                                     _ptr(x_packed), 0, None, 0, res, None, 0, None, 0), "l1_solve_batch(group)")
        return x_packed, results_to_dict(res)

    def info(self) -> dict:
        inf = Info()
        _check(load().l1_get_info(self._h, C.byref(inf)), "l1_get_info")
        return {k: (list(getattr(inf, k)) if k.startswith("sweep_") else getattr(inf, k))
                for k, _ in Info._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().l1_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lipschitz_static(A, max_iter: int = 1000, rtol: float = 1e-6, stream=None,
                     return_status: bool = False):
    """Power-iteration estimate of ||A||_2^2 without any allocation.

    ``A`` is a device-resident m x n FP32 column-major tensor (m <= 8192,
    n <= 65536) on the current device.  For callers that may not allocate
    device memory; every call shares one static scratch array per GPU, so
    calls that can overlap on the GPU must be serialised.  The call
    synchronises its stream, so it must not run inside a stream capture.  A
    handle's L is 1.01 times this estimate.  With ``return_status`` the
    result is ``(rho, converged, iterations)``."""
    import torch
    if not isinstance(A, torch.Tensor) or A.dtype != torch.float32:
        raise TypeError(f"lipschitz_static: A must be a float32 torch tensor, got "
                        f"{getattr(A, 'dtype', type(A).__name__)}")
    if not A.is_cuda:
        raise TypeError("lipschitz_static: A must be a CUDA tensor")
    if A.dim() != 2:
        raise ValueError("lipschitz_static: A must be 2-D")
    if A.device.index is not None and A.device.index != torch.cuda.current_device():
        raise ValueError(f"lipschitz_static: A is on cuda:{A.device.index} but cuda:"
                         f"{torch.cuda.current_device()} is current")
    L = load()
    m, n = A.shape
    rho = C.c_double(0.0)
    status = C.c_int32(-1)
    iters = C.c_int32(0)
    st = _current_stream() if stream is None else C.c_void_p(stream)
    _check(L.l1_lipschitz_static(_ptr(A), m, n, _ld(A), max_iter, rtol, st, C.byref(rho),
                                 C.byref(status), C.byref(iters)), "l1_lipschitz_static")
    if return_status:
        return rho.value, status.value == CONVERGED, iters.value
    return rho.value


def align_batch(B, b, tol: float = 1e-6, max_outer: int = 10000, xi0: float = 0.0, stream=None):
    """l1_align_batch: the alignment step of §II-B for count problems,
    min ||e||_1 s.t. b_k = B_k w + e, w unpenalised (reading R16).

    ``B`` is a CUDA float32 tensor of shape (count, p, m) (problem k's
    column j is B[k, j]), ``b`` of shape (count, m).  Returns (w, e, results)
    with w of shape (count, p) and e of shape (count, m)."""
    import torch
    for name, t in (("B", B), ("b", b)):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or not t.is_cuda:
            raise TypeError(f"align_batch: {name} must be a float32 CUDA tensor")
    if B.dim() != 3 or b.dim() != 2 or b.shape[0] != B.shape[0] or b.shape[1] != B.shape[2]:
        raise ValueError("align_batch: B must be (count, p, m) and b (count, m)")
    B = B.contiguous()
    b = b.contiguous()
    count, p, m = B.shape
    w = torch.empty((count, p), dtype=torch.float32, device=B.device)
    e = torch.empty((count, m), dtype=torch.float32, device=B.device)
    res = (Result * count)()
    st = _current_stream() if stream is None else C.c_void_p(stream)
    _check(load().l1_align_batch(_ptr(B), m, p, m, m * p, _ptr(b), m, count, float(tol), int(max_outer),
                                 float(xi0), st, _ptr(w), _ptr(e), res), "l1_align_batch")
    return w, e, results_to_dict(res)


def _cuda_tensor(t, dtype, name: str, dims: int):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != dtype or not t.is_cuda:
        raise TypeError(f"{name} must be a {dtype} CUDA tensor")
    if t.dim() != dims:
        raise ValueError(f"{name} must have {dims} dimensions")
    if t.device.index is not None and t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on cuda:{t.device.index} but cuda:{torch.cuda.current_device()} is current")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


def align_warp(img, tau, rows: int, cols: int, stream=None):
    """l1_align_warp: b = y o tau and J = d(y o tau)/d tau on the rows x cols
    canonical frame (§II-B, reading R19) for each task.

    ``img``: CUDA float32 (count, H, W); ``tau``: CUDA float64 (count, 4) as
    (a, b, tx, ty).  Returns (b of shape (count, rows*cols), J of shape
    (count, 4, rows*cols))."""
    import torch
    pi = _cuda_tensor(img, torch.float32, "align_warp: img", 3)
    pt = _cuda_tensor(tau, torch.float64, "align_warp: tau", 2)
    count, H, W = img.shape
    if tau.shape != (count, 4):
        raise ValueError("align_warp: tau must be (count, 4)")
    m = rows * cols
    B = torch.empty((count, 4, m), dtype=torch.float32, device=img.device)
    b = torch.empty((count, m), dtype=torch.float32, device=img.device)
    st = _current_stream() if stream is None else C.c_void_p(stream)
    _check(load().l1_align_warp(pi, H, W, H * W, pt, count, rows, cols, 0, st, _ptr(B), m, 4 * m, _ptr(b), m, None),
           "l1_align_warp")
    return b, -B


def align_images(img, A, tau, rows: int, cols: int, tol: float = 1e-3, max_outer: int = 5000,
                 tau_tol: float = 0.05, max_align: int = 30, stream=None):
    """l1_align_images: the face-alignment loop of §II-B (reading R19).

    ``img``: CUDA float32 (count, H, W) query images; ``A``: CUDA float32
    (count, n, rows*cols), task k's training image j at A[k, j]; ``tau``:
    CUDA float64 (count, 4), the starting transformations, overwritten with
    the final ones.  Returns {"iters", "status"} as numpy arrays."""
    import torch
    pi = _cuda_tensor(img, torch.float32, "align_images: img", 3)
    pa = _cuda_tensor(A, torch.float32, "align_images: A", 3)
    pt = _cuda_tensor(tau, torch.float64, "align_images: tau", 2)
    count, H, W = img.shape
    if A.shape[0] != count or A.shape[2] != rows * cols or tau.shape != (count, 4):
        raise ValueError("align_images: A must be (count, n, rows*cols) and tau (count, 4)")
    n = A.shape[1]
    iters = (C.c_int32 * count)()
    status = (C.c_int32 * count)()
    st = _current_stream() if stream is None else C.c_void_p(stream)
    _check(load().l1_align_images(pi, H, W, H * W, pa, n, n * rows * cols, rows, cols, count, pt, float(tol),
                                  int(max_outer), float(tau_tol), int(max_align), st, iters, status),
           "l1_align_images")
    return {"iters": np.array(iters[:], dtype=np.int32), "status": np.array(status[:], dtype=np.int32)}


def _colmajor(t):
    """CUDA tensor -> column-major FP32 copy (the layout the C ABI reads)."""
    t = t.detach().to(dtype=__import__("torch").float32)
    return t.t().contiguous().t()


def unrolled_palm(A, b, K: int, J: int = 10, ckpt_every: int = 20, xi: float = 0.0,
                  lipschitz: float = 0.0):
    """x = K unrolled PALM steps (P1 mode) on CUDA tensors A (m x n) and b
    (m x N), differentiable with respect to A and b through l1_backward.

    xi (0: 2m/||b||_1 per column) and L (0: power iteration x 1.01) are
    held constant.  The autograd glue only moves pointers; every step runs in
    the library's kernels."""
    import torch

    class _Unrolled(torch.autograd.Function):
        @staticmethod
        def forward(ctx, A_, b_):
            s = Solver(_colmajor(A_), mode=P1, solver=PALM, xi0=xi, lipschitz=lipschitz,
                       unroll_K=K, unroll_J=J, ckpt_every=ckpt_every,
                       stream=torch.cuda.current_stream(A_.device).cuda_stream)
            x, _, res = s.solve(_colmajor(b_), 0.0, 1)
            ctx.solver = s
            ctx.results = res
            return x.contiguous()

        @staticmethod
        def backward(ctx, gx):
            s = ctx.solver
            gb, gA = s.backward(_colmajor(gx), want_b=ctx.needs_input_grad[1],
                                want_A=ctx.needs_input_grad[0])
            s.close()
            return gA, gb

    squeeze = b.dim() == 1
    x = _Unrolled.apply(A, b.reshape(b.shape[0], -1))
    return x.reshape(-1) if squeeze else x


def results_to_dict(res) -> dict:
    """Column arrays of an l1_result array."""
    out = {}
    for f in RESULT_FIELDS:
        out[f] = np.array([getattr(r, f) for r in res])
    return out
