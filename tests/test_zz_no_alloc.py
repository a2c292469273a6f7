"""The allocation-free entry point l1_lipschitz_static against the estimate a
solver handle makes (l1_setup, which allocates).

l1_lipschitz_static serves callers that may not allocate device memory (their
memory belongs to their own pool allocator, or they must not stall the device
in cudaMalloc/cudaFree); its scratch is one static array per GPU.  This file
sorts last so that a run stopping at its first failure has already run every
other test; it passes alone in a fresh process as well.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RHO_TOL = 1e-5  # relative, as the objective tolerance of the parity tests


@pytest.fixture(scope="module")
def l1():
    import paper_1007_3753_gb300 as pkg
    from paper_1007_3753_gb300 import build
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    pkg.load()
    return pkg


def _dev_colmajor(a, ld=None):
    """numpy m x n -> column-major FP32 CUDA tensor with leading dimension ld."""
    m, n = a.shape
    ld = ld or m
    buf = torch.zeros((n, ld), dtype=torch.float32, device="cuda")
    buf[:, :m] = torch.from_numpy(np.ascontiguousarray(a.T, dtype=np.float32)).cuda()
    return buf[:, :m].t()


def _handle_rho(l1, a):
    s = l1.Solver(np.asfortranarray(a, dtype=np.float32), mode=l1.QP_LAMBDA, solver=l1.PALM, lam=1e-2)
    try:
        return s.info()["lipschitz"] / 1.01
    finally:
        s.close()


def test_static_matches_handle_on_consecutive_calls(l1):
    rng = np.random.default_rng(9100)
    a1 = rng.standard_normal((300, 500)) / np.sqrt(300)
    a2 = rng.standard_normal((1024, 1200)) / np.sqrt(1024)
    d1, d2 = _dev_colmajor(a1), _dev_colmajor(a2, ld=1040)  # the second with a padded lda
    rho1 = l1.lipschitz_static(d1)
    rho2 = l1.lipschitz_static(d2)   # second call in a row; the scratch holds the first call's state
    rho1_again = l1.lipschitz_static(d1)
    torch.cuda.synchronize()
    ref1, ref2 = _handle_rho(l1, a1), _handle_rho(l1, a2)
    print(f"static {rho1:.9g} {rho2:.9g}  handle {ref1:.9g} {ref2:.9g}")
    assert abs(rho1 - ref1) <= RHO_TOL * ref1
    assert abs(rho2 - ref2) <= RHO_TOL * ref2
    assert rho1_again == rho1  # deterministic; nothing of the previous call leaks in
    # the estimate is a Rayleigh quotient: at most sigma_max^2, and close to it
    for rho, a in ((rho1, a1), (rho2, a2)):
        s2 = np.linalg.norm(a, 2) ** 2
        assert rho <= s2 * (1 + 1e-5) and rho >= s2 * (1 - 1e-2)


def test_static_rejects_sizes_beyond_the_scratch(l1):
    lib = l1.load()
    rho = C.c_double(0.0)
    tall = torch.zeros((2, 8193), dtype=torch.float32, device="cuda").t()   # 8193 x 2
    wide = torch.zeros((65537, 1), dtype=torch.float32, device="cuda").t()  # 1 x 65537
    for t, ld in ((tall, 8193), (wide, 1)):
        m, n = t.shape
        rc = lib.l1_lipschitz_static(C.c_void_p(t.data_ptr()), m, n, ld, 100, 1e-6, None, C.byref(rho),
                                     None, None)
        assert rc == l1.ERR_INVALID_ARG
        assert b"static scratch" in lib.l1_last_error()
    # a host pointer is refused, not dereferenced
    host = np.zeros((4, 4), dtype=np.float32, order="F")
    rc = lib.l1_lipschitz_static(C.c_void_p(host.ctypes.data), 4, 4, 4, 100, 1e-6, None, C.byref(rho),
                                 None, None)
    assert rc == l1.ERR_INVALID_ARG


def test_static_reports_an_unconverged_estimate(l1):
    """When max_iter runs out before the stopping rule fires the call still
    returns L1_OK, but the status says so (and the estimate is low).  Two
    top singular values 1 and 0.999 make the power iteration slow."""
    rng = np.random.default_rng(9101)
    m, n = 200, 120
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sv = np.linspace(0.5, 0.999, n)
    sv[-1] = 1.0
    a = (U * sv) @ V.T
    d = _dev_colmajor(a)
    rho1, conv1, it1 = l1.lipschitz_static(d, max_iter=1, rtol=1e-12, return_status=True)
    assert not conv1 and it1 == 1
    assert rho1 < 1.0
    rho, conv, it = l1.lipschitz_static(d, max_iter=20000, rtol=1e-9, return_status=True)
    assert conv and 1 < it <= 20000
    assert abs(rho - 1.0) <= 1e-3
    # the capture refusal and the device check fire before anything is enqueued
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin(capture_error_mode="thread_local")
        try:
            with pytest.raises(l1.L1Error):
                l1.lipschitz_static(d, stream=s.cuda_stream)
        finally:
            g.capture_end()
