"""The C-ABI library on the host: it builds, loads, exports every symbol the
header declares, the ctypes mirrors of its structs have the C layout, and
argument checks that fire before any CUDA call behave as documented."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1007_3753_gb300 as l1
from paper_1007_3753_gb300 import build as l1build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "l1alm.h")


@pytest.fixture(scope="module")
def lib():
    l1build.build()
    return l1.load()


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"L1_API\s+[\w\s\*]+?\b(l1_\w+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert names == sorted(l1.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", l1.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = sorted(set(re.findall(r"\sT\s(l1_\w+)", out)))
    assert exported == names
    for nm_ in names:
        assert hasattr(lib, nm_)


def test_struct_layouts_match_header(tmp_path):
    prog = tmp_path / "probe.c"
    prog.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "l1alm.h"
int main(void) {
  printf("%zu %zu %zu\n", sizeof(l1_options), sizeof(l1_result), sizeof(l1_info));
  printf("%zu %zu %zu %zu\n", offsetof(l1_options, lambda), offsetof(l1_options, class_offsets),
         offsetof(l1_options, stream), offsetof(l1_options, unroll_K));
  printf("%zu %zu\n", offsetof(l1_result, rel_change), offsetof(l1_result, param));
  return 0;
}
''')
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    vals = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                        check=True).stdout.split()))
    assert vals[:3] == [C.sizeof(l1.Options), C.sizeof(l1.Result), C.sizeof(l1.Info)]
    assert vals[3:7] == [l1.Options.lambda_.offset, l1.Options.class_offsets.offset,
                         l1.Options.stream.offset, l1.Options.unroll_K.offset]
    assert vals[7:] == [l1.Result.rel_change.offset, l1.Result.param.offset]


def test_host_side_argument_checks(lib):
    o = l1.Options()
    lib.l1_options_init(C.byref(o))
    assert o.solver == l1.DALM and o.inner_max == 50 and o.check_every == 16
    h = C.c_void_p()
    A = np.ones((4, 8), dtype=np.float32, order="F")
    # null A, bad sizes, lda < m, unknown mode: rejected before any CUDA call
    assert lib.l1_setup(None, 4, 8, 4, l1.P1, C.byref(o), C.byref(h)) == l1.ERR_INVALID_ARG
    assert lib.l1_setup(A.ctypes.data, 0, 8, 4, l1.P1, C.byref(o), C.byref(h)) == l1.ERR_INVALID_ARG
    assert lib.l1_setup(A.ctypes.data, 4, 8, 3, l1.P1, C.byref(o), C.byref(h)) == l1.ERR_INVALID_ARG
    assert lib.l1_setup(A.ctypes.data, 4, 8, 4, 9, C.byref(o), C.byref(h)) == l1.ERR_INVALID_ARG
    o.lambda_ = 0.0
    assert lib.l1_setup(A.ctypes.data, 4, 8, 4, l1.QP_LAMBDA, C.byref(o), C.byref(h)) == l1.ERR_INVALID_ARG
    off = np.array([0, 3, 8], dtype=np.int32)
    o.class_count = 2
    o.class_offsets = off.ctypes.data_as(C.POINTER(C.c_int32))
    bad = np.array([0, 5, 7], dtype=np.int32)  # does not end at n
    o.class_offsets = bad.ctypes.data_as(C.POINTER(C.c_int32))
    assert lib.l1_setup(A.ctypes.data, 4, 8, 4, l1.CAB, C.byref(o), C.byref(h)) == l1.ERR_INVALID_ARG
    assert not h.value
    res = (l1.Result * 1)()
    assert lib.l1_solve_batch(None, None, 4, 1, 1e-6, 10, None, 8, None, 0, res, None, 0, None, 0) == l1.ERR_INVALID_ARG
    assert lib.l1_backward(None, None, 1, None, None) == l1.ERR_INVALID_ARG
    assert lib.l1_destroy(None) == l1.OK
    assert lib.l1_status_string(l1.ERR_NOT_SPD) == b"L1_ERR_NOT_SPD"
    assert lib.l1_status_string(l1.ERR_UNSUPPORTED) == b"L1_ERR_UNSUPPORTED"


def test_refused_combinations_before_any_cuda_call(lib):
    """Requests the library does not implement return L1_ERR_UNSUPPORTED and
    malformed ones L1_ERR_INVALID_ARG, from the argument checks alone."""
    A = np.ones((4, 8), dtype=np.float32, order="F")
    h = C.c_void_p()

    def setup(mode, **kw):
        o = l1.Options()
        lib.l1_options_init(C.byref(o))
        for k, v in kw.items():
            setattr(o, k, v)
        rc = lib.l1_setup(A.ctypes.data, 4, 8, 4, mode, C.byref(o), C.byref(h))
        assert not h.value
        return rc
    U, I = l1.ERR_UNSUPPORTED, l1.ERR_INVALID_ARG
    assert setup(l1.P1_2, solver=l1.DALM, epsilon=0.1) == U      # R10 is a PALM
    assert setup(l1.P1_2, solver=l1.PALM, epsilon=0.0) == I      # no radius
    for kw in (dict(solver=l1.PALM), dict(unroll_K=5, solver=l1.PALM)):
        assert setup(l1.CAB, precision=l1.A_BF16, **kw) == U, kw  # low precision: batched DALM only
    assert setup(l1.CAB, precision=l1.A_FP8E4M3, engine=l1.ENGINE_TC) == U  # FP8: CUDA-core sweeps only
    assert setup(l1.CAB, engine=l1.ENGINE_TC, tc_pieces=1) == U       # a one-piece panel cannot converge
    assert setup(l1.CAB, engine=l1.ENGINE_TC, tc_pieces_y=1) == U
    assert setup(l1.CAB, engine=l1.ENGINE_TC, tc_pieces=4) == I
    assert setup(l1.CAB, engine=l1.ENGINE_TC, tc_min_cols=-1) == I
    assert setup(l1.QP_LAMBDA, precision=l1.A_FP8E4M3, lambda_=0.1) == U
    assert setup(l1.CAB, solver=l1.PALM, engine=l1.ENGINE_TC) == U
    assert setup(l1.QP_LAMBDA, engine=l1.ENGINE_TC, lambda_=0.1) == U
    assert setup(l1.CAB, solver=l1.PALM, unroll_K=5) == U       # unrolled PALM is P1
    assert setup(l1.P1, solver=l1.DALM, unroll_K=5) == U
    assert setup(l1.P1, solver=l1.PALM, unroll_K=-1) == I
    # DALM with a CG y-step (R15): one step, FP32, tensor cores
    assert setup(l1.CAB, cg_steps=-1) == I
    assert setup(l1.CAB, cg_steps=2) == U
    assert setup(l1.CAB, solver=l1.PALM, cg_steps=1) == U
    assert setup(l1.CAB, engine=l1.ENGINE_SIMT, cg_steps=1) == U
    assert setup(l1.CAB, precision=l1.A_BF16, cg_steps=1) == U
    # FISTA with continuation (R17): (QP_lambda) only
    assert setup(l1.QP_LAMBDA, lambda_=0.1, lambda0=-1.0) == I
    assert setup(l1.QP_LAMBDA, lambda_=0.1, lambda0=1.0, cont_rho=1.5) == I
    assert setup(l1.P1, lambda0=1.0) == U
    # AMP (R18): P1 on the FP32 CUDA-core sweeps
    assert setup(l1.P1, solver=l1.AMP, tau0=-1.0) == I
    assert setup(l1.P1, solver=l1.DALM, tau0=1.0) == U
    assert setup(l1.CAB, solver=l1.AMP) == U
    assert setup(l1.QP_LAMBDA, solver=l1.AMP, lambda_=0.1) == U
    assert setup(l1.P1, solver=l1.AMP, precision=l1.A_BF16) == U
    assert setup(l1.P1, solver=l1.AMP, unroll_K=5) == U
    assert setup(l1.P1, solver=7) == I
    assert setup(l1.P1, precision=9) == I
    assert setup(l1.P1, engine=9) == I
    flat = np.array([0, 3, 3, 8], dtype=np.int32)  # an empty class
    assert setup(l1.CAB, class_count=3, class_offsets=flat.ctypes.data_as(C.POINTER(C.c_int32))) == I
    # groups: (QP_lambda) only, FP32 or BF16, positive sizes
    ms = np.array([4, 6], dtype=np.int64)
    ns = np.array([8, 12], dtype=np.int64)
    o = l1.Options()
    lib.l1_options_init(C.byref(o))
    o.lambda_ = 0.1
    P64 = C.POINTER(C.c_int64)
    args = (ms.ctypes.data_as(P64), ns.ctypes.data_as(P64))
    assert lib.l1_setup_group(None, *args, 2, l1.CAB, C.byref(o), C.byref(h)) == I
    assert lib.l1_setup_group(None, *args, 0, l1.QP_LAMBDA, C.byref(o), C.byref(h)) == I
    o.precision = l1.A_FP8E4M3
    assert lib.l1_setup_group(None, *args, 2, l1.QP_LAMBDA, C.byref(o), C.byref(h)) == U
    o.precision = l1.A_FP32
    ms[1] = 0
    assert lib.l1_setup_group(None, *args, 2, l1.QP_LAMBDA, C.byref(o), C.byref(h)) == I
    o.lambda_ = 0.0
    assert lib.l1_setup_group(None, *args, 2, l1.QP_LAMBDA, C.byref(o), C.byref(h)) == I
    assert not h.value
    # the allocation-free entry point checks its arguments and its size limit first
    rho = C.c_double(0.0)
    st, it = C.c_int32(-1), C.c_int32(-1)
    args = (None, C.byref(rho), C.byref(st), C.byref(it))
    assert lib.l1_lipschitz_static(None, 4, 8, 4, 10, 1e-6, *args) == I
    assert lib.l1_lipschitz_static(A.ctypes.data, 4, 8, 3, 10, 1e-6, *args) == I
    assert lib.l1_lipschitz_static(A.ctypes.data, 1 << 20, 8, 1 << 20, 10, 1e-6, *args) == I
    assert (st.value, it.value) == (-1, -1)  # nothing written on a refused call


def test_static_wrapper_refuses_other_dtypes_before_any_launch(lib):
    """lipschitz_static reads FP32: a BF16 (or FP64, or host) tensor is refused
    in Python before the library is called, so no kernel reads past a buffer."""
    torch = pytest.importorskip("torch")
    for dt in (torch.bfloat16, torch.float16, torch.float64):
        with pytest.raises(TypeError):
            l1.lipschitz_static(torch.zeros((8, 4), dtype=dt).t())
    with pytest.raises(TypeError):
        l1.lipschitz_static(torch.zeros((8, 4), dtype=torch.float32).t())  # host tensor
    with pytest.raises(TypeError):
        l1.lipschitz_static(np.zeros((4, 8), dtype=np.float32, order="F"))


def test_product_path_has_no_cpu_fallback():
    """The package never imports the oracle and has no host compute path."""
    pkg = os.path.join(ROOT, "paper_1007_3753_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "l1_oracle" not in src, f


def test_buffers_other_than_float32_are_refused_before_any_call(lib):
    """Every buffer of the C ABI holds FP32: the binding refuses tensors and
    arrays of another dtype before the call (the library would otherwise read
    past the end of a BF16 buffer)."""
    torch = pytest.importorskip("torch")
    for dt in (torch.bfloat16, torch.float16, torch.float64):
        with pytest.raises(TypeError):
            l1.Solver(torch.zeros((8, 4), dtype=dt).t(), mode=l1.P1, solver=l1.DALM)
        with pytest.raises(TypeError):
            l1._ptr(torch.zeros(4, dtype=dt))
    for dt in (np.float64, np.float16, np.int32):
        with pytest.raises(TypeError):
            l1._ptr(np.zeros(4, dtype=dt))
    assert l1._ptr(np.zeros(4, dtype=np.float32)) is not None
    assert l1._ptr(torch.zeros(4, dtype=torch.float32)) is not None


def test_alignment_loop_argument_checks(lib):
    """l1_align_warp and l1_align_images refuse null pointers, too-small
    images, strides and sizes before any CUDA call (host pointers serve as
    stand-ins: nothing is dereferenced)."""
    I = l1.ERR_INVALID_ARG
    img = np.zeros(16, dtype=np.float32)
    tau = np.zeros(4, dtype=np.float64)
    B = np.zeros(64, dtype=np.float32)
    b = np.zeros(16, dtype=np.float32)
    pi, pt, pB, pb = img.ctypes.data, tau.ctypes.data, B.ctypes.data, b.ctypes.data
    # l1_align_warp(img, H, W, img_stride, tau, count, rows, cols, col0, stream, B, ldB, strideB, b, strideb, active)
    assert lib.l1_align_warp(None, 4, 4, 16, pt, 1, 2, 2, 0, None, pB, 4, 16, pb, 4, None) == I
    assert lib.l1_align_warp(pi, 1, 4, 16, pt, 1, 2, 2, 0, None, pB, 4, 16, pb, 4, None) == I   # H < 2
    assert lib.l1_align_warp(pi, 4, 4, 15, pt, 1, 2, 2, 0, None, pB, 4, 16, pb, 4, None) == I   # img_stride
    assert lib.l1_align_warp(pi, 4, 4, 16, pt, 0, 2, 2, 0, None, pB, 4, 16, pb, 4, None) == I   # count
    assert lib.l1_align_warp(pi, 4, 4, 16, pt, 70000, 2, 2, 0, None, pB, 4, 16, pb, 4, None) == I
    assert lib.l1_align_warp(pi, 4, 4, 16, pt, 1, 2, 2, 0, None, pB, 3, 16, pb, 4, None) == I   # ldB < m
    assert lib.l1_align_warp(pi, 4, 4, 16, pt, 1, 2, 2, 1, None, pB, 4, 16, pb, 4, None) == I   # strideB
    assert lib.l1_align_warp(pi, 4, 4, 16, pt, 1, 2, 2, 0, None, pB, 4, 16, pb, 3, None) == I   # strideb
    it = (C.c_int32 * 1)()
    stt = (C.c_int32 * 1)()
    # l1_align_images(img, H, W, img_stride, A, n, A_stride, rows, cols, count, tau, tol, max_outer,
    #                 tau_tol, max_align, stream, iters, status)
    A = np.zeros(64, dtype=np.float32)
    pA = A.ctypes.data
    assert lib.l1_align_images(pi, 4, 4, 16, None, 2, 32, 4, 4, 1, pt, 1e-3, 10, 1e-2, 5, None, it, stt) == I
    assert lib.l1_align_images(pi, 4, 4, 16, pA, 29, 16 * 29, 4, 4, 1, pt, 1e-3, 10, 1e-2, 5, None, it, stt) == I
    assert lib.l1_align_images(pi, 4, 4, 16, pA, 2, 31, 4, 4, 1, pt, 1e-3, 10, 1e-2, 5, None, it, stt) == I
    assert lib.l1_align_images(pi, 4, 4, 16, pA, 2, 32, 4, 4, 1, pt, -1.0, 10, 1e-2, 5, None, it, stt) == I
    assert lib.l1_align_images(pi, 4, 4, 16, pA, 2, 32, 4, 4, 1, pt, 1e-3, 10, 1e-2, 0, None, it, stt) == I
    assert lib.l1_align_images(pi, 4, 4, 16, pA, 2, 32, 4, 4, 1, pt, 1e-3, 10, 1e-2, 5, None, None, stt) == I
