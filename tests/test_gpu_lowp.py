"""A held in BF16 or FP8 e4m3 for the batched DALM sweeps, followed by the
FP32 refinement phase (l1_options.precision, refine).

The low-precision phase changes the iteration's path, so the trajectory is
not compared with the oracle's; the limit is.  Exact recovery (§VI-A, the
200 x 400 instances with a 20-sparse x0) fixes the limit independently of
any solver: after refinement x must equal x0 within the parity tolerance,
while the low-precision answer alone must not (the refinement does the
work).  On the cross-and-bouquet workload the class labels must equal the
FP64 oracle's.
"""
import numpy as np
import pytest

import oracle
import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

X_TOL = 1e-4


@pytest.fixture(scope="module")
def l1():
    import paper_1007_3753_gb300 as pkg
    from paper_1007_3753_gb300 import build
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    pkg.load()
    return pkg


def _rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_lowp_refined_exact_recovery(l1, prec):
    p = l1.A_BF16 if prec == "bf16" else l1.A_FP8E4M3
    errs, errs_raw, iters = [], [], []
    for seed in range(6):
        pr = synthetic.p1_instance(200, 400, 20, seed=seed)
        A, b, x0 = pr["A"], pr["b"], pr["x0"]
        B = np.asfortranarray(np.stack([b, 2.0 * b, -b], 1), dtype=np.float32)  # x0, 2 x0, -x0
        X0 = np.stack([x0, 2.0 * x0, -x0], 1)
        s = l1.Solver(A, mode=l1.P1, solver=l1.DALM, precision=p)
        x, _, res = s.solve(B, tol=1e-6, max_iter=4000)
        assert np.all(res["status"] == l1.CONVERGED)
        errs += [_rel(x[:, j], X0[:, j]) for j in range(3)]
        iters += list(res["iters"])
        raw = l1.Solver(A, mode=l1.P1, solver=l1.DALM, precision=p, refine=False)
        xr, _, _ = raw.solve(B, tol=1e-6, max_iter=4000)
        errs_raw += [_rel(xr[:, j], X0[:, j]) for j in range(3)]
        s.close()
        raw.close()
    print(f"{prec}: refined max err {max(errs):.2e} (iters {min(iters)}..{max(iters)}), "
          f"unrefined min err {min(errs_raw):.2e}")
    assert max(errs) <= X_TOL
    assert min(errs_raw) > 10 * X_TOL


@pytest.mark.parametrize("prec", ["bf16", "fp8", "bf16-tc"])
def test_lowp_cab_labels_match_oracle(l1, prec):
    p = l1.A_FP8E4M3 if prec == "fp8" else l1.A_BF16
    eng = dict(engine=l1.ENGINE_TC, tc_min_cols=1) if prec == "bf16-tc" else {}
    pr = synthetic.cab_problem(256, 8, 12, 24, corrupt=0.3, seed=1300)
    A, B, off = pr["A"], pr["B"].astype(np.float32), pr["offsets"]
    s = l1.Solver(A, mode=l1.CAB, solver=l1.DALM, class_offsets=off, precision=p, **eng)
    x, _, res = s.solve(B, tol=1e-4, max_iter=20000)
    assert np.all(res["status"] == l1.CONVERGED)
    worst = 0.0
    for j in range(B.shape[1]):
        b = B[:, j].astype(np.float64)
        w, _, _ = oracle.dalm(A, b, cab=True, tol=1e-4, max_iter=200000)
        n = A.shape[1]
        lab = oracle.classify(A, off, b, w[:n], w[n:])[0]
        assert res["label"][j] == lab, j
        fo = np.abs(w).sum()
        worst = max(worst, abs(res["primal_obj"][j] - fo) / fo)
    print(f"{prec} CAB: labels equal, objective rel. err max {worst:.2e}")
    s.close()


def test_lowp_rejected_where_unsupported(l1):
    A = synthetic.gaussian_dictionary(16, 32, synthetic.rng(2))
    for kw in (dict(mode=l1.CAB, solver=l1.PALM), dict(mode=l1.QP_LAMBDA, solver=l1.PALM, lam=0.1)):
        with pytest.raises(l1.L1Error) as e:
            l1.Solver(A, precision=l1.A_BF16, **kw)
        assert e.value.code == l1.ERR_UNSUPPORTED
    with pytest.raises(l1.L1Error) as e:
        l1.Solver(A, mode=l1.CAB, solver=l1.DALM, precision=l1.A_FP8E4M3, engine=l1.ENGINE_TC)
    assert e.value.code == l1.ERR_UNSUPPORTED
