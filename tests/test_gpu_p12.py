"""P1,2 (Eq. 2) by PALM with the e-step replaced by the projection of
b - A x + theta/xi onto the eps-ball (reading R10), against the FP64 oracle:
the same number of outer and inner steps element by element, and the
constraint ||b - A x|| <= eps at convergence."""
import concurrent.futures as cf

import numpy as np
import pytest

import oracle
import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

X_TOL = 1e-4
OBJ_TOL = 1e-5


@pytest.fixture(scope="module")
def l1():
    import paper_1007_3753_gb300 as pkg
    from paper_1007_3753_gb300 import build
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    pkg.load()
    return pkg


def _instance(N, seed=1500, m=128, n=256, k=12, noise=0.01):
    g = synthetic.rng(seed)
    A = synthetic.gaussian_dictionary(m, n, g)
    X0 = np.zeros((n, N))
    for j in range(N):
        X0[g.choice(n, k, replace=False), j] = g.standard_normal(k)
    B = np.asfortranarray(A @ X0 + noise * g.standard_normal((m, N))).astype(np.float32)
    return A, B


def _pmap(f, it):
    with cf.ThreadPoolExecutor(8) as ex:
        return list(ex.map(f, it))


@pytest.mark.parametrize("N", [1, 11])
def test_p12_palm_matches_oracle_fixed_iterations(l1, N):
    A, B = _instance(N)
    eps = 0.05
    L = oracle.lipschitz(A)
    outer, inner = 12, 20
    s = l1.Solver(A, mode=l1.P1_2, solver=l1.PALM, epsilon=eps, lipschitz=L, inner_max=inner)
    x, _, res = s.solve(B, tol=0.0, max_iter=outer)
    outs = _pmap(lambda j: oracle.palm(A, B[:, j].astype(np.float64), mode=oracle.MODE_P12, tol=0.0,
                                       max_outer=outer, inner_max=inner, L=L, epsilon=eps), range(N))
    ex = eo = 0.0
    for j, (xo, _, _, st) in enumerate(outs):
        assert res["iters"][j] == outer and res["inner_iters"][j] == st["inner_total"]
        ex = max(ex, np.linalg.norm(x[:, j] - xo) / np.linalg.norm(xo))
        fo = np.abs(xo).sum()
        eo = max(eo, abs(res["primal_obj"][j] - fo) / fo)
    print(f"P1,2 N={N}: x rel. err max {ex:.2e}, objective rel. err max {eo:.2e}")
    assert ex <= X_TOL and eo <= OBJ_TOL
    s.close()


def test_p12_converges_to_the_ball(l1):
    A, B = _instance(6, seed=1600)
    eps = 0.05
    s = l1.Solver(A, mode=l1.P1_2, solver=l1.PALM, epsilon=eps)
    x, _, res = s.solve(B, tol=1e-6, max_iter=2000)
    assert np.all(res["status"] == l1.CONVERGED)
    for j in range(B.shape[1]):
        r = np.linalg.norm(B[:, j] - A @ x[:, j])
        assert r <= eps * (1 + 1e-3), (j, r)
        assert abs(res["resid"][j] - r) <= 1e-4 * eps
        xo, _, _, _ = oracle.palm(A, B[:, j].astype(np.float64), mode=oracle.MODE_P12, tol=1e-6, epsilon=eps,
                                  max_outer=2000)
        assert abs(res["primal_obj"][j] - np.abs(xo).sum()) <= 1e-4 * np.abs(xo).sum()
    # weak duality of Eq. 2
    assert np.all(res["gap"] >= -1e-4 * res["primal_obj"])
    s.close()


def test_p12_requires_palm_and_eps(l1):
    A, _ = _instance(1)
    with pytest.raises(l1.L1Error) as e:
        l1.Solver(A, mode=l1.P1_2, solver=l1.DALM, epsilon=0.1)
    assert e.value.code == l1.ERR_UNSUPPORTED
    with pytest.raises(l1.L1Error) as e:
        l1.Solver(A, mode=l1.P1_2, solver=l1.PALM)
    assert e.value.code == l1.ERR_INVALID_ARG
