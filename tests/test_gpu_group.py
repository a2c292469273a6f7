"""Uneven batches of (QP_lambda) instances (one persistent launch) against the
FP64 oracle's FISTA (Eq. 18), in FP32 and BF16 dictionary storage, and the
optimality conditions (Eq. 12) at the sizes of the 8192-instance workload."""
import concurrent.futures as cf

import numpy as np
import pytest

import oracle
import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def l1():
    import paper_1007_3753_gb300 as pkg
    from paper_1007_3753_gb300 import build
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    pkg.load()
    return pkg


def _instances(count, seed, m_lo, m_hi):
    ms, ns = synthetic.qp_group_sizes(count, seed=seed, m_lo=m_lo, m_hi=m_hi)
    inst = [synthetic.qp_instance(int(m), int(n), seed=seed + 1 + i) for i, (m, n) in enumerate(zip(ms, ns))]
    return ms, ns, inst


def _oracle_all(As, b, boff, lam, L, tol, max_iter):
    def one(i):
        A = np.asfortranarray(As[i])
        return oracle.fista_qp(A, b[boff[i]:boff[i + 1]].astype(np.float64), lam, L=L, tol=tol,
                               max_iter=max_iter)[0]
    with cf.ThreadPoolExecutor(8) as ex:
        return list(ex.map(one, range(len(As))))


@pytest.mark.parametrize("bf16", [False, True])
def test_group_trajectory_matches_oracle(l1, bf16):
    """A fixed number of FISTA steps (Eq. 18) with one step size 1/L shared by
    both sides (L from an SVD, an upper bound for every instance), compared
    element by element: FP32 arithmetic against the FP64 oracle."""
    ms, ns, inst = _instances(29, 700, 24, 160)
    lam, steps = 5e-3, 300
    As = [p["A"] for p in inst]
    if bf16:  # the oracle solves the problem the BF16 dictionaries define
        # (torch's host conversion: round to nearest even)
        As = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)
              .to(torch.float32).numpy().astype(np.float64) for a in As]
    L = 1.01 * max(np.linalg.norm(a, 2) ** 2 for a in As)
    b = np.concatenate([p["b"] for p in inst]).astype(np.float32)
    g = l1.Group([p["A"] for p in inst], ms, ns, lam, lipschitz=L,
                 precision=l1.A_BF16 if bf16 else l1.A_FP32)
    x, res = g.solve(b, 0.0, steps)
    assert np.all(res["status"] == l1.MAX_ITER) and np.all(res["iters"] == steps)
    outs = _oracle_all(As, b, g.boff, lam, L, 0.0, steps)
    worst_x = worst_o = 0.0
    for i, xo in enumerate(outs):
        xg = x[g.xoff[i]:g.xoff[i + 1]]
        A, bi = As[i], b[g.boff[i]:g.boff[i + 1]].astype(np.float64)
        worst_x = max(worst_x, np.linalg.norm(xg - xo) / np.linalg.norm(xo))
        Fo = 0.5 * np.sum((bi - A @ xo) ** 2) + lam * np.abs(xo).sum()
        worst_o = max(worst_o, abs(res["primal_obj"][i] - Fo) / Fo)
    print(f"group bf16={bf16}: x rel. err max {worst_x:.2e}, objective rel. err max {worst_o:.2e}")
    assert worst_x <= 1e-4 and worst_o <= 1e-5
    g.close()


def test_group_converged_objective(l1):
    """Run to the stopping rule (§VI-C) with each instance's own power-iteration
    L: the objectives agree with the oracle's converged ones.  The iterates are
    only compared loosely: at a relative change of 1e-6 a FISTA iterate is
    still ~2e-4 from the limit, and the two sides stop a few steps apart."""
    ms, ns, inst = _instances(29, 700, 24, 160)
    lam, tol = 5e-3, 1e-6
    b = np.concatenate([p["b"] for p in inst]).astype(np.float32)
    g = l1.Group([p["A"] for p in inst], ms, ns, lam, precision=l1.A_FP32)
    x, res = g.solve(b, tol, 200000)
    assert np.all(res["status"] == l1.CONVERGED)
    outs = _oracle_all([p["A"] for p in inst], b, g.boff, lam, None, tol, 400000)
    for i, xo in enumerate(outs):
        xg = x[g.xoff[i]:g.xoff[i + 1]]
        A, bi = inst[i]["A"], b[g.boff[i]:g.boff[i + 1]].astype(np.float64)
        Fo = 0.5 * np.sum((bi - A @ xo) ** 2) + lam * np.abs(xo).sum()
        assert abs(res["primal_obj"][i] - Fo) <= 1e-5 * Fo, i
        assert np.linalg.norm(xg - xo) <= 1e-3 * np.linalg.norm(xo), i
    g.close()


def test_group_kkt_at_workload_sizes(l1):
    """Instances drawn from the 8192-instance recipe (m in [256, 4096]); at any
    size the FISTA limit satisfies |A^T (b - A x)| <= lambda, with equality and
    the sign of x on the support (Eq. 12)."""
    ms, ns = synthetic.qp_group_sizes(8192, seed=4000)
    pick = np.argsort(ms)[np.linspace(0, 8191, 6).astype(int)]  # stratified over m
    inst = [synthetic.qp_instance(int(ms[i]), int(ns[i]), seed=4000 + 1 + int(i)) for i in pick]
    lam = 1e-3
    g = l1.Group([p["A"] for p in inst], ms[pick], ns[pick], lam, precision=l1.A_FP32)
    b = np.concatenate([p["b"] for p in inst]).astype(np.float32)
    x, res = g.solve(b, 1e-8, 100000)
    for k, p in enumerate(inst):
        xg = x[g.xoff[k]:g.xoff[k + 1]].astype(np.float64)
        c = p["A"].T @ (p["b"] - p["A"] @ xg)
        supp = xg != 0
        assert np.max(np.abs(c)) <= lam * 1.02, (k, np.max(np.abs(c)) / lam)
        assert np.max(np.abs(c[supp] - lam * np.sign(xg[supp])), initial=0.0) <= 0.02 * lam, k
    g.close()


def test_group_chunked_load_matches_one_shot(l1):
    """l1_group_load of instances in two calls (each estimating L for its own
    range) gives the solve of a handle set up with every dictionary at once."""
    ms, ns, inst = _instances(12, 900, 24, 96)
    As = [p["A"] for p in inst]
    b = np.concatenate([p["b"] for p in inst]).astype(np.float32)
    g1 = l1.Group(As, ms, ns, 5e-3)
    g2 = l1.Group(None, ms, ns, 5e-3)
    g2.load(0, As[:5])
    g2.load(5, As[5:])
    x1, r1 = g1.solve(b, 0.0, 300)
    x2, r2 = g2.solve(b, 0.0, 300)
    for i in range(len(ms)):
        a, c = x1[g1.xoff[i]:g1.xoff[i + 1]], x2[g2.xoff[i]:g2.xoff[i + 1]]
        assert np.linalg.norm(a - c) <= 1e-5 * np.linalg.norm(a), i
    assert np.allclose(r1["param"], r2["param"], rtol=1e-5)
    g1.close()
    g2.close()
