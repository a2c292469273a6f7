"""Unrolled PALM (reading R11 of Algorithm 1, P1 mode) and its adjoint on the
GPU against the FP64 oracle's forward and reverse sweep (which the CPU pins
check against finite differences and the adjoint identity).

Tolerances: x and both gradients within 1e-4 relative (the forward
tolerance of every parity test).  The reverse sweep runs the K steps
backwards in FP32, so its rounding error is about K x 2^-24 times the
conditioning of a step (measured: below 1e-6 at K = 200); a soft-threshold
argument within FP32 rounding of its threshold could flip its mask between
the two precisions, which none of these seeded cases does.
"""
import concurrent.futures as cf

import numpy as np
import pytest

import oracle
import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

X_TOL = 1e-4
G_TOL = 1e-4


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
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300)


def _xi(b32, m):
    return 2.0 * m / np.abs(b32.astype(np.float64)).sum()


def _oracle_cols(A, B32, G, L, K, J, cols):
    """Per column j in cols: oracle x_K and gradients for the adjoint G[:, j]
    (x_target is chosen so that x_K - x_target = G[:, j])."""
    m = A.shape[0]

    def one(j):
        b = B32[:, j].astype(np.float64)
        xi = _xi(B32[:, j], m)
        x = oracle.unrolled_palm(A, b, xi, L, K, J, np.zeros(A.shape[1]), grad=False)[0]
        _, _, gA, gb = oracle.unrolled_palm(A, b, xi, L, K, J, x - G[:, j])
        return x, gA, gb
    with cf.ThreadPoolExecutor(8) as ex:
        return list(ex.map(one, cols))


@pytest.mark.parametrize("K,J,C", [(25, 10, 7), (20, 4, 20), (9, 9, 3)])
def test_unrolled_forward_and_adjoint_match_oracle(l1, K, J, C):
    m, n, N = 64, 128, 7
    p = synthetic.unrolled_instance(m, n, N, k=6, seed=5100 + K)
    A, B32 = p["A"], p["B"].astype(np.float32)
    A32 = A.astype(np.float32).astype(np.float64)
    L = 1.01 * np.linalg.norm(A32, 2) ** 2
    s = l1.Solver(A, mode=l1.P1, solver=l1.PALM, lipschitz=L, unroll_K=K, unroll_J=J, ckpt_every=C)
    x, _, res = s.solve(B32, 0.0, 1)
    assert np.all(res["status"] == l1.MAX_ITER) and np.all(res["inner_iters"] == K)
    G = np.asfortranarray(np.random.default_rng(K).standard_normal((n, N)), dtype=np.float32)
    gb, gA = s.backward(G)
    outs = _oracle_cols(A32, B32, G.astype(np.float64), L, K, J, range(N))
    gA_o = sum(o[1] for o in outs)
    ex = max(_rel(x[:, j], outs[j][0]) for j in range(N))
    eb = max(_rel(gb[:, j], outs[j][2]) for j in range(N))
    eA = _rel(gA, gA_o)
    print(f"K={K} J={J} C={C}: x {ex:.2e}  grad_b {eb:.2e}  grad_A {eA:.2e}")
    assert ex <= X_TOL and eb <= G_TOL and eA <= G_TOL
    # the objective the forward reports
    assert np.allclose(res["primal_obj"], np.abs(x).sum(axis=0), rtol=1e-5)
    s.close()


def test_unrolled_at_workload_size_sampled(l1):
    """A 1024 x 2048, N = 256, K = 200, J = 10, checkpoints every 20 steps.
    grad_x is nonzero on two sampled columns only, so grad_A is the oracle's
    sum over those two; the other columns' grad_b must be exactly zero."""
    m, n, N, K, J, C = 1024, 2048, 256, 200, 10, 20
    p = synthetic.unrolled_instance(m, n, N, k=50, seed=5000)
    A, B32, Xt = p["A"], p["B"].astype(np.float32), p["X_target"]
    A32 = A.astype(np.float32).astype(np.float64)
    L = 1.01 * np.linalg.norm(A32, 2) ** 2
    s = l1.Solver(A, mode=l1.P1, solver=l1.PALM, lipschitz=L, unroll_K=K, unroll_J=J, ckpt_every=C)
    x, _, res = s.solve(B32, 0.0, 1)
    cols = [3, 200]
    G = np.zeros((n, N), dtype=np.float32, order="F")
    for j in cols:
        G[:, j] = x[:, j] - Xt[:, j]
    gb, gA = s.backward(G)
    outs = _oracle_cols(A32, B32, G.astype(np.float64), L, K, J, cols)
    ex = max(_rel(x[:, j], o[0]) for j, o in zip(cols, outs))
    eb = max(_rel(gb[:, j], o[2]) for j, o in zip(cols, outs))
    eA = _rel(gA, outs[0][1] + outs[1][1])
    print(f"workload: x {ex:.2e}  grad_b {eb:.2e}  grad_A {eA:.2e}")
    assert ex <= X_TOL and eb <= G_TOL and eA <= G_TOL
    others = [j for j in range(N) if j not in cols]
    assert not np.any(gb[:, others])
    s.close()


def test_autograd_function_matches_backward(l1):
    m, n, N, K = 48, 96, 5, 30
    p = synthetic.unrolled_instance(m, n, N, k=5, seed=5200)
    A = torch.tensor(p["A"], dtype=torch.float32, device="cuda", requires_grad=True)
    b = torch.tensor(p["B"], dtype=torch.float32, device="cuda", requires_grad=True)
    xt = torch.tensor(p["X_target"], dtype=torch.float32, device="cuda")
    L = 1.01 * float(np.linalg.norm(p["A"].astype(np.float32).astype(np.float64), 2) ** 2)
    x = l1.unrolled_palm(A, b, K, J=10, ckpt_every=8, lipschitz=L)
    loss = 0.5 * ((x - xt) ** 2).sum()
    loss.backward()
    # the same gradients through the C ABI directly
    s = l1.Solver(p["A"], mode=l1.P1, solver=l1.PALM, lipschitz=L, unroll_K=K, unroll_J=10, ckpt_every=8)
    x2, _, _ = s.solve(p["B"].astype(np.float32), 0.0, 1)
    assert np.array_equal(x.detach().cpu().numpy(), x2)
    gb, gA = s.backward(np.asfortranarray(x2 - p["X_target"].astype(np.float32)))
    assert np.array_equal(b.grad.cpu().numpy(), gb)
    assert np.array_equal(A.grad.cpu().numpy(), gA)
    s.close()


def test_backward_errors(l1):
    A = synthetic.gaussian_dictionary(16, 32, synthetic.rng(1))
    plain = l1.Solver(A, mode=l1.P1, solver=l1.PALM)
    with pytest.raises(l1.L1Error) as e:
        plain.backward(np.zeros((32, 1), dtype=np.float32, order="F"))
    assert e.value.code == l1.ERR_NO_TAPE
    s = l1.Solver(A, mode=l1.P1, solver=l1.PALM, unroll_K=5)
    with pytest.raises(l1.L1Error) as e:
        s.backward(np.zeros((32, 1), dtype=np.float32, order="F"))  # no forward yet
    assert e.value.code == l1.ERR_NO_TAPE
    s.solve(np.ones((16, 2), dtype=np.float32, order="F"), 0.0, 1)
    with pytest.raises(l1.L1Error) as e:
        s.backward(np.zeros((32, 3), dtype=np.float32, order="F"))  # N differs
    assert e.value.code == l1.ERR_INVALID_ARG
    gb, gA = s.backward(np.zeros((32, 2), dtype=np.float32, order="F"))
    assert not np.any(gb) and not np.any(gA)
    for kw in (dict(mode=l1.CAB, solver=l1.PALM), dict(mode=l1.P1, solver=l1.DALM)):
        with pytest.raises(l1.L1Error) as e:
            l1.Solver(A, unroll_K=5, **kw)
        assert e.value.code == l1.ERR_UNSUPPORTED
    plain.close()
    s.close()
