"""l1_align_batch (the convex alignment step of §II-B, reading R16) on the
GPU against the FP64 oracle's orc_palm_align: trajectories after the same
number of iterations, the answer at the stopping tolerance, recovery of a
planted w0 under 10 % gross errors, and the singular case."""
import numpy as np
import pytest

import oracle

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


def _problems(count, m, p, frac, seed):
    """Tall B_k with unit Gaussian columns, w0 ~ N(0, 1), a fraction `frac`
    of the entries of e0 large (5 N(0, 1)), b_k = B_k w0 + e0."""
    g = np.random.default_rng(seed)
    B = g.standard_normal((count, p, m))
    B /= np.linalg.norm(B, axis=2, keepdims=True)
    w0 = g.standard_normal((count, p))
    e0 = np.zeros((count, m))
    for k in range(count):
        idx = g.choice(m, int(frac * m), replace=False)
        e0[k, idx] = 5.0 * g.standard_normal(idx.size)
    b = np.einsum("kpm,kp->km", B, w0) + e0
    return B.astype(np.float32), b.astype(np.float32), w0, e0


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def test_align_matches_oracle_at_fixed_iterations(l1):
    B, b, _, _ = _problems(6, 1200, 11, 0.1, seed=1)
    w, e, res = l1.align_batch(torch.from_numpy(B).cuda(), torch.from_numpy(b).cuda(), tol=0.0, max_outer=40)
    w, e = w.cpu().numpy(), e.cpu().numpy()
    assert (res["iters"] == 40).all()
    for k in range(B.shape[0]):
        Bk = np.asfortranarray(B[k].T.astype(np.float64))
        wo, eo, _, st = oracle.palm_align(Bk, b[k].astype(np.float64), tol=0.0, max_outer=40)
        xw, xe = _rel(w[k], wo), _rel(e[k], eo)
        print(k, "w err", xw, "e err", xe)
        assert xw <= 1e-4 and xe <= 1e-4
        assert abs(res["primal_obj"][k] - np.abs(eo).sum()) <= 1e-5 * np.abs(eo).sum()
        assert abs(res["param"][k] - st["param"]) <= 1e-12 * st["param"]


def test_align_recovers_the_planted_transform(l1):
    """3000 iterations (the relative-change rule can stop this iteration
    early while theta is still catching up, as the oracle's pins note)."""
    B, b, w0, e0 = _problems(64, 1200, 11, 0.1, seed=2)
    w, e, res = l1.align_batch(torch.from_numpy(B).cuda(), torch.from_numpy(b).cuda(), tol=0.0, max_outer=3000)
    w = w.cpu().numpy()
    errs = [_rel(w[k], w0[k]) for k in range(64)]
    print("max rel. error of w against the planted w0", max(errs))
    assert max(errs) <= 1e-4


def test_align_at_the_stopping_tolerance(l1):
    """Every sampled problem stops within one iteration of the oracle and
    agrees with the oracle's iterate at the GPU's stopping iteration."""
    B, b, _, _ = _problems(8, 1200, 11, 0.1, seed=4)
    tol = 1e-6
    w, e, res = l1.align_batch(torch.from_numpy(B).cuda(), torch.from_numpy(b).cuda(), tol=tol, max_outer=5000)
    w, e = w.cpu().numpy(), e.cpu().numpy()
    assert (res["status"] == l1.CONVERGED).all()
    for k in range(B.shape[0]):
        Bk = np.asfortranarray(B[k].T.astype(np.float64))
        bk = b[k].astype(np.float64)
        wo, eo, _, st = oracle.palm_align(Bk, bk, tol=tol, max_outer=5000)
        kg = int(res["iters"][k])
        assert abs(kg - st["iters"]) <= 1, (k, kg, st["iters"])
        if kg != st["iters"]:
            wo, eo, _, _ = oracle.palm_align(Bk, bk, tol=0.0, max_outer=kg)
        assert _rel(w[k], wo) <= 1e-4 and _rel(e[k], eo) <= 1e-4, k


def test_align_flags_a_singular_dictionary(l1):
    B, b, _, _ = _problems(2, 300, 4, 0.1, seed=3)
    B[1, 3] = B[1, 2]  # two equal columns: B^T B singular
    w, e, res = l1.align_batch(torch.from_numpy(B).cuda(), torch.from_numpy(b).cuda(), tol=1e-6, max_outer=2000)
    assert res["status"][0] == l1.CONVERGED
    assert res["status"][1] == l1.NONFINITE
    assert np.isnan(w.cpu().numpy()[1]).all()
