"""The seeded input generators against the workload recipes they state:
§VI-A instances, the cross-and-bouquet model of §II-A (Eq. 5) with the
corruption of §VI-B, the uneven (QP_lambda) batch, batches of P1 right-hand
sides and the synthetic alignment tasks of §VI-C.  CPU only."""
import numpy as np

import synthetic


def _unit_cols(A):
    return np.allclose(np.linalg.norm(A, axis=0), 1.0, atol=1e-12)


def test_p1_instance_recipe():
    p = synthetic.p1_instance(200, 400, 20, seed=3)
    A, x0, b = p["A"], p["x0"], p["b"]
    assert A.shape == (200, 400) and A.flags.f_contiguous and _unit_cols(A)
    assert np.count_nonzero(x0) == 20 and set(np.abs(x0[x0 != 0])) == {1.0}
    assert np.array_equal(np.flatnonzero(x0), p["support"])
    assert np.allclose(b, A @ x0, rtol=0, atol=1e-12)
    u = synthetic.p1_instance(200, 400, 20, seed=3, entries="uniform10")["x0"]
    assert np.count_nonzero(u) == 20 and np.max(np.abs(u)) <= 10.0
    # the same seed gives the same instance, another seed another one
    assert np.array_equal(synthetic.p1_instance(200, 400, 20, seed=3)["A"], A)
    assert not np.array_equal(synthetic.p1_instance(200, 400, 20, seed=4)["A"], A)


def test_cab_problem_recipe():
    m, C, per, N = 256, 5, 12, 40
    p = synthetic.cab_problem(m, C, per, N, corrupt=0.3, seed=11)
    A, B, off, lab, bad = p["A"], p["B"], p["offsets"], p["labels"], p["corrupted"]
    assert A.shape == (m, C * per) and _unit_cols(A) and np.all(A >= -0.05)
    assert list(off) == [per * c for c in range(C + 1)]
    assert B.shape == (m, N) and np.all((lab >= 0) & (lab < C))
    assert np.all(bad.sum(axis=0) == int(np.floor(0.3 * m)))  # floor(p m) entries per vector
    assert np.all((B >= 0.0) & (B <= 1.0))  # peak-1 nonnegative signal, U[0,1] errors
    # the uncorrupted part of a test vector lies in its class's training span
    # (rank-9 subspace spanned by 12 columns that carry 1 % noise)
    for j in range(N):
        Ac = A[:, off[lab[j]]:off[lab[j] + 1]]
        keep = ~bad[:, j]
        coef, *_ = np.linalg.lstsq(Ac[keep], B[keep, j], rcond=None)
        assert np.linalg.norm(Ac[keep] @ coef - B[keep, j]) <= 0.05 * np.linalg.norm(B[keep, j])
    assert np.array_equal(synthetic.cab_problem(m, C, per, N, seed=11)["B"], B)


def test_qp_group_recipe():
    ms, ns = synthetic.qp_group_sizes(8192, seed=4000)
    assert ms.min() >= 256 and ms.max() <= 4096
    assert np.all(ns % 8 == 0)
    r = ns / ms
    assert r.min() >= 2.0 - 4.0 / 256 and r.max() <= 4.0 + 4.0 / 256
    # log-uniform m and n/m: E[m n] = E[m^2] E[n/m]
    e_m2 = (4096 ** 2 - 256 ** 2) / (2 * np.log(4096 / 256))
    e_r = (4.0 - 2.0) / np.log(2.0)
    assert abs(np.mean(ms.astype(float) * ns) / (e_m2 * e_r) - 1.0) <= 0.05
    q = synthetic.qp_instance(300, 680, seed=9)
    assert q["A"].shape == (300, 680) and _unit_cols(q["A"])
    assert np.count_nonzero(q["x0"]) == 30
    resid = q["b"] - q["A"] @ q["x0"]
    assert 0.5 * 0.01 <= np.std(resid) <= 1.5 * 0.01


def test_unrolled_instance_recipe():
    p = synthetic.unrolled_instance(64, 128, 6, k=5, seed=2)
    A, X, B = p["A"], p["X_target"], p["B"]
    assert A.shape == (64, 128) and _unit_cols(A) and X.shape == (128, 6) and B.shape == (64, 6)
    assert np.all(np.count_nonzero(X, axis=0) == 5)
    assert np.std(B - A @ X) <= 0.02


def test_p1_batch_recipe():
    p = synthetic.p1_batch(100, 300, 10, 7, seed=4)
    A, X0, B = p["A"], p["X0"], p["B"]
    assert A.shape == (100, 300) and _unit_cols(A)
    assert X0.shape == (300, 7) and B.shape == (100, 7) and B.flags.f_contiguous
    assert all(np.count_nonzero(X0[:, j]) == 10 for j in range(7))
    assert np.max(np.abs(X0)) <= 10.0
    assert np.allclose(B, A @ X0, rtol=0, atol=1e-12)
    q = synthetic.p1_batch(100, 300, 10, 7, seed=4)
    assert np.array_equal(q["B"], B)
    r = synthetic.p1_batch(100, 300, 10, 2, seed=4, entries="pm1")["X0"]
    assert set(np.abs(r[r != 0])) == {1.0}


def test_alignment_images_recipe():
    """§VI-C on synthetic faces: 40 x 30 frame, 7 training images of full
    rank, an 80 x 60 query that shows the face at the true similarity (at
    the pixels outside the occluded block it equals a nonnegative mix of the
    training images), a square block of 10 % of the face area replaced, and
    the two perturbations of the start (4 pixels along x; 15 degrees about
    the frame centre)."""
    d = synthetic.alignment_images(3, "translation", seed=11)
    rows, cols = d["rows"], d["cols"]
    m = rows * cols
    assert (rows, cols) == (40, 30) and d["A"].shape == (3, m, 7) and d["img"].shape == (3, 80, 60)
    t = d["tau_true"][0]
    assert np.array_equal(t, [1.0, 0.0, 15.0, 20.0])
    assert np.allclose(d["tau_init"] - d["tau_true"], [0.0, 0.0, 4.0, 0.0])
    for k in range(3):
        A = d["A"][k]
        assert np.linalg.matrix_rank(A) == 7 and np.all(A > 0)
        b = d["img"][k][20:60, 15:45].ravel()  # the face at the true similarity
        side = int(round(np.sqrt(0.1 * m)))
        keep = np.ones(m, dtype=bool)
        for _ in range(8):  # least squares, trimming the worst-fitting pixels
            c, *_ = np.linalg.lstsq(A[keep], b[keep], rcond=None)
            r = np.abs(b - A @ c)
            keep = r <= np.sort(r)[m - side * side - 1]
        off = np.flatnonzero(r > 1e-9)
        assert side * side * 0.5 <= off.size <= side * side  # only the occluded block misfits
        rr, cc = off // cols, off % cols
        assert rr.max() - rr.min() < side and cc.max() - cc.min() < side  # and it is a square block
        assert np.all(c > -1e-9) and abs(c.sum() - 1.0) < 1e-6  # a convex mix of the illuminations
    rot = synthetic.alignment_images(1, "rotation", seed=11)
    a, bb, tx, ty = rot["tau_init"][0]
    assert np.isclose(np.degrees(np.arctan2(bb, a)), 15.0) and np.isclose(a * a + bb * bb, 1.0)
    cu, cv = (cols - 1) / 2.0, (rows - 1) / 2.0
    assert np.allclose([a * cu - bb * cv + tx, bb * cu + a * cv + ty], [cu + 15.0, cv + 20.0])
    assert np.array_equal(synthetic.alignment_images(1, "rotation", seed=11)["img"], rot["img"])
