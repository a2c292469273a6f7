"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (stated by the task for floating point):
  ||x - x_oracle|| / ||x_oracle|| <= 1e-4, objective relative error <= 1e-5,
  class labels identical.
Two kinds of comparison:
  * after the same number of iterations (tol = 0 runs exactly max_iter
    iterations on both sides): the trajectories agree;
  * at the stopping tolerance (check_at_tolerance): every sampled column is
    compared, none is left out.  The relative-change rule fixes the answer only
    up to the iteration at which it fires, and one iteration moves w by
    rel_change * ||w|| (just below tol * ||w||), so two correct runs whose
    rounding differs can stop one iteration apart.  Each GPU column must stop
    within one iteration of the oracle's own stop, and its x must agree with
    the oracle's iterate at the GPU's stopping iteration to the tolerances
    above.
"""
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


def _dev(a):
    """numpy (m x N) -> column-major FP32 CUDA tensor."""
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32).T)).cuda()
    return t.t()


def _pmap(fn, items):
    with cf.ThreadPoolExecutor(max_workers=8) as ex:
        return list(ex.map(fn, items))


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


class Errs:
    """Collects per-column errors and asserts once, reporting the worst."""

    def __init__(self, what):
        self.what, self.x, self.obj = what, [], []

    def add(self, xg, xo, obj_g=None):
        self.x.append(_rel(xg, xo))
        if obj_g is not None:
            oo = np.abs(xo).sum()
            self.obj.append(abs(obj_g - oo) / oo if oo > 0 else abs(obj_g))

    def check(self):
        xs, os_ = np.array(self.x), np.array(self.obj or [0.0])
        msg = (f"{self.what}: x rel. err max {xs.max():.2e} median {np.median(xs):.2e}; "
               f"objective rel. err max {os_.max():.2e} median {np.median(os_):.2e}")
        print(msg)
        assert xs.max() <= X_TOL and os_.max() <= OBJ_TOL, msg


def check_at_tolerance(what, res, x, cols, run_oracle, max_stop_diff=1):
    """The at-tolerance parity check described above.  run_oracle(j, tol_on,
    iters) runs the oracle on column j: with tol_on at the solve's tol (and
    its max_iter), else exactly `iters` iterations; it returns (w, stats)."""
    first = _pmap(lambda j: run_oracle(j, True, 0), cols)
    need = [(k, j) for k, (j, (w, st)) in enumerate(zip(cols, first)) if res["iters"][j] != st["iters"]]
    again = dict(zip([k for k, _ in need],
                     _pmap(lambda kj: run_oracle(kj[1], False, int(res["iters"][kj[1]])), need)))
    ex = Errs(what)
    stops = []
    for k, (j, (w, st)) in enumerate(zip(cols, first)):
        stops.append(int(res["iters"][j]) - int(st["iters"]))
        w_at = again[k][0] if k in again else w
        ex.add(x[:, j], w_at, res["primal_obj"][j])
    print(f"{what}: GPU stop - oracle stop per column {stops}")
    assert max(abs(d) for d in stops) <= max_stop_diff, stops
    ex.check()
    return first


# ------------------------------------------------------------ CAB (Eq. 5)

@pytest.mark.parametrize("N", [1, 5, 37])
def test_cab_dalm_matches_oracle_fixed_iterations(l1, N):
    p = synthetic.cab_problem(256, 10, 30, N, seed=11)
    A, B, off = p["A"], p["B"], p["offsets"]
    n = A.shape[1]
    iters = 300
    s = l1.Solver(_dev(A), mode=l1.CAB, solver=l1.DALM, class_offsets=off)
    x, y, res = s.solve(_dev(B), tol=0.0, max_iter=iters, want_y=True)
    x = x.cpu().numpy()
    y = y.cpu().numpy()
    assert np.all(res["iters"] == iters) and np.all(res["status"] == l1.MAX_ITER)
    outs = _pmap(lambda j: oracle.dalm(A, B[:, j], cab=True, tol=0.0, max_iter=iters), range(N))
    ex, ey = Errs(f"CAB DALM N={N} x"), Errs(f"CAB DALM N={N} y")
    for j, (w, yo, st) in enumerate(outs):
        ex.add(x[:, j], w, res["primal_obj"][j])
        ey.add(y[:, j], yo)
        lab, slab, r, _ = oracle.classify(A, off, B[:, j], w[:n], w[n:])
        srt = np.sort(r)
        if srt[1] - srt[0] > 1e-6 * srt[1]:  # well-posed label
            assert res["label"][j] == lab, j
        assert res["sci_label"][j] == slab, j
    ex.check()
    ey.check()
    s.close()


def test_cab_dalm_matches_oracle_at_tolerance(l1):
    p = synthetic.cab_problem(256, 10, 30, 24, seed=12)
    A, B, off = p["A"], p["B"], p["offsets"]
    tol = 1e-3
    s = l1.Solver(_dev(A), mode=l1.CAB, solver=l1.DALM, class_offsets=off)
    x, _, res = s.solve(_dev(B), tol=tol, max_iter=20000)
    x = x.cpu().numpy()
    assert np.all(res["status"] == l1.CONVERGED)

    def run(j, tol_on, iters):
        w, _, st = oracle.dalm(A, B[:, j], cab=True, tol=tol if tol_on else 0.0,
                               max_iter=20000 if tol_on else iters)
        return w, st
    check_at_tolerance("CAB DALM at tol 1e-3", res, x, list(range(24)), run)
    s.close()


@pytest.mark.parametrize("N", [1, 13])
def test_cab_palm_matches_oracle_fixed_iterations(l1, N):
    p = synthetic.cab_problem(192, 6, 30, N, seed=13)
    A, B, off = p["A"], p["B"], p["offsets"]
    L = oracle.lipschitz(A)
    outer, inner = 12, 20
    s = l1.Solver(_dev(A), mode=l1.CAB, solver=l1.PALM, class_offsets=off, lipschitz=L,
                  inner_max=inner)
    x, y, res = s.solve(_dev(B), tol=0.0, max_iter=outer, want_y=True)
    x = x.cpu().numpy()
    n = A.shape[1]
    outs = _pmap(lambda j: oracle.palm(A, B[:, j], mode=oracle.MODE_CAB, tol=0.0, max_outer=outer,
                                       inner_max=inner, L=L), range(N))
    ex = Errs(f"CAB PALM N={N}")
    for j, (xo, eo, th, st) in enumerate(outs):
        assert res["iters"][j] == outer and res["inner_iters"][j] == st["inner_total"]
        ex.add(x[:, j], np.concatenate([xo, eo]), res["primal_obj"][j])
    ex.check()
    s.close()


# ------------------------------------------------- basis pursuit (Eq. 1)

def test_p1_exact_recovery_200x400(l1):
    """§VI-A setting at FP32: both solvers recover x0 and track the oracle."""
    for seed in range(6):
        pr = synthetic.p1_instance(200, 400, 20, seed=seed)
        A, b, x0 = pr["A"], pr["b"], pr["x0"]
        L = oracle.lipschitz(A)
        for solver in (l1.DALM, l1.PALM):
            s = l1.Solver(_dev(A), mode=l1.P1, solver=solver, lipschitz=L)
            x, _, res = s.solve(_dev(b.reshape(-1, 1)), tol=1e-6, max_iter=2000)
            x = x.cpu().numpy()[:, 0]
            assert res["status"][0] == l1.CONVERGED
            assert _rel(x, x0) <= X_TOL, (seed, solver, _rel(x, x0))
            if solver == l1.DALM:
                w, _, st = oracle.dalm(A, b, cab=False, tol=1e-6)
            else:
                w, _, _, st = oracle.palm(A, b, mode=oracle.MODE_P1, tol=1e-6, L=L)
            assert _rel(x, w) <= X_TOL
            s.close()


def test_p1_dalm_batch_fixed_iterations(l1):
    pr = synthetic.p1_instance(200, 400, 20, seed=3)
    A = pr["A"]
    g = np.random.default_rng(0)
    B = np.stack([A @ np.where(g.random(400) < 0.05, g.standard_normal(400), 0) for _ in range(19)], 1)
    iters = 80
    s = l1.Solver(_dev(A), mode=l1.P1, solver=l1.DALM)
    x, _, res = s.solve(_dev(B), tol=0.0, max_iter=iters)
    x = x.cpu().numpy()
    for j in range(19):
        w, _, _ = oracle.dalm(A, B[:, j], cab=False, tol=0.0, max_iter=iters)
        assert _rel(x[:, j], w) <= X_TOL
    s.close()


def test_p1_dalm_rejects_singular(l1):
    A = np.random.default_rng(1).standard_normal((8, 20))
    A = np.vstack([A, A[:2]])  # A A^T singular
    with pytest.raises(l1.L1Error) as ei:
        l1.Solver(_dev(A), mode=l1.P1, solver=l1.DALM)
    assert ei.value.code == l1.ERR_NOT_SPD


# ------------------------------------------------------------ QP (Eq. 3)

@pytest.mark.parametrize("N", [1, 9])
def test_qp_fista_matches_oracle(l1, N):
    g = np.random.default_rng(4)
    inst = synthetic.qp_instance(128, 320, seed=40)
    A = inst["A"]
    B = np.stack([inst["b"]] + [A @ np.where(g.random(320) < 0.04, g.standard_normal(320), 0)
                                + 0.01 * g.standard_normal(128) for _ in range(N - 1)], 1)
    lam = 1e-2
    L = oracle.lipschitz(A)
    s = l1.Solver(_dev(A), mode=l1.QP_LAMBDA, lam=lam, lipschitz=L)
    x, _, res = s.solve(_dev(B), tol=1e-7, max_iter=20000)
    x = x.cpu().numpy()
    for j in range(N):
        xo, st = oracle.fista_qp(A, B[:, j], lam, L=L, tol=1e-7, max_iter=20000)
        assert _rel(x[:, j], xo) <= X_TOL, (j, _rel(x[:, j], xo), res["iters"][j], st["iters"])
        F = 0.5 * np.sum((B[:, j] - A @ xo) ** 2) + lam * np.abs(xo).sum()
        assert abs(res["primal_obj"][j] - F) <= OBJ_TOL * F
        assert res["gap"][j] >= -1e-6 * F
    s.close()


# ------------------------------------------------------------ edge cases

def test_edge_cases(l1):
    p = synthetic.cab_problem(64, 4, 8, 6, seed=14)
    A, B = p["A"], p["B"].copy()
    B[:, 1] = 0.0          # b = 0: every iterate stays 0
    B[3, 4] = np.nan       # poisoned column
    s = l1.Solver(_dev(A), mode=l1.CAB, solver=l1.DALM)
    x, _, res = s.solve(_dev(B), tol=1e-6, max_iter=50)
    x = x.cpu().numpy()
    assert res["status"][1] == l1.CONVERGED and res["iters"][1] == 1 and np.all(x[:, 1] == 0)
    assert res["status"][4] == l1.NONFINITE
    for j in (0, 2, 3, 5):  # neighbours of the poisoned column are unaffected
        w, _, st = oracle.dalm(A, B[:, j], cab=True, tol=1e-6, max_iter=50)
        assert res["iters"][j] == st["iters"]
        assert _rel(x[:, j], w) <= X_TOL
    # host numpy in, host numpy out (the library copies)
    xh, _, resh = s.solve(np.asfortranarray(B[:, [0, 2]]), tol=1e-6, max_iter=50)
    assert isinstance(xh, np.ndarray) and _rel(xh[:, 0], x[:, 0]) <= 1e-6
    # a second, larger solve regrows the workspace
    Bb = np.tile(p["B"], (1, 12))
    x2, _, res2 = s.solve(_dev(Bb), tol=1e-6, max_iter=50)
    assert _rel(x2.cpu().numpy()[:, 0], x[:, 0]) <= 1e-6
    # the old workspace is released: a handle that grew to this width holds
    # as much device memory as one that started there
    s2 = l1.Solver(_dev(A), mode=l1.CAB, solver=l1.DALM)
    s2.solve(_dev(Bb), tol=1e-6, max_iter=50)
    assert s.info()["device_bytes"] == s2.info()["device_bytes"]
    s2.close()
    s.close()


# ------------------------------------- the benchmarked launch configuration

def test_bench_configuration_cuda_cores_fixed_iterations(l1):
    """Full 1024 x 1200 (+I) cross-and-bouquet batch of 1024 right-hand sides
    on the CUDA-core sweeps, 300 iterations, a sample of columns against the
    oracle's same 300 iterations.  (At the stopping tolerance, after ~1800
    iterations, the FP32 products of these sweeps drift from the FP64
    trajectory by up to ~7e-5 in x and ~1.3e-5 in the objective, measured;
    DALM therefore runs on the tensor-core engine by default, whose products
    track it to ~4e-6 -- see test_bench_configuration_tensor_core_engine.)"""
    import bench
    cfg = bench.CAB1024
    p = bench.cab_workload(cfg)
    A, B, off = p["A"], p["B"], p["offsets"]
    iters = 300
    s = l1.Solver(_dev(A), mode=l1.CAB, solver=l1.DALM, class_offsets=off, engine=l1.ENGINE_SIMT)
    x, _, res = s.solve(_dev(B), tol=0.0, max_iter=iters)
    x = x.cpu().numpy()
    sample = [0, 1, 2, 3, 511, 767, 1022, 1023]
    outs = _pmap(lambda j: oracle.dalm(A, B[:, j], cab=True, tol=0.0, max_iter=iters), sample)
    ex = Errs("bench configuration sample (CUDA cores, 300 iterations)")
    for j, (w, _, _) in zip(sample, outs):
        ex.add(x[:, j], w, res["primal_obj"][j])
    ex.check()
    s.close()


# ------------------------------------------------ tensor-core (tcgen05) engine

@pytest.mark.parametrize("N,pieces", [(40, 3), (200, 3), (200, 2)])
def test_cab_dalm_tensor_core_engine_matches_oracle(l1, N, pieces):
    """BF16 tcgen05 sweeps (A and the panels as aligned BF16 pieces, the
    leading product summed exactly) against the FP64 oracle after a fixed
    iteration count: ragged M tiles (256 and 300 rows), a ragged 128-column
    tile, two tiles; three pieces (FP32-level) and two (16-bit) per operand."""
    p = synthetic.cab_problem(256, 10, 30, N, seed=21)
    A, B, off = p["A"], p["B"], p["offsets"]
    n = A.shape[1]
    iters = 300
    s = l1.Solver(_dev(A), mode=l1.CAB, solver=l1.DALM, class_offsets=off, engine=l1.ENGINE_TC,
                  tc_min_cols=1, tc_pieces=pieces, tc_pieces_y=pieces)
    x, y, res = s.solve(_dev(B), tol=0.0, max_iter=iters, want_y=True)
    x = x.cpu().numpy()
    y = y.cpu().numpy()
    assert np.all(res["iters"] == iters)
    cols = list(range(0, N, max(1, N // 12)))
    outs = _pmap(lambda j: oracle.dalm(A, B[:, j], cab=True, tol=0.0, max_iter=iters), cols)
    ex, ey = Errs(f"TC CAB DALM N={N} pieces={pieces} x"), Errs(f"TC CAB DALM N={N} pieces={pieces} y")
    for j, (w, yo, st) in zip(cols, outs):
        ex.add(x[:, j], w, res["primal_obj"][j])
        ey.add(y[:, j], yo)
        lab, slab, r, _ = oracle.classify(A, off, B[:, j], w[:n], w[n:])
        assert res["label"][j] == lab and res["sci_label"][j] == slab
    if pieces == 3:
        ex.check()
        ey.check()
    else:
        # 16-bit products: reported, and held to a looser bound
        print(f"two pieces: x err max {max(ex.x):.2e}, y err max {max(ey.x):.2e}")
        assert max(ex.x) <= 1e-2
    s.close()


def test_p1_dalm_tensor_core_engine_matches_oracle(l1):
    """P1 (B = A, no identity block) on the tensor-core engine."""
    pr = synthetic.p1_instance(200, 400, 20, seed=3)
    A = pr["A"]
    g = np.random.default_rng(0)
    B = np.stack([A @ np.where(g.random(400) < 0.05, g.standard_normal(400), 0) for _ in range(19)], 1)
    iters = 80
    s = l1.Solver(_dev(A), mode=l1.P1, solver=l1.DALM, engine=l1.ENGINE_TC, tc_min_cols=1)
    x, _, res = s.solve(_dev(B), tol=0.0, max_iter=iters)
    x = x.cpu().numpy()
    ex = Errs("TC P1 DALM")
    for j in range(19):
        w, _, _ = oracle.dalm(A, B[:, j], cab=False, tol=0.0, max_iter=iters)
        ex.add(x[:, j], w)
    ex.check()
    s.close()


def test_tensor_core_engine_at_tolerance_with_fallback(l1):
    """At the stopping tolerance: 300 columns start on the tensor-core sweeps
    and, as columns retire, the set falls below tc_min_cols and continues on
    the CUDA-core sweeps (state converted); every sampled column is checked."""
    p = synthetic.cab_problem(256, 10, 30, 300, seed=22)
    A, B, off = p["A"], p["B"], p["offsets"]
    tol = 1e-3
    s = l1.Solver(_dev(A), mode=l1.CAB, solver=l1.DALM, class_offsets=off, engine=l1.ENGINE_TC,
                  tc_min_cols=160)
    x, _, res = s.solve(_dev(B), tol=tol, max_iter=20000)
    x = x.cpu().numpy()
    assert np.all(res["status"] == l1.CONVERGED)
    its = np.sort(res["iters"])
    print("iterations: first retire", its[0], "median", its[150], "last", its[-1])
    cols = [int(j) for j in np.argsort(res["iters"])[::25]]  # spread over early and late retirements

    def run(j, tol_on, iters):
        w, _, st = oracle.dalm(A, B[:, j], cab=True, tol=tol if tol_on else 0.0,
                               max_iter=20000 if tol_on else iters)
        return w, st
    check_at_tolerance("TC engine at tol 1e-3 with fallback", res, x, cols, run)
    s.close()


def test_bench_configuration_tensor_core_engine(l1):
    import bench
    cfg = bench.CAB1024
    p = bench.cab_workload(cfg)
    A, B, off = p["A"], p["B"], p["offsets"]
    n = A.shape[1]
    s = l1.Solver(_dev(A), mode=l1.CAB, solver=l1.DALM, class_offsets=off, engine=l1.ENGINE_TC)
    x, _, res = s.solve(_dev(B), tol=cfg["tol"], max_iter=cfg["max_iter"])
    x = x.cpu().numpy()
    assert np.mean(res["status"] == l1.CONVERGED) >= 0.99
    assert np.mean(res["label"] == p["labels"]) >= 0.99
    sample = [0, 1, 2, 3, 511, 767, 1022, 1023]

    def run(j, tol_on, iters):
        w, _, st = oracle.dalm(A, B[:, j], cab=True, tol=cfg["tol"] if tol_on else 0.0,
                               max_iter=cfg["max_iter"] if tol_on else iters)
        return w, st
    first = check_at_tolerance("TC bench configuration sample", res, x, sample, run)
    for j, (w, st) in zip(sample, first):
        lab, slab, r, _ = oracle.classify(A, off, B[:, j], w[:n], w[n:])
        assert res["label"][j] == lab
    s.close()


# ------------------------------------------------------------ warm start

@pytest.mark.parametrize("engine", ["simt", "tc"])
def test_dalm_warm_start_continues_the_iteration(l1, engine):
    """A DALM solve stopped after k1 iterations and resumed from its (x, y)
    for k2 more equals k1 + k2 iterations of the oracle (and of an
    uninterrupted solve)."""
    p = synthetic.cab_problem(256, 10, 30, 140, seed=31)
    A, B, off = p["A"], p["B"], p["offsets"]
    eng = dict(engine=l1.ENGINE_TC, tc_min_cols=1) if engine == "tc" else dict(engine=l1.ENGINE_SIMT)
    s = l1.Solver(_dev(A), mode=l1.CAB, solver=l1.DALM, class_offsets=off, **eng)
    k1, k2 = 120, 80
    x1, y1, _ = s.solve(_dev(B), tol=0.0, max_iter=k1, want_y=True)
    x2, y2, r2 = s.solve(_dev(B), tol=0.0, max_iter=k2, want_y=True, x_init=x1, y_init=y1)
    xf, _, _ = s.solve(_dev(B), tol=0.0, max_iter=k1 + k2)
    x2, xf = x2.cpu().numpy(), xf.cpu().numpy()
    cols = [0, 7, 70, 139]
    outs = _pmap(lambda j: oracle.dalm(A, B[:, j], cab=True, tol=0.0, max_iter=k1 + k2), cols)
    ex = Errs(f"DALM warm start ({engine})")
    for j, (w, _, _) in zip(cols, outs):
        ex.add(x2[:, j], w, r2["primal_obj"][j])
        assert _rel(x2[:, j], xf[:, j]) <= 1e-5
    ex.check()
    s.close()


def test_palm_warm_start_continues_the_iteration(l1):
    """CAB PALM (fixed xi) resumed from (x, e, theta) after k1 outer
    iterations equals k1 + k2 outer iterations of the oracle."""
    p = synthetic.cab_problem(192, 6, 30, 9, seed=32)
    A, B, off = p["A"], p["B"], p["offsets"]
    L = oracle.lipschitz(A)
    inner = 20
    s = l1.Solver(_dev(A), mode=l1.CAB, solver=l1.PALM, class_offsets=off, lipschitz=L, inner_max=inner)
    k1, k2 = 5, 7
    x1, y1, _ = s.solve(_dev(B), tol=0.0, max_iter=k1, want_y=True)
    x2, _, r2 = s.solve(_dev(B), tol=0.0, max_iter=k2, want_y=True, x_init=x1, y_init=y1)
    x2 = x2.cpu().numpy()
    outs = _pmap(lambda j: oracle.palm(A, B[:, j], mode=oracle.MODE_CAB, tol=0.0, max_outer=k1 + k2,
                                       inner_max=inner, L=L), range(9))
    ex = Errs("PALM warm start")
    for j, (xo, eo, th, st) in enumerate(outs):
        ex.add(x2[:, j], np.concatenate([xo, eo]), r2["primal_obj"][j])
    ex.check()
    s.close()


def test_graph_replay_is_deterministic(l1):
    """The polling chunks are captured as CUDA graphs on the first solve and
    replayed afterwards; replays (and a solve after the workspace grew, which
    drops the cached graphs) give bit-identical results."""
    p = synthetic.cab_problem(192, 6, 30, 40, seed=21)
    A, B, off = p["A"], p["B"], p["offsets"]
    s = l1.Solver(_dev(A), mode=l1.CAB, solver=l1.DALM, class_offsets=off)
    x1, _, r1 = s.solve(_dev(B), tol=1e-4, max_iter=3000)
    x2, _, r2 = s.solve(_dev(B), tol=1e-4, max_iter=3000)
    assert torch.equal(x1, x2) and np.array_equal(r1["iters"], r2["iters"])
    # a wider batch grows the workspace (the cached graphs point into the old
    # one and are dropped); its sweeps split K differently, so the first 40
    # columns agree to rounding, not bit for bit
    big = np.concatenate([B, B[:, :30]], axis=1)
    x3, _, r3 = s.solve(_dev(big), tol=1e-4, max_iter=3000)
    a, b = x3[:, :40].cpu().numpy(), x1.cpu().numpy()
    assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b)
    assert np.array_equal(r3["label"][:40], r1["label"])
    assert np.array_equal(r3["label"][40:], r1["label"][:30])
    s.close()


@pytest.mark.parametrize("engine", ["simt", "tc"])
def test_profiled_solve_reports_sweep_times(l1, engine):
    """l1_options.profile times every sweep with CUDA events, whether the
    chunk is replayed from a graph (CUDA-core sweeps) or launched directly
    (tensor-core engine); the profiled solve equals the unprofiled one."""
    p = synthetic.cab_problem(192, 6, 30, 40, seed=23)
    A, B, off = p["A"], p["B"], p["offsets"]
    eng = l1.ENGINE_TC if engine == "tc" else l1.ENGINE_SIMT
    s0 = l1.Solver(_dev(A), mode=l1.CAB, solver=l1.DALM, class_offsets=off, engine=eng)
    s1 = l1.Solver(_dev(A), mode=l1.CAB, solver=l1.DALM, class_offsets=off, engine=eng, profile=True)
    x0, _, r0 = s0.solve(_dev(B), tol=0.0, max_iter=64)
    x1, _, r1 = s1.solve(_dev(B), tol=0.0, max_iter=64)
    assert torch.equal(x0, x1)
    info = s1.info()
    assert all(v > 0 for v in info["sweep_launches"][:3]) and all(v > 0 for v in info["sweep_ms"][:3])
    s0.close()
    s1.close()


# ---------------------------------------- the plain per-instance FP32 solver

def test_plain_per_instance_solver_tracks_the_oracle(l1):
    """l1_solve_plain (one right-hand side, one simple FP32 kernel per step,
    the FP32 inverse without its low part) against the oracle after a fixed
    iteration count, and to the stopping rule with the oracle's labels."""
    p = synthetic.cab_problem(256, 10, 30, 3, seed=41)
    A, B, off = p["A"], p["B"], p["offsets"]
    n = A.shape[1]
    s = l1.Solver(_dev(A), mode=l1.CAB, solver=l1.DALM, class_offsets=off)
    errs = []
    for j in range(3):
        x, r = s.solve_plain(_dev(B[:, j:j + 1])[:, 0].contiguous(), 0.0, 300)
        w, _, _ = oracle.dalm(A, B[:, j], cab=True, tol=0.0, max_iter=300)
        assert r["iters"] == 300 and r["status"] == l1.MAX_ITER
        errs.append(_rel(x.cpu().numpy(), w))
        x, r = s.solve_plain(B[:, j].astype(np.float32), 1e-3, 20000)  # host in, host out
        assert r["status"] == l1.CONVERGED
        wo, _, st = oracle.dalm(A, B[:, j], cab=True, tol=1e-3, max_iter=20000)
        assert abs(r["iters"] - st["iters"]) <= 2
        lab = oracle.classify(A, off, B[:, j], wo[:n], wo[n:])[0]
        assert oracle.classify(A, off, B[:, j], x[:n].astype(np.float64), x[n:].astype(np.float64))[0] == lab
    print(f"plain per-instance FP32 solver, 300 iterations: x rel. err max {max(errs):.2e}")
    assert max(errs) <= 1e-3
    s.close()


def test_4096_workload_against_stored_oracle_answers(l1):
    """The 4096 x 4000 (+ identity) cross-and-bouquet workload (100 classes x
    40 columns, 4096 test vectors, seed 3000) on the default engine, at the
    stopping tolerance, against FP64-oracle answers stored for 8 sampled
    columns (an oracle solve of this size takes minutes): every sampled column
    must stop within one iteration of the oracle, agree with the oracle's
    iterate at its own stop and carry the oracle's label.  Then 200 fixed
    iterations of 4 of those columns, solved as a batch of 4 on the tensor
    cores, against the oracle's iterate after 200 iterations."""
    import bench
    cfg = bench.CAB4096
    p = bench.cab_workload(cfg)
    A, B, off = p["A"], p["B"], p["offsets"]
    g = bench.golden_oracle(p)
    cols = sorted(g)
    s = l1.Solver(_dev(A), mode=l1.CAB, solver=l1.DALM, class_offsets=off)
    x, _, res = s.solve(_dev(B), tol=cfg["tol"], max_iter=cfg["max_iter"])
    x = x.cpu().numpy()
    assert np.mean(res["status"] == l1.CONVERGED) >= 0.99
    assert np.mean(res["label"] == p["labels"]) >= 0.99
    d = bench.verify_columns(cols, x[:, cols], res["iters"][cols], res["primal_obj"][cols], res["label"][cols],
                             lambda j: g[j]["stop"], lambda j, k: g[j]["at"].get(k), lambda j: g[j]["label"])
    print("4096 workload, stored oracle sample:", {k: v for k, v in d.items() if k != "per_instance"})
    print([(q["col"], q["stop_gpu_minus_oracle"], q["rel_err_x"], q["rel_err_obj"]) for q in d["per_instance"]])
    assert d["within_bar"] == d["of"] == len(cols), d["per_instance"]

    gz = np.load(bench.GOLDEN4096)
    fc = [int(j) for j in gz["fixed_cols"]]
    s4 = l1.Solver(_dev(A), mode=l1.CAB, solver=l1.DALM, class_offsets=off, engine=l1.ENGINE_TC, tc_min_cols=1)
    x4, _, r4 = s4.solve(_dev(B[:, fc]), tol=0.0, max_iter=int(gz["fixed_iters"]))
    x4 = x4.cpu().numpy()
    assert (r4["iters"] == int(gz["fixed_iters"])).all()
    ex = Errs("4096 workload, 200 fixed iterations, batch of 4 on the tensor cores")
    for k in range(len(fc)):
        ex.add(x4[:, k], gz["w_fixed"][:, k].astype(np.float64), r4["primal_obj"][k])
    ex.check()
    s.close()
    s4.close()


def test_split_autotuner_records_choices_and_keeps_parity(l1):
    """l1_setup's autotuner times the tile strategies (fused or deferred
    epilogue, split-K) of the three tensor-core sweep shapes (A u: m x n, the
    y-step: m x m, A^T y: n x m) at widths up to 4096 and keeps the fastest;
    tune=False keeps the fixed rule.  A narrow batch solved on either handle
    matches the oracle after the same iterations."""
    p = synthetic.cab_problem(1024, 40, 30, 6, corrupt=0.3, seed=11)
    A, B = p["A"], p["B"]
    m, n = A.shape
    s = l1.Solver(_dev(A), mode=l1.CAB, solver=l1.DALM, engine=l1.ENGINE_TC, tc_min_cols=1)
    t = s.tuning()
    print("split-K choices:", t)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert len(t) > 0
    for e in t:
        assert (e["M"], e["K"]) in {(m, n), (m, m), (n, m)}
        assert 1 <= e["ksplit"] <= 16 and e["us"] >= 0 and e["deferred"] in (0, 1) and e["bn"] in (64, 128)
        assert e["ksplit"] == 1 or e["deferred"] == 1
        assert e["bn"] == 128 or e["deferred"] == 1
        # split-K slices fill at most four waves of one CTA per SM
        assert e["ksplit"] * e["tiles"] * (128 // e["bn"]) <= 4 * sms or e["ksplit"] == 1
    s0 = l1.Solver(_dev(A), mode=l1.CAB, solver=l1.DALM, engine=l1.ENGINE_TC, tc_min_cols=1, tune=False)
    assert s0.tuning() == []
    iters = 120
    xa, _, _ = s.solve(_dev(B), tol=0.0, max_iter=iters)
    xb, _, _ = s0.solve(_dev(B), tol=0.0, max_iter=iters)
    xa, xb = xa.cpu().numpy(), xb.cpu().numpy()
    ex = Errs("narrow TC batch, tuned and fixed split-K, 120 iterations")
    for j in range(B.shape[1]):
        w, _, _ = oracle.dalm(A, B[:, j], cab=True, tol=0.0, max_iter=iters)
        ex.add(xa[:, j], w)
        ex.add(xb[:, j], w)
    ex.check()
    s.close()
    s0.close()


def test_qp_fista_with_continuation_matches_oracle(l1):
    """FISTA with fixed-point continuation (reading R17) for a batch of
    (QP_lambda) problems on one Gaussian dictionary: lambda falls by 0.95 per
    step from lambda_0 = max_j ||A^T b_j||_inf to lambda = 1e-3 lambda_0.
    After the same number of steps (tol = 0) and at the stopping tolerance
    (stop within one step of the oracle's) the GPU follows orc_fista_cont;
    it stops in fewer steps than plain FISTA at the same lambda."""
    pr = synthetic.p1_instance(200, 400, 20, seed=0)
    A = pr["A"]
    g = np.random.default_rng(5)
    N = 6
    X0 = np.zeros((400, N))
    for j in range(N):
        X0[g.choice(400, 20, replace=False), j] = g.choice([-1.0, 1.0], 20)
    B = A @ X0
    lam0 = float(np.max(np.abs(A.T @ B)))
    lam = 1e-3 * lam0
    L = oracle.lipschitz(A)
    s = l1.Solver(_dev(A), mode=l1.QP_LAMBDA, lam=lam, lipschitz=L, lam0=lam0)
    x, _, res = s.solve(_dev(B), tol=0.0, max_iter=120)
    x = x.cpu().numpy()
    ex = Errs("FISTA with continuation, 120 steps")
    for j in range(N):
        w, _ = oracle.fista_cont(A, B[:, j], lam, lam0=lam0, L=L, tol=0.0, max_iter=120)
        ex.add(x[:, j], w)
    ex.check()
    tol = 1e-6
    x, _, res = s.solve(_dev(B), tol=tol, max_iter=20000)
    x = x.cpu().numpy()
    assert (res["status"] == l1.CONVERGED).all()
    s_plain = l1.Solver(_dev(A), mode=l1.QP_LAMBDA, lam=lam, lipschitz=L)
    _, _, res_plain = s_plain.solve(_dev(B), tol=tol, max_iter=20000)
    print("steps: continuation", res["iters"], "plain", res_plain["iters"])
    assert np.all(res["iters"] < res_plain["iters"])

    # at the stopping tolerance: every column stops within one step of the
    # oracle and agrees with the oracle's iterate at its own stop (the
    # objective here is (QP_lambda)'s, 1/2 ||b - A x||^2 + lambda ||x||_1)
    ex = Errs("FISTA with continuation at tol 1e-6")
    stops = []
    for j in range(N):
        w, st = oracle.fista_cont(A, B[:, j], lam, lam0=lam0, L=L, tol=tol, max_iter=20000)
        kg = int(res["iters"][j])
        stops.append(kg - st["iters"])
        if kg != st["iters"]:
            w, _ = oracle.fista_cont(A, B[:, j], lam, lam0=lam0, L=L, tol=0.0, max_iter=kg)
        ex.add(x[:, j], w)
        F = 0.5 * np.sum((B[:, j] - A @ w) ** 2) + lam * np.abs(w).sum()
        ex.obj.append(abs(res["primal_obj"][j] - F) / F)
    print("GPU stop - oracle stop", stops)
    assert max(abs(d) for d in stops) <= 1
    ex.check()
    s.close()
    s_plain.close()
