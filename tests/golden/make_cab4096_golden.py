"""Writes cab4096_dalm_oracle.npz: FP64-oracle answers for a sample of the
4096 x 4000 (+ identity) cross-and-bouquet workload (100 classes x 40
columns, 4096 test vectors, seed 3000), which the oracle needs hours of CPU
time to produce at run time.  Only the oracle (oracle/) and the input
generator (synthetic/) are called; nothing comes from the CUDA path.

For each sampled test vector j it stores
  * the DALM iterate at the oracle's own stop (relative-change rule of §VI-C
    at tol = 1e-4, Algorithm 2 from w = 0, y = 0) and the stopping iteration
    k_j, with the iterates one step before and after it (as FP16 differences
    from the stopped one: they differ by about tol), so that a run stopping
    within one iteration of the oracle can be compared with the oracle's
    iterate at its own stopping iteration;
  * the iterate after exactly K_FIXED iterations (tol = 0), for a trajectory
    comparison at a fixed iteration count;
  * the class labels of the stopped iterate (minimum per-class residual and
    the SCI rule, §II-A, Eq. 40);
  * checksums of the generated inputs, so that a machine whose generator
    output differs is noticed.

Run:  python tests/golden/make_cab4096_golden.py   (about half an hour on 8 cores)
"""
from __future__ import annotations

import os
import sys
import time
from concurrent.futures import ProcessPoolExecutor
from multiprocessing import get_context

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

CFG = dict(m=4096, classes=100, per_class=40, N=4096, corrupt=0.3, seed=3000, tol=1e-4, max_iter=10000)
SAMPLE = [0, 1, 517, 1024, 2047, 2900, 3583, 4095]
K_FIXED = 200
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cab4096_dalm_oracle.npz")


def problem():
    import synthetic
    return synthetic.cab_problem(CFG["m"], CFG["classes"], CFG["per_class"], CFG["N"], corrupt=CFG["corrupt"],
                                 seed=CFG["seed"])


def job(args):
    import oracle
    j, kind, iters = args
    p = problem()
    A, b = p["A"], p["B"][:, j]
    t = time.time()
    if kind == "tol":
        w, y, st = oracle.dalm(A, b, cab=True, tol=CFG["tol"], max_iter=CFG["max_iter"])
    else:
        w, y, st = oracle.dalm(A, b, cab=True, tol=0.0, max_iter=iters)
    return j, kind, iters, w, st, time.time() - t


def main():
    p = problem()
    A, B, off = p["A"], p["B"], p["offsets"]
    n = A.shape[1]
    ctx = get_context("spawn")
    workers = min(8, os.cpu_count() or 1)
    with ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as ex:
        first = list(ex.map(job, [(j, "tol", 0) for j in SAMPLE] + [(j, "fixed", K_FIXED) for j in SAMPLE[:4]]))
        stops = {j: st["iters"] for j, kind, _, _, st, _ in first if kind == "tol"}
        conv = {j: st["converged"] for j, kind, _, _, st, _ in first if kind == "tol"}
        nbrs = list(ex.map(job, [(j, "at", stops[j] + d) for j in SAMPLE for d in (-1, 1)]))
    import oracle
    w_stop = {j: w for j, kind, _, w, _, _ in first if kind == "tol"}
    w_fixed = {j: w for j, kind, _, w, _, _ in first if kind == "fixed"}
    w_at = {(j, it): w for j, kind, it, w, _, _ in nbrs}
    ws = np.stack([w_stop[j] for j in SAMPLE], 1)
    dm = np.stack([w_at[(j, stops[j] - 1)] - w_stop[j] for j in SAMPLE], 1)
    dp = np.stack([w_at[(j, stops[j] + 1)] - w_stop[j] for j in SAMPLE], 1)
    # the stored FP16 differences must reproduce the neighbours to well below
    # the 1e-4 comparison bar
    for k, j in enumerate(SAMPLE):
        for d, it in ((dm, stops[j] - 1), (dp, stops[j] + 1)):
            rec = ws[:, k].astype(np.float32).astype(np.float64) + d[:, k].astype(np.float16).astype(np.float64)
            err = np.linalg.norm(rec - w_at[(j, it)]) / np.linalg.norm(w_at[(j, it)])
            assert err < 1e-6, (j, it, err)
    labels = [oracle.classify(A, off, B[:, j], w_stop[j][:n], w_stop[j][n:])[:2] for j in SAMPLE]
    np.savez_compressed(
        OUT, cols=np.array(SAMPLE, np.int32), stop_iters=np.array([stops[j] for j in SAMPLE], np.int32),
        converged=np.array([conv[j] for j in SAMPLE], np.int32),
        w_stop=ws.astype(np.float32), d_before=dm.astype(np.float16), d_after=dp.astype(np.float16),
        fixed_cols=np.array(SAMPLE[:4], np.int32), fixed_iters=np.int32(K_FIXED),
        w_fixed=np.stack([w_fixed[j] for j in SAMPLE[:4]], 1).astype(np.float32),
        label=np.array([a for a, _ in labels], np.int32), sci_label=np.array([b for _, b in labels], np.int32),
        a_sum=np.float64(A.sum()), a_sq=np.float64((A * A).sum()),
        b_sums=np.array([B[:, j].sum() for j in SAMPLE], np.float64),
        tol=np.float64(CFG["tol"]), max_iter=np.int32(CFG["max_iter"]), seed=np.int32(CFG["seed"]))
    print("wrote", OUT, "stops", [stops[j] for j in SAMPLE],
          "oracle seconds", [round(t) for *_, t in first])


if __name__ == "__main__":
    main()
