#!/usr/bin/env python3
"""Benchmark of the batched cross-and-bouquet DALM solve (one JSON line).

Workload (the robust-classification setting of §VI-B at the stated sizes):
dictionary [A I] with A 1024 x 1200 = 40 classes x 30 columns, each class a
rank-9 nonnegative subspace plus 1 % noise, unit columns; 1024 test vectors
with 30 % of their entries replaced by uniform [0, 1] gross errors; DALM
(Algorithm 2) in FP32, every test vector stopped by the relative-change rule
of §VI-C at tol, then classified by the minimum per-class residual.

A step is one l1_solve_batch over the 1024 right-hand sides (all sweeps,
per-column stopping, finalisation and classification).  `value` counts the
converged solves per second with the inputs resident in HBM; `e2e` repeats the
measurement through the same C-ABI call with pinned host buffers (the copies
in and out are inside the timed region).  L2 is flushed (a 512 MiB write)
before every timed step; the flush is outside the step's CUDA events.

--impl reference times the FP64 CPU oracle (the same algorithm, plain C) on
the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic  # noqa: E402

# the cross-and-bouquet workloads (tests import them to check parity in the
# same launch shape): 40 classes x 30 columns at m = 1024 in FP32, and
# 100 classes x 40 columns at m = 4096 with A held in BF16 pieces on the
# tensor cores
CAB1024 = dict(m=1024, classes=40, per_class=30, N=1024, corrupt=0.3, seed=1000,
               tol=1e-4, max_iter=10000, solver="DALM")
CAB4096 = dict(m=4096, classes=100, per_class=40, N=4096, corrupt=0.3, seed=3000,
               tol=1e-4, max_iter=10000, solver="DALM")
BENCH = dict(CAB1024)


def cab_workload(cfg, rank: int = 0):
    return synthetic.cab_problem(cfg["m"], cfg["classes"], cfg["per_class"], cfg["N"],
                                 corrupt=cfg["corrupt"], seed=cfg["seed"] + rank)
METRIC = "solves/sec at rel. err <=1e-4 vs FP64 oracle"
L2_FLUSH_BYTES = 512 << 20
FP32_SIMT_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x FMA x max clock
TF32_PER_BF16 = 1.1 / 2.25  # nominal dense tensor rates of the part
# ncu dram__bytes_read.sum + dram__bytes_write.sum of one full-batch launch
# (all 1024 columns active, cold cache) of each CUDA-core sweep of this
# build, and the algorithmic bytes of that launch
SIMT_TRAFFIC = {"A_u": (18.42e6, 18.2e6), "Finv_r": (21.12e6, 21.0e6), "At_y": (19.27e6, 19.1e6)}
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def measured_peaks() -> dict:
    """Measured peaks of this machine's GPUs, else the stated fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {k: float(d[k]) for k in FALLBACK_PEAKS}
    except (OSError, KeyError, ValueError):
        return dict(FALLBACK_PEAKS)


def reduce_over_ranks(dist, time_value: float, count: int, device: str = "cuda"):
    """Whole-job figures of a replicated run: the slowest rank's time and the
    sum of the ranks' converged solves (dist None: this process only)."""
    if dist is None:
        return time_value, count
    import torch
    t = torch.tensor([time_value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([count], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), int(c.item())


def workload(rank: int = 0):
    return synthetic.cab_problem(BENCH["m"], BENCH["classes"], BENCH["per_class"], BENCH["N"],
                                 corrupt=BENCH["corrupt"], seed=BENCH["seed"] + rank)


def config_dict(extra=None):
    d = {"workload": f"cab_dalm_m{BENCH['m']}_n{BENCH['classes'] * BENCH['per_class']}_N{BENCH['N']}",
         "m": BENCH["m"], "n": BENCH["classes"] * BENCH["per_class"], "classes": BENCH["classes"],
         "rhs_per_gpu": BENCH["N"], "solver": BENCH["solver"], "tol": BENCH["tol"],
         "max_iter": BENCH["max_iter"], "corrupt_fraction": BENCH["corrupt"],
         "l2": (f"flushed (512 MiB write) before each timed step; A ({BENCH['m'] * BENCH['classes'] * BENCH['per_class'] * 4 / 1e6:.1f} MB FP32) "
                "and F (the inverse of A A^T + I) stay in L2 within a solve when they fit (129 MB)")}
    if extra:
        d.update(extra)
    return d


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm_, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm_)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def run_cpu_oracle(p, cols, threads, tol, max_iter):
    import concurrent.futures as cf

    import oracle
    oracle.build()
    A, B = p["A"], p["B"]

    def one(j):
        return oracle.dalm(A, B[:, j], cab=True, tol=tol, max_iter=max_iter)

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        outs = list(ex.map(one, cols))
    dt = time.perf_counter() - t0
    conv = sum(1 for _, _, st in outs if st["converged"])
    return conv, dt, outs


def oracle_agreement(p, cols, x_gpu, obj_gpu, label_gpu, outs, bar=1e-4):
    """Per sampled test vector j: ||x_gpu - w_j|| / ||w_j|| and the relative
    objective error against the oracle's w_j = [x; e] (same tol and
    max_iter), and whether the class labels agree.  x_gpu holds the sampled
    columns of the GPU solve in the order of cols."""
    import oracle
    A, B, off = p["A"], p["B"], p["offsets"]
    n = A.shape[1]
    ex, eo, labels = [], [], 0
    for k, (j, (w, _, _)) in enumerate(zip(cols, outs)):
        nw = np.linalg.norm(w)
        ex.append(float(np.linalg.norm(np.asarray(x_gpu[:, k], np.float64) - w) / nw) if nw > 0 else 0.0)
        f = float(np.abs(w).sum())
        eo.append(abs(float(obj_gpu[k]) - f) / f if f > 0 else 0.0)
        labels += int(oracle.classify(A, off, B[:, j], w[:n], w[n:])[0] == int(label_gpu[k]))
    return {"sample": f"test vectors {cols[0]}..{cols[-1]} of the last timed solve, oracle at the same tol/max_iter",
            "max_rel_err_x": max(ex), "max_rel_err_obj": max(eo),
            "within_bar": sum(1 for e in ex if e <= bar), "bar": bar, "of": len(ex),
            "labels_equal": labels}


def bench_reference(args, rank, world):
    """FP64 CPU oracle on the host cores (the comparison arm)."""
    if rank != 0:
        return 0
    p = workload(0)
    threads = min(os.cpu_count() or 1, 16)
    sample = list(range(threads))  # one instance per core per step
    for _ in range(max(0, min(args.warmup, 1))):
        pass  # the oracle has no warm-up state
    total_conv, total_t = 0, 0.0
    for _ in range(args.steps):
        conv, dt, _ = run_cpu_oracle(p, sample, threads, BENCH["tol"], BENCH["max_iter"])
        total_conv += conv
        total_t += dt
    value = total_conv / total_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict({"sample": f"{len(sample)} of {BENCH['N']} test vectors per step"}),
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": threads, "kind": "oracle",
                             "sample": f"{len(sample)} test vectors per step, one per thread"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def bench_ours(args, rank, world):
    import torch

    import paper_1007_3753_gb300 as l1
    from paper_1007_3753_gb300 import build

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()
    l1.load()
    p = workload(rank)
    A, B, off = p["A"], p["B"], p["offsets"]
    m, n = A.shape
    N = B.shape[1]
    stream = torch.cuda.current_stream()
    A_d = torch.from_numpy(np.ascontiguousarray(A.T, dtype=np.float32)).cuda().t()
    B_d = torch.from_numpy(np.ascontiguousarray(B.T, dtype=np.float32)).cuda().t()
    x_d = torch.empty((N, n + m), dtype=torch.float32, device="cuda").t()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    solver = l1.DALM if BENCH["solver"] == "DALM" else l1.PALM
    engine = l1.ENGINE_TC if args.engine == "tc" else l1.ENGINE_SIMT
    # two handles on the same dictionary: the last timed step runs on the one
    # that times every sweep with CUDA events (the roofline), the others on
    # the one without events
    prec = {"fp32": l1.A_FP32, "bf16": l1.A_BF16, "fp8": l1.A_FP8E4M3}[args.precision]
    s = l1.Solver(A_d, mode=l1.CAB, solver=solver, class_offsets=off, profile=False, engine=engine,
                  precision=prec, stream=stream.cuda_stream)
    sp = l1.Solver(A_d, mode=l1.CAB, solver=solver, class_offsets=off, profile=True, engine=engine,
                   precision=prec, stream=stream.cuda_stream)
    setup_ms = s.info()["setup_ms"]
    tol, max_iter = BENCH["tol"], BENCH["max_iter"]

    for _ in range(args.warmup):
        s.solve(B_d, tol, max_iter, x=x_d)
        sp.solve(B_d, tol, max_iter, x=x_d)
    torch.cuda.synchronize()
    info0, infop0 = s.info(), sp.info()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    barrier()
    if sampler:
        sampler.start()
    step_ms, conv, iters, labels_ok = [], 0, [], 0
    check_cols = min(os.cpu_count() or 1, 16, N)
    for step in range(args.steps):
        flush.fill_(1.0)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h = sp if step == args.steps - 1 else s
        ev0.record(stream)
        _, _, res = h.solve(B_d, tol, max_iter, x=x_d)
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        conv += int(np.sum(res["status"] == l1.CONVERGED))
        iters.append(float(np.mean(res["iters"])))
        labels_ok += int(np.sum(res["label"] == p["labels"]))
    barrier()
    clocks = sampler.stop() if sampler else None
    # the first columns of the last timed solve, for the comparison with the
    # oracle below (later calls reuse x_d)
    x_check = x_d[:, :check_cols].cpu().numpy()
    res_check = {k: np.asarray(res[k][:check_cols]) for k in ("primal_obj", "label")}
    info1, infop1 = s.info(), sp.info()
    total_ms = sum(step_ms)
    total_ms, conv = reduce_over_ranks(dist, total_ms, conv)
    value = conv / (total_ms / 1e3)

    # ---- end to end through the same call with pinned host buffers
    Bh = torch.from_numpy(np.ascontiguousarray(B.T, dtype=np.float32)).pin_memory().t()
    xh = torch.empty((N, n + m), dtype=torch.float32).pin_memory().t()
    s.solve(Bh, tol, max_iter, x=xh)  # warm
    barrier()
    t0 = time.perf_counter()
    e2e_conv = 0
    for _ in range(args.steps):
        _, _, res = s.solve(Bh, tol, max_iter, x=xh)
        e2e_conv += int(np.sum(res["status"] == l1.CONVERGED))
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s, e2e_conv = reduce_over_ranks(dist, e2e_s, e2e_conv)

    if rank != 0:
        s.close()
        sp.close()
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # ---- roofline of the dominant sweep over the timed region
    names = ["A_u", "Finv_r", "At_y", "other"]
    d_ms = [infop1["sweep_ms"][k] - infop0["sweep_ms"][k] for k in range(4)]
    d_fl = [infop1["sweep_flop"][k] - infop0["sweep_flop"][k] for k in range(4)]
    d_ln = [infop1["sweep_launches"][k] - infop0["sweep_launches"][k] for k in range(4)]
    k = int(np.argmax(d_ms))
    achieved = d_fl[k] / (d_ms[k] / 1e3) / 1e12 if d_ms[k] > 0 else 0.0
    # with --engine tc, A u and A^T y run on tcgen05 and the y-step stays on
    # the compensated CUDA-core sweep (the library's default tc_sweeps)
    on_tc = args.engine == "tc" and names[k] in ("A_u", "At_y")
    if on_tc:
        # split-TF32 tcgen05 sweeps: 3 TF32 products per FP32 product (6 for the
        # y-step); peak = measured sustained BF16 x the nominal TF32/BF16 ratio
        peaks = measured_peaks()
        terms = [3, 6, 3, 1][k]
        peak = peaks["bf16_tflops_sustained"] * TF32_PER_BF16
        roofline = {"bound": "tensor", "kernel": f"sweep {names[k]} (gemm_tc_kernel, tcgen05 kind::tf32)",
                    "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": None,
                    "peak_note": (f"of measured: bf16_tflops_sustained {peaks['bf16_tflops_sustained']} x "
                                  f"{TF32_PER_BF16:.4f} (nominal TF32 1.1 / BF16 2.25 PFLOP/s); "
                                  f"achieved counts algorithmic FP32 FLOPs 2*M*K*N"),
                    "executed_tf32_tflops": achieved * terms, "executed_frac": achieved * terms / peak,
                    "launches": d_ln[k], "avg_launch_us": 1e3 * d_ms[k] / max(1, d_ln[k]),
                    "share_of_sweep_time": d_ms[k] / max(1e-9, sum(d_ms))}
    else:
        # the y-step multiplies by the FP32 pair F_hi + F_lo: two products per
        # algorithmic one
        terms = [1, 2, 1, 1][k]
        default_size = (BENCH["m"], BENCH["classes"], BENCH["per_class"], BENCH["N"]) == (1024, 40, 30, 1024)
        tr = SIMT_TRAFFIC.get(names[k]) if default_size and args.precision == "fp32" else None
        roofline = {"bound": "alu", "kernel": f"sweep {names[k]} (gemm_simt_kernel / split-K pair)",
                    "achieved": achieved, "peak": FP32_SIMT_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP32_SIMT_PEAK_TFLOPS, "traffic": tr[0] if tr else None,
                    "traffic_note": ("bytes of one full-batch launch (N = 1024, cold cache) from ncu; "
                                     f"algorithmic bytes of that launch {tr[1]:.3g}") if tr else None,
                    "peak_note": "FP32 FMA: 152 SMs x 128 lanes x 2 FLOP x 2070 MHz (derived, no measured FP32 peak)",
                    "executed_tflops": achieved * terms, "executed_frac": achieved * terms / FP32_SIMT_PEAK_TFLOPS,
                    "launches": d_ln[k], "avg_launch_us": 1e3 * d_ms[k] / max(1, d_ln[k]),
                    "share_of_sweep_time": d_ms[k] / max(1e-9, sum(d_ms))}

    # ---- the dominant sweep at full width: 100 iterations with every column
    # active (the timed solves above also contain the narrow launches of the
    # last columns, which are latency-bound)
    fw0 = sp.info()
    sp.solve(B_d, 0.0, 100, x=x_d)
    torch.cuda.synchronize()
    fw1 = sp.info()
    fms = fw1["sweep_ms"][k] - fw0["sweep_ms"][k]
    ffl = fw1["sweep_flop"][k] - fw0["sweep_flop"][k]
    fach = ffl / (fms / 1e3) / 1e12 if fms > 0 else 0.0
    fterms = [3, 6, 3, 1][k] if on_tc else [1, 2, 1, 1][k]
    fpeak = roofline["peak"]
    roofline_full = {"bound": roofline["bound"], "kernel": roofline["kernel"], "achieved": fach,
                     "peak": fpeak, "unit": "TFLOP/s", "frac": fach / fpeak,
                     "executed_frac": fach * fterms / fpeak,
                     "note": f"100 iterations, all {N} columns active, same handle and events"}

    # ---- the same solver one right-hand side at a time (no batching): the
    # first 16 test vectors, each its own l1_solve_batch with N = 1
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    single_conv = 0
    n_single = min(16, N)
    for j in range(n_single):
        _, _, r1 = s.solve(B_d[:, j:j + 1], tol, max_iter)
        single_conv += int(r1["status"][0] == l1.CONVERGED)
    torch.cuda.synchronize()
    single_rate = single_conv / (time.perf_counter() - t0)
    per_instance = {"value": single_rate, "unit": "solves/s",
                    "sample": f"first {n_single} test vectors, one l1_solve_batch each (N = 1)",
                    "batched_over_per_instance": value / single_rate if single_rate > 0 else None}

    # ---- CPU oracle on a bounded sample of the same workload
    cpu = None
    agreement = None
    if not args.no_cpu_baseline:
        threads = min(os.cpu_count() or 1, 16)
        sample = list(range(min(threads, N)))
        c_conv, c_dt, outs = run_cpu_oracle(p, sample, threads, tol, max_iter)
        cpu = {"value": c_conv / c_dt, "unit": "solves/s", "cores": threads, "kind": "oracle",
               "sample": f"first {len(sample)} of {N} test vectors, one per thread, same tol/max_iter"}
        try:
            agreement = oracle_agreement(p, sample, x_check, res_check["primal_obj"], res_check["label"],
                                         outs)
        except Exception as exc:  # reported in the line, never fatal to it
            agreement = {"error": f"{type(exc).__name__}: {exc}"}

    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "ms_per_step_median": statistics.median(step_ms),  # rank 0's own steps
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else f"{args.precision} A, f32 arithmetic",
            "data": "synthetic",
            "config": config_dict({"parallelism": f"replicas{world}" if world > 1 else "single",
                                   "engine": args.engine, "precision": args.precision, "setup_ms": setup_ms,
                                   "mean_iters": statistics.mean(iters),
                                   "label_accuracy_vs_planted": labels_ok / (args.steps * N)}),
            "e2e": {"value": e2e_conv / e2e_s, "unit": "solves/s",
                    "h2d_bytes_per_step": 4 * m * N,
                    "d2h_bytes_per_step": 4 * (n + m) * N + 72 * N},
            "gpu_launches": int((info1["gpu_launches"] - info0["gpu_launches"]) +
                                (infop1["gpu_launches"] - infop0["gpu_launches"])),
            "roofline": roofline, "roofline_full_width": roofline_full, "cpu_baseline": cpu,
            "per_instance_gpu": per_instance, "oracle_agreement": agreement, "clocks": clocks}
    print(json.dumps(line), flush=True)
    s.close()
    sp.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


# uneven batch of independent (QP_lambda) problems (Eq. 3): m log-uniform in
# [256, 4096], n/m log-uniform in [2, 4], Gaussian unit-column A, m/10-sparse
# x0, b = A x0 + N(0, 0.01^2), lambda = 1e-3; A stored in BF16
GROUP = dict(count=8192, seed=4000, lam=1e-3, tol=1e-5, max_iter=5000)


def bench_group(args, rank, world):
    """--workload qp-group: FISTA over the uneven batch in one persistent
    launch per solve (l1_setup_group).  The dictionaries (71e9 entries, 142.5 GB
    in BF16) are drawn on the device by torch from per-instance seeds and
    streamed into the handle with l1_group_load; the timed region is the solve
    alone, with every dictionary resident in HBM."""
    import torch

    import paper_1007_3753_gb300 as l1
    from paper_1007_3753_gb300 import build

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    build.build()
    l1.load()
    count = args.count or GROUP["count"]
    ms, ns = synthetic.qp_group_sizes(count, seed=GROUP["seed"] + 100000 * rank)
    stream = torch.cuda.current_stream()
    t0 = time.time()
    g = l1.Group(None, ms, ns, GROUP["lam"], precision=l1.A_BF16, stream=stream.cuda_stream)
    b = torch.empty(int(g.boff[-1]), dtype=torch.float32, device="cuda")
    gen = torch.Generator(device="cuda")
    first, chunk, chunk_bytes = 0, [], 0
    for i in range(count):
        m, n = int(ms[i]), int(ns[i])
        gen.manual_seed(GROUP["seed"] + 1 + i + 100000 * rank)
        At = torch.randn((n, m), device="cuda", generator=gen)  # row j = column j of A
        At /= At.norm(dim=1, keepdim=True)
        k = max(1, m // 10)
        x0 = torch.zeros(n, device="cuda")
        x0[torch.randperm(n, device="cuda", generator=gen)[:k]] = torch.randn(k, device="cuda", generator=gen)
        b[int(g.boff[i]):int(g.boff[i + 1])] = At.t() @ x0 + 0.01 * torch.randn(m, device="cuda", generator=gen)
        chunk.append(At.t())  # column-major m x n view
        chunk_bytes += 4 * m * n
        if chunk_bytes >= (4 << 30) or i == count - 1:
            g.load(first, chunk)
            torch.cuda.synchronize()
            first, chunk, chunk_bytes = i + 1, [], 0
    setup_s = time.time() - t0
    tol, max_iter = GROUP["tol"], (args.max_iter or GROUP["max_iter"])
    for _ in range(args.warmup):
        g.solve(b, tol, max_iter)
    torch.cuda.synchronize()
    info0 = g.info()
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
    step_ms, conv, a_bytes = [], 0, 0.0
    mn = ms.astype(np.float64) * ns.astype(np.float64)
    for _ in range(args.steps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        _, res = g.solve(b, tol, max_iter)
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        conv += int(np.sum(res["status"] == l1.CONVERGED))
        # every FISTA step of instance i reads its BF16 dictionary once
        a_bytes += float(np.sum(res["iters"] * mn)) * 2.0
    clocks = sampler.stop() if sampler else None
    info1 = g.info()
    total_ms = sum(step_ms)
    peaks = measured_peaks()
    achieved = a_bytes / (total_ms / 1e3) / 1e9
    line = {"metric": "QP_lambda solves/sec (uneven batch, FISTA to the relative-change rule)",
            "value": conv / (total_ms / 1e3), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16 A, f32 arithmetic", "data": "synthetic",
            "config": {"workload": f"qp_group_{count}_bf16", "instances": count, "lambda": GROUP["lam"],
                       "tol": tol, "max_iter": max_iter, "sum_mn": float(mn.sum()),
                       "a_bytes_bf16": float(mn.sum()) * 2.0, "setup_s": setup_s,
                       "mean_iters": float(np.mean(res["iters"])), "max_iters": int(np.max(res["iters"])),
                       "l2": "A (GBs) far larger than L2; every step streams it from HBM"},
            "gpu_launches": int(info1["gpu_launches"] - info0["gpu_launches"]),
            "roofline": {"bound": "hbm", "kernel": "group_kernel (persistent cooperative FISTA)",
                         "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                         "peak_note": "of measured hbm_gbs; achieved counts sum_i iters_i m_i n_i x 2 B (BF16 A)"},
            "clocks": clocks}
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.close()
    return 0


# unrolled PALM and its adjoint (reading R11): A 1024 x 2048 Gaussian with unit
# columns, N = 256 targets with 50 nonzeros, K = 200 inner steps, a
# multiplier step every J = 10, checkpoints every 20 steps
UNROLL = dict(m=1024, n=2048, N=256, k=50, K=200, J=10, ckpt=20, seed=5000)


def bench_unrolled(args, rank, world):
    """--workload unrolled: one step = the unrolled forward (l1_solve_batch)
    plus the adjoint (l1_backward with grad_x = x - x_target), device-resident."""
    import torch

    import paper_1007_3753_gb300 as l1
    from paper_1007_3753_gb300 import build

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    build.build()
    l1.load()
    u = UNROLL
    p = synthetic.unrolled_instance(u["m"], u["n"], u["N"], k=u["k"], seed=u["seed"] + rank)
    m, n, N, K, J = u["m"], u["n"], u["N"], u["K"], u["J"]
    stream = torch.cuda.current_stream()

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32).T)).cuda().t()
    A_d, B_d, Xt_d = dev(p["A"]), dev(p["B"]), dev(p["X_target"])
    s = l1.Solver(A_d, mode=l1.P1, solver=l1.PALM, unroll_K=K, unroll_J=J, ckpt_every=u["ckpt"],
                  stream=stream.cuda_stream)
    x_d = torch.empty((N, n), dtype=torch.float32, device="cuda").t()
    gb = torch.empty((N, m), dtype=torch.float32, device="cuda").t()
    gA = torch.empty((n, m), dtype=torch.float32, device="cuda").t()

    def step():
        s.solve(B_d, 0.0, 1, x=x_d)
        gx = (x_d - Xt_d).t().contiguous().t()
        s.backward(gx, grad_b=gb, grad_A=gA)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    info0 = s.info()
    step_ms = []
    for _ in range(args.steps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        step()
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
    info1 = s.info()
    total_ms = sum(step_ms)
    # executed FP32 flops per step: every sweep is 2 m n N; forward K steps x 2
    # sweeps + (K/J - 1) multiplier sweeps + 1 residual sweep; backward the
    # recomputation (forward again, less the residual sweep), K x 2 reverse
    # sweeps, K/J - 1 multiplier adjoints, and grad_A as 2 m n N per step x 2
    # plus 2 m n N per multiplier adjoint
    sweep = 2.0 * m * n * N
    n_outer = -(-K // J)
    fwd = (2 * K + (n_outer - 1) + 1) * sweep
    bwd = (2 * K + (n_outer - 1)) * sweep + 2 * K * sweep + (n_outer - 1) * sweep + (2 * K + (n_outer - 1)) * sweep
    flop = fwd + bwd
    achieved = flop / (total_ms / args.steps / 1e3) / 1e12
    line = {"metric": "unrolled PALM forward + adjoint samples/sec", "value": N * args.steps / (total_ms / 1e3),
            "unit": "samples/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"unrolled_palm_m{m}_n{n}_N{N}_K{K}", "J": J, "ckpt_every": u["ckpt"],
                       "device_bytes": info1["device_bytes"], "flop_per_step": flop},
            "gpu_launches": int(info1["gpu_launches"] - info0["gpu_launches"]),
            "roofline": {"bound": "alu", "kernel": "whole step (CUDA-core sweeps and rank_update_kernel)",
                         "achieved": achieved, "peak": FP32_SIMT_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP32_SIMT_PEAK_TFLOPS, "traffic": None,
                         "peak_note": "FP32 FMA: 152 SMs x 128 lanes x 2 FLOP x 2070 MHz (derived)"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()
    return 0


# basis pursuit (Eq. 1) of §VI-A: A 200 x 400 Gaussian with unit columns,
# x0 20-sparse with +-1 entries, b = A x0, tol 1e-6; 20 seeded instances
P1 = dict(m=200, n=400, k=20, count=20, tol=1e-6, max_iter=5000)


def bench_p1(args, rank, world):
    """--workload p1: the 20 instances as one batch of right-hand sides
    sharing A (one dictionary, as the batched API requires): instance j is
    x0_j on the seed-0 dictionary; DALM and PALM; exact recovery checked.
    P1,2 runs on the same x0 with noise added to b."""
    import torch

    import paper_1007_3753_gb300 as l1
    from paper_1007_3753_gb300 import build

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    build.build()
    l1.load()
    u = P1
    base = synthetic.p1_instance(u["m"], u["n"], u["k"], seed=0)
    A = base["A"]
    X0 = np.stack([synthetic.p1_instance(u["m"], u["n"], u["k"], seed=s0)["x0"] for s0 in range(u["count"])], 1)
    B = np.asfortranarray(A @ X0).astype(np.float32)
    stream = torch.cuda.current_stream()
    B_d = torch.from_numpy(np.ascontiguousarray(B.T)).cuda().t()
    out = {}
    for name, solver in (("DALM", l1.DALM), ("PALM", l1.PALM)):
        s = l1.Solver(A, mode=l1.P1, solver=solver, stream=stream.cuda_stream)
        for _ in range(args.warmup):
            s.solve(B_d, u["tol"], u["max_iter"])
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        conv = 0
        for _ in range(args.steps):
            x, _, res = s.solve(B_d, u["tol"], u["max_iter"])
            conv += int(np.sum(res["status"] == l1.CONVERGED))
        ev1.record(stream)
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1)
        xh = x.cpu().numpy()
        err = max(np.linalg.norm(xh[:, j] - X0[:, j]) / np.linalg.norm(X0[:, j]) for j in range(u["count"]))
        out[name] = {"solves_per_s": conv / (ms / 1e3), "ms_per_batch": ms / args.steps,
                     "mean_iters": float(np.mean(res["iters"])), "max_rel_err_vs_x0": float(err)}
        s.close()
    # P1,2 (Eq. 2, PALM with the eps-ball e-step): the same x0 with Gaussian
    # noise of standard deviation 0.01 added to b, eps = 1.1 x 0.01 sqrt(m)
    g = np.random.default_rng(7)
    sigma = 0.01
    eps = 1.1 * sigma * np.sqrt(u["m"])
    Bn = np.asfortranarray(A @ X0 + sigma * g.standard_normal((u["m"], u["count"]))).astype(np.float32)
    Bn_d = torch.from_numpy(np.ascontiguousarray(Bn.T)).cuda().t()
    s = l1.Solver(A, mode=l1.P1_2, solver=l1.PALM, epsilon=eps, stream=stream.cuda_stream)
    for _ in range(args.warmup):
        s.solve(Bn_d, u["tol"], u["max_iter"])
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    conv = 0
    for _ in range(args.steps):
        x, _, res = s.solve(Bn_d, u["tol"], u["max_iter"])
        conv += int(np.sum(res["status"] == l1.CONVERGED))
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    xh = x.cpu().numpy()
    err = max(np.linalg.norm(xh[:, j] - X0[:, j]) / np.linalg.norm(X0[:, j]) for j in range(u["count"]))
    out["PALM_P1_2"] = {"solves_per_s": conv / (ms / 1e3), "ms_per_batch": ms / args.steps,
                        "mean_iters": float(np.mean(res["iters"])), "max_rel_err_vs_x0": float(err),
                        "epsilon": float(eps), "max_resid_over_eps": float(np.max(res["resid"]) / eps)}
    s.close()
    line = {"metric": "P1 solves/sec (exact recovery, 20 instances per batch)",
            "value": out["DALM"]["solves_per_s"], "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "p1_m200_n400_k20_batch20", "tol": u["tol"], "solvers": out}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--tol", type=float, default=None)
    ap.add_argument("--max-iter", type=int, default=None)
    ap.add_argument("--engine", choices=["tc", "simt"], default="simt")
    ap.add_argument("--workload", choices=["cab", "qp-group", "unrolled", "p1"], default="cab")
    ap.add_argument("--count", type=int, default=None, help="qp-group: number of instances")
    ap.add_argument("--m", type=int, default=None, help="cab: rows of A")
    ap.add_argument("--classes", type=int, default=None, help="cab: classes")
    ap.add_argument("--per-class", type=int, default=None, help="cab: columns per class")
    ap.add_argument("--N", type=int, default=None, help="cab: right-hand sides")
    ap.add_argument("--precision", choices=["fp32", "bf16", "fp8"], default="fp32",
                    help="cab: stored precision of A (bf16 / fp8 add the FP32 refinement phase)")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="cab: skip the CPU oracle leg")
    args = ap.parse_args()
    for key, val in (("m", args.m), ("classes", args.classes), ("per_class", args.per_class), ("N", args.N)):
        if val is not None:
            BENCH[key] = val
    if args.tol is not None:
        BENCH["tol"] = args.tol
    if args.max_iter is not None:
        BENCH["max_iter"] = args.max_iter
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return bench_reference(args, rank, world)
    if args.workload == "qp-group":
        return bench_group(args, rank, world)
    if args.workload == "unrolled":
        return bench_unrolled(args, rank, world)
    if args.workload == "p1":
        return bench_p1(args, rank, world)
    return bench_ours(args, rank, world)


if __name__ == "__main__":
    sys.exit(main())
