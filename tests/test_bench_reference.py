"""bench.py --impl reference (the FP64 oracle on the host cores, no GPU):
one JSON line with the fields the benchmark contract asks for; and the
host logic that decides which sampled GPU columns count as verified."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "cab1024", "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=900,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "e2e", "cpu_baseline"):
        assert key in d, key
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["config"]["workload"] == "cab_dalm_m1024_n1200_N1024"


def test_verify_columns_counts_only_columns_within_the_bar():
    """The comparison bench.py makes between sampled GPU columns and the
    oracle: the oracle's own iterates (cast to FP32) verify; a planted 1e-3
    perturbation, a stop two iterations away from the oracle's, or a wrong
    label do not."""
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import synthetic
    p = synthetic.cab_problem(48, 3, 4, 4, corrupt=0.2, seed=77)
    A, B, off = p["A"], p["B"], p["offsets"]
    n = A.shape[1]
    cols = [0, 1, 2, 3]
    tol = 1e-6
    outs = [oracle.dalm(A, B[:, j], cab=True, tol=tol, max_iter=20000) for j in cols]
    stops = {j: st["iters"] for j, (_, _, st) in zip(cols, outs)}
    ws = {j: w for j, (w, _, _) in zip(cols, outs)}

    def at(j, k):
        return ws[j] if k == stops[j] else oracle.dalm(A, B[:, j], cab=True, tol=0.0, max_iter=k)[0]

    labels = {j: oracle.classify(A, off, B[:, j], ws[j][:n], ws[j][n:])[0] for j in cols}
    x = np.stack([ws[j] for j in cols], 1).astype(np.float32)
    obj = np.array([np.abs(ws[j]).sum() for j in cols])
    its = np.array([stops[j] for j in cols])
    lab = np.array([labels[j] for j in cols])
    d = bench.verify_columns(cols, x, its, obj, lab, lambda j: stops[j], at, lambda j: labels[j])
    assert d["within_bar"] == 4 and d["labels_equal"] == 4 and d["max_rel_err_x"] <= 1e-6
    # one iteration later is still an answer of the rule, compared with the
    # oracle's iterate there
    its1 = its.copy()
    its1[0] += 1
    x1 = x.copy()
    x1[:, 0] = at(0, stops[0] + 1)
    obj1 = obj.copy()
    obj1[0] = np.abs(at(0, stops[0] + 1)).sum()
    assert bench.verify_columns(cols, x1, its1, obj1, lab, lambda j: stops[j], at,
                                lambda j: labels[j])["within_bar"] == 4
    x2 = x.copy()
    x2[:, 1] *= 1.001
    its2 = its.copy()
    its2[2] += 2
    lab2 = lab.copy()
    lab2[3] = (lab2[3] + 1) % 3
    d = bench.verify_columns(cols, x2, its2, obj, lab2, lambda j: stops[j], at, lambda j: labels[j])
    assert d["within_bar"] == 1 and not d["per_instance"][1]["verified"]
    assert d["per_instance"][2]["rel_err_x"] is None and d["labels_equal"] == 3


def test_reference_arm_of_the_other_workloads_says_unavailable():
    """The oracle arm is timed on the cross-and-bouquet workloads; on the
    others --impl reference prints its one-line reason and exits 0."""
    for w in ("qp-group", "unrolled", "p1", "align", "amp", "align-images"):
        out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", w,
                              "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=300, cwd=ROOT)
        assert out.returncode == 0, out.stderr[-2000:]
        d = json.loads([ln for ln in out.stdout.splitlines() if ln.startswith("{")][-1])
        assert d["impl"] == "reference" and w in d["unavailable"]
