"""bench.py --impl reference (the FP64 oracle on the host cores, no GPU):
one JSON line with the fields the benchmark contract asks for."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
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
    assert d["config"]["workload"].startswith("cab_dalm_")


def test_oracle_agreement_reports_errors_and_labels():
    """The comparison bench.py makes between the sampled GPU columns and the
    oracle: zero error for the oracle's own answers (cast to FP32), and a
    planted perturbation of one column is reported against the 1e-4 bar."""
    import numpy as np

    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import synthetic
    p = synthetic.cab_problem(48, 3, 4, 4, corrupt=0.2, seed=77)
    cols = [0, 1, 2]
    conv, dt, outs = bench.run_cpu_oracle(p, cols, 3, 1e-6, 20000)
    assert conv == 3
    A, B, off = p["A"], p["B"], p["offsets"]
    n = A.shape[1]
    x = np.stack([w for w, _, _ in outs], 1).astype(np.float32)
    obj = np.array([np.abs(w).sum() for w, _, _ in outs])
    lab = np.array([oracle.classify(A, off, B[:, j], w[:n], w[n:])[0] for j, (w, _, _) in zip(cols, outs)])
    d = bench.oracle_agreement(p, cols, x, obj, lab, outs)
    assert d["max_rel_err_x"] <= 1e-6 and d["max_rel_err_obj"] <= 1e-12
    assert d["within_bar"] == 3 and d["labels_equal"] == 3 and d["of"] == 3
    x[:, 1] *= 1.001
    d = bench.oracle_agreement(p, cols, x, obj, lab, outs)
    assert 9e-4 <= d["max_rel_err_x"] <= 1.1e-3 and d["within_bar"] == 2
