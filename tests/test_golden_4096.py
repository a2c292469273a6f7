"""The stored FP64-oracle answers for the 4096 x 4000 (+ identity)
cross-and-bouquet workload: this machine's generator reproduces the inputs
they were made for, each stored stop satisfies the relative-change rule of
§VI-C (the step into it is below tol), and each stored label is the class
the test vector was drawn from."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_stored_answers_match_generator_and_stopping_rule():
    import bench
    p = bench.cab_workload(bench.CAB4096)
    g = bench.golden_oracle(p)  # raises if the inputs differ
    gz = np.load(bench.GOLDEN4096)
    tol = float(gz["tol"])
    assert len(g) == 8
    for j, e in g.items():
        ko = e["stop"]
        assert 1 < ko < int(gz["max_iter"])
        w, wb = e["at"][ko], e["at"][ko - 1]
        # stored w is FP32 and the neighbours FP16 differences: rounding of
        # about 1e-7 relative, far below tol
        assert np.linalg.norm(w - wb) / np.linalg.norm(wb) < tol * 1.01
        assert 0 <= e["label"] < bench.CAB4096["classes"]
        assert e["label"] == p["labels"][j]
