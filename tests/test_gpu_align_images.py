"""The image side of the face-alignment loop (§II-B, reading R19) on the GPU
(l1_align_warp, l1_align_images) against the oracle (oracle.warp_jacobian,
oracle.align_images) on the same FP32-rounded synthetic faces.

  * the warp and its Jacobian, element by element, at transformations that
    put the sample points off the pixel grid, and where every point is
    clamped (J = 0);
  * the whole loop from 4 pixels of translation and 15 degrees of rotation:
    the same tasks succeed, the final transformations agree to a tenth of a
    pixel and the step counts to three (one task in sixteen may differ);
  * a task whose convex step is singular stops with L1_NONFINITE.
"""
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


def _r32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _task_tensors(d):
    img = torch.from_numpy(np.ascontiguousarray(d["img"], dtype=np.float32)).cuda()
    # task k's training image j at A[k, j] (m values, pixel (u, v) at v cols + u)
    A = torch.from_numpy(np.ascontiguousarray(np.transpose(d["A"], (0, 2, 1)), dtype=np.float32)).cuda()
    return img, A


def test_warp_and_jacobian_match_the_oracle(l1):
    d = synthetic.alignment_images(12, "rotation", seed=7200)
    rows, cols = d["rows"], d["cols"]
    g = np.random.default_rng(1)
    tau = d["tau_init"] + g.normal(0.0, [0.02, 0.02, 1.5, 1.5], (12, 4))
    tau[11] = [1.0, 0.0, -500.0, -500.0]  # every point clamped to the corner
    img, _ = _task_tensors(d)
    b, J = l1.align_warp(img, torch.from_numpy(tau).cuda(), rows, cols)
    b, J = b.cpu().numpy(), J.cpu().numpy()
    worst_b = worst_j = 0.0
    for k in range(12):
        bo, Jo = oracle.warp_jacobian(_r32(d["img"][k]), tau[k], rows, cols)
        worst_b = max(worst_b, np.max(np.abs(b[k] - bo)) / np.max(np.abs(bo)))
        worst_j = max(worst_j, np.max(np.abs(J[k].T - Jo)) / max(np.max(np.abs(Jo)), 1e-30))
        if k == 11:
            assert np.all(J[k] == 0.0) and np.all(Jo == 0.0)
    print(f"warp: b rel. err {worst_b:.2e}, J rel. err {worst_j:.2e}")
    assert worst_b <= 1e-6 and worst_j <= 1e-6


@pytest.mark.parametrize("kind", ["translation", "rotation"])
def test_alignment_loop_matches_the_oracle(l1, kind):
    d = synthetic.alignment_images(16, kind, seed=7100)
    rows, cols = d["rows"], d["cols"]
    img, A = _task_tensors(d)
    tau = torch.from_numpy(d["tau_init"].copy()).cuda()
    res = l1.align_images(img, A, tau, rows, cols)
    tg = tau.cpu().numpy()
    ok_gpu = ok_orc = 0
    off = []
    for k in range(16):
        to, steps, conv = oracle.align_images(_r32(d["A"][k]), _r32(d["img"][k]), d["tau_init"][k], rows, cols)
        e_orc = oracle.corner_shift(to - d["tau_true"][k], rows, cols)
        e_gpu = oracle.corner_shift(tg[k] - d["tau_true"][k], rows, cols)
        ok_orc += e_orc < 1.0
        ok_gpu += e_gpu < 1.0
        if e_orc < 1.0:
            diff = oracle.corner_shift(tg[k] - to, rows, cols)
            if not (diff <= 0.1 and res["status"][k] == l1.CONVERGED and abs(int(res["iters"][k]) - steps) <= 3):
                off.append((k, diff, int(res["status"][k]), int(res["iters"][k]), steps))
    print(f"{kind}: success GPU {ok_gpu}/16, oracle {ok_orc}/16, mean steps {res['iters'].mean():.2f}, "
          f"tasks off the oracle's path {off}")
    # the convex steps are FP32 on the GPU and FP64 in the oracle, both to the
    # relative change 1e-3: one task in sixteen may take a different path
    assert len(off) <= 1
    assert ok_gpu >= ok_orc - 1 and ok_gpu >= 12


def test_singular_step_stops_the_task(l1):
    """Task 1 has no training images (A = 0) on a constant query: B = [0, -J]
    with J = 0 is singular, the convex step reports it and the task stops
    with L1_NONFINITE after one step; task 0 aligns as usual."""
    d = synthetic.alignment_images(2, "translation", seed=7300)
    d["A"][1] = 0.0
    d["img"][1] = 0.5
    img, A = _task_tensors(d)
    tau = torch.from_numpy(d["tau_init"].copy()).cuda()
    res = l1.align_images(img, A, tau, d["rows"], d["cols"])
    assert res["status"][1] == l1.NONFINITE and res["iters"][1] == 1
    assert np.all(np.isfinite(tau.cpu().numpy()))
    assert res["status"][0] != l1.NONFINITE
