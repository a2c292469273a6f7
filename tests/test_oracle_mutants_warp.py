"""Planted mistakes in the numpy part of the oracle (the image side of the
alignment loop, reading R19), on the CPU.

Each mutant is one plausible slip in ``oracle.warp_jacobian`` or
``oracle.align_images`` -- a wrong sign, swapped coordinates, a dropped
clamp or term, a wrong update.  The mutated function is compiled from the
edited source and put in place of the original for the duration of the
check; at least one of the pins of ``tests/test_oracle_pins.py`` on the
alignment loop must then fail.  The unmodified source, handled the same way,
must pass them all (the control).
"""
import inspect
import textwrap

import numpy as np
import pytest

import oracle
import test_oracle_pins as pins

PIN_TESTS = (pins.test_warp_is_exact_on_pixel_grids_and_affine_images,
             pins.test_warp_jacobian_matches_finite_differences,
             pins.test_alignment_loop_recovers_the_transformation)

# (id, function, text in its source, mistaken text)
MUTANTS = [
    ("x_sign_of_b", "warp_jacobian", "x = a * u - bb * v + tx", "x = a * u + bb * v + tx"),
    ("y_swapped_uv", "warp_jacobian", "y = bb * u + a * v + ty", "y = bb * v + a * u + ty"),
    ("no_clamp", "warp_jacobian", "xc = np.clip(x, 0.0, W - 1.0)", "xc = x"),
    ("cell_weights_swapped", "warp_jacobian",
     "val = (1.0 - fy) * ((1.0 - fx) * p00 + fx * p01) + fy * ((1.0 - fx) * p10 + fx * p11)",
     "val = (1.0 - fx) * ((1.0 - fy) * p00 + fy * p01) + fx * ((1.0 - fy) * p10 + fy * p11)"),
    ("slope_x_wrong_row", "warp_jacobian",
     "(1.0 - fy) * (p01 - p00) + fy * (p11 - p10)", "(1.0 - fy) * (p10 - p00) + fy * (p11 - p01)"),
    ("jacobian_b_sign", "warp_jacobian", "-gx * v + gy * u", "gx * v + gy * u"),
    ("jacobian_a_missing_v", "warp_jacobian", "gx * u + gy * v", "gx * u"),
    ("clamped_slope_kept", "warp_jacobian",
     "gx = np.where((x >= 0.0) & (x <= W - 1.0), (1.0 - fy) * (p01 - p00) + fy * (p11 - p10), 0.0)",
     "gx = (1.0 - fy) * (p01 - p00) + fy * (p11 - p10)"),
    ("update_sign", "align_images", "tau = tau + dtau", "tau = tau - dtau"),
    ("jacobian_not_negated", "align_images", "np.hstack([A, -J])", "np.hstack([A, J])"),
]


def _swap(name, src):
    ns = dict(vars(oracle))
    exec(compile(textwrap.dedent(src), f"<mutant {name}>", "exec"), ns)
    return ns[name]


def _run_pins():
    failed = []
    for t in PIN_TESTS:
        try:
            t()
        except AssertionError:
            failed.append(t.__name__)
        except (ValueError, FloatingPointError, IndexError, np.linalg.LinAlgError, RuntimeError):
            failed.append(t.__name__)
    return failed


def test_control_passes_every_alignment_pin(monkeypatch):
    for name in ("warp_jacobian", "align_images"):
        monkeypatch.setattr(oracle, name, _swap(name, inspect.getsource(getattr(oracle, name))))
    assert _run_pins() == []


@pytest.mark.parametrize("mid", [m[0] for m in MUTANTS])
def test_mutant_fails_an_alignment_pin(monkeypatch, mid):
    _, name, old, new = next(m for m in MUTANTS if m[0] == mid)
    src = inspect.getsource(getattr(oracle, name))
    assert src.count(old) == 1, f"{mid}: the text to mutate must occur exactly once"
    # the oracle's own align_images looks warp_jacobian up in the module, so
    # replacing the module attribute reaches it too
    monkeypatch.setattr(oracle, name, _swap(name, src.replace(old, new)))
    failed = _run_pins()
    assert failed, f"{mid}: every alignment pin passed on the planted mistake"
    print(f"{mid}: caught by {failed[0]}")
