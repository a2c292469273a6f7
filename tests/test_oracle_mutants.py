"""Planted mistakes in the oracle, on the CPU.

Each mutant below is one plausible slip in ``oracle/l1_oracle.c`` -- a
dropped term, a wrong sign, a wrong index or bound, a transposed operand --
and at least one pin of ``tests/test_oracle_pins.py`` must fail on it.  The
mutated source is compiled into a temporary library and loaded by a child
pytest through ``L1_ORACLE_LIB`` (the pins not marked slow).  The
unmodified source, built and loaded the same way, must pass every one of
them (the control), so a broken harness cannot pass for a caught mutant.

Mistakes that change only the path of an iteration and not its limit are
caught, where the iteration is FISTA, by the O(1/k^2) rate of §IV-A and the
potential function of its proof.  Path-only readings outside FISTA (which
norm the relative change divides by, which inner iterate becomes x_{k+1})
are seen by no pin; the GPU trajectory comparisons hold the CUDA path to the
same readings.
"""
import concurrent.futures as cf
import os
import re
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "l1_oracle.c")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# (id, the passage the mistaken line restates, text in the source, mistaken text)
MUTANTS = [
    # helpers
    ("soft_sign", "R9 soft threshold",
     "if (v < -a) return v + a;", "if (v < -a) return v - a;"),
    ("soft_no_shrink", "R9 soft threshold",
     "if (v > a) return v - a;", "if (v > a) return v;"),
    ("clamp_half_box", "Eq. 38 projection onto [-1, 1]",
     "(v < -1.0 ? -1.0 : v)", "(v < 0.0 ? 0.0 : v)"),
    ("matvec_transposed", "A x",
     "for (int i = 0; i < m; ++i) y[i] += col[i] * xj;",
     "for (int i = 0; i < m; ++i) y[i] += A[j + (size_t)i * n] * xj;"),
    ("tvec_wrong_stride", "A^T y",
     "x[j] = dot(A + (size_t)j * m, y, m);", "x[j] = dot(A + (size_t)j, y, m);"),
    ("lipschitz_norm_not_squared", "R4 L = ||A||_2^2",
     "const double rho_new = dot(u, u, m);", "const double rho_new = nrm2(u, m);"),
    # FISTA, Eq. 18
    ("fista_gradient_sign", "Eq. 18 gradient step",
     "x[j] = soft(y[j] + g[j] / L, lambda / L);", "x[j] = soft(y[j] - g[j] / L, lambda / L);"),
    ("fista_threshold_unscaled", "Eq. 18 threshold lambda/L",
     "x[j] = soft(y[j] + g[j] / L, lambda / L);", "x[j] = soft(y[j] + g[j] / L, lambda);"),
    ("fista_no_momentum", "Eq. 18 momentum (t_k - 1)/t_{k+1}",
     "    const double mu = (t - 1.0) / t_new;\n    double d2",
     "    const double mu = 0.0;\n    double d2"),
    ("fista_momentum_index", "Eq. 18 momentum (t_k - 1)/t_{k+1}",
     "    const double mu = (t - 1.0) / t_new;\n    double d2",
     "    const double mu = t / t_new;\n    double d2"),
    ("fista_extrapolate_from_old", "Eq. 18 y_{k+1} = x_k + mu (x_k - x_{k-1})",
     "y[j] = x[j] + mu * dj;", "y[j] = xp[j] + mu * dj;"),
    ("fista_t_update", "Eq. 18 t_{k+1}",
     "    const double t_new = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));\n    const double mu = (t - 1.0) / t_new;\n    double d2",
     "    const double t_new = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t));\n    const double mu = (t - 1.0) / t_new;\n    double d2"),
    # FISTA with continuation, reading R17
    ("fista_cont_below_target", "R17 lambda_{k+1} = max(rho lambda_k, lambda)",
     "lam = rho * lam > lambda ? rho * lam : lambda;", "lam = rho * lam;"),
    ("fista_cont_stops_early", "R17 the rule applies once lambda_k = lambda",
     "if (lam <= lambda && rel < tol) { conv = 1; break; }", "if (rel < 1e3 * tol) { conv = 1; break; }"),
    # AMP, §IV / reading R18
    ("amp_no_onsager", "§IV z-step: the term (eta/delta) z_k",
     "z[i] = b[i] - r[i] + (eta / delta) * z[i];", "z[i] = b[i] - r[i];"),
    ("amp_delta_inverted", "§IV delta = m/n",
     "const double delta = (double)m / (double)n;", "const double delta = (double)n / (double)m;"),
    ("amp_tau_without_delta", "§IV tau_{k+1} = (tau_k / delta) eta_k",
     "tau = tau / delta * eta;", "tau = tau * eta;"),
    ("amp_v_sign", "§IV x-step soft(A^T z + x, tau)",
     "for (int j = 0; j < n; ++j) v[j] += x[j];", "for (int j = 0; j < n; ++j) v[j] -= x[j];"),
    ("amp_derivative_everywhere", "R18 average derivative of soft(., tau)",
     "if (fabs(v[j]) > tau) ++above;", "++above;"),
    # PALM, Algorithm 1 / Eq. 33 / reading R10
    ("palm_e_multiplier_sign", "Algorithm 1 e-step",
     "e_new[i] = soft(b[i] - Ax[i] + theta[i] / xi, 1.0 / xi);",
     "e_new[i] = soft(b[i] - Ax[i] - theta[i] / xi, 1.0 / xi);"),
    ("palm_e_threshold", "Algorithm 1 e-step threshold 1/xi",
     "e_new[i] = soft(b[i] - Ax[i] + theta[i] / xi, 1.0 / xi);",
     "e_new[i] = soft(b[i] - Ax[i] + theta[i] / xi, xi);"),
    ("p12_unit_ball", "R10 projection onto the eps-ball",
     "const double s = (vn > o->epsilon) ? o->epsilon / vn : 1.0;",
     "const double s = (vn > o->epsilon) ? 1.0 / vn : 1.0;"),
    ("p12_no_multiplier", "R10 projection of b - A x + theta/xi",
     "for (int i = 0; i < m; ++i) e_new[i] = b[i] - Ax[i] + theta[i] / xi;",
     "for (int i = 0; i < m; ++i) e_new[i] = b[i] - Ax[i];"),
    ("palm_c_e_sign", "Algorithm 1 inner target b - e + theta/xi",
     "c[i] = b[i] - e_new[i] + theta[i] / xi;", "c[i] = b[i] + e_new[i] + theta[i] / xi;"),
    ("palm_c_no_multiplier", "Algorithm 1 inner target b - e + theta/xi",
     "c[i] = b[i] - e_new[i] + theta[i] / xi;", "c[i] = b[i] - e_new[i];"),
    ("palm_inner_threshold", "Algorithm 1 inner threshold 1/(xi L)",
     "soft(z[j] + g[j] / L, 1.0 / (xi * L))", "soft(z[j] + g[j] / L, 1.0 / L)"),
    ("palm_inner_no_momentum", "Algorithm 1 inner FISTA momentum",
     "            const double mu = (t - 1.0) / t_new;\n            double d2 = 0.0;\n            for (int j = 0; j < n; ++j) {\n                const double dj = w_new[j] - w[j];",
     "            const double mu = 0.0;\n            double d2 = 0.0;\n            for (int j = 0; j < n; ++j) {\n                const double dj = w_new[j] - w[j];"),
    ("palm_inner_momentum_index", "Algorithm 1 inner FISTA momentum",
     "            const double mu = (t - 1.0) / t_new;\n            double d2 = 0.0;",
     "            const double mu = t / t_new;\n            double d2 = 0.0;"),
    ("palm_theta_sign", "Algorithm 1 multiplier update",
     "theta[i] += xi * (b[i] - Ax[i] - e_new[i]);", "theta[i] -= xi * (b[i] - Ax[i] - e_new[i]);"),
    ("palm_theta_no_e", "Algorithm 1 multiplier update",
     "theta[i] += xi * (b[i] - Ax[i] - e_new[i]);", "theta[i] += xi * (b[i] - Ax[i]);"),
    ("palm_xi0_inverted", "§V-A xi = 2m/||b||_1",
     "double xi0 = o->xi0 > 0.0 ? o->xi0 : (b1 > 0.0 ? 2.0 * m / b1 : 1.0);",
     "double xi0 = o->xi0 > 0.0 ? o->xi0 : (b1 > 0.0 ? 2.0 * b1 / m : 1.0);"),
    # DALM, Algorithm 2 / Eqs. 38-39 / reading R1
    ("dalm_z_sign", "Eq. 38 z-update",
     "z[j] = clamp1(bty[j] + w[j] / beta);", "z[j] = clamp1(bty[j] - w[j] / beta);"),
    ("dalm_rhs_sign", "Eq. 39 right-hand side",
     "v[j] = z[j] - w[j] / beta;", "v[j] = z[j] + w[j] / beta;"),
    ("dalm_rhs_b_unscaled", "Eq. 39 right-hand side",
     "rhs[i] += b[i] / beta;", "rhs[i] += b[i];"),
    ("dalm_w_sign", "Algorithm 2 w-update",
     "const double dj = -beta * (z[j] - bty[j]);", "const double dj = beta * (z[j] - bty[j]);"),
    ("dalm_gram_no_identity", "R1 B B^T = A A^T + I",
     "if (cab) g[k] += 1.0;", "if (cab) g[k] += 0.0;"),
    ("cholesky_wrong_index", "Cholesky factor",
     "for (int i = j; i < m; ++i) gj[i] -= rk[i] * rjk;",
     "for (int i = j; i < m; ++i) gj[i] -= rk[i] * rk[i];"),
    ("cholesky_solve_transposed", "back substitution with R^T",
     "s -= R[k + (size_t)i * m] * y[k];", "s -= R[i + (size_t)k * m] * y[k];"),
    ("cg_step_length_inverted", "CG y-step of §V-B: alpha = r^T r / p^T B B^T p",
     "const double alpha = rr / pq;", "const double alpha = pq / rr;"),
    ("cg_residual_sign", "CG y-step of §V-B: residual update",
     "r[i] -= alpha * q[i]; }", "r[i] += alpha * q[i]; }"),
    ("cg_no_conjugation", "CG y-step of §V-B: conjugate direction",
     "for (int i = 0; i < m; ++i) p[i] = r[i] + gamma * p[i];",
     "for (int i = 0; i < m; ++i) p[i] = r[i];"),
    ("cab_operator_sign", "R1 B = [A I]",
     "if (cab) for (int i = 0; i < m; ++i) out[i] += v[n + i];",
     "if (cab) for (int i = 0; i < m; ++i) out[i] -= v[n + i];"),
    ("cab_adjoint_dropped", "R1 B^T = [A^T; I]",
     "if (cab) for (int i = 0; i < m; ++i) out[n + i] = y[i];",
     "if (cab) for (int i = 0; i < m; ++i) out[n + i] = 0.0;"),
    # the alignment step of §II-B, reading R16
    # (a wrong e threshold alone only rescales ||e||_1, the one term of this
    # objective, so it leaves the minimiser unchanged: not a mistake a limit
    # can show)
    ("align_e_multiplier_sign", "R16 e-step",
     "e_next[i] = soft(b[i] - Bw[i] + theta[i] / xi, 1.0 / xi);",
     "e_next[i] = soft(b[i] - Bw[i] - theta[i] / xi, 1.0 / xi);"),
    ("align_rhs_e_sign", "R16 least-squares target b - e + theta/xi",
     "t[i] = b[i] - e_next[i] + theta[i] / xi;", "t[i] = b[i] + e_next[i] + theta[i] / xi;"),
    ("align_theta_no_e", "R16 multiplier update",
     "theta[i] += xi * (b[i] - Bw[i] - e_next[i]);", "theta[i] += xi * (b[i] - Bw[i]);"),
    ("align_gram_diagonal", "R16 B^T B",
     "G[i + (size_t)k * p] = dot(B + (size_t)i * m, B + (size_t)k * m, m);",
     "G[i + (size_t)k * p] = dot(B + (size_t)i * m, B + (size_t)i * m, m);"),
    # classification, §II-A and Eq. 40
    ("classify_keeps_error", "§II-A residual of b - e",
     "v[i] = b[i] - (e ? e[i] : 0.0);", "v[i] = b[i];"),
    ("classify_argmax", "§II-A label = argmin residual",
     "if (resid[c] < resid[best]) best = c;", "if (resid[c] > resid[best]) best = c;"),
    ("sci_signed_mass", "Eq. 40 ||delta_i(x)||_1",
     "l1 += fabs(xj);", "l1 += xj;"),
    # unrolled PALM and its reverse sweep, reading R11
    ("unrolled_theta_unscaled", "R11 multiplier update",
     "theta[i] += xi * (b[i] - r[i]);", "theta[i] += (b[i] - r[i]);"),
    ("unrolled_c_sign", "R11 inner target b + theta/xi",
     "for (int i = 0; i < m; ++i) c[i] = b[i] + theta[i] / xi;",
     "for (int i = 0; i < m; ++i) c[i] = b[i] - theta[i] / xi;"),
    ("unrolled_momentum_index", "R11 forward FISTA momentum",
     "            const double mu = (t - 1.0) / t_new;\n            Mu[s] = mu;",
     "            const double mu = t / t_new;\n            Mu[s] = mu;"),
    ("unrolled_mask_dropped", "reverse of the soft threshold",
     "vbar[j] = (fabs(v[j]) > thr) ? wn_bar : 0.0;", "vbar[j] = wn_bar;"),
    ("unrolled_gradA_sign", "reverse of v = z + A^T (c - A z)/L",
     "grad_A[i + (size_t)j * m] += (rs[i] * vbar[j] - q[i] * zs[j]) / L;",
     "grad_A[i + (size_t)j * m] += (rs[i] * vbar[j] + q[i] * zs[j]) / L;"),
    ("unrolled_z0_adjoint_dropped", "reverse of z_0 = w_0 = x",
     "xbar[j] = wbar[j] + zbar[j];", "xbar[j] = wbar[j];"),
    ("unrolled_momentum_adjoint", "reverse of z' = (1 + mu) w' - mu w",
     "wbar[j] = -mu * zbar[j];", "wbar[j] = mu * zbar[j];"),
]

PER_MUTANT_TIMEOUT_S = 600


def _has_timeout_plugin() -> bool:
    try:
        import pytest_timeout  # noqa: F401
        return True
    except ImportError:
        return False


def _run_pins(lib_path: str) -> tuple[int, str]:
    env = dict(os.environ, L1_ORACLE_LIB=lib_path, OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "pytest", PINS, "-x", "-q", "-p", "no:cacheprovider",
           "-m", "not gpu and not slow"]
    if _has_timeout_plugin():
        cmd += ["--timeout", "300"]
    try:
        p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=PER_MUTANT_TIMEOUT_S)
    except subprocess.TimeoutExpired:
        return -1, "child pytest exceeded its time limit"
    return p.returncode, p.stdout + p.stderr


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    with open(SRC) as f:
        src = f.read()
    d = tmp_path_factory.mktemp("mutants")
    jobs = {}

    def compile_variant(name, text):
        path = os.path.join(d, name + ".c")
        with open(path, "w") as f:
            f.write(text)
        return oracle.compile_source(path, os.path.join(d, name + ".so"))
    jobs["control"] = compile_variant("control", src)
    for mid, _, old, new in MUTANTS:
        assert src.count(old) == 1, f"{mid}: the text to mutate must occur exactly once"
        jobs[mid] = compile_variant(mid, src.replace(old, new))
    with cf.ThreadPoolExecutor(max(1, min(8, os.cpu_count() or 1))) as ex:
        futs = {mid: ex.submit(_run_pins, so) for mid, so in jobs.items()}
        return {mid: f.result() for mid, f in futs.items()}


def test_control_passes_every_pin(outcomes):
    rc, out = outcomes["control"]
    assert rc == 0, out[-3000:]


@pytest.mark.parametrize("mid", [m[0] for m in MUTANTS])
def test_mutant_fails_a_pin(outcomes, mid):
    rc, out = outcomes[mid]
    caught = re.findall(r"FAILED \S+::(\S+)", out)
    assert rc != 0, f"{mid}: every pin passed on the planted mistake"
    assert rc == 1 and caught, f"{mid}: the child pytest did not run to a test failure\n{out[-3000:]}"
    print(f"{mid}: caught by {caught[0]}")
