/*
 * FP64 CPU oracle for the augmented Lagrangian l1 solvers of
 *   A. Y. Yang, Z. Zhou, A. Ganesh, S. S. Sastry, Y. Ma,
 *   "Fast l1-Minimization Algorithms for Robust Face Recognition".
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously correct
 * restatement of the paper's algorithms that the CUDA library is checked
 * against.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header or constant with the
 * CUDA library.
 *
 * Conventions
 *   - Matrices are column-major: A[i + j*m] is row i, column j of A (m x n).
 *   - All arithmetic is IEEE double.  No BLAS, no blocking, no reordering:
 *     every product is a plain loop in the order the definition states.
 *   - Equation numbers follow the paper's LaTeX source order:
 *       Eq. 1 (P1), Eq. 2 (P1,2), Eq. 3 (QP_lambda), Eq. 5 (CAB model),
 *       Eq. 10 (LP form), Eq. 11 (l1 subdifferential), Eq. 18 (FISTA),
 *       Eq. 33 (method of multipliers), Eq. 35 (ALM for CAB),
 *       Eq. 38 (dual z-update), Eq. 39 (dual y-system), Eq. 40 (SCI);
 *     Algorithm 1 = PALM for CAB, Algorithm 2 = DALM for CAB.
 *
 * Readings of passages the paper leaves open (each also listed in the design
 * notes):
 *   R1  Algorithm 2 writes "A z" in the y-step and "A^T y" in the w-step; the
 *       operator there is B = [A I] (Eq. 39 with A -> B, x -> w, §V-B).
 *   R2  DALM's beta is not given: default beta = ||b||_1 / m per instance.
 *   R3  P1 PALM lets xi_k grow (§V-A): xi_0 = 2m/||b||_1, xi_{k+1} =
 *       min(growth * xi_k, xi_max * xi_0), growth 1.2, xi_max 1e4.  CAB
 *       keeps xi fixed at 2m/||b||_1 (§V-A, below Eq. 34).
 *   R4  L in Algorithm 1 is the Lipschitz constant ||A||_2^2 of the smooth
 *       term's gradient (§IV-A), estimated by power iteration on A^T A and
 *       multiplied by a safety factor (1.01 by default).
 *   R5  Inner loop (Algorithm 1 leaves its test open): stop when ||w_{l+1} - w_l|| <=
 *       inner_tol * ||w_l|| (with ||w_l|| = 0 only an exact zero step
 *       stops), or after inner_max steps.
 *   R6  Outer stopping rule: ||w_{k+1} - w_k|| / ||w_k|| < tol (§VI-C), where
 *       w = [x; e] for CAB and w = x otherwise.  A zero step counts as 0,
 *       a nonzero step from a zero iterate as +infinity.
 *   R7  x_{k+1} <- w_l takes the last inner iterate computed.
 *   R8  FISTA restarts with t = 1, z = w = x_k each outer iteration.
 *   R9  soft(v, a) = sign(v) max(|v| - a, 0), sign(0) = 0.
 *   R10 P1,2 (Eq. 2) has no algorithm in the paper: it is Algorithm 1 with
 *       the e-step replaced by the projection of b - A x + theta/xi onto the
 *       l2 ball of radius epsilon (the minimiser of the same augmented
 *       Lagrangian over ||e|| <= epsilon).
 *   R11 Unrolled PALM (differentiation): K inner FISTA steps in total, a
 *       multiplier update after every J inner steps, no early exit; xi and L
 *       are constants (no gradient flows through them).
 *   R15 The inexact y-step §V-B mentions (a single conjugate-gradient step
 *       instead of the exact solve): CG on (B B^T) y = B z - (B w - b)/beta
 *       started from the previous y; cg_steps = 1 is that variant.
 *   R16 The alignment step of §II-B solved by PALM: Algorithm 1 with the
 *       x-step replaced by the exact least-squares minimiser over the
 *       unpenalised w, and xi fixed at 2m/||b||_1.
 *   R17 FISTA with fixed-point continuation (the setup of the comparison in
 *       §VI-A): iteration k of Eq. 18 uses lambda_k, lambda_1 = lambda_0 given,
 *       lambda_{k+1} = max(rho lambda_k, lambda) with rho = 0.95; t and the
 *       extrapolation carry over when lambda changes; the stopping rule (R6
 *       on x) is applied only once lambda_k has reached lambda.
 *   R18 AMP (§IV, the message-passing iteration for P1): x_0 = 0, z_0 = b,
 *       delta = m/n; the paper gives no initial threshold.  The first x-step
 *       sees v = A^T b, which for a Gaussian dictionary with unit columns is
 *       x_0's target plus noise of standard deviation about ||b||_2/sqrt(m)
 *       (the picture the AMP derivation rests on), so by default tau_0 is
 *       1.5 ||b||_2 / sqrt(m), a threshold at one and a half noise deviations
 *       (half of ||A^T b||_inf, tried first, lets the first step keep too few
 *       entries, the count then drives tau below the noise and the iteration
 *       diverges on many Gaussian instances); the average derivative of
 *       soft(., tau) at v is the fraction of entries with |v_i| > tau; the
 *       rule R6 on x is applied after each x-step, and a stopped iteration
 *       keeps z_k and tau_k (the ones that produced the returned x); an
 *       iterate that is not finite stops it (converged = -1).
 *   R19 The image side of the alignment loop of §II-B (restated in numpy in
 *       oracle/__init__.py): tau is a similarity (a, b, tx, ty) mapping the
 *       canonical pixel (u, v) to (a u - b v + tx, b u + a v + ty); y o tau is
 *       the bilinear interpolant of the query, the point clamped to the image;
 *       J is the interpolant's slope in its cell (0 where clamped) times the
 *       derivative of the point in tau; no intensity normalisation; the loop
 *       adds dtau (the last four entries of w) to tau and stops once dtau
 *       moves no corner of the canonical frame by tau_tol pixels or more.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_NOT_SPD (-2)
#define ORC_ERR_NOMEM (-3)

#define ORC_MODE_P1 0
#define ORC_MODE_P12 1
#define ORC_MODE_QP 2
#define ORC_MODE_CAB 3

typedef struct {
    int iters;          /* outer iterations (PALM) or iterations (DALM, FISTA) */
    int inner_total;    /* total inner FISTA steps (PALM) */
    int converged;      /* 1 when the stopping rule R6 was met */
    double rel_change;  /* last value of the stopping quantity */
    double param;       /* xi_0 (PALM), beta (DALM), lambda/L (FISTA) used */
} orc_stats;

typedef struct {
    int mode;           /* ORC_MODE_P1, ORC_MODE_P12 or ORC_MODE_CAB */
    double tol;         /* outer tolerance (R6) */
    int max_outer;      /* outer iteration cap */
    int inner_max;      /* inner FISTA cap (R5) */
    double inner_tol;   /* inner tolerance (R5) */
    double xi0;         /* <= 0: 2m/||b||_1 */
    double xi_growth;   /* R3: P1 and P1,2 only */
    double xi_max;      /* R3: cap as a multiple of xi_0 */
    double L;           /* Lipschitz constant (R4), > 0 */
    double epsilon;     /* P1,2 radius */
} orc_palm_opts;

/* ---------------------------------------------------------------- helpers */

static double dot(const double* a, const double* b, int n) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

static double nrm2(const double* a, int n) { return sqrt(dot(a, a, n)); }

static double nrm1(const double* a, int n) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += fabs(a[i]);
    return s;
}

/* y = A x, A m x n column-major */
static void mat_vec(const double* A, int m, int n, const double* x, double* y) {
    for (int i = 0; i < m; ++i) y[i] = 0.0;
    for (int j = 0; j < n; ++j) {
        const double xj = x[j];
        const double* col = A + (size_t)j * m;
        for (int i = 0; i < m; ++i) y[i] += col[i] * xj;
    }
}

/* x = A^T y */
static void mat_tvec(const double* A, int m, int n, const double* y, double* x) {
    for (int j = 0; j < n; ++j) x[j] = dot(A + (size_t)j * m, y, m);
}

/* R9: proximal operator of a*||.||_1 (§IV, soft-thresholding) */
static double soft(double v, double a) {
    if (v > a) return v - a;
    if (v < -a) return v + a;
    return 0.0;
}

/* projection onto [-1, 1] (Eq. 38) */
static double clamp1(double v) { return v > 1.0 ? 1.0 : (v < -1.0 ? -1.0 : v); }

/* R6: relative change with the zero conventions */
static double rel_change(double diff, double base) {
    if (diff == 0.0) return 0.0;
    if (base == 0.0) return INFINITY;
    return diff / base;
}

static void* zalloc(size_t count) { return calloc(count ? count : 1, sizeof(double)); }

/* ---------------------------------------------------- Lipschitz constant */

/* R4: power iteration on A^T A from v = 1/sqrt(n).  The Rayleigh quotient
 * ||A v||^2 (||v|| = 1) is a lower bound of ||A||_2^2 that increases to it;
 * stop when it changes by <= rtol relative, then scale by `safety`. */
double orc_lipschitz(const double* A, int m, int n, int max_iter, double rtol,
                     double safety, int* iters_out) {
    double* v = (double*)zalloc(n);
    double* u = (double*)zalloc(m);
    double* g = (double*)zalloc(n);
    if (!v || !u || !g) { free(v); free(u); free(g); return -1.0; }
    for (int j = 0; j < n; ++j) v[j] = 1.0 / sqrt((double)n);
    double rho = 0.0;
    int it = 0;
    for (it = 1; it <= max_iter; ++it) {
        mat_vec(A, m, n, v, u);
        const double rho_new = dot(u, u, m);
        mat_tvec(A, m, n, u, g);
        const double gn = nrm2(g, n);
        if (gn == 0.0) { rho = rho_new; break; }
        for (int j = 0; j < n; ++j) v[j] = g[j] / gn;
        const int done = it > 1 && fabs(rho_new - rho) <= rtol * rho_new;
        rho = rho_new;
        if (done) break;
    }
    if (iters_out) *iters_out = it > max_iter ? max_iter : it;
    free(v); free(u); free(g);
    return safety * rho;
}

/* ------------------------------------------------ FISTA for (QP_lambda) */

/* One step of Eq. 18 (§IV-A) on F(x) = 1/2 ||b - A x||^2 + lambda ||x||_1:
 *   x_k     = soft(y_k - grad f(y_k)/L, lambda/L),  grad f(y) = A^T (A y - b)
 *   t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
 *   y_{k+1} = x_k + (t_k - 1)/t_{k+1} (x_k - x_{k-1}),
 * from y = y_k, xp = x_{k-1}, *tp = t_k; leaves x = x_k, y = y_{k+1},
 * xp = x_k, *tp = t_{k+1}; returns the relative change of x (R6).  r and g
 * are m- and n-vectors of scratch. */
static double fista_step(const double* A, int m, int n, const double* b, double lambda, double L,
                         double* y, double* xp, double* r, double* g, double* x, double* tp) {
    const double t = *tp;
    mat_vec(A, m, n, y, r);
    for (int i = 0; i < m; ++i) r[i] = b[i] - r[i];      /* r = b - A y */
    mat_tvec(A, m, n, r, g);                               /* g = -grad f(y) */
    for (int j = 0; j < n; ++j) x[j] = soft(y[j] + g[j] / L, lambda / L);
    const double t_new = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    const double mu = (t - 1.0) / t_new;
    double d2 = 0.0;
    for (int j = 0; j < n; ++j) {
        const double dj = x[j] - xp[j];
        d2 += dj * dj;
        y[j] = x[j] + mu * dj;
    }
    const double rel = rel_change(sqrt(d2), nrm2(xp, n));
    memcpy(xp, x, sizeof(double) * n);
    *tp = t_new;
    return rel;
}

/* FISTA (Eq. 18) for (QP_lambda) with y_1 = x_0 = 0, t_1 = 1; stops on R6
 * applied to x. */
int orc_fista_qp(const double* A, int m, int n, const double* b, double lambda,
                 double L, double tol, int max_iter, double* x, orc_stats* st) {
    if (!A || !b || !x || m <= 0 || n <= 0 || !(L > 0.0) || lambda < 0.0) return ORC_ERR_ARG;
    double* y = (double*)zalloc(n);
    double* xp = (double*)zalloc(n);
    double* r = (double*)zalloc(m);
    double* g = (double*)zalloc(n);
    if (!y || !xp || !r || !g) { free(y); free(xp); free(r); free(g); return ORC_ERR_NOMEM; }
    double t = 1.0, rel = INFINITY;
    int k = 0, conv = 0;
    for (k = 1; k <= max_iter; ++k) {
        rel = fista_step(A, m, n, b, lambda, L, y, xp, r, g, x, &t);
        if (rel < tol) { conv = 1; break; }
    }
    if (st) {
        st->iters = k > max_iter ? max_iter : k;
        st->inner_total = st->iters;
        st->converged = conv;
        st->rel_change = rel;
        st->param = lambda / L;
    }
    free(y); free(xp); free(r); free(g);
    return ORC_OK;
}

/* FISTA with continuation (R17): the steps of Eq. 18 with the threshold
 * lambda_k / L of a geometrically decreasing lambda_k, from lambda_0 down to
 * lambda; the rule R6 is applied once lambda_k = lambda. */
int orc_fista_cont(const double* A, int m, int n, const double* b, double lambda0, double lambda,
                   double rho, double L, double tol, int max_iter, double* x, orc_stats* st) {
    if (!A || !b || !x || m <= 0 || n <= 0 || !(L > 0.0) || lambda < 0.0 || lambda0 < lambda ||
        !(rho > 0.0 && rho <= 1.0))
        return ORC_ERR_ARG;
    double* y = (double*)zalloc(n);
    double* xp = (double*)zalloc(n);
    double* r = (double*)zalloc(m);
    double* g = (double*)zalloc(n);
    if (!y || !xp || !r || !g) { free(y); free(xp); free(r); free(g); return ORC_ERR_NOMEM; }
    double t = 1.0, rel = INFINITY, lam = lambda0;
    int k = 0, conv = 0;
    for (k = 1; k <= max_iter; ++k) {
        rel = fista_step(A, m, n, b, lam, L, y, xp, r, g, x, &t);
        if (lam <= lambda && rel < tol) { conv = 1; break; }
        lam = rho * lam > lambda ? rho * lam : lambda;
    }
    if (st) {
        st->iters = k > max_iter ? max_iter : k;
        st->inner_total = st->iters;
        st->converged = conv;
        st->rel_change = rel;
        st->param = lambda / L;
    }
    free(y); free(xp); free(r); free(g);
    return ORC_OK;
}

/* ------------------------------------------------------------------- AMP */

/* Approximate message passing for P1 (§IV, reading R18):
 *   x_{k+1} = soft(A^T z_k + x_k, tau_k)
 *   eta_k   = average over i of d soft(v, tau_k)/dv at v = A^T z_k + x_k
 *   z_{k+1} = b - A x_{k+1} + (eta_k / delta) z_k
 *   tau_{k+1} = (tau_k / delta) eta_k,          delta = m / n.
 * tau0 <= 0 takes 1.5 ||b||_2 / sqrt(m).  On return z and *tau hold the z_k
 * and tau_k of the last x-step (NULL to skip). */
int orc_amp(const double* A, int m, int n, const double* b, double tau0, double tol, int max_iter,
            double* x, double* z_out, double* tau_out, orc_stats* st) {
    if (!A || !b || !x || m <= 0 || n <= 0 || max_iter < 0) return ORC_ERR_ARG;
    double* z = (double*)zalloc(m);
    double* v = (double*)zalloc(n);
    double* xn = (double*)zalloc(n);
    double* r = (double*)zalloc(m);
    if (!z || !v || !xn || !r) { free(z); free(v); free(xn); free(r); return ORC_ERR_NOMEM; }
    const double delta = (double)m / (double)n;
    memset(x, 0, sizeof(double) * n);
    memcpy(z, b, sizeof(double) * m);
    double tau = tau0;
    if (!(tau > 0.0)) tau = 1.5 * nrm2(b, m) / sqrt((double)m);
    double rel = INFINITY;
    int k = 0, conv = 0;
    for (k = 1; k <= max_iter; ++k) {
        mat_tvec(A, m, n, z, v);
        for (int j = 0; j < n; ++j) v[j] += x[j];             /* v = A^T z_k + x_k */
        int above = 0;
        for (int j = 0; j < n; ++j) {
            xn[j] = soft(v[j], tau);
            if (fabs(v[j]) > tau) ++above;
        }
        const double eta = (double)above / (double)n;
        double d2 = 0.0;
        for (int j = 0; j < n; ++j) d2 += (xn[j] - x[j]) * (xn[j] - x[j]);
        rel = rel_change(sqrt(d2), nrm2(x, n));
        memcpy(x, xn, sizeof(double) * n);
        if (!isfinite(d2) || !isfinite(tau)) { conv = -1; break; }
        if (rel < tol) { conv = 1; break; }
        if (k == max_iter) break;
        mat_vec(A, m, n, x, r);
        int finite = 1;
        for (int i = 0; i < m; ++i) {
            z[i] = b[i] - r[i] + (eta / delta) * z[i];
            if (!isfinite(z[i])) finite = 0;
        }
        tau = tau / delta * eta;
        if (!finite) { conv = -1; break; }
    }
    if (z_out) memcpy(z_out, z, sizeof(double) * m);
    if (tau_out) *tau_out = tau;
    if (st) {
        st->iters = k > max_iter ? max_iter : k;
        st->inner_total = st->iters;
        st->converged = conv;
        st->rel_change = rel;
        st->param = tau;
    }
    free(z); free(v); free(xn); free(r);
    return ORC_OK;
}

/* ------------------------------------------------------------------- PALM */

/* Primal ALM.  CAB mode is Algorithm 1 (§V-A) on min ||x||_1 + ||e||_1
 * s.t. b = A x + e; P1 mode is Eq. 33 with e = 0 and the inner argmin by FISTA
 * (§V-A: the subproblem has the (QP_lambda) form); P1,2 mode follows R10.
 *   step 3: e_{k+1} = shrink(b - A x_k + theta_k/xi, 1/xi)
 *   steps 4-7: FISTA from t = 1, z = w = x_k:
 *       w_{l+1} = shrink(z_l + A^T(b - A z_l - e_{k+1} + theta_k/xi)/L, 1/(xi L))
 *       t_{l+1} = (1 + sqrt(1 + 4 t_l^2))/2
 *       z_{l+1} = w_{l+1} + (t_l - 1)/t_{l+1} (w_{l+1} - w_l)
 *   step 8: x_{k+1} = w_l, theta_{k+1} = theta_k + xi (b - A x_{k+1} - e_{k+1}).
 * Inputs x, e, theta are ignored on entry (cold start x = 0, e = b for CAB,
 * theta = 0); on return they hold the final iterates. */
int orc_palm(const double* A, int m, int n, const double* b, const orc_palm_opts* o,
             double* x, double* e, double* theta, orc_stats* st) {
    if (!A || !b || !o || !x || !theta || m <= 0 || n <= 0 || !(o->L > 0.0)) return ORC_ERR_ARG;
    if (o->mode != ORC_MODE_P1 && o->mode != ORC_MODE_P12 && o->mode != ORC_MODE_CAB) return ORC_ERR_ARG;
    if ((o->mode != ORC_MODE_P1) && !e) return ORC_ERR_ARG;
    const int has_e = o->mode != ORC_MODE_P1;
    double* e_loc = has_e ? e : (double*)zalloc(m);
    double* e_new = (double*)zalloc(m);
    double* c = (double*)zalloc(m);
    double* r = (double*)zalloc(m);
    double* g = (double*)zalloc(n);
    double* w = (double*)zalloc(n);
    double* w_new = (double*)zalloc(n);
    double* z = (double*)zalloc(n);
    double* Ax = (double*)zalloc(m);
    if (!e_loc || !e_new || !c || !r || !g || !w || !w_new || !z || !Ax) {
        if (!has_e) free(e_loc);
        free(e_new); free(c); free(r); free(g); free(w); free(w_new); free(z); free(Ax);
        return ORC_ERR_NOMEM;
    }
    const double L = o->L;
    const double b1 = nrm1(b, m);
    double xi0 = o->xi0 > 0.0 ? o->xi0 : (b1 > 0.0 ? 2.0 * m / b1 : 1.0);
    double xi = xi0;
    const double growth = (o->mode == ORC_MODE_CAB) ? 1.0 : (o->xi_growth > 0.0 ? o->xi_growth : 1.0);
    const double xi_cap = (o->xi_max > 0.0 ? o->xi_max : 1.0) * xi0;

    /* Algorithm 1, input line: x_1 = 0, e_1 = b, theta_1 = 0 */
    for (int j = 0; j < n; ++j) x[j] = 0.0;
    for (int i = 0; i < m; ++i) { theta[i] = 0.0; e_loc[i] = (o->mode == ORC_MODE_CAB) ? b[i] : 0.0; }

    int k = 0, conv = 0, inner_total = 0;
    double rel = INFINITY;
    for (k = 1; k <= o->max_outer; ++k) {
        /* step 3 */
        mat_vec(A, m, n, x, Ax);
        if (o->mode == ORC_MODE_CAB) {
            for (int i = 0; i < m; ++i) e_new[i] = soft(b[i] - Ax[i] + theta[i] / xi, 1.0 / xi);
        } else if (o->mode == ORC_MODE_P12) {
            for (int i = 0; i < m; ++i) e_new[i] = b[i] - Ax[i] + theta[i] / xi;
            const double vn = nrm2(e_new, m);
            const double s = (vn > o->epsilon) ? o->epsilon / vn : 1.0;
            for (int i = 0; i < m; ++i) e_new[i] *= s;
        } else {
            for (int i = 0; i < m; ++i) e_new[i] = 0.0;
        }
        /* steps 4-7 */
        for (int i = 0; i < m; ++i) c[i] = b[i] - e_new[i] + theta[i] / xi;
        double t = 1.0;
        memcpy(z, x, sizeof(double) * n);
        memcpy(w, x, sizeof(double) * n);
        for (int l = 1; l <= o->inner_max; ++l) {
            mat_vec(A, m, n, z, r);
            for (int i = 0; i < m; ++i) r[i] = c[i] - r[i];
            mat_tvec(A, m, n, r, g);
            for (int j = 0; j < n; ++j) w_new[j] = soft(z[j] + g[j] / L, 1.0 / (xi * L));
            const double t_new = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
            const double mu = (t - 1.0) / t_new;
            double d2 = 0.0;
            for (int j = 0; j < n; ++j) {
                const double dj = w_new[j] - w[j];
                d2 += dj * dj;
                z[j] = w_new[j] + mu * dj;
            }
            const double base = nrm2(w, n);
            memcpy(w, w_new, sizeof(double) * n);
            t = t_new;
            ++inner_total;
            const double d = sqrt(d2);
            if (d == 0.0 || (base > 0.0 && d <= o->inner_tol * base)) break;
        }
        /* step 8 */
        mat_vec(A, m, n, w, Ax);
        for (int i = 0; i < m; ++i) theta[i] += xi * (b[i] - Ax[i] - e_new[i]);
        double d2 = 0.0, base2 = 0.0;
        for (int j = 0; j < n; ++j) { const double dj = w[j] - x[j]; d2 += dj * dj; base2 += x[j] * x[j]; }
        if (has_e) {
            for (int i = 0; i < m; ++i) { const double di = e_new[i] - e_loc[i]; d2 += di * di; base2 += e_loc[i] * e_loc[i]; }
        }
        rel = rel_change(sqrt(d2), sqrt(base2));
        memcpy(x, w, sizeof(double) * n);
        memcpy(e_loc, e_new, sizeof(double) * m);
        if (growth != 1.0) { xi = growth * xi; if (xi > xi_cap) xi = xi_cap; }
        if (rel < o->tol) { conv = 1; break; }
    }
    if (st) {
        st->iters = k > o->max_outer ? o->max_outer : k;
        st->inner_total = inner_total;
        st->converged = conv;
        st->rel_change = rel;
        st->param = xi0;
    }
    if (!has_e) free(e_loc);
    free(e_new); free(c); free(r); free(g); free(w); free(w_new); free(z); free(Ax);
    return ORC_OK;
}

/* ------------------------------------------------------------------- DALM */

/* Cholesky factor G = R R^T of the m x m SPD matrix G (column-major, lower
 * triangle used), in place into the lower triangle.  Returns ORC_ERR_NOT_SPD
 * when a pivot is not positive beyond rounding: d <= 16 m eps G_jj, the
 * size of the rounding error the subtraction can leave on a singular
 * matrix. */
static int cholesky_lower(double* G, int m) {
    for (int j = 0; j < m; ++j) {
        /* column j: G(i, j) - sum over k = 0, ..., j-1 of R(i, k) R(j, k) for
         * i >= j, each sum taken in that order of k (k outside i so that the
         * inner loop walks down contiguous columns) */
        double* gj = G + (size_t)j * m;
        const double gjj = gj[j];
        for (int k = 0; k < j; ++k) {
            const double* rk = G + (size_t)k * m;
            const double rjk = rk[j];
            for (int i = j; i < m; ++i) gj[i] -= rk[i] * rjk;
        }
        const double d = gj[j];
        if (!(d > 16.0 * m * 2.220446049250313e-16 * gjj)) return ORC_ERR_NOT_SPD;
        const double rjj = sqrt(d);
        gj[j] = rjj;
        for (int i = j + 1; i < m; ++i) gj[i] = gj[i] / rjj;
    }
    return ORC_OK;
}

/* solve R R^T y = rhs with the lower factor R (forward then back substitution) */
static void cholesky_solve(const double* R, int m, const double* rhs, double* y) {
    /* forward: y(i) = (rhs(i) - sum over k < i of R(i, k) y(k)) / R(i, i), the
     * sum taken in increasing k; column k is applied to all rows below it
     * once y(k) is known, so the inner loop walks down a contiguous column */
    for (int i = 0; i < m; ++i) y[i] = rhs[i];
    for (int k = 0; k < m; ++k) {
        const double* rk = R + (size_t)k * m;
        y[k] = y[k] / rk[k];
        const double yk = y[k];
        for (int i = k + 1; i < m; ++i) y[i] -= rk[i] * yk;
    }
    for (int i = m - 1; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < m; ++k) s -= R[k + (size_t)i * m] * y[k];
        y[i] = s / R[i + (size_t)i * m];
    }
}

/* B = [A I] (cab = 1) or B = A (cab = 0): v (length n or n+m) -> B v */
static void b_vec(const double* A, int m, int n, int cab, const double* v, double* out) {
    mat_vec(A, m, n, v, out);
    if (cab) for (int i = 0; i < m; ++i) out[i] += v[n + i];
}

/* y -> B^T y */
static void b_tvec(const double* A, int m, int n, int cab, const double* y, double* out) {
    mat_tvec(A, m, n, y, out);
    if (cab) for (int i = 0; i < m; ++i) out[n + i] = y[i];
}

/* cg_steps conjugate-gradient steps on (B B^T) y = rhs, starting from the
 * y passed in (the previous iterate), with B B^T applied as B (B^T p); the
 * inexact alternative to the exact y-step that §V-B mentions (one step
 * there).  r, p, q have length m, t length n (+ m for CAB). */
static void cg_ystep(const double* A, int m, int n, int cab, const double* rhs, int cg_steps,
                     double* y, double* r, double* p, double* q, double* t) {
    b_tvec(A, m, n, cab, y, t);
    b_vec(A, m, n, cab, t, q);
    for (int i = 0; i < m; ++i) { r[i] = rhs[i] - q[i]; p[i] = r[i]; }
    double rr = dot(r, r, m);
    for (int s = 0; s < cg_steps && rr > 0.0; ++s) {
        b_tvec(A, m, n, cab, p, t);
        b_vec(A, m, n, cab, t, q);
        const double pq = dot(p, q, m);
        if (!(pq > 0.0)) break;
        const double alpha = rr / pq;
        for (int i = 0; i < m; ++i) { y[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        const double rr_next = dot(r, r, m);
        const double gamma = rr_next / rr;
        for (int i = 0; i < m; ++i) p[i] = r[i] + gamma * p[i];
        rr = rr_next;
    }
}

/* Dual ALM, Algorithm 2 (§V-B) with reading R1:
 *   z_{k+1} = P_[-1,1](B^T y_k + w_k / beta)                    (Eq. 38)
 *   y_{k+1} = (B B^T)^{-1} (B z_{k+1} - (B w_k - b) / beta)     (Eq. 39)
 *   w_{k+1} = w_k - beta (z_{k+1} - B^T y_{k+1}),
 * from w_1 = 0, y_1 = 0.  With cg_steps = 0 the y-step is exact: B B^T =
 * A A^T (+ I for CAB) is factored once by Cholesky, and P1 with singular
 * A A^T returns ORC_ERR_NOT_SPD (§V-B assumes A A^T invertible).  With
 * cg_steps > 0 it takes that many conjugate-gradient steps from y_k
 * instead (cg_ystep).  w has length n (+ m for CAB): x = w[0:n], e = w[n:]. */
int orc_dalm(const double* A, int m, int n, int cab, const double* b, double beta,
             double tol, int max_iter, int cg_steps, double* w, double* y, orc_stats* st) {
    if (!A || !b || !w || !y || m <= 0 || n <= 0 || cg_steps < 0) return ORC_ERR_ARG;
    const int nb = cab ? n + m : n;
    double* G = (double*)zalloc(cg_steps ? 4 * (size_t)m : (size_t)m * m);
    double* z = (double*)zalloc(nb);
    double* v = (double*)zalloc(nb);
    double* bty = (double*)zalloc(nb);
    double* rhs = (double*)zalloc(m);
    if (!G || !z || !v || !bty || !rhs) { free(G); free(z); free(v); free(bty); free(rhs); return ORC_ERR_NOMEM; }
    /* G = A A^T (+ I) for the exact y-step; CG needs four m-vectors instead */
    if (cg_steps == 0) {
        /* G(i, k) = sum over j = 0, 1, ..., n-1 of A(i, j) A(k, j), summed in
         * that order for every (i, k); the loops run j outside i so that the
         * innermost one walks down contiguous columns */
        for (int k = 0; k < m; ++k) {
            double* g = G + (size_t)k * m;
            for (int i = 0; i < m; ++i) g[i] = 0.0;
            for (int j = 0; j < n; ++j) {
                const double* col = A + (size_t)j * m;
                const double akj = col[k];
                for (int i = 0; i < m; ++i) g[i] += col[i] * akj;
            }
            if (cab) g[k] += 1.0;
        }
        if (cholesky_lower(G, m) != ORC_OK) {
            free(G); free(z); free(v); free(bty); free(rhs);
            return ORC_ERR_NOT_SPD;
        }
    }
    if (!(beta > 0.0)) { const double b1 = nrm1(b, m); beta = b1 > 0.0 ? b1 / m : 1.0; }
    for (int j = 0; j < nb; ++j) { w[j] = 0.0; bty[j] = 0.0; }
    for (int i = 0; i < m; ++i) y[i] = 0.0;
    int k = 0, conv = 0;
    double rel = INFINITY;
    for (k = 1; k <= max_iter; ++k) {
        for (int j = 0; j < nb; ++j) z[j] = clamp1(bty[j] + w[j] / beta);
        /* B z - (B w - b)/beta = B (z - w/beta) + b/beta */
        for (int j = 0; j < nb; ++j) v[j] = z[j] - w[j] / beta;
        b_vec(A, m, n, cab, v, rhs);
        for (int i = 0; i < m; ++i) rhs[i] += b[i] / beta;
        if (cg_steps == 0) cholesky_solve(G, m, rhs, y);
        else cg_ystep(A, m, n, cab, rhs, cg_steps, y, G, G + m, G + 2 * (size_t)m, v);
        b_tvec(A, m, n, cab, y, bty);
        double d2 = 0.0, base2 = 0.0;
        for (int j = 0; j < nb; ++j) {
            const double dj = -beta * (z[j] - bty[j]);
            d2 += dj * dj;
            base2 += w[j] * w[j];
            w[j] += dj;
        }
        rel = rel_change(sqrt(d2), sqrt(base2));
        if (rel < tol) { conv = 1; break; }
    }
    if (st) {
        st->iters = k > max_iter ? max_iter : k;
        st->inner_total = st->iters;
        st->converged = conv;
        st->rel_change = rel;
        st->param = beta;
    }
    free(G); free(z); free(v); free(bty); free(rhs);
    return ORC_OK;
}

/* ------------------------------------------- alignment l1 step (§II-B) */

/* The convex step of the face-alignment loop (§II-B, the last displayed
 * problem there): min ||e||_1 s.t. b = B w + e with B = [A_i, -J_i] tall and
 * w (coefficients and the transformation update) not penalised.  Reading R16:
 * Algorithm 1 with its x-step replaced by the exact minimiser of the
 * augmented Lagrangian over the unpenalised w, a least-squares solve with
 * B^T B factored once by Cholesky:
 *   e_{k+1} = shrink(b - B w_k + theta_k/xi, 1/xi)
 *   w_{k+1} = (B^T B)^{-1} B^T (b - e_{k+1} + theta_k/xi)
 *   theta_{k+1} = theta_k + xi (b - B w_{k+1} - e_{k+1}),
 * from w = 0, e = b, theta = 0, xi fixed at 2m/||b||_1 (as for CAB, §V-A)
 * unless xi0 > 0, stopping on R6 with w = [w; e].  B is m x p column-major;
 * returns ORC_ERR_NOT_SPD when B^T B is singular. */
int orc_palm_align(const double* B, int m, int p, const double* b, double tol, int max_outer,
                   double xi0, double* w, double* e, double* theta, orc_stats* st) {
    if (!B || !b || !w || !e || !theta || m <= 0 || p <= 0) return ORC_ERR_ARG;
    double* G = (double*)zalloc((size_t)p * p);
    double* Bw = (double*)zalloc(m);
    double* t = (double*)zalloc(m);
    double* rhs = (double*)zalloc(p);
    double* w_next = (double*)zalloc(p);
    double* e_next = (double*)zalloc(m);
    if (!G || !Bw || !t || !rhs || !w_next || !e_next) {
        free(G); free(Bw); free(t); free(rhs); free(w_next); free(e_next);
        return ORC_ERR_NOMEM;
    }
    for (int i = 0; i < p; ++i)
        for (int k = 0; k < p; ++k) G[i + (size_t)k * p] = dot(B + (size_t)i * m, B + (size_t)k * m, m);
    if (cholesky_lower(G, p) != ORC_OK) {
        free(G); free(Bw); free(t); free(rhs); free(w_next); free(e_next);
        return ORC_ERR_NOT_SPD;
    }
    const double b1 = nrm1(b, m);
    const double xi = xi0 > 0.0 ? xi0 : (b1 > 0.0 ? 2.0 * m / b1 : 1.0);
    for (int j = 0; j < p; ++j) w[j] = 0.0;
    for (int i = 0; i < m; ++i) { e[i] = b[i]; theta[i] = 0.0; Bw[i] = 0.0; }
    int k = 0, conv = 0;
    double rel = INFINITY;
    for (k = 1; k <= max_outer; ++k) {
        for (int i = 0; i < m; ++i) e_next[i] = soft(b[i] - Bw[i] + theta[i] / xi, 1.0 / xi);
        for (int i = 0; i < m; ++i) t[i] = b[i] - e_next[i] + theta[i] / xi;
        mat_tvec(B, m, p, t, rhs);
        cholesky_solve(G, p, rhs, w_next);
        mat_vec(B, m, p, w_next, Bw);
        for (int i = 0; i < m; ++i) theta[i] += xi * (b[i] - Bw[i] - e_next[i]);
        double d2 = 0.0, base2 = 0.0;
        for (int j = 0; j < p; ++j) { const double d = w_next[j] - w[j]; d2 += d * d; base2 += w[j] * w[j]; }
        for (int i = 0; i < m; ++i) { const double d = e_next[i] - e[i]; d2 += d * d; base2 += e[i] * e[i]; }
        rel = rel_change(sqrt(d2), sqrt(base2));
        memcpy(w, w_next, sizeof(double) * p);
        memcpy(e, e_next, sizeof(double) * m);
        if (rel < tol) { conv = 1; break; }
    }
    if (st) {
        st->iters = k > max_outer ? max_outer : k;
        st->inner_total = st->iters;
        st->converged = conv;
        st->rel_change = rel;
        st->param = xi;
    }
    free(G); free(Bw); free(t); free(rhs); free(w_next); free(e_next);
    return ORC_OK;
}

/* --------------------------------------------------------- classification */

/* Per-class residuals r_i = ||b - e - A delta_i(x)||_2 (the SRC rule of §II-A
 * with the CAB error term removed; delta_i keeps the entries of class i),
 * label = argmin_i r_i (lowest index on ties), and the SCI rule of Eq. 40:
 * argmax_i (C ||delta_i(x)||_1 / ||x||_1 - 1)/(C - 1), i.e. argmax_i
 * ||delta_i(x)||_1 (lowest index on ties).  e may be NULL (no error term).
 * offsets has C+1 entries; class i owns columns offsets[i]..offsets[i+1]-1. */
int orc_classify(const double* A, int m, int n, const int* offsets, int C,
                 const double* b, const double* x, const double* e,
                 double* resid, double* sci, int* label, int* sci_label) {
    if (!A || !offsets || !b || !x || !resid || !label || C <= 0) return ORC_ERR_ARG;
    if (offsets[0] != 0 || offsets[C] != n) return ORC_ERR_ARG;
    double* v = (double*)zalloc(m);
    if (!v) return ORC_ERR_NOMEM;
    const double x1 = nrm1(x, n);
    int best = 0, best_sci = 0;
    double best_l1 = -1.0;
    for (int c = 0; c < C; ++c) {
        for (int i = 0; i < m; ++i) v[i] = b[i] - (e ? e[i] : 0.0);
        double l1 = 0.0;
        for (int j = offsets[c]; j < offsets[c + 1]; ++j) {
            const double xj = x[j];
            l1 += fabs(xj);
            for (int i = 0; i < m; ++i) v[i] -= A[i + (size_t)j * m] * xj;
        }
        resid[c] = nrm2(v, m);
        if (sci) sci[c] = (C > 1 && x1 > 0.0) ? (C * l1 / x1 - 1.0) / (C - 1.0) : 0.0;
        if (resid[c] < resid[best]) best = c;
        if (l1 > best_l1) { best_l1 = l1; best_sci = c; }
    }
    *label = best;
    if (sci_label) *sci_label = best_sci;
    free(v);
    return ORC_OK;
}

/* ---------------------------------------------- unrolled PALM and adjoint */

/* Forward of R11 for one right-hand side (P1 mode, e = 0):
 *   x = 0, theta = 0; for each of the K/J outer blocks:
 *     c = b + theta/xi; t = 1; z = w = x
 *     J times: r = c - A z; v = z + A^T r / L; w' = soft(v, 1/(xi L));
 *              t' = (1 + sqrt(1 + 4 t^2))/2; z = w' + (t-1)/t' (w' - w);
 *              w = w'; t = t'
 *     x = w; theta = theta + xi (b - A x)
 * and loss = 1/2 ||x - x_target||^2.  The reverse sweep is plain reverse-mode
 * differentiation of exactly these statements (soft-threshold derivative 1
 * where |v| > 1/(xi L), else 0; xi, L held constant).  grad_A (m x n) and
 * grad_b (m) are ACCUMULATED into (callers zero them); either may be NULL. */
int orc_unrolled_palm(const double* A, int m, int n, const double* b, double xi,
                      double L, int K, int J, const double* x_target,
                      double* x_out, double* loss, double* grad_A, double* grad_b) {
    if (!A || !b || !x_target || m <= 0 || n <= 0 || K <= 0 || J <= 0 || !(L > 0.0) || !(xi > 0.0))
        return ORC_ERR_ARG;
    const int n_outer = (K + J - 1) / J;
    /* tapes: per inner step z (n), w_old (n), v (n), r (m), mu; per outer x (n) */
    double* Zs = (double*)zalloc((size_t)K * n);
    double* Ws = (double*)zalloc((size_t)K * n);
    double* Vs = (double*)zalloc((size_t)K * n);
    double* Rs = (double*)zalloc((size_t)K * m);
    double* Mu = (double*)zalloc(K);
    double* Xs = (double*)zalloc((size_t)n_outer * n);
    double* x = (double*)zalloc(n);
    double* theta = (double*)zalloc(m);
    double* c = (double*)zalloc(m);
    double* z = (double*)zalloc(n);
    double* w = (double*)zalloc(n);
    double* g = (double*)zalloc(n);
    double* r = (double*)zalloc(m);
    double* q = (double*)zalloc(m);
    double* xbar = (double*)zalloc(n);
    double* wbar = (double*)zalloc(n);
    double* zbar = (double*)zalloc(n);
    double* vbar = (double*)zalloc(n);
    double* tbar = (double*)zalloc(m);
    double* cbar = (double*)zalloc(m);
    double* tmp = (double*)zalloc(n);
    int rc = ORC_OK;
    if (!Zs || !Ws || !Vs || !Rs || !Mu || !Xs || !x || !theta || !c || !z || !w || !g || !r ||
        !q || !xbar || !wbar || !zbar || !vbar || !tbar || !cbar || !tmp) { rc = ORC_ERR_NOMEM; goto done; }

    const double thr = 1.0 / (xi * L);
    int s = 0;
    for (int o = 0; o < n_outer; ++o) {
        for (int i = 0; i < m; ++i) c[i] = b[i] + theta[i] / xi;
        double t = 1.0;
        memcpy(z, x, sizeof(double) * n);
        memcpy(w, x, sizeof(double) * n);
        const int steps = (o == n_outer - 1) ? K - o * J : J;
        for (int l = 0; l < steps; ++l, ++s) {
            memcpy(Zs + (size_t)s * n, z, sizeof(double) * n);
            memcpy(Ws + (size_t)s * n, w, sizeof(double) * n);
            mat_vec(A, m, n, z, r);
            for (int i = 0; i < m; ++i) r[i] = c[i] - r[i];
            memcpy(Rs + (size_t)s * m, r, sizeof(double) * m);
            mat_tvec(A, m, n, r, g);
            double* v = Vs + (size_t)s * n;
            for (int j = 0; j < n; ++j) v[j] = z[j] + g[j] / L;
            const double t_new = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
            const double mu = (t - 1.0) / t_new;
            Mu[s] = mu;
            for (int j = 0; j < n; ++j) {
                const double wn = soft(v[j], thr);
                z[j] = wn + mu * (wn - w[j]);
                w[j] = wn;
            }
            t = t_new;
        }
        memcpy(x, w, sizeof(double) * n);
        memcpy(Xs + (size_t)o * n, x, sizeof(double) * n);
        mat_vec(A, m, n, x, r);
        for (int i = 0; i < m; ++i) theta[i] += xi * (b[i] - r[i]);
    }
    if (x_out) memcpy(x_out, x, sizeof(double) * n);
    double l2 = 0.0;
    for (int j = 0; j < n; ++j) { const double d = x[j] - x_target[j]; l2 += d * d; xbar[j] = d; }
    if (loss) *loss = 0.5 * l2;
    if (!grad_A && !grad_b) goto done;

    /* reverse sweep; tbar holds the adjoint of theta after the current outer
     * block's update (zero for the last block: its update feeds nothing). */
    for (int i = 0; i < m; ++i) tbar[i] = 0.0;
    s = K - 1;
    for (int o = n_outer - 1; o >= 0; --o) {
        const double* xo = Xs + (size_t)o * n;
        /* theta_{o+1} = theta_o + xi (b - A x_o) */
        if (o < n_outer - 1) {
            if (grad_b) for (int i = 0; i < m; ++i) grad_b[i] += xi * tbar[i];
            mat_tvec(A, m, n, tbar, tmp);
            for (int j = 0; j < n; ++j) xbar[j] -= xi * tmp[j];
            if (grad_A)
                for (int j = 0; j < n; ++j)
                    for (int i = 0; i < m; ++i) grad_A[i + (size_t)j * m] -= xi * tbar[i] * xo[j];
        }
        /* x_o = w at the end of the inner block; z at the end feeds nothing */
        memcpy(wbar, xbar, sizeof(double) * n);
        for (int j = 0; j < n; ++j) zbar[j] = 0.0;
        for (int i = 0; i < m; ++i) cbar[i] = 0.0;
        const int steps = (o == n_outer - 1) ? K - o * J : J;
        for (int l = steps - 1; l >= 0; --l, --s) {
            const double mu = Mu[s];
            const double* v = Vs + (size_t)s * n;
            const double* zs = Zs + (size_t)s * n;
            const double* rs = Rs + (size_t)s * m;
            /* z' = (1 + mu) w' - mu w ; w' = soft(v) */
            for (int j = 0; j < n; ++j) {
                const double wn_bar = wbar[j] + (1.0 + mu) * zbar[j];
                vbar[j] = (fabs(v[j]) > thr) ? wn_bar : 0.0;
                wbar[j] = -mu * zbar[j];
            }
            /* v = z + A^T (c - A z) / L */
            mat_vec(A, m, n, vbar, q);
            mat_tvec(A, m, n, q, tmp);
            for (int j = 0; j < n; ++j) zbar[j] = vbar[j] - tmp[j] / L;
            for (int i = 0; i < m; ++i) cbar[i] += q[i] / L;
            if (grad_A)
                for (int j = 0; j < n; ++j)
                    for (int i = 0; i < m; ++i)
                        grad_A[i + (size_t)j * m] += (rs[i] * vbar[j] - q[i] * zs[j]) / L;
        }
        /* z_0 = w_0 = x_{o-1} */
        for (int j = 0; j < n; ++j) xbar[j] = wbar[j] + zbar[j];
        /* c = b + theta_o / xi ; theta_o = theta_{o-1} + ... (carried by tbar) */
        if (grad_b) for (int i = 0; i < m; ++i) grad_b[i] += cbar[i];
        for (int i = 0; i < m; ++i) tbar[i] += cbar[i] / xi;
    }
done:
    free(Zs); free(Ws); free(Vs); free(Rs); free(Mu); free(Xs); free(x); free(theta); free(c);
    free(z); free(w); free(g); free(r); free(q); free(xbar); free(wbar); free(zbar); free(vbar);
    free(tbar); free(cbar); free(tmp);
    return rc;
}
