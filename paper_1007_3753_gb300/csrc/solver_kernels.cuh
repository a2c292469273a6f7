// Fused epilogues and per-column controllers of the batched PALM / DALM /
// FISTA sweeps.  Every panel is column-major with one problem per column;
// m-length panels use leading dimension ldm, n-length panels ldn.
#pragma once

#include "common.cuh"
#include "dalm_tc.cuh"
#include "gemm_simt.cuh"

namespace l1 {

// Per-column solver state (struct of arrays, N entries each).
struct Cols {
    int N;
    // float
    float* beta;   // DALM penalty
    float* binv;   // 1 / beta
    float* xi;     // PALM penalty of the current outer step
    float* xicap;  // PALM: cap of the xi schedule
    float* mu;     // FISTA momentum (t_l - 1) / t_{l+1} of the next inner step
    // int
    int32_t* active;
    int32_t* status;
    int32_t* iters;  // outer iterations (PALM) / iterations
    int32_t* inner;  // total inner steps
    int32_t* phase;  // PalmPhase
    int32_t* l;      // inner steps in the current outer iteration
    int32_t* label;
    int32_t* sci_label;
    // double
    double* t;     // FISTA t_l
    double* rel;   // last relative change
    double* de2;   // PALM: ||e_{k+1} - e_k||^2 of the current outer iteration
    double* e2;    // PALM: ||e_k||^2
    double* b1;    // ||b||_1
    double* fin;   // [N][8] final metrics
    float* smax;   // max |B^T y| (finalize)
    int32_t* orig; // original column of each slot (compaction)
};

// Results of retired columns, in the caller's column order.
struct Home {
    int N;
    float* Wx;      // x (n x N, ldn)
    float* We;      // e (m x N, ldm)
    float* Y;       // dual iterate (m x N, ldm)
    int32_t* status;
    int32_t* iters;
    int32_t* inner;
    double* rel;
    double* param;  // beta (DALM), xi_0 (PALM), lambda/L (FISTA)
    float* xi;      // PALM: xi of the last outer step (final multiplier step)
};

// xi used by an outer step: the schedule of §V-A (growth then cap) applies
// from the second outer step on; the first keeps xi_0.
__device__ __forceinline__ float xi_for_phase(int ph, float xi, float growth, float cap) {
    return ph == PH_OUTER ? fminf(growth * xi, cap) : xi;
}

// ------------------------------------------------------------ DALM epilogues
// Algorithm 2 (§V-B) with B = [A I] (CAB) or B = A (P1).  Panel U holds
// z_{k+1} - w_k/beta, so the right-hand side of Eq. 39 is
//   B z_{k+1} - (B w_k - b)/beta = A U_x (+ U_e) + b/beta.

// G1: R = A U_x (+ U_e) + b / beta
struct EpiDalmRhs {
    static constexpr int NRED = 0;
    float* R;
    const float* Ue;
    const float* B;
    const float* binv;
    const int32_t* active;
    int64_t ldm;
    int cab;
    __device__ void operator()(int i, int j, float acc, double*) const {
        if (!active[j]) return;
        const int64_t o = (int64_t)j * ldm + i;
        float v = fmaf(B[o], binv[j], acc);
        if (cab) v += Ue[o];
        R[o] = v;
    }
};

// G2: y_{k+1} = (B B^T)^{-1} R; for CAB the identity block of B^T y_{k+1}
// is y_{k+1} itself, so the e-part of the w-step and the next z - w/beta
// are formed here:  z_e = U_e + w_e/beta,  w_e' = w_e - beta (z_e - y),
// U_e' = clamp(y + w_e'/beta) - w_e'/beta.  red: ||dw_e||^2, ||w_e||^2.
struct EpiDalmY {
    static constexpr int NRED = 2;
    float* Y;
    float* We;
    float* Ue;
    const float* beta;
    const float* binv;
    const int32_t* active;
    int64_t ldm;
    int cab;
    __device__ void operator()(int i, int j, float acc, double* red) const {
        if (!active[j]) return;
        const int64_t o = (int64_t)j * ldm + i;
        Y[o] = acc;
        if (!cab) return;
        const float bi = binv[j], be = beta[j];
        const float we = We[o];
        const float z = fmaf(we, bi, Ue[o]);
        const float dw = -be * (z - acc);
        const float wn = we + dw;
        We[o] = wn;
        const float wb = wn * bi;
        Ue[o] = clamp_unit(acc + wb) - wb;
        red[0] += (double)dw * dw;
        red[1] += (double)we * we;
    }
};

// G3: s = A^T y_{k+1}; the x-part of the w-step and the next z - w/beta.
// red: ||dw_x||^2, ||w_x||^2.
struct EpiDalmS {
    static constexpr int NRED = 2;
    float* Wx;
    float* Ux;
    const float* beta;
    const float* binv;
    const int32_t* active;
    int64_t ldn;
    __device__ void operator()(int i, int j, float acc, double* red) const {
        if (!active[j]) return;
        const int64_t o = (int64_t)j * ldn + i;
        const float bi = binv[j], be = beta[j];
        const float w = Wx[o];
        const float z = fmaf(w, bi, Ux[o]);
        const float dw = -be * (z - acc);
        const float wn = w + dw;
        Wx[o] = wn;
        const float wb = wn * bi;
        const float u = clamp_unit(acc + wb) - wb;
        Ux[o] = u;
        red[0] += (double)dw * dw;
        red[1] += (double)w * w;
    }
};

// The state of the tensor-core engine (V, Z) -> the state of the CUDA-core
// sweeps (U = z - w/beta = Z - W/beta), in place: the active slots, or with
// inactive_only the frozen ones (before they are written home).
__global__ void tc_state_to_simt_kernel(float* U, const float* Z, const float* W, const float* binv,
                                        const int32_t* active, int64_t ld, int rows, int inactive_only) {
    const int j = blockIdx.y;
    if ((active[j] != 0) == (inactive_only != 0)) return;
    const float bi = binv[j];
    const int64_t o = (int64_t)j * ld;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x)
        U[o + i] = Z[o + i] - W[o + i] * bi;
}

// DALM state from (w, y) with acc = (A^T y)_j (a warm start, or the restart
// of a refinement phase): z = clamp(acc + w/beta) -- or, with have_u, the
// carried U gives z = U + w/beta -- then U = z - w/beta in place, or for the
// tensor-core engine (tc) Z = z and V = z - (acc + w/beta) in U's place.
__device__ __forceinline__ void dalm_restart_elem(float* U, float* Z, float w, float bi, float acc, int64_t o,
                                                  int have_u, int tc) {
    const float wb = w * bi;
    const float z = have_u ? U[o] + wb : clamp_unit(acc + wb);
    if (tc) {
        Z[o] = z;
        U[o] = z - (acc + wb);
    } else {
        U[o] = z - wb;
    }
}

struct EpiDalmRestart {
    static constexpr int NRED = 0;
    float* Ux;
    float* Zx;
    const float* Wx;
    const float* binv;
    const int32_t* active;
    int64_t ldn;
    int have_u;
    int tc;
    __device__ void operator()(int i, int j, float acc, double*) const {
        if (!active[j]) return;
        const int64_t o = (int64_t)j * ldn + i;
        dalm_restart_elem(Ux, Zx, Wx[o], binv[j], acc, o, have_u, tc);
    }
};

// the e-part of the same (B^T y there is y itself)
__global__ void dalm_restart_e_kernel(float* Ue, float* Ze, const float* We, const float* Y, const float* binv,
                                      const int32_t* active, int64_t ldm, int m, int have_u, int tc) {
    const int j = blockIdx.y;
    if (!active[j]) return;
    const float bi = binv[j];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const int64_t o = (int64_t)j * ldm + i;
        dalm_restart_elem(Ue, Ze, We[o], bi, Y[o], o, have_u, tc);
    }
}

// ------------------------------------------------------------ PALM epilogues
// Algorithm 1 (§V-A) as a per-column state machine over two sweeps per inner
// FISTA step:  G_A: A V  (V = z_l, or x_{k+1} at an outer step),
//              G_At: A^T R.
struct PalmParams {
    int mode;       // L1_P1, L1_CAB or L1_QP_LAMBDA
    float growth;   // xi schedule growth (1 for CAB and QP)
    float Linv;     // 1 / L
};

// G_A epilogue.  Inner phase: r = c - A z_l.  Outer phase (acc = A x_{k+1}):
// step 8 of the previous outer iteration theta += xi (b - A x - e), then the
// schedule xi -> xi', then step 3 e = shrink(b - A x + theta/xi', 1/xi'),
// c = b - e + theta/xi' and the first inner residual r = c - A x.
// red (outer phase only): ||e_{k+1} - e_k||^2, ||e_k||^2.
struct EpiPalmA {
    static constexpr int NRED = 3;
    float* R;
    float* Cc;
    float* E;
    float* TH;
    const float* B;
    Cols c;
    PalmParams p;
    int64_t ldm;
    __device__ void operator()(int i, int j, float acc, double* red) const {
        if (!c.active[j]) return;
        const int64_t o = (int64_t)j * ldm + i;
        const int ph = c.phase[j];
        if (ph == PH_INNER) {
            R[o] = Cc[o] - acc;
            return;
        }
        const float xi = c.xi[j];
        const float b = B[o];
        float th = TH[o];
        const float e_old = E[o];
        if (ph == PH_OUTER) th = fmaf(xi, b - acc - e_old, th);
        const float xin = xi_for_phase(ph, xi, p.growth, c.xicap[j]);
        const float thx = th / xin;
        if (p.mode == L1_P1_2) {
            // R10: e is the projection of v = b - A x + theta/xi onto the
            // eps-ball; its scale needs ||v||, so v is stored here and
            // p12_fixup_kernel scales it (and corrects c and r) before the
            // next sweep.  red: ||v||^2, ||e_k||^2, v . e_k
            const float v = b - acc + thx;
            TH[o] = th;
            E[o] = v;
            const float cc = b + thx;
            Cc[o] = cc;
            R[o] = cc - acc;
            red[0] += (double)v * v;
            red[1] += (double)e_old * e_old;
            red[2] += (double)v * e_old;
            return;
        }
        float e_new = 0.0f;
        if (p.mode == L1_CAB) e_new = soft_thr(b - acc + thx, 1.0f / xin);
        TH[o] = th;
        E[o] = e_new;
        const float cc = b - e_new + thx;
        Cc[o] = cc;
        R[o] = cc - acc;
        const float de = e_new - e_old;
        red[0] += (double)de * de;
        red[1] += (double)e_old * e_old;
    }
};

// G_At epilogue: one FISTA step of Algorithm 1 steps 6-7 (Eq. 18 for QP):
//   w' = shrink(z + g/L, 1/(xi L)), z' = w' + mu (w' - w),   g = A^T r.
// red: ||w' - w||^2, ||w||^2, ||w' - x_k||^2, ||x_k||^2.
struct EpiPalmAt {
    static constexpr int NRED = 4;
    float* W;
    float* V;
    const float* X;
    Cols c;
    PalmParams p;
    int64_t ldn;
    __device__ void operator()(int i, int j, float acc, double* red) const {
        if (!c.active[j]) return;
        const int64_t o = (int64_t)j * ldn + i;
        const int ph = c.phase[j];
        const float xin = xi_for_phase(ph, c.xi[j], p.growth, c.xicap[j]);
        const float thr = p.Linv / xin;
        const float z = V[o], w = W[o], x = X[o];
        const float wn = soft_thr(fmaf(acc, p.Linv, z), thr);
        const float mu = c.mu[j];
        const float dw = wn - w;
        W[o] = wn;
        V[o] = fmaf(mu, dw, wn);
        const float dx = wn - x;
        red[0] += (double)dw * dw;
        red[1] += (double)w * w;
        red[2] += (double)dx * dx;
        red[3] += (double)x * x;
    }
};

// ------------------------------------------------------------ AMP epilogues
// Approximate message passing for P1 (§IV, reading R18).  x lives in Wx and
// z in Y; per column, tau_k is c.t (FP64) with its FP32 copy in c.xi, and
// the z-step coefficient (n/m) <eta'> in c.mu.

// x-step (acc = A^T z_k): v = acc + x_k, x_{k+1} = soft(v, tau_k).
// red: ||x_{k+1} - x_k||^2, ||x_k||^2, the count of |v_i| > tau_k (the
// entries where soft(., tau_k) has derivative 1).
struct EpiAmpX {
    static constexpr int NRED = 3;
    float* Wx;
    const float* tau;
    const int32_t* active;
    int64_t ldn;
    __device__ void operator()(int i, int j, float acc, double* red) const {
        if (!active[j]) return;
        const int64_t o = (int64_t)j * ldn + i;
        const float x = Wx[o];
        const float v = acc + x;
        const float t = tau[j];
        const float xn = soft_thr(v, t);
        Wx[o] = xn;
        const float dx = xn - x;
        red[0] += (double)dx * dx;
        red[1] += (double)x * x;
        red[2] += fabsf(v) > t ? 1.0 : 0.0;
    }
};

// z-step (acc = A x_{k+1}): z_{k+1} = b - A x_{k+1} + coef_j z_k.
struct EpiAmpZ {
    static constexpr int NRED = 0;
    float* Y;
    const float* B;
    const float* coef;
    const int32_t* active;
    int64_t ldm;
    __device__ void operator()(int i, int j, float acc, double*) const {
        if (!active[j]) return;
        const int64_t o = (int64_t)j * ldm + i;
        Y[o] = fmaf(coef[j], Y[o], B[o] - acc);
    }
};


// ------------------------------------------------------------- controllers
// One 128-thread block per column: sums the row-block partials in index
// order, applies the stopping rules, and (PALM) restarts FISTA.

__device__ __forceinline__ double block_sum_128(double v, double* sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) s = sh[0] + sh[1] + sh[2] + sh[3];
    return s;  // valid in thread 0
}

// sum of part[p][j][r] over p < np, in a fixed order
__device__ __forceinline__ double sum_parts(const double* part, int np, int N, int j, int r,
                                            double* sh) {
    double v = 0.0;
    for (int p = threadIdx.x; p < np; p += blockDim.x) v += part[((int64_t)p * N + j) * kPartStride + r];
    return block_sum_128(v, sh);
}

// DALM controller: one warp per column (kCtrlCols columns per 128-thread
// block) adds the row-block partials of ||dw||^2 and ||w||^2 (lane p takes
// row blocks p, p + 32, ...; then a fixed warp tree) and applies the
// relative-change rule of §VI-C.
constexpr int kCtrlCols = 4;

__global__ void ctrl_dalm_kernel(Cols c, const double* part_e, int np_e, const double* part_x,
                                 int np_x, double tol, int max_iter) {
    const int j = blockIdx.x * kCtrlCols + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (j >= c.N || !c.active[j]) return;
    double d2 = 0.0, w2 = 0.0;
    for (int p = lane; p < np_x; p += 32) {
        const double* q = part_x + ((int64_t)p * c.N + j) * kPartStride;
        d2 += q[0];
        w2 += q[1];
    }
    if (part_e) {
        for (int p = lane; p < np_e; p += 32) {
            const double* q = part_e + ((int64_t)p * c.N + j) * kPartStride;
            d2 += q[0];
            w2 += q[1];
        }
    }
    d2 = warp_sum(d2);
    w2 = warp_sum(w2);
    if (lane != 0) return;
    const int it = c.iters[j] + 1;
    c.iters[j] = it;
    c.inner[j] = it;
    const double rel = rel_change(sqrt(d2), sqrt(w2));
    c.rel[j] = rel;
    if (!isfinite(d2) || !isfinite(w2)) {
        c.status[j] = L1_NONFINITE;
        c.active[j] = 0;
    } else if (rel < tol) {
        c.status[j] = L1_CONVERGED;
        c.active[j] = 0;
    } else if (it >= max_iter) {
        c.status[j] = L1_MAX_ITER;
        c.active[j] = 0;
    }
}

// tau_0 per column (one 128-thread block each): the given tau0, else
// 1.5 ||b||_2 / sqrt(m) (R18: the first x-step sees A^T b as the target
// plus noise of deviation about ||b||_2 / sqrt(m))
__global__ void amp_init_kernel(Cols c, const float* B, int64_t ldm, int m, double tau0) {
    __shared__ double sh[4];
    const int j = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double b = B[(int64_t)j * ldm + i];
        s += b * b;
    }
    s = block_sum_128(s, sh);
    if (threadIdx.x != 0) return;
    const double t = tau0 > 0.0 ? tau0 : 1.5 * sqrt(s) / sqrt((double)m);
    c.t[j] = t;
    c.xi[j] = (float)t;
    c.mu[j] = 0.0f;
}

// AMP controller (after the x-step), one warp per column: the relative
// change of x (R6); for a column that goes on, with eta = count / n and
// delta = m / n, the z-step coefficient eta / delta = count / m and
// tau_{k+1} = tau_k count / m.  A stopped column keeps z_k and tau_k.
__global__ void ctrl_amp_kernel(Cols c, const double* part, int np, int m, double tol, int max_iter) {
    const int j = blockIdx.x * kCtrlCols + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (j >= c.N || !c.active[j]) return;
    double d2 = 0.0, x2 = 0.0, cnt = 0.0;
    for (int p = lane; p < np; p += 32) {
        const double* q = part + ((int64_t)p * c.N + j) * kPartStride;
        d2 += q[0];
        x2 += q[1];
        cnt += q[2];
    }
    d2 = warp_sum(d2);
    x2 = warp_sum(x2);
    cnt = warp_sum(cnt);
    if (lane != 0) return;
    const int it = c.iters[j] + 1;
    c.iters[j] = it;
    c.inner[j] = it;
    const double rel = rel_change(sqrt(d2), sqrt(x2));
    c.rel[j] = rel;
    if (!isfinite(d2) || !isfinite(x2)) {
        c.status[j] = L1_NONFINITE;
        c.active[j] = 0;
    } else if (rel < tol) {
        c.status[j] = L1_CONVERGED;
        c.active[j] = 0;
    } else if (it >= max_iter) {
        c.status[j] = L1_MAX_ITER;
        c.active[j] = 0;
    } else {
        const double r = cnt / m;
        const double tn = c.t[j] * r;
        c.t[j] = tn;
        c.xi[j] = (float)tn;
        c.mu[j] = (float)r;
    }
}

// DALM with a CG y-step (reading R15): alpha_j = ||d||^2 / ||B^T d||^2 from
// the row-block partials of ||d||^2 (part_d) and ||A^T d||^2 (part_q); for
// CAB B^T d = [A^T d; d].  Inactive columns get 0.
__global__ void cg_alpha_kernel(Cols c, const double* part_d, int np_d, const double* part_q, int np_q, int cab,
                                float* alpha) {
    __shared__ double sh[4];
    const int j = blockIdx.x;
    if (!c.active[j]) {
        if (threadIdx.x == 0) alpha[j] = 0.0f;
        return;
    }
    const double dd = sum_parts(part_d, np_d, c.N, j, 0, sh);
    const double qq = sum_parts(part_q, np_q, c.N, j, 0, sh);
    if (threadIdx.x == 0) {
        const double den = qq + (cab ? dd : 0.0);
        alpha[j] = den > 0.0 ? (float)(dd / den) : 0.0f;
    }
}

// PALM / FISTA controller (after G_At).  Outer rule of §VI-C on w = [x; e];
// inner rule: ||w_{l+1} - w_l|| <= inner_tol ||w_l|| or inner_max steps.
// Restarting FISTA (t = 1, z = w = x_{k+1}) copies W into X and V.
__global__ void ctrl_palm_kernel(Cols c, PalmParams p, const double* part_A, int np_A,
                                 const double* part_At, int np_At, float* W, float* X, float* V,
                                 int64_t ldn, int n, double tol, double inner_tol, int inner_max,
                                 int max_iter) {
    __shared__ double sh[4];
    __shared__ int restart;
    const int j = blockIdx.x;
    if (!c.active[j]) return;
    const int ph = c.phase[j];
    double de2 = 0.0, e2 = 0.0;
    if (ph != PH_INNER && p.mode == L1_P1_2) {
        de2 = c.de2[j];  // from p12_fixup_kernel
        e2 = c.e2[j];
    } else if (ph != PH_INNER && p.mode != L1_QP_LAMBDA) {
        de2 = sum_parts(part_A, np_A, c.N, j, 0, sh);
        e2 = sum_parts(part_A, np_A, c.N, j, 1, sh);
    }
    const double d2 = sum_parts(part_At, np_At, c.N, j, 0, sh);
    const double w2 = sum_parts(part_At, np_At, c.N, j, 1, sh);
    const double dx2 = sum_parts(part_At, np_At, c.N, j, 2, sh);
    const double x2 = sum_parts(part_At, np_At, c.N, j, 3, sh);
    if (threadIdx.x == 0) {
        restart = 0;
        if (ph != PH_INNER) {
            c.xi[j] = xi_for_phase(ph, c.xi[j], p.growth, c.xicap[j]);
            c.phase[j] = PH_INNER;
            c.de2[j] = de2;
            c.e2[j] = e2;
        }
        const int l = c.l[j] + 1;
        c.l[j] = l;
        const int tot = c.inner[j] + 1;
        c.inner[j] = tot;
        const double t = c.t[j];
        const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        const double tnn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tn * tn));
        c.t[j] = tn;
        c.mu[j] = (float)((tn - 1.0) / tnn);
        const bool finite = isfinite(d2) && isfinite(w2);
        if (p.mode == L1_QP_LAMBDA) {
            // FISTA of Eq. 18: one loop, the outer rule applies to x_k; with
            // continuation (R17, growth > 1) lambda = 1/xi falls by the factor
            // 1/growth per step down to its target 1/xicap, and the rule
            // applies once it is there
            c.iters[j] = tot;
            const double rel = rel_change(sqrt(d2), sqrt(w2));
            c.rel[j] = rel;
            const bool at_target = !(p.growth > 1.0f) || c.xi[j] >= c.xicap[j];
            if (!finite) { c.status[j] = L1_NONFINITE; c.active[j] = 0; }
            else if (at_target && rel < tol) { c.status[j] = L1_CONVERGED; c.active[j] = 0; }
            else if (tot >= max_iter) { c.status[j] = L1_MAX_ITER; c.active[j] = 0; }
            if (!at_target) c.xi[j] = fminf(c.xi[j] * p.growth, c.xicap[j]);
        } else {
            const double d = sqrt(d2), base = sqrt(w2);
            const bool inner_done = d == 0.0 || (base > 0.0 && d <= inner_tol * base) || l >= inner_max;
            if (!finite) {
                c.status[j] = L1_NONFINITE;
                c.active[j] = 0;
            } else if (inner_done) {
                const int k = c.iters[j] + 1;
                c.iters[j] = k;
                const double rel = rel_change(sqrt(dx2 + c.de2[j]), sqrt(x2 + c.e2[j]));
                c.rel[j] = rel;
                if (rel < tol) { c.status[j] = L1_CONVERGED; c.active[j] = 0; }
                else if (k >= max_iter) { c.status[j] = L1_MAX_ITER; c.active[j] = 0; }
                else {
                    c.phase[j] = PH_OUTER;
                    c.l[j] = 0;
                    c.t[j] = 1.0;
                    c.mu[j] = 0.0f;  // t_1 = 1: the first step has no momentum
                    restart = 1;
                }
            }
        }
    }
    __syncthreads();
    if (restart) {
        const int64_t o = (int64_t)j * ldn;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const float w = W[o + i];
            X[o + i] = w;
            V[o + i] = w;
        }
    }
}

// P1,2 outer step (R10), between the two sweeps: e = min(1, eps/||v||) v,
// c -= e, r -= e, and ||e_{k+1} - e_k||^2 = s^2||v||^2 - 2 s v.e_k + ||e_k||^2
// for the outer rule.  One 128-thread block per column in its outer phase.
__global__ void p12_fixup_kernel(Cols c, const double* part_A, int np_A, float* E, float* Cc, float* R,
                                 int64_t ldm, int m, double eps) {
    __shared__ double sh[4];
    __shared__ float s_sh;
    const int j = blockIdx.x;
    if (!c.active[j] || c.phase[j] == PH_INNER) return;
    const double vv = sum_parts(part_A, np_A, c.N, j, 0, sh);
    const double ee = sum_parts(part_A, np_A, c.N, j, 1, sh);
    const double ve = sum_parts(part_A, np_A, c.N, j, 2, sh);
    if (threadIdx.x == 0) {
        const double nv = sqrt(vv);
        const double sc = nv > eps ? eps / nv : 1.0;
        c.de2[j] = fmax(0.0, sc * sc * vv - 2.0 * sc * ve + ee);
        c.e2[j] = ee;
        s_sh = (float)sc;
    }
    __syncthreads();
    const float sc = s_sh;
    const int64_t o = (int64_t)j * ldm;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const float e = sc * E[o + i];
        E[o + i] = e;
        Cc[o + i] -= e;
        R[o + i] -= e;
    }
}

// ------------------------------------------------------------- compaction
// Stable partition of the slots: newpos[s] = rank of s among the active slots
// (or -1), *count = number of active slots.  One block of 1024 threads.
__global__ void compact_scan_kernel(const int32_t* active, int N, int32_t* newpos, int32_t* count) {
    __shared__ int warp_tot[32];
    __shared__ int base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int c0 = 0; c0 < N; c0 += blockDim.x) {
        const int s = c0 + threadIdx.x;
        const int f = (s < N && active[s]) ? 1 : 0;
        int incl = f;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) warp_tot[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int t = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += v;
            }
            warp_tot[lane] = t;  // inclusive prefix over warps
        }
        __syncthreads();
        const int warp_off = wid > 0 ? warp_tot[wid - 1] : 0;
        if (s < N) newpos[s] = f ? base + warp_off + incl - 1 : -1;
        __syncthreads();
        if (threadIdx.x == 0) base += warp_tot[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = base;
}

// Move the active slots of one panel to their new positions (dst is a
// second buffer) and write retiring slots to the home panel (nullable).
__global__ void compact_panel_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                     float* __restrict__ home, int64_t ld, int rows, int N,
                                     const int32_t* __restrict__ newpos,
                                     const int32_t* __restrict__ orig) {
    const int s = blockIdx.y;
    if (s >= N) return;
    const int np = newpos[s];
    const float* col = src + (int64_t)s * ld;
    if (np >= 0) {
        float* d = dst + (int64_t)np * ld;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) d[i] = col[i];
    } else if (home) {
        float* d = home + (int64_t)orig[s] * ld;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) d[i] = col[i];
    }
}

// Same for the per-slot scalars; retiring slots write their results home.
__global__ void compact_cols_kernel(Cols src, Cols dst, Home home, int N, const int32_t* newpos,
                                    int solver, double xi_max) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const int np = newpos[s];
    if (np >= 0) {
        dst.beta[np] = src.beta[s];
        dst.binv[np] = src.binv[s];
        dst.xi[np] = src.xi[s];
        dst.xicap[np] = src.xicap[s];
        dst.mu[np] = src.mu[s];
        dst.active[np] = src.active[s];
        dst.status[np] = src.status[s];
        dst.iters[np] = src.iters[s];
        dst.inner[np] = src.inner[s];
        dst.phase[np] = src.phase[s];
        dst.l[np] = src.l[s];
        dst.t[np] = src.t[s];
        dst.rel[np] = src.rel[s];
        dst.de2[np] = src.de2[s];
        dst.e2[np] = src.e2[s];
        dst.b1[np] = src.b1[s];
        dst.orig[np] = src.orig[s];
    } else {
        const int o = src.orig[s];
        home.status[o] = src.status[s];
        home.iters[o] = src.iters[s];
        home.inner[o] = src.inner[s];
        home.rel[o] = src.rel[s];
        home.xi[o] = src.xi[s];
        home.param[o] = solver == L1_DALM  ? (double)src.beta[s]
                        : solver == L1_AMP ? src.t[s]
                                           : (double)src.xicap[s] / xi_max;
    }
}

// number of columns still active -> *count
__global__ void count_active_kernel(const int32_t* active, int N, int32_t* count) {
    __shared__ int sh[32];
    int v = 0;
    for (int j = threadIdx.x; j < N; j += blockDim.x) v += active[j] != 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        *count = s;
    }
}

// ------------------------------------------------------------- finalisation
// F1 (rows of A, acc = A x): r = b - A x - e.  PALM applies its last
// multiplier step theta += xi r (Algorithm 1 step 8) so the dual estimate
// matches the returned x.  QP keeps r in R for the dual point.
// red: ||r||^2, b^T y (P1/CAB) or b^T r (QP), ||e||_1, ||y||^2 (unused).
struct EpiFinalA {
    static constexpr int NRED = 4;
    float* R;
    float* Y;
    const float* E;  // nullable
    const float* B;
    const float* xi; // PALM only (nullable)
    float* smax;     // CAB: max |y| (the identity block of B^T y)
    int64_t ldm;
    int mode;
    __device__ void operator()(int i, int j, float acc, double* red) const {
        const int64_t o = (int64_t)j * ldm + i;
        const float b = B[o];
        const float e = E ? E[o] : 0.0f;
        const float r = b - acc - e;
        if (mode == L1_P1_2) {
            // the constraint of Eq. 2 is on b - A x
            const double rb = (double)b - (double)acc;
            red[0] += rb * rb;
        } else {
            red[0] += (double)r * r;
        }
        red[2] += fabs((double)e);
        if (mode == L1_QP_LAMBDA) {
            R[o] = r;
            red[1] += (double)b * r;
            return;
        }
        float y = Y[o];
        if (xi) {
            y = fmaf(xi[j], r, y);
            Y[o] = y;
        }
        red[1] += (double)b * y;
        red[3] += (double)y * y;
        if (mode == L1_CAB) atomicMax(reinterpret_cast<int*>(smax + j), __float_as_int(fabsf(y)));
    }
};

// F2 (rows of A^T, acc = A^T y or A^T r): max |acc|, ||x||_1.
struct EpiFinalAt {
    static constexpr int NRED = 1;
    const float* Wx;
    float* smax;
    int64_t ldn;
    __device__ void operator()(int i, int j, float acc, double* red) const {
        atomicMax(reinterpret_cast<int*>(smax + j), __float_as_int(fabsf(acc)));
        red[0] += fabs((double)Wx[(int64_t)j * ldn + i]);
    }
};

// fin[j][0..7] = primal, dual, gap, resid, x1, e1, -, -
__global__ void final_metrics_kernel(int N, const float* smax_arr, double* fin, const double* part_A,
                                     int np_A, const double* part_At, int np_At, int mode, double lambda) {
    __shared__ double sh[4];
    const int j = blockIdx.x;
    const double r2 = sum_parts(part_A, np_A, N, j, 0, sh);
    const double by = sum_parts(part_A, np_A, N, j, 1, sh);
    const double e1 = sum_parts(part_A, np_A, N, j, 2, sh);
    const double y2 = sum_parts(part_A, np_A, N, j, 3, sh);
    const double x1 = sum_parts(part_At, np_At, N, j, 0, sh);
    if (threadIdx.x != 0) return;
    const double smax = (double)smax_arr[j];
    double primal, dual;
    if (mode == L1_QP_LAMBDA) {
        // dual of Eq. 3: max b^T u - 1/2||u||^2 s.t. ||A^T u||_inf <= lambda,
        // feasible point u = s r with s = min(1, lambda / ||A^T r||_inf)
        primal = 0.5 * r2 + lambda * x1;
        const double s = smax > 0.0 ? fmin(1.0, lambda / smax) : 1.0;
        dual = s * by - 0.5 * s * s * r2;
    } else if (mode == L1_P1_2) {
        // dual of Eq. 2: max b^T y - eps ||y|| s.t. ||A^T y||_inf <= 1, made
        // feasible by scaling (lambda carries eps here)
        primal = x1;
        dual = (by - lambda * sqrt(y2)) / fmax(1.0, smax);
    } else {
        // dual of Eq. 1 / Eq. 5: max b^T y s.t. ||B^T y||_inf <= 1 (§V-B),
        // made feasible by scaling
        primal = x1 + e1;
        dual = by / fmax(1.0, smax);
    }
    double* f = fin + (int64_t)j * 8;
    f[0] = primal;
    f[1] = dual;
    f[2] = primal - dual;
    f[3] = sqrt(r2);
    f[4] = x1;
    f[5] = e1;
}

// ----------------------------------------------------------- classification
// Per-class residual ||b - e - A delta_c(x)||_2 (§II-A) and the l1 mass
// ||delta_c(x)||_1 of the SCI rule (Eq. 40).
//
// classify_tile_kernel<JT>: one block per (class, JT test vectors); the
// class's coefficients of those vectors sit in shared memory (class size x
// JT floats), and each thread walks rows i = t, t + blockDim, ...: it reads
// the class's entries of row i from the column-major A (consecutive threads,
// consecutive rows: coalesced), forms the JT products in FP32, and adds the
// squared residuals b_ij - e_ij - (A delta_c(x_j))_i of its rows in FP32;
// the threads' sums are added over each warp in FP32 and over the warps in
// FP64, in a fixed order.  Blocks of one column tile run back to back, so the
// tile's b and e are read from HBM once for all classes.
template <int JT>
__global__ void __launch_bounds__(256) classify_tile_kernel(const float* A_cm, int64_t ldm, int m,
                                                            const int32_t* offsets, const float* B,
                                                            const float* E, const float* Wx, int64_t ldn,
                                                            int N, double* resid2, double* l1mass) {
    extern __shared__ float xs[];  // [class size][JT]
    __shared__ float wsum[8][JT];
    const int cls = blockIdx.x, j0 = blockIdx.y * JT;
    const int c0 = offsets[cls], csz = offsets[cls + 1] - c0;
    for (int idx = threadIdx.x; idx < csz * JT; idx += blockDim.x) {
        const int jj = idx / csz, k = idx % csz;
        xs[k * JT + jj] = j0 + jj < N ? Wx[(int64_t)(j0 + jj) * ldn + c0 + k] : 0.0f;
    }
    __syncthreads();
    float q[JT];
#pragma unroll
    for (int jj = 0; jj < JT; ++jj) q[jj] = 0.0f;
    const float* Ac = A_cm + (int64_t)c0 * ldm;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        float sacc[JT];
#pragma unroll
        for (int jj = 0; jj < JT; ++jj) sacc[jj] = 0.0f;
        for (int k = 0; k < csz; ++k) {
            const float a = Ac[(int64_t)k * ldm + i];
            const float* xk = xs + k * JT;
#pragma unroll
            for (int jj = 0; jj < JT; ++jj) sacc[jj] = fmaf(a, xk[jj], sacc[jj]);
        }
#pragma unroll
        for (int jj = 0; jj < JT; ++jj) {
            if (j0 + jj < N) {
                const int64_t o = (int64_t)(j0 + jj) * ldm + i;
                const float v = B[o] - (E ? E[o] : 0.0f) - sacc[jj];
                q[jj] = fmaf(v, v, q[jj]);
            }
        }
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int jj = 0; jj < JT; ++jj) {
        const float sv = warp_sum_f(q[jj]);
        if (lane == 0) wsum[w][jj] = sv;
    }
    __syncthreads();
    if (threadIdx.x < JT && j0 + (int)threadIdx.x < N) {
        const int jj = threadIdx.x;
        double r2 = 0.0, l1v = 0.0;
        for (int ww = 0; ww < 8; ++ww) r2 += (double)wsum[ww][jj];
        for (int k = 0; k < csz; ++k) l1v += fabs((double)xs[k * JT + jj]);
        resid2[(int64_t)cls * N + j0 + jj] = r2;
        l1mass[(int64_t)cls * N + j0 + jj] = l1v;
    }
}

// Classes too large for classify_tile_kernel's shared memory: one block per
// (class, column); A is read row-major so a class's columns in one row are
// contiguous.
__global__ void classify_resid_kernel(const float* A_rm, int64_t lda_rm, int m,
                                      const int32_t* offsets, const float* B, const float* E,
                                      const float* Wx, int64_t ldm, int64_t ldn, int N,
                                      double* resid2, double* l1mass) {
    __shared__ double sh[8];
    const int cls = blockIdx.x, j = blockIdx.y;
    const int c0 = offsets[cls], c1 = offsets[cls + 1];
    const float* x = Wx + (int64_t)j * ldn;
    double acc = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        // the class's part of row i in FP32 (FP64 arithmetic runs at a small
        // fraction of the FP32 rate on this part; a class has tens of
        // columns), the residual's square summed in FP64
        const float* arow = A_rm + (int64_t)i * lda_rm;
        float s = 0.0f;
        for (int k = c0; k < c1; ++k) s = fmaf(arow[k], x[k], s);
        const float v = B[(int64_t)j * ldm + i] - (E ? E[(int64_t)j * ldm + i] : 0.0f) - s;
        acc += (double)v * v;
    }
    double l1v = 0.0;
    for (int k = c0 + threadIdx.x; k < c1; k += blockDim.x) l1v += fabs((double)x[k]);
    // block reductions (fixed order)
    acc = warp_sum(acc);
    l1v = warp_sum(l1v);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { sh[w] = acc; sh[4 + w] = l1v; }
    __syncthreads();
    if (threadIdx.x == 0) {
        resid2[(int64_t)cls * N + j] = sh[0] + sh[1] + sh[2] + sh[3];
        l1mass[(int64_t)cls * N + j] = sh[4] + sh[5] + sh[6] + sh[7];
    }
}

__global__ void classify_argmin_kernel(const double* resid2, const double* l1mass, int C, int N,
                                       int32_t* label, int32_t* sci_label) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    int best = 0, bsci = 0;
    double br = resid2[j], bl = l1mass[j];
    for (int cls = 1; cls < C; ++cls) {
        const double r = resid2[(int64_t)cls * N + j];
        const double l = l1mass[(int64_t)cls * N + j];
        if (r < br) { br = r; best = cls; }
        if (l > bl) { bl = l; bsci = cls; }
    }
    label[j] = best;
    sci_label[j] = bsci;
}

}  // namespace l1
