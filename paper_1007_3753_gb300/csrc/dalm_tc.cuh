// DALM on the BF16 tensor-core engine: the epilogues of its three sweeps and
// the launches (instantiated in dalm_tc.cu, apart from the rest of the
// solver so that the two compile in parallel).
#pragma once

#include "common.cuh"
#include "tc16.cuh"

namespace l1 {

// ------------------------------------- DALM epilogues of the tensor-core engine
// Algorithm 2 with B = [A I] (CAB) or B = A (P1), the y-step of Eq. 39 taken
// as a correction of the previous dual iterate:
//   y_{k+1} = y_k + (B B^T)^{-1} d,   d = B z_{k+1} - (B w_k - b)/beta - B B^T y_k
//                                      = B V + b/beta,  V = z_{k+1} - w_k/beta - B^T y_k,
// which is the step of Eq. 39 in exact arithmetic.  Its fixed point does not
// depend on how exactly the inverse is applied, and d vanishes as the
// iteration converges, so the rounding of the inverse's product shrinks with
// it.  V = clamp(v) - v with v = B^T y_k + w_k/beta.  Panels: V_x (FP32 and
// BF16 pieces), V_e, Z = z_{k+1}, W, Y.  Each functor returns the value whose
// BF16 pieces the next sweep reads (0 for frozen columns); its per-column
// reduction terms are FP32 (summed over 32 rows in FP32, above that in FP64).

// Each functor has two halves so that the epilogue can issue the state loads
// of several columns before the first store: load(i, j) reads what element
// (i, j) needs (whether or not its column is active), apply(i, j, acc, st,
// red) does the rest and returns the value for the piece sink.

// T1 (rows of A, acc = A V_x): d = acc (+ V_e) + b / beta
struct EpiTcD {
    static constexpr int NRED = 0;
    struct State {
        float b, ve;
        int act;
    };
    const float* Ve;
    const float* B;
    const float* binv;
    const int32_t* active;
    int64_t ldm;
    int cab;
    __device__ State load(int i, int j) const {
        const int64_t o = (int64_t)j * ldm + i;
        return State{B[o], cab ? Ve[o] : 0.0f, active[j]};
    }
    __device__ float apply(int, int j, float acc, const State& st, float*) const {
        if (!st.act) return 0.0f;
        return fmaf(st.b, binv[j], acc) + st.ve;
    }
};

// T2 (rows of F, acc = F d): y' = y + acc.  CAB: the e-part of the w-step
// (B^T y' is y' there): w_e' = w_e - beta (z_e - y'), z_e' = clamp(v),
// V_e = z_e' - v with v = y' + w_e'/beta.  red: ||dw_e||^2, ||w_e||^2.
// Returns y'.
struct EpiTcY {
    static constexpr int NRED = 2;
    struct State {
        float y, we, ze;
        int act;
    };
    float* Y;
    float* We;
    float* Ze;
    float* Ve;
    const float* beta;
    const float* binv;
    const int32_t* active;
    int64_t ldm;
    int cab;
    __device__ State load(int i, int j) const {
        const int64_t o = (int64_t)j * ldm + i;
        return State{Y[o], cab ? We[o] : 0.0f, cab ? Ze[o] : 0.0f, active[j]};
    }
    __device__ float apply(int i, int j, float acc, const State& st, float* red) const {
        if (!st.act) return 0.0f;
        const int64_t o = (int64_t)j * ldm + i;
        const float y = st.y + acc;
        Y[o] = y;
        if (cab) {
            const float dw = -beta[j] * (st.ze - y);
            const float wn = st.we + dw;
            We[o] = wn;
            const float v = fmaf(wn, binv[j], y);
            const float z = clamp_unit(v);
            Ze[o] = z;
            Ve[o] = z - v;
            red[0] += dw * dw;
            red[1] += st.we * st.we;
        }
        return y;
    }
};

// T3 (rows of A^T, acc = A^T y'): the x-part of the w-step,
// w_x' = w_x - beta (z_x - acc), z_x' = clamp(v), V_x = z_x' - v with
// v = acc + w_x'/beta.  red: ||dw_x||^2, ||w_x||^2.  Returns V_x.
struct EpiTcS {
    static constexpr int NRED = 2;
    struct State {
        float w, z;
        int act;
    };
    float* Wx;
    float* Zx;
    float* Vx;
    const float* beta;
    const float* binv;
    const int32_t* active;
    int64_t ldn;
    __device__ State load(int i, int j) const {
        const int64_t o = (int64_t)j * ldn + i;
        return State{Wx[o], Zx[o], active[j]};
    }
    __device__ float apply(int i, int j, float acc, const State& st, float* red) const {
        if (!st.act) return 0.0f;
        const int64_t o = (int64_t)j * ldn + i;
        const float dw = -beta[j] * (st.z - acc);
        const float wn = st.w + dw;
        Wx[o] = wn;
        const float v = fmaf(wn, binv[j], acc);
        const float z = clamp_unit(v);
        Zx[o] = z;
        const float vx = z - v;
        Vx[o] = vx;
        red[0] += dw * dw;
        red[1] += st.w * st.w;
        return vx;
    }
};

// ---------------------------------------- DALM with a conjugate-gradient y-step
// One CG step on (B B^T) y = B z_{k+1} - (B w_k - b)/beta from y_k (§V-B's
// inexact alternative to the factor; reading R15): its residual is
// r_0 = B V + b/beta = d (the same d as above), p = d, and
// y_{k+1} = y_k + alpha d with alpha = ||d||^2 / (d^T B B^T d)
//                                    = ||d||^2 / ||B^T d||^2.

// T1' (rows of A, acc = A V_x): d as in EpiTcD, also stored in FP32 (the
// y-step adds alpha d); red: ||d||^2.
struct EpiCgD {
    static constexpr int NRED = 1;
    struct State {
        float b, ve;
        int act;
    };
    float* D;
    const float* Ve;
    const float* B;
    const float* binv;
    const int32_t* active;
    int64_t ldm;
    int cab;
    __device__ State load(int i, int j) const {
        const int64_t o = (int64_t)j * ldm + i;
        return State{B[o], cab ? Ve[o] : 0.0f, active[j]};
    }
    __device__ float apply(int i, int j, float acc, const State& st, float* red) const {
        if (!st.act) return 0.0f;
        const float d = fmaf(st.b, binv[j], acc) + st.ve;
        D[(int64_t)j * ldm + i] = d;
        red[0] += d * d;
        return d;
    }
};

// T2' (rows of A^T, acc = A^T d): red: ||A^T d||^2 (the identity block of
// B^T d is d itself, whose square is T1's term).  Nothing is stored.
struct EpiCgQ {
    static constexpr int NRED = 1;
    struct State {
        int act;
    };
    const int32_t* active;
    __device__ State load(int, int j) const { return State{active[j]}; }
    __device__ float apply(int, int, float acc, const State& st, float* red) const {
        if (st.act) red[0] += acc * acc;
        return 0.0f;
    }
};

// ------------------------------------- AMP epilogues of the tensor-core engine
// Approximate message passing for P1 (§IV, reading R18): x in Wx, z in Y;
// the A^T z sweep reads the BF16 pieces of z and the A x sweep those of x,
// which these functors return.  Per column: tau_k (FP32 copy) and the z-step
// coefficient (n/m) <eta'>, both set by ctrl_amp_kernel.

// AX (rows of A^T, acc = A^T z_k): x_{k+1} = soft(acc + x_k, tau_k).
// red: ||x_{k+1} - x_k||^2, ||x_k||^2, the count of |v_i| > tau_k.
struct EpiTcAmpX {
    static constexpr int NRED = 3;
    struct State {
        float x;
        int act;
    };
    float* Wx;
    const float* tau;
    const int32_t* active;
    int64_t ldn;
    __device__ State load(int i, int j) const { return State{Wx[(int64_t)j * ldn + i], active[j]}; }
    __device__ float apply(int i, int j, float acc, const State& st, float* red) const {
        if (!st.act) return 0.0f;
        const float v = acc + st.x;
        const float t = tau[j];
        const float xn = soft_thr(v, t);
        Wx[(int64_t)j * ldn + i] = xn;
        const float dx = xn - st.x;
        red[0] += dx * dx;
        red[1] += st.x * st.x;
        red[2] += fabsf(v) > t ? 1.0f : 0.0f;
        return xn;
    }
};

// AZ (rows of A, acc = A x_{k+1}): z_{k+1} = b - acc + coef_j z_k.
struct EpiTcAmpZ {
    static constexpr int NRED = 0;
    struct State {
        float z, b;
        int act;
    };
    float* Y;
    const float* B;
    const float* coef;
    const int32_t* active;
    int64_t ldm;
    __device__ State load(int i, int j) const {
        const int64_t o = (int64_t)j * ldm + i;
        return State{Y[o], B[o], active[j]};
    }
    __device__ float apply(int i, int j, float acc, const State& st, float*) const {
        if (!st.act) return 0.0f;
        const float zn = fmaf(coef[j], st.z, st.b - acc);
        Y[(int64_t)j * ldm + i] = zn;
        return zn;
    }
};

int tc_sweep(Handle* h, int M, int N, int K, const tc16::Operands& op, const tc16::Terms& tl, const EpiTcAmpX& epi,
             const tc16::PieceOut& po, double* part, const int32_t* active);
int tc_sweep(Handle* h, int M, int N, int K, const tc16::Operands& op, const tc16::Terms& tl, const EpiTcAmpZ& epi,
             const tc16::PieceOut& po, double* part, const int32_t* active);
int tc_sweep(Handle* h, int M, int N, int K, const tc16::Operands& op, const tc16::Terms& tl, const EpiTcD& epi,
             const tc16::PieceOut& po, double* part, const int32_t* active);
int tc_sweep(Handle* h, int M, int N, int K, const tc16::Operands& op, const tc16::Terms& tl, const EpiCgD& epi,
             const tc16::PieceOut& po, double* part, const int32_t* active);
int tc_sweep(Handle* h, int M, int N, int K, const tc16::Operands& op, const tc16::Terms& tl, const EpiCgQ& epi,
             const tc16::PieceOut& po, double* part, const int32_t* active);
// The y-epilogue (EpiTcY) applied to acc = alpha_j S(i, j) (S: m x N, leading
// dimension lds) instead of a sweep's sums: the CG y-step.  Returns the
// number of row blocks.
int tc_scaled_y(Handle* h, int M, int N, const float* S, int64_t lds, const float* alpha, const EpiTcY& epi,
                const tc16::PieceOut& po, double* part, const int32_t* active);
int tc_sweep(Handle* h, int M, int N, int K, const tc16::Operands& op, const tc16::Terms& tl, const EpiTcY& epi,
             const tc16::PieceOut& po, double* part, const int32_t* active);
int tc_sweep(Handle* h, int M, int N, int K, const tc16::Operands& op, const tc16::Terms& tl, const EpiTcS& epi,
             const tc16::PieceOut& po, double* part, const int32_t* active);

}  // namespace l1
