// l1_align_batch: the convex step of the face-alignment loop (§II-B): for
// each problem k, min ||e||_1 s.t. b_k = B_k w + e, with B_k tall (m x p,
// p <= 32: training images of one subject beside the negated Jacobian of the
// transformation) and w not penalised.  Reading R16: Algorithm 1 with its
// x-step replaced by the exact minimiser of the augmented Lagrangian over w,
//   e_{j+1}     = shrink(b - B w_j + theta_j/xi, 1/xi)
//   w_{j+1}     = (B^T B)^{-1} B^T (b - e_{j+1} + theta_j/xi)
//   theta_{j+1} = theta_j + xi (b - B w_{j+1} - e_{j+1}),
// from w = 0, e = b, theta = 0, xi = 2m/||b||_1 (or xi0), stopping on the
// relative change of [w; e] (§VI-C).
//
// One CTA per problem runs the whole loop: B_k, b, e, theta and B w in
// shared memory (the problem is touched in HBM once), (B^T B)^{-1} formed in
// FP64 in the CTA (Gauss-Jordan on p x p with the Cholesky pivot test), the
// products B^T t and B w in FP32 over the rows, the p-vector solve and every
// reduction of the stopping rule in FP64.
#include <cmath>

#include "common.cuh"

namespace l1 {
namespace {

constexpr int kAThreads = 256;
constexpr int kAWarps = kAThreads / 32;
constexpr int kAMaxP = 32;

__device__ __forceinline__ float soft_a(float v, float a) { return v > a ? v - a : (v < -a ? v + a : 0.0f); }

struct AlignOut {
    int32_t status, iters;
    double rel, l1e, param;
};

// dynamic shared memory: Bs[m * p] (column-major), bv[m], ev[m], th[m],
// bw[m] (floats); then doubles: G[p * p], Gi[p * p], rhs[p], wv[p], red[...]
__global__ void __launch_bounds__(kAThreads) align_kernel(const float* __restrict__ B, int m, int p, int64_t ldB,
                                                          int64_t strideB, const float* __restrict__ b,
                                                          int64_t strideb, double tol, int max_outer, double xi0,
                                                          float* __restrict__ w_out, float* __restrict__ e_out,
                                                          AlignOut* __restrict__ out,
                                                          const int32_t* __restrict__ active) {
    extern __shared__ __align__(16) unsigned char asm_raw[];
    const int k = blockIdx.x, t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (active != nullptr && !active[k]) return;  // the whole CTA, before any barrier
    double* G = reinterpret_cast<double*>(asm_raw);
    double* Gi = G + kAMaxP * kAMaxP;
    double* rhs = Gi + kAMaxP * kAMaxP;
    double* wv = rhs + kAMaxP;
    double* red = wv + kAMaxP;  // [4][kAWarps]
    float* Bs = reinterpret_cast<float*>(red + 4 * kAWarps);
    float* bv = Bs + (size_t)m * p;
    float* ev = bv + m;
    float* th = ev + m;
    float* bw = th + m;
    __shared__ float rhs_f[kAMaxP];
    __shared__ int flag;

    const float* Bk = B + (size_t)k * strideB;
    const float* bk = b + (size_t)k * strideb;
    for (int j = 0; j < p; ++j)
        for (int i = t; i < m; i += kAThreads) Bs[(size_t)j * m + i] = Bk[(size_t)j * ldB + i];
    double b1 = 0.0;
    for (int i = t; i < m; i += kAThreads) {
        const float v = bk[i];
        bv[i] = v;
        ev[i] = v;  // e_1 = b
        th[i] = 0.0f;
        bw[i] = 0.0f;
        b1 += fabs((double)v);
    }
    b1 = warp_sum(b1);
    if (lane == 0) red[warp] = b1;
    __syncthreads();
    // G = B^T B (FP32 products, FP64 sums): one warp per entry of the upper triangle
    for (int q = warp; q < p * p; q += kAWarps) {
        const int r = q / p, c = q % p;
        if (c < r) continue;
        double s = 0.0;
        for (int i = lane; i < m; i += 32) s += (double)Bs[(size_t)r * m + i] * Bs[(size_t)c * m + i];
        s = warp_sum(s);
        if (lane == 0) {
            G[r * kAMaxP + c] = s;
            G[c * kAMaxP + r] = s;
        }
    }
    __syncthreads();
    // (B^T B)^{-1} by Gauss-Jordan without pivoting (the matrix is SPD; a
    // pivot below 16 p eps G_jj marks it singular), FP64, one thread
    if (t == 0) {
        double bsum = 0.0;
        for (int w = 0; w < kAWarps; ++w) bsum += red[w];
        red[3 * kAWarps] = bsum;
        flag = 1;
        double d0[kAMaxP];
        for (int r = 0; r < p; ++r) {
            d0[r] = G[r * kAMaxP + r];
            for (int c = 0; c < p; ++c) Gi[r * kAMaxP + c] = (r == c) ? 1.0 : 0.0;
        }
        for (int j = 0; j < p && flag; ++j) {
            // the pivot is the Schur complement's diagonal, as in a Cholesky
            // factorisation: below 16 p eps of the original diagonal, B^T B
            // is singular to working precision
            const double piv = G[j * kAMaxP + j];
            if (!(piv > 16.0 * p * 2.220446049250313e-16 * d0[j])) {
                flag = 0;
                break;
            }
            const double inv = 1.0 / piv;
            for (int c = 0; c < p; ++c) {
                G[j * kAMaxP + c] *= inv;
                Gi[j * kAMaxP + c] *= inv;
            }
            for (int r = 0; r < p; ++r) {
                if (r == j) continue;
                const double f = G[r * kAMaxP + j];
                if (f == 0.0) continue;
                for (int c = 0; c < p; ++c) {
                    G[r * kAMaxP + c] -= f * G[j * kAMaxP + c];
                    Gi[r * kAMaxP + c] -= f * Gi[j * kAMaxP + c];
                }
            }
        }
    }
    if (t < p) wv[t] = 0.0;
    __syncthreads();
    if (!flag) {
        if (t == 0) out[k] = AlignOut{L1_NONFINITE, 0, NAN, NAN, NAN};
        for (int j = t; j < p; j += kAThreads) w_out[(size_t)k * p + j] = NAN;
        for (int i = t; i < m; i += kAThreads) e_out[(size_t)k * m + i] = NAN;
        return;
    }
    const double bsum = red[3 * kAWarps];
    const double xi = xi0 > 0.0 ? xi0 : (bsum > 0.0 ? 2.0 * m / bsum : 1.0);
    const float fxi = (float)xi, fxinv = (float)(1.0 / xi);
    int it = 0, status = L1_MAX_ITER;
    double rel = INFINITY;
    for (it = 1; it <= max_outer; ++it) {
        // e-step and t = b - e + theta/xi (kept in bw, which the w-step refills)
        double de2 = 0.0, e2 = 0.0;
        for (int i = t; i < m; i += kAThreads) {
            const float c = bv[i] + th[i] * fxinv;
            const float en = soft_a(c - bw[i], fxinv);
            const float eo = ev[i];
            de2 += (double)(en - eo) * (en - eo);
            e2 += (double)eo * eo;
            ev[i] = en;
            bw[i] = c - en;
        }
        de2 = warp_sum(de2);
        e2 = warp_sum(e2);
        if (lane == 0) {
            red[warp] = de2;
            red[kAWarps + warp] = e2;
        }
        __syncthreads();
        // B^T t: one warp per column
        for (int j = warp; j < p; j += kAWarps) {
            float s = 0.0f;
            for (int i = lane; i < m; i += 32) s = fmaf(Bs[(size_t)j * m + i], bw[i], s);
            s = warp_sum_f(s);
            if (lane == 0) rhs_f[j] = s;
        }
        __syncthreads();
        // w-step in FP64 by p threads; the w part of the stopping rule
        double dw2 = 0.0, w2 = 0.0, wn = 0.0;
        if (t < p) {
            for (int c = 0; c < p; ++c) wn += Gi[t * kAMaxP + c] * (double)rhs_f[c];
            const double wo = wv[t];
            dw2 = (wn - wo) * (wn - wo);
            w2 = wo * wo;
        }
        __syncthreads();  // every thread has read wv
        if (t < p) wv[t] = wn;
        if (warp == 0) {
            dw2 = warp_sum(dw2);
            w2 = warp_sum(w2);
            if (lane == 0) {
                red[2 * kAWarps] = dw2;
                red[2 * kAWarps + 1] = w2;
            }
        }
        __syncthreads();
        // B w and the multiplier step
        float wf[kAMaxP];
#pragma unroll
        for (int j = 0; j < kAMaxP; ++j) wf[j] = j < p ? (float)wv[j] : 0.0f;
        for (int i = t; i < m; i += kAThreads) {
            float s = 0.0f;
#pragma unroll
            for (int j = 0; j < kAMaxP; ++j)
                if (j < p) s = fmaf(Bs[(size_t)j * m + i], wf[j], s);
            bw[i] = s;
            th[i] = fmaf(fxi, bv[i] - s - ev[i], th[i]);
        }
        // relative change of [w; e] (every thread sums the warp partials in
        // the same order)
        double d2 = red[2 * kAWarps], base2 = red[2 * kAWarps + 1];
        for (int w = 0; w < kAWarps; ++w) {
            d2 += red[w];
            base2 += red[kAWarps + w];
        }
        rel = rel_change(sqrt(d2), sqrt(base2));
        __syncthreads();  // red is rewritten by the next e-step
        if (!isfinite(d2) || !isfinite(base2)) {
            status = L1_NONFINITE;
            break;
        }
        if (rel < tol) {
            status = L1_CONVERGED;
            break;
        }
    }
    // outputs: w, e, ||e||_1
    double l1e = 0.0;
    for (int i = t; i < m; i += kAThreads) {
        const float v = ev[i];
        e_out[(size_t)k * m + i] = v;
        l1e += fabs((double)v);
    }
    if (t < p) w_out[(size_t)k * p + t] = (float)wv[t];
    l1e = warp_sum(l1e);
    if (lane == 0) red[warp] = l1e;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < kAWarps; ++w) s += red[w];
        out[k] = AlignOut{status, it > max_outer ? max_outer : it, rel, s, xi};
    }
}

}  // namespace

size_t align_smem_bytes(int m, int p) {
    return sizeof(double) * (2 * kAMaxP * kAMaxP + 2 * kAMaxP + 4 * kAWarps) + sizeof(float) * ((size_t)m * p + 4 * (size_t)m);
}

}  // namespace l1

using namespace l1;

namespace l1 {

// l1_align_batch over the problems whose flag in active (device, count
// entries; NULL: all) is set; the others are not touched (their CTAs return
// at once) and their res entries are zero.
int align_batch_run(const float* B, int64_t m, int64_t p, int64_t ldB, int64_t strideB, const float* b,
                    int64_t strideb, int64_t count, double tol, int32_t max_outer, double xi0, void* stream, float* w,
                    float* e, l1_result* res, const int32_t* active);

}  // namespace l1

extern "C" L1_API int l1_align_batch(const float* B, int64_t m, int64_t p, int64_t ldB, int64_t strideB,
                                     const float* b, int64_t strideb, int64_t count, double tol, int32_t max_outer,
                                     double xi0, void* stream, float* w, float* e, l1_result* res) {
    return align_batch_run(B, m, p, ldB, strideB, b, strideb, count, tol, max_outer, xi0, stream, w, e, res, nullptr);
}

int l1::align_batch_run(const float* B, int64_t m, int64_t p, int64_t ldB, int64_t strideB, const float* b,
                        int64_t strideb, int64_t count, double tol, int32_t max_outer, double xi0, void* stream,
                        float* w, float* e, l1_result* res, const int32_t* active) {
    if (!B || !b || !w || !e || !res || m <= 0 || p <= 0 || p > kAMaxP || p >= m || ldB < m ||
        strideB < ldB * p || strideb < m || count <= 0 || count > (1 << 30) || max_outer <= 0 || !(tol >= 0.0))
        return L1_ERR_INVALID_ARG;
    const size_t smem = align_smem_bytes((int)m, (int)p);
    if (smem > 200 * 1024) {
        set_last_error("l1_align_batch: m x p too large for one CTA's shared memory");
        return L1_ERR_INVALID_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    AlignOut* dout = nullptr;
    if (cudaMalloc(&dout, sizeof(AlignOut) * (size_t)count) != cudaSuccess) {
        cudaGetLastError();
        return L1_ERR_OOM;
    }
    int rc = L1_OK;
    std::vector<AlignOut> hout((size_t)count);
    do {
        if (active != nullptr && cudaMemsetAsync(dout, 0, sizeof(AlignOut) * (size_t)count, s) != cudaSuccess) {
            rc = L1_ERR_CUDA;
            break;
        }
        if (cudaFuncSetAttribute(align_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess) {
            rc = L1_ERR_CUDA;
            break;
        }
        align_kernel<<<(unsigned)count, kAThreads, smem, s>>>(B, (int)m, (int)p, ldB, strideB, b, strideb, tol,
                                                              max_outer, xi0, w, e, dout, active);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(hout.data(), dout, sizeof(AlignOut) * (size_t)count, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            rc = L1_ERR_CUDA;
            break;
        }
    } while (false);
    if (rc == L1_ERR_CUDA) set_last_error(std::string("l1_align_batch: ") + cudaGetErrorString(cudaGetLastError()));
    cudaFree(dout);
    if (rc != L1_OK) return rc;
    for (int64_t k = 0; k < count; ++k) {
        l1_result r{};
        r.status = hout[k].status;
        r.iters = r.inner_iters = hout[k].iters;
        r.label = r.sci_label = -1;
        r.rel_change = hout[k].rel;
        r.primal_obj = hout[k].l1e;
        r.dual_obj = r.gap = r.resid = NAN;
        r.param = hout[k].param;
        res[k] = r;
    }
    return L1_OK;
}
