// l1_solve_plain: DALM (Algorithm 2, reading R1) for ONE right-hand side in
// plain FP32, one simple kernel per step and the stopping rule (§VI-C) read
// on the host after every iteration.  It is the unbatched, unfused baseline
// the batched solver is measured against: no panels, no fused epilogues, no
// tensor cores, no graphs.  It uses the handle's FP32 layouts of A and the
// FP32 (B B^T)^{-1} (high part only).
#include <cmath>

#include "common.cuh"

namespace l1 {
namespace {

constexpr int kThreads = 256;

// out(i) = sum_k M(i, k) v(k) for a row-major M (rows of length K, pitch ld):
// one warp per row, FP32 accumulation
__global__ void plain_gemv_kernel(const float* __restrict__ Mrm, int64_t ld, int rows, int K,
                                  const float* __restrict__ v, float* __restrict__ out) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= rows) return;
    const float* row = Mrm + (int64_t)warp * ld;
    float s = 0.0f;
    for (int k = lane; k < K; k += 32) s = fmaf(row[k], v[k], s);
    s = warp_sum_f(s);
    if (lane == 0) out[warp] = s;
}

// z = P_[-1,1](B^T y + w/beta) (Eq. 38), u = z - w/beta
__global__ void plain_z_kernel(const float* bty, const float* w, float binv, int len, float* z, float* u) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    const float wb = w[i] * binv;
    const float zi = clamp_unit(bty[i] + wb);
    z[i] = zi;
    u[i] = zi - wb;
}

// right-hand side of Eq. 39: B u + b/beta (the identity block of B adds u_e)
__global__ void plain_rhs_kernel(float* r, const float* u_e, const float* b, float binv, int m) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    float v = fmaf(b[i], binv, r[i]);
    if (u_e) v += u_e[i];
    r[i] = v;
}

// the identity block of B^T y
__global__ void plain_copy_kernel(const float* src, float* dst, int len) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) dst[i] = src[i];
}

// w-step: dw = -beta (z - B^T y), w += dw; per-block partials of ||dw||^2,
// ||w||^2 and ||w'||_1 (FP64, summed in block order by plain_sum_kernel)
__global__ void plain_w_kernel(const float* z, const float* bty, float beta, int len, float* w, double* part) {
    __shared__ double sh[3][kThreads / 32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double d2 = 0.0, w2 = 0.0, w1 = 0.0;
    if (i < len) {
        const float wi = w[i];
        const float dw = -beta * (z[i] - bty[i]);
        const float wn = wi + dw;
        w[i] = wn;
        d2 = (double)dw * dw;
        w2 = (double)wi * wi;
        w1 = fabs((double)wn);
    }
    d2 = warp_sum(d2);
    w2 = warp_sum(w2);
    w1 = warp_sum(w1);
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = d2;
        sh[1][threadIdx.x >> 5] = w2;
        sh[2][threadIdx.x >> 5] = w1;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int k = 0; k < kThreads / 32; ++k) s += sh[threadIdx.x][k];
        part[(int64_t)blockIdx.x * 3 + threadIdx.x] = s;
    }
}

__global__ void plain_sum_kernel(const double* part, int nblk, int nvals, double* out) {
    const int r = threadIdx.x;
    if (r >= nvals) return;
    double s = 0.0;
    for (int k = 0; k < nblk; ++k) s += part[(int64_t)k * nvals + r];
    out[r] = s;
}

// ||b||_1 (beta = ||b||_1 / m, reading R2)
__global__ void plain_l1_kernel(const float* b, int m, double* out) {
    __shared__ double sh[kThreads / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) s += fabs((double)b[i]);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kThreads / 32; ++k) t += sh[k];
        *out = t;
    }
}

}  // namespace
}  // namespace l1

using namespace l1;

extern "C" L1_API int l1_solve_plain(l1_handle hh, const float* b, double tol, int32_t max_iter, float* x,
                                     l1_result* res) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !b || !x || !res || max_iter <= 0 || !(tol >= 0.0)) return L1_ERR_INVALID_ARG;
    if (h->grp || h->opt.unroll_K > 0 || !h->F || (h->mode != L1_CAB && h->mode != L1_P1)) return L1_ERR_UNSUPPORTED;
    const int m = (int)h->m, n = (int)h->n;
    const bool cab = h->mode == L1_CAB;
    const int len = cab ? n + m : n;
    cudaStream_t s = h->stream;
    const int nblk = (len + kThreads - 1) / kThreads;
    float* buf = nullptr;
    double* dbuf = nullptr;
    double hsum[4] = {0.0, 0.0, 0.0, 0.0};
    // w, z, u, bty (len each), b, r, y (m each)
    const size_t nf = 4 * (size_t)len + 3 * (size_t)m;
    L1_CUDA_TRY(cudaMalloc(&buf, sizeof(float) * nf));
    if (cudaMalloc(&dbuf, sizeof(double) * (3 * (size_t)nblk + 4)) != cudaSuccess) {
        cudaFree(buf);
        set_last_error("l1_solve_plain: allocation failed");
        return L1_ERR_OOM;
    }
    float *w = buf, *z = w + len, *u = z + len, *bty = u + len, *bd = bty + len, *r = bd + m, *y = r + m;
    double* part = dbuf;
    double* sums = dbuf + 3 * (size_t)nblk;
    int rc = L1_OK;
    l1_result out{};
    out.label = out.sci_label = -1;
    do {
        if (cudaMemcpyAsync(bd, b, sizeof(float) * m, cudaMemcpyDefault, s) != cudaSuccess ||
            cudaMemsetAsync(w, 0, sizeof(float) * len, s) != cudaSuccess ||
            cudaMemsetAsync(bty, 0, sizeof(float) * len, s) != cudaSuccess) {
            rc = L1_ERR_CUDA;
            break;
        }
        plain_l1_kernel<<<1, kThreads, 0, s>>>(bd, m, sums);
        ++h->launches;
        if (cudaMemcpyAsync(hsum, sums, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            rc = L1_ERR_CUDA;
            break;
        }
        const double beta = hsum[0] > 0.0 ? hsum[0] / m : 1.0;
        const float fb = (float)beta, fbi = (float)(1.0 / beta);
        const int gl = (len + kThreads - 1) / kThreads, gm = (m + kThreads - 1) / kThreads;
        out.status = L1_MAX_ITER;
        out.param = beta;
        int it = 0;
        double rel = INFINITY;
        for (it = 1; it <= max_iter; ++it) {
            // Algorithm 2: z-step, y-step through (B B^T)^{-1}, w-step
            plain_z_kernel<<<gl, kThreads, 0, s>>>(bty, w, fbi, len, z, u);
            plain_gemv_kernel<<<(m * 32 + kThreads - 1) / kThreads, kThreads, 0, s>>>(h->A_rm, h->ldn, m, n, u, r);
            plain_rhs_kernel<<<gm, kThreads, 0, s>>>(r, cab ? u + n : nullptr, bd, fbi, m);
            plain_gemv_kernel<<<(m * 32 + kThreads - 1) / kThreads, kThreads, 0, s>>>(h->F, h->ldm, m, m, r, y);
            plain_gemv_kernel<<<(n * 32 + kThreads - 1) / kThreads, kThreads, 0, s>>>(h->A_cm, h->ldm, n, m, y, bty);
            if (cab) plain_copy_kernel<<<gm, kThreads, 0, s>>>(y, bty + n, m);
            plain_w_kernel<<<nblk, kThreads, 0, s>>>(z, bty, fb, len, w, part);
            plain_sum_kernel<<<1, 32, 0, s>>>(part, nblk, 3, sums);
            h->launches += cab ? 8 : 7;
            if (cudaMemcpyAsync(hsum, sums, sizeof(double) * 3, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                rc = L1_ERR_CUDA;
                break;
            }
            rel = rel_change(std::sqrt(hsum[0]), std::sqrt(hsum[1]));
            if (!std::isfinite(hsum[0]) || !std::isfinite(hsum[1])) {
                out.status = L1_NONFINITE;
                break;
            }
            if (rel < tol) {
                out.status = L1_CONVERGED;
                break;
            }
        }
        if (rc != L1_OK) break;
        out.iters = out.inner_iters = it > max_iter ? max_iter : it;
        out.rel_change = rel;
        out.primal_obj = hsum[2];
        out.dual_obj = out.gap = out.resid = NAN;
        if (cudaMemcpyAsync(x, w, sizeof(float) * len, cudaMemcpyDefault, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            rc = L1_ERR_CUDA;
    } while (false);
    if (rc == L1_ERR_CUDA) set_last_error(std::string("l1_solve_plain: ") + cudaGetErrorString(cudaGetLastError()));
    cudaFree(buf);
    cudaFree(dbuf);
    if (rc == L1_OK) *res = out;
    return rc;
}
