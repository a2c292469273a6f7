// The image side of the face-alignment loop of §II-B (reading R19): the warp
// b = y o tau of a query image by a similarity tau and its Jacobian
// J = d(y o tau)/d tau as CUDA kernels (l1_align_warp), and the loop itself
// (l1_align_images): per task, b and J at the current tau, the convex step
// min ||e||_1 s.t. b = [A, -J] w + e of l1_align_batch, tau <- tau + dtau
// with dtau the last four entries of w, until the step moves no corner of
// the canonical frame by tau_tol pixels or more.
//
// tau = (a, b, tx, ty): canonical pixel (u, v) (column u < cols, row v <
// rows, vector index v cols + u) lies at x = a u - b v + tx, y = b u + a v +
// ty of the query image (H x W, row-major, pixel (y, x) at y W + x).  y o tau
// is the bilinear interpolant of the query there, the point first clamped to
// [0, W-1] x [0, H-1], the cell the one with lower corner (min(floor(x),
// W-2), min(floor(y), H-2)); its x- (y-) derivative is the interpolant's
// slope in that cell, and 0 where x (y) was clamped.  Coordinates, weights
// and sums are FP64, the pixels FP32.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace l1 {

// l1_align_batch restricted to the problems whose device flag is set (align.cu)
int align_batch_run(const float* B, int64_t m, int64_t p, int64_t ldB, int64_t strideB, const float* b,
                    int64_t strideb, int64_t count, double tol, int32_t max_outer, double xi0, void* stream, float* w,
                    float* e, l1_result* res, const int32_t* active);

namespace {

constexpr int kWarpThreads = 256;

// One thread per (canonical pixel, task): b_k and the four columns col0 ..
// col0 + 3 of B_k set to -J (the convex step's B = [A, -J]).
__global__ void __launch_bounds__(kWarpThreads)
warp_kernel(const float* __restrict__ img, int H, int W, int64_t img_stride, const double* __restrict__ tau, int rows,
            int cols, int col0, float* __restrict__ B, int64_t ldB, int64_t strideB, float* __restrict__ b,
            int64_t strideb, const int32_t* __restrict__ active) {
    const int64_t k = blockIdx.y;
    const int r = blockIdx.x * kWarpThreads + threadIdx.x;
    const int m = rows * cols;
    if (r >= m || (active != nullptr && !active[k])) return;
    const double u = (double)(r % cols), v = (double)(r / cols);
    const double ta = tau[4 * k + 0], tb = tau[4 * k + 1], tx = tau[4 * k + 2], ty = tau[4 * k + 3];
    const double x = __dadd_rn(__dadd_rn(__dmul_rn(ta, u), -__dmul_rn(tb, v)), tx);
    const double y = __dadd_rn(__dadd_rn(__dmul_rn(tb, u), __dmul_rn(ta, v)), ty);
    const double xc = fmin(fmax(x, 0.0), (double)(W - 1)), yc = fmin(fmax(y, 0.0), (double)(H - 1));
    const int x0 = min((int)floor(xc), W - 2), y0 = min((int)floor(yc), H - 2);
    const double fx = xc - x0, fy = yc - y0;
    const float* q = img + k * img_stride + (int64_t)y0 * W + x0;
    const double p00 = q[0], p01 = q[1], p10 = q[W], p11 = q[W + 1];
    const double val = (1.0 - fy) * ((1.0 - fx) * p00 + fx * p01) + fy * ((1.0 - fx) * p10 + fx * p11);
    const double gx = (x >= 0.0 && x <= (double)(W - 1)) ? (1.0 - fy) * (p01 - p00) + fy * (p11 - p10) : 0.0;
    const double gy = (y >= 0.0 && y <= (double)(H - 1)) ? (1.0 - fx) * (p10 - p00) + fx * (p11 - p01) : 0.0;
    b[k * strideb + r] = (float)val;
    float* Bk = B + k * strideB + (int64_t)col0 * ldB + r;
    // dx/dtau = (u, -v, 1, 0), dy/dtau = (v, u, 0, 1)
    Bk[0] = (float)-(gx * u + gy * v);
    Bk[ldB] = (float)-(-gx * v + gy * u);
    Bk[2 * ldB] = (float)-gx;
    Bk[3 * ldB] = (float)-gy;
}

// The training images of each task into the first n columns of B_k.
__global__ void copy_train_kernel(const float* __restrict__ A, int64_t A_stride, int m, int n, float* __restrict__ B,
                                  int64_t ldB, int64_t strideB) {
    const int64_t k = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)m * n) return;
    const int c = (int)(i / m), r = (int)(i % m);
    B[k * strideB + (int64_t)c * ldB + r] = A[k * A_stride + i];
}

// tau <- tau + dtau (dtau = w[n .. n+3]) for the active tasks, and the
// loop's stopping rule: the largest corner displacement of dtau below
// tau_tol -> converged; a convex step that failed or a dtau that is not
// finite -> L1_NONFINITE; max_align steps -> L1_MAX_ITER.
__global__ void tau_update_kernel(double* __restrict__ tau, const float* __restrict__ w, int p, int n, int rows,
                                  int cols, const int32_t* __restrict__ step_status, double tau_tol, int max_align,
                                  int count, int32_t* __restrict__ active, int32_t* __restrict__ iters,
                                  int32_t* __restrict__ status) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count || !active[k]) return;
    const int it = iters[k] + 1;
    iters[k] = it;
    double d[4];
    bool finite = step_status[k] != L1_NONFINITE;
    for (int t = 0; t < 4; ++t) {
        d[t] = (double)w[(int64_t)k * p + n + t];
        finite = finite && isfinite(d[t]);
    }
    if (!finite) {
        status[k] = L1_NONFINITE;
        active[k] = 0;
        return;
    }
    for (int t = 0; t < 4; ++t) tau[4 * k + t] += d[t];
    double shift = 0.0;
    const double cu[4] = {0.0, (double)(cols - 1), 0.0, (double)(cols - 1)};
    const double cv[4] = {0.0, 0.0, (double)(rows - 1), (double)(rows - 1)};
    for (int c = 0; c < 4; ++c) {
        const double dx = d[0] * cu[c] - d[1] * cv[c] + d[2], dy = d[1] * cu[c] + d[0] * cv[c] + d[3];
        shift = fmax(shift, sqrt(dx * dx + dy * dy));
    }
    if (shift < tau_tol) {
        status[k] = L1_CONVERGED;
        active[k] = 0;
    } else if (it >= max_align) {
        status[k] = L1_MAX_ITER;
        active[k] = 0;
    }
}

__global__ void count_flags_kernel(const int32_t* __restrict__ active, int count, int32_t* __restrict__ out) {
    __shared__ int sh[32];
    int s = 0;
    for (int k = threadIdx.x; k < count; k += blockDim.x) s += active[k] != 0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        *out = t;
    }
}

bool warp_args_ok(const float* img, int64_t H, int64_t W, int64_t img_stride, const double* tau, int64_t count,
                  int32_t rows, int32_t cols) {
    return img && tau && H >= 2 && W >= 2 && H <= (1 << 15) && W <= (1 << 15) && img_stride >= H * W &&
           count > 0 && count <= 65535 && rows > 0 && cols > 0 && (int64_t)rows * cols <= (1 << 20);
}

}  // namespace
}  // namespace l1

using namespace l1;

extern "C" L1_API int l1_align_warp(const float* img, int64_t H, int64_t W, int64_t img_stride, const double* tau,
                                    int64_t count, int32_t rows, int32_t cols, int32_t col0, void* stream, float* B,
                                    int64_t ldB, int64_t strideB, float* b, int64_t strideb,
                                    const int32_t* active) {
    const int64_t m = (int64_t)rows * cols;
    if (!warp_args_ok(img, H, W, img_stride, tau, count, rows, cols) || !B || !b || col0 < 0 || ldB < m ||
        strideB < ldB * (col0 + 4) || strideb < m)
        return L1_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    dim3 grid((unsigned)((m + kWarpThreads - 1) / kWarpThreads), (unsigned)count);
    warp_kernel<<<grid, kWarpThreads, 0, s>>>(img, (int)H, (int)W, img_stride, tau, rows, cols, col0, B, ldB, strideB,
                                             b, strideb, active);
    if (cudaGetLastError() != cudaSuccess) {
        set_last_error("l1_align_warp: launch failed");
        return L1_ERR_CUDA;
    }
    return L1_OK;
}

extern "C" L1_API int l1_align_images(const float* img, int64_t H, int64_t W, int64_t img_stride, const float* A,
                                      int32_t n, int64_t A_stride, int32_t rows, int32_t cols, int64_t count,
                                      double* tau, double tol, int32_t max_outer, double tau_tol, int32_t max_align,
                                      void* stream, int32_t* iters, int32_t* status) {
    const int64_t m = (int64_t)rows * cols;
    const int p = n + 4;
    if (!warp_args_ok(img, H, W, img_stride, tau, count, rows, cols) || !A || !iters || !status || n <= 0 ||
        p > 32 || p >= m || A_stride < m * n || !(tol >= 0.0) || max_outer <= 0 || !(tau_tol >= 0.0) ||
        max_align <= 0)
        return L1_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t ldB = m, strideB = m * p;
    float *B = nullptr, *b = nullptr, *w = nullptr, *e = nullptr;
    int32_t *flags = nullptr;  // active, iters, status, step status [count each], count of active
    const size_t need_f = (size_t)count * (strideB + 2 * m + p);
    if (cudaMalloc(&B, sizeof(float) * need_f) != cudaSuccess ||
        cudaMalloc(&flags, sizeof(int32_t) * (4 * (size_t)count + 1)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(B);
        return L1_ERR_OOM;
    }
    b = B + (size_t)count * strideB;
    e = b + (size_t)count * m;
    w = e + (size_t)count * m;
    int32_t* d_active = flags;
    int32_t* d_iters = flags + count;
    int32_t* d_status = flags + 2 * count;
    int32_t* d_step = flags + 3 * count;
    int32_t* d_count = flags + 4 * count;
    int rc = L1_OK;
    std::vector<l1_result> res((size_t)count);
    std::vector<int32_t> hstep((size_t)count), hact((size_t)count, 1), hstat((size_t)count, L1_MAX_ITER);
    do {
        if (cudaMemcpyAsync(d_active, hact.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(d_status, hstat.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, s) !=
                cudaSuccess ||
            cudaMemsetAsync(d_iters, 0, sizeof(int32_t) * count, s) != cudaSuccess) {
            rc = L1_ERR_CUDA;
            break;
        }
        copy_train_kernel<<<dim3((unsigned)((m * n + 255) / 256), (unsigned)count), 256, 0, s>>>(A, A_stride, (int)m,
                                                                                                n, B, ldB, strideB);
        if (cudaGetLastError() != cudaSuccess) {
            rc = L1_ERR_CUDA;
            break;
        }
        for (int j = 0; j < max_align && rc == L1_OK; ++j) {
            rc = l1_align_warp(img, H, W, img_stride, tau, count, rows, cols, n, stream, B, ldB, strideB, b, m,
                               d_active);
            if (rc) break;
            // the convex steps of the tasks still active
            rc = align_batch_run(B, m, p, ldB, strideB, b, m, count, tol, max_outer, 0.0, stream, w, e, res.data(),
                                 d_active);
            if (rc) break;
            for (int64_t k = 0; k < count; ++k) hstep[k] = res[k].status;
            if (cudaMemcpyAsync(d_step, hstep.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, s) !=
                cudaSuccess) {
                rc = L1_ERR_CUDA;
                break;
            }
            tau_update_kernel<<<(unsigned)((count + 127) / 128), 128, 0, s>>>(tau, w, p, n, rows, cols, d_step,
                                                                             tau_tol, max_align, (int)count, d_active,
                                                                             d_iters, d_status);
            count_flags_kernel<<<1, 1024, 0, s>>>(d_active, (int)count, d_count);
            int32_t left = 0;
            if (cudaGetLastError() != cudaSuccess ||
                cudaMemcpyAsync(&left, d_count, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                rc = L1_ERR_CUDA;
                break;
            }
            if (left == 0) break;
        }
        if (rc) break;
        if (cudaMemcpyAsync(iters, d_iters, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(status, d_status, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            rc = L1_ERR_CUDA;
    } while (false);
    if (rc == L1_ERR_CUDA) set_last_error(std::string("l1_align_images: ") + cudaGetErrorString(cudaGetLastError()));
    cudaFree(B);
    cudaFree(flags);
    return rc;
}
