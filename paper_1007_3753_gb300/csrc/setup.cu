// One-time work of l1_setup (§V): layouts of A, the Lipschitz constant of
// Algorithm 1 step 6, and DALM's factor of B B^T (Eq. 39).
#include <cstdio>

#include "common.cuh"
#include "gemm_simt.cuh"
#include "setup.cuh"

namespace l1 {

// ------------------------------------------------------------ layouts of A
// src: column-major m x n with leading dimension lda (FP32, device).
// A_cm: column-major, ld = ldm (rows of A^T contiguous: K-major operand of A^T y)
// A_rm: row-major,    ld = ldn (rows of A contiguous:   K-major operand of A u)
// Padding entries are zero (the sweeps run K to a multiple of 4).
__global__ void copy_cm_kernel(const float* __restrict__ src, int64_t lda, int m, int n,
                               float* __restrict__ dst, int64_t ldm) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)ldm * n;
    if (idx >= total) return;
    const int64_t j = idx / ldm, i = idx % ldm;
    dst[idx] = i < m ? src[j * lda + i] : 0.0f;
}

__global__ void transpose_kernel(const float* __restrict__ src, int64_t lds, int m, int n,
                                 float* __restrict__ dst, int64_t ldd) {
    // dst[i * ldd + j] = src[j * lds + i]; 32x32 tiles through shared memory
    __shared__ float tile[32][33];
    const int j0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int j = j0 + r, i = i0 + threadIdx.x;
        tile[r][threadIdx.x] = (i < m && j < n) ? src[(int64_t)j * lds + i] : 0.0f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = i0 + r, j = j0 + threadIdx.x;
        if (i < m && j < ldd) dst[(int64_t)i * ldd + j] = (j < n) ? tile[threadIdx.x][r] : 0.0f;
    }
}

int make_layouts(Handle* h, const float* A_dev, int64_t lda) {
    const int m = (int)h->m, n = (int)h->n;
    {
        const int64_t total = h->ldm * n;
        copy_cm_kernel<<<(unsigned)((total + 255) / 256), 256, 0, h->stream>>>(A_dev, lda, m, n, h->A_cm, h->ldm);
        L1_LAUNCH_CHECK(h);
    }
    {
        dim3 grid((unsigned)((h->ldn + 31) / 32), (unsigned)((m + 31) / 32));
        transpose_kernel<<<grid, dim3(32, 8), 0, h->stream>>>(A_dev, lda, m, n, h->A_rm, h->ldn);
        L1_LAUNCH_CHECK(h);
    }
    return L1_OK;
}

// ------------------------------------------------ low-precision copies of A
// One block per row of a layout (rows x cols, leading dimension ld, the
// padding zero).  BF16: round to nearest even.  FP8 e4m3: scale = max |row|
// / 448 (the largest finite e4m3), q = e4m3(a / scale) rounded to nearest
// with saturation; an all-zero row keeps scale 1.
__global__ void quantize_rows_kernel(const float* __restrict__ src, int rows, int64_t ld, int prec,
                                     void* dst, float* scale) {
    __shared__ float sh[32];
    const int r = blockIdx.x;
    if (r >= rows) return;
    const float* row = src + (int64_t)r * ld;
    float sc = 1.0f;
    if (prec == L1_A_FP8E4M3) {
        float mx = 0.0f;
        for (int64_t k = threadIdx.x; k < ld; k += blockDim.x) mx = fmaxf(mx, fabsf(row[k]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
        __syncthreads();
        if (threadIdx.x == 0) {
            float m2 = 0.0f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m2 = fmaxf(m2, sh[w]);
            sh[0] = m2 > 0.0f ? m2 / 448.0f : 1.0f;
        }
        __syncthreads();
        sc = sh[0];
        if (threadIdx.x == 0) scale[r] = sc;
        uint8_t* d = static_cast<uint8_t*>(dst) + (int64_t)r * ld;
        for (int64_t k = threadIdx.x; k < ld; k += blockDim.x)
            d[k] = (uint8_t)__nv_cvt_float_to_fp8(row[k] / sc, __NV_SATFINITE, __NV_E4M3);
    } else {
        __nv_bfloat16* d = static_cast<__nv_bfloat16*>(dst) + (int64_t)r * ld;
        for (int64_t k = threadIdx.x; k < ld; k += blockDim.x) d[k] = __float2bfloat16_rn(row[k]);
    }
}

int make_lowp(Handle* h) {
    const int prec = h->opt.precision;
    const size_t es = prec == L1_A_FP8E4M3 ? 1 : 2;
    L1_TRY(dev_alloc(h, &h->A_rm_lp, es * (size_t)h->ldn * h->m));
    L1_TRY(dev_alloc(h, &h->A_cm_lp, es * (size_t)h->ldm * h->n));
    if (prec == L1_A_FP8E4M3) {
        L1_TRY(dev_alloc_t(h, &h->A_rm_scale, (size_t)h->m));
        L1_TRY(dev_alloc_t(h, &h->A_cm_scale, (size_t)h->n));
    }
    quantize_rows_kernel<<<(unsigned)h->m, 256, 0, h->stream>>>(h->A_rm, (int)h->m, h->ldn, prec, h->A_rm_lp,
                                                                 h->A_rm_scale);
    L1_LAUNCH_CHECK(h);
    quantize_rows_kernel<<<(unsigned)h->n, 256, 0, h->stream>>>(h->A_cm, (int)h->n, h->ldm, prec, h->A_cm_lp,
                                                                 h->A_cm_scale);
    L1_LAUNCH_CHECK(h);
    return L1_OK;
}

// ----------------------------------------------------- Lipschitz constant
// Power iteration on A^T A (reading of "L" in Algorithm 1 step 6 as the
// Lipschitz constant ||A||_2^2 of the smooth term's gradient, §IV-A):
// v <- A^T A v / ||A^T A v||, Rayleigh quotient rho = ||A v||^2 for ||v|| = 1.
struct EpiStore {
    static constexpr int NRED = 1;
    float* out;
    int64_t ld;
    __device__ void operator()(int i, int j, float acc, double* red) const {
        out[(int64_t)j * ld + i] = acc;
        red[0] += (double)acc * acc;
    }
};

__global__ void fill_kernel(float* p, int64_t count, float v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) p[i] = v;
}

__global__ void scale_vec_kernel(float* p, int n, const double* sumsq) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double s = *sumsq;
    if (i < n && s > 0.0) p[i] = (float)((double)p[i] / sqrt(s));
}

__global__ void sum_parts_kernel(const double* part, int np, double* out) {
    __shared__ double sh[32];
    double v = 0.0;
    for (int p = threadIdx.x; p < np; p += blockDim.x) v += part[(int64_t)p * kPartStride];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        *out = s;
    }
}

int power_iteration(Handle* h, int max_iter, double rtol, double* L_out) {
    const int m = (int)h->m, n = (int)h->n;
    float *v = nullptr, *u = nullptr;
    double *part = nullptr, *sums = nullptr, *hs = nullptr;
    const int np = std::max(sweep_row_blocks(m, 1), sweep_row_blocks(n, 1));
    int rc = L1_OK;
    cudaStream_t s = h->stream;
    if (cudaMalloc(&v, sizeof(float) * h->ldn) != cudaSuccess ||
        cudaMalloc(&u, sizeof(float) * h->ldm) != cudaSuccess ||
        cudaMalloc(&part, sizeof(double) * kPartStride * np) != cudaSuccess ||
        cudaMalloc(&sums, sizeof(double) * 2) != cudaSuccess ||
        cudaMallocHost(&hs, sizeof(double) * 2) != cudaSuccess) {
        rc = L1_ERR_OOM;
    }
    double rho = 0.0;
    if (rc == L1_OK) {
        cudaMemsetAsync(v, 0, sizeof(float) * h->ldn, s);
        cudaMemsetAsync(u, 0, sizeof(float) * h->ldm, s);
        fill_kernel<<<(n + 255) / 256, 256, 0, s>>>(v, n, (float)(1.0 / std::sqrt((double)n)));
        ++h->launches;
        for (int it = 1; it <= max_iter; ++it) {
            int np1 = launch_sweep(h, m, 1, n, h->A_rm, h->ldn, v, h->ldn, EpiStore{u, h->ldm}, part, nullptr);
            if (np1 < 0) { rc = np1; break; }
            sum_parts_kernel<<<1, 256, 0, s>>>(part, np1, sums);
            ++h->launches;
            int np2 = launch_sweep(h, n, 1, m, h->A_cm, h->ldm, u, h->ldm, EpiStore{v, h->ldn}, part, nullptr);
            if (np2 < 0) { rc = np2; break; }
            sum_parts_kernel<<<1, 256, 0, s>>>(part, np2, sums + 1);
            ++h->launches;
            scale_vec_kernel<<<(n + 255) / 256, 256, 0, s>>>(v, n, sums + 1);
            ++h->launches;
            if (cudaMemcpyAsync(hs, sums, sizeof(double) * 2, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                set_last_error(std::string("power iteration: ") + cudaGetErrorString(cudaGetLastError()));
                rc = L1_ERR_CUDA;
                break;
            }
            const double rho_new = hs[0];
            const bool done = it > 1 && std::fabs(rho_new - rho) <= rtol * rho_new;
            rho = rho_new;
            if (hs[1] == 0.0 || done) break;
        }
    }
    if (v) cudaFree(v);
    if (u) cudaFree(u);
    if (part) cudaFree(part);
    if (sums) cudaFree(sums);
    if (hs) cudaFreeHost(hs);
    *L_out = rho;
    return rc;
}

// ------------------------------------------------------- FP64 factor of B B^T
// C(i, k) = sum_j X(i, j) X(k, j) with X(i, j) = Xp[i * si + j * sj], FP64
// accumulation; 16 x 16 output tile per block, j staged through shared memory.
template <class T>
__global__ void syrk64_kernel(const T* __restrict__ Xp, int64_t si, int64_t sj, int rows, int K,
                              double* __restrict__ C, int64_t ldc, double diag_add) {
    __shared__ double a[16][17], b[16][17];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = blockIdx.y * 16 + ty, k = blockIdx.x * 16 + tx;
    double acc = 0.0;
    for (int j0 = 0; j0 < K; j0 += 16) {
        const int ia = blockIdx.y * 16 + ty, ja = j0 + tx;
        a[ty][tx] = (ia < rows && ja < K) ? (double)Xp[ia * si + (int64_t)ja * sj] : 0.0;
        const int kb = blockIdx.x * 16 + ty;
        b[ty][tx] = (kb < rows && ja < K) ? (double)Xp[kb * si + (int64_t)ja * sj] : 0.0;
        __syncthreads();
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) acc += a[ty][jj] * b[tx][jj];
        __syncthreads();
    }
    if (i < rows && k < rows) C[(int64_t)k * ldc + i] = acc + (i == k ? diag_add : 0.0);
}

// Right-looking Cholesky, column k: pivot check and scaling of column k.
// A pivot that is not positive beyond rounding (d <= 16 m eps G_kk of the
// original matrix) marks the matrix as not SPD.
__global__ void chol_pivot_kernel(double* G, int m, int k, const double* diag0, int* flag) {
    __shared__ double piv;
    if (threadIdx.x == 0) {
        const double d = G[(int64_t)k * m + k];
        const double thr = 16.0 * m * 2.220446049250313e-16 * diag0[k];
        if (!(d > thr)) {
            *flag = 1;
            piv = 1.0;
        } else {
            piv = sqrt(d);
        }
        G[(int64_t)k * m + k] = piv;
    }
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) G[(int64_t)k * m + i] /= piv;
}

// trailing update G[i][j] -= G[i][k] G[j][k] for k < j <= i
__global__ void chol_update_kernel(double* G, int m, int k) {
    const int j = k + 1 + blockIdx.y * blockDim.y + threadIdx.y;
    if (j >= m) return;
    const double gjk = G[(int64_t)k * m + j];
    for (int i = j + blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        G[(int64_t)j * m + i] -= G[(int64_t)k * m + i] * gjk;
}

__global__ void diag_copy_kernel(const double* G, int m, double* d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) d[i] = G[(int64_t)i * m + i];
}

__global__ void eye_kernel(double* X, int m) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)m * m) return;
    const int64_t c = idx / m, r = idx % m;
    X[idx] = (r == c) ? 1.0 : 0.0;
}

// forward substitution L X = I, right-looking over k with X kept unscaled:
// X[i][c] -= (L[i][k] / L[k][k]) X[k][c] for i > k, c <= k
__global__ void trinv_update_kernel(const double* Lf, double* X, int m, int k) {
    const int c = blockIdx.y * blockDim.y + threadIdx.y;
    if (c > k) return;
    const double xk = X[(int64_t)c * m + k] / Lf[(int64_t)k * m + k];
    for (int i = k + 1 + blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        X[(int64_t)c * m + i] -= Lf[(int64_t)k * m + i] * xk;
}

__global__ void trinv_scale_kernel(const double* Lf, double* X, int m) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)m * m) return;
    const int64_t c = idx / m, r = idx % m;
    X[idx] = (r >= c) ? X[idx] / Lf[r * m + r] : 0.0;
}

// FP64 -> FP32 pair: hi = fl32(v), lo = fl32(v - hi), so hi + lo carries
// about 48 bits of v.  The y-step of DALM multiplies by (B B^T)^{-1}, whose
// condition number amplifies the rounding of a plain FP32 copy.
__global__ void to_f32_split_kernel(const double* src, int m, float* hi, float* lo, int64_t ldd) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = ldd * m;
    if (idx >= total) return;
    const int64_t c = idx / ldd, r = idx % ldd;
    const double v = (r < m) ? src[c * m + r] : 0.0;
    const float h = (float)v;
    hi[idx] = h;
    lo[idx] = (float)(v - (double)h);
}

int dalm_factor(Handle* h, double diag_add) {
    const int m = (int)h->m, n = (int)h->n;
    cudaStream_t s = h->stream;
    double *G = nullptr, *X = nullptr, *d0 = nullptr;
    int* flag = nullptr;
    int hflag = 0;
    int rc = L1_OK;
    const size_t mm = (size_t)m * m;
    if (cudaMalloc(&G, sizeof(double) * mm) != cudaSuccess || cudaMalloc(&X, sizeof(double) * mm) != cudaSuccess ||
        cudaMalloc(&d0, sizeof(double) * m) != cudaSuccess || cudaMalloc(&flag, sizeof(int)) != cudaSuccess) {
        rc = L1_ERR_OOM;
    }
    if (rc == L1_OK) {
        cudaMemsetAsync(flag, 0, sizeof(int), s);
        // G = A A^T (+ I), FP64 accumulation from the FP32 dictionary
        dim3 g16((m + 15) / 16, (m + 15) / 16);
        syrk64_kernel<float><<<g16, dim3(16, 16), 0, s>>>(h->A_rm, h->ldn, 1, m, n, G, m, diag_add);
        ++h->launches;
        diag_copy_kernel<<<(m + 255) / 256, 256, 0, s>>>(G, m, d0);
        ++h->launches;
        for (int k = 0; k < m; ++k) {
            chol_pivot_kernel<<<1, 256, 0, s>>>(G, m, k, d0, flag);
            const int rem = m - k - 1;
            if (rem > 0) {
                dim3 blk(128, 2);
                dim3 grd((unsigned)std::min(8, (rem + 127) / 128), (unsigned)((rem + 1) / 2));
                chol_update_kernel<<<grd, blk, 0, s>>>(G, m, k);
            }
            h->launches += 2;
        }
        // inverse of the factor, then F = L^{-T} L^{-1} = (B B^T)^{-1}
        eye_kernel<<<(unsigned)((mm + 255) / 256), 256, 0, s>>>(X, m);
        ++h->launches;
        for (int k = 0; k < m - 1; ++k) {
            dim3 blk(128, 2);
            const int rem = m - k - 1;
            dim3 grd((unsigned)std::min(8, (rem + 127) / 128), (unsigned)((k + 2) / 2));
            trinv_update_kernel<<<grd, blk, 0, s>>>(G, X, m, k);
            ++h->launches;
        }
        trinv_scale_kernel<<<(unsigned)((mm + 255) / 256), 256, 0, s>>>(G, X, m);
        ++h->launches;
        // F(i, k) = sum_j Linv(j, i) Linv(j, k): X(i, j) = Linv(j, i) = X[i*m + j]
        syrk64_kernel<double><<<g16, dim3(16, 16), 0, s>>>(X, m, 1, m, m, G, m, 0.0);
        ++h->launches;
        to_f32_split_kernel<<<(unsigned)((h->ldm * m + 255) / 256), 256, 0, s>>>(G, m, h->F, h->F_lo, h->ldm);
        ++h->launches;
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            set_last_error(std::string("dalm factor: ") + cudaGetErrorString(e));
            rc = L1_ERR_CUDA;
        } else if (hflag) {
            rc = L1_ERR_NOT_SPD;
        }
    }
    if (G) cudaFree(G);
    if (X) cudaFree(X);
    if (d0) cudaFree(d0);
    if (flag) cudaFree(flag);
    return rc;
}

}  // namespace l1
