// CUDA-core FP32 sweeps with fused epilogues: OUT(M x N) = Aop(M x K) X(K x N).
//
// Operand layouts (the only two the solvers need):
//   Aop is K-major: element (i, k) at Aop[i * lda + k]   (row-major M x K)
//   X   is column-major K x N: element (k, j) at X[j * ldx + k]
// lda and ldx are multiples of 4 floats and the entries between K and the
// padded leading dimension are zero in both operands, so the K loop runs to
// round_up(K, 4) with 128-bit loads and no tail case.
//
// The epilogue functor E is called once per output element with the FP32
// accumulator:  e(i, j, acc, red)  where red points to E::NRED doubles that
// the element may add per-column reduction terms to.  Each kernel reduces
// those terms over its rows in a fixed order (warp shuffles, then shared
// memory) and writes one partial per (row block, column):
//   part[(row_block * N + j) * 4 + r],  r < E::NRED.
// The controller kernels sum the row blocks in index order, so every
// reduction is deterministic.
#pragma once

#include "common.cuh"

namespace l1 {

constexpr int kPartStride = 4;  // doubles per (row block, column) partial

// ------------------------------------------------------------------- GEMV
// N <= NC columns (NC in 1..8): one warp per row, 128-bit loads along K.
// This is the single-right-hand-side path: each element of Aop is read once
// per call, so the kernel is bound by the bandwidth of wherever Aop lives.
constexpr int kGemvWarps = 4;
constexpr int kGemvRowsPerWarp = 1;

// Aop2 (nullable) is the low part of a split operand Aop + Aop2 (same
// layout): its products go to a separate accumulator that is added last, so
// the small terms are not absorbed by the large ones.
template <int NC, class E>
__global__ void __launch_bounds__(kGemvWarps * 32)
gemv_kernel(int M, int N, int K, const float* __restrict__ Aop, const float* __restrict__ Aop2,
            int64_t lda, const float* __restrict__ X, int64_t ldx, E epi, double* __restrict__ part) {
    constexpr int NR = E::NRED > 0 ? E::NRED : 1;
    __shared__ double red_s[kGemvWarps][NC][NR];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Kp = (K + 3) & ~3;
    double red[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) red[r] = 0.0;
    const int row0 = (blockIdx.x * kGemvWarps + warp) * kGemvRowsPerWarp;
    for (int rr = 0; rr < kGemvRowsPerWarp; ++rr) {
        const int i = row0 + rr;
        if (i >= M) break;
        float acc[NC], acc2[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = acc2[c] = 0.0f;
        const float* arow = Aop + (int64_t)i * lda;
        const float* arow2 = Aop2 ? Aop2 + (int64_t)i * lda : nullptr;
        for (int k = lane * 4; k < Kp; k += 128) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(arow + k));
            float4 a2 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (arow2) a2 = __ldg(reinterpret_cast<const float4*>(arow2 + k));
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                if (c < N) {
                    const float4 x = __ldg(reinterpret_cast<const float4*>(X + (int64_t)c * ldx + k));
                    acc[c] = fmaf(a.x, x.x, acc[c]);
                    acc[c] = fmaf(a.y, x.y, acc[c]);
                    acc[c] = fmaf(a.z, x.z, acc[c]);
                    acc[c] = fmaf(a.w, x.w, acc[c]);
                    if (arow2) {
                        acc2[c] = fmaf(a2.x, x.x, acc2[c]);
                        acc2[c] = fmaf(a2.y, x.y, acc2[c]);
                        acc2[c] = fmaf(a2.z, x.z, acc2[c]);
                        acc2[c] = fmaf(a2.w, x.w, acc2[c]);
                    }
                }
            }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = warp_sum_f(acc[c]) + warp_sum_f(acc2[c]);
        // lane c applies the epilogue of column c
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            if (lane == c && c < N) {
                double rloc[NR];
#pragma unroll
                for (int r = 0; r < NR; ++r) rloc[r] = 0.0;
                epi(i, c, acc[c], rloc);
#pragma unroll
                for (int r = 0; r < NR; ++r) red[r] += rloc[r];
            }
        }
    }
    if constexpr (E::NRED > 0) {
        // lane c holds the sums of column c for this warp's rows
#pragma unroll
        for (int c = 0; c < NC; ++c)
            if (lane == c)
#pragma unroll
                for (int r = 0; r < NR; ++r) red_s[warp][c][r] = red[r];
        __syncthreads();
        if (threadIdx.x < NC * NR) {
            const int c = threadIdx.x / NR, r = threadIdx.x % NR;
            if (c < N) {
                double s = 0.0;
                for (int w = 0; w < kGemvWarps; ++w) s += red_s[w][c][r];
                part[((int64_t)blockIdx.x * N + c) * kPartStride + r] = s;
            }
        }
    }
}

// --------------------------------------------------------------- tiled GEMM
// 64 x 64 output tile per 256-thread CTA, 4 x 4 per thread, K step 16,
// double-buffered shared memory.
constexpr int kBM = 64, kBN = 64, kBK = 16;

template <class E, bool SPLIT>
__global__ void __launch_bounds__(256)
gemm_simt_kernel(int M, int N, int K, const float* __restrict__ Aop, const float* __restrict__ Aop2,
                 int64_t lda, const float* __restrict__ X, int64_t ldx, E epi,
                 double* __restrict__ part, const int32_t* __restrict__ active) {
    constexpr int NR = E::NRED > 0 ? E::NRED : 1;
    __shared__ __align__(16) float As[2][kBK][kBM];
    __shared__ __align__(16) float As2[SPLIT ? 2 : 1][SPLIT ? kBK : 1][SPLIT ? kBM : 4];
    __shared__ __align__(16) float Xs[2][kBK][kBN];
    __shared__ double red_s[8][kBN][NR];
    __shared__ int any_active;

    const int t = threadIdx.x;
    const int tc = t & 15, tr = t >> 4;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;

    if (active != nullptr) {
        if (t == 0) any_active = 0;
        __syncthreads();
        if (t < kBN && n0 + t < N && active[n0 + t]) any_active = 1;
        __syncthreads();
        if (!any_active) {
            // every column of this tile is frozen: nothing to compute, but the
            // partials must still be defined for the controller
            if constexpr (E::NRED > 0) {
                if (t < kBN && n0 + t < N)
                    for (int r = 0; r < NR; ++r)
                        part[((int64_t)blockIdx.y * N + n0 + t) * kPartStride + r] = 0.0;
            }
            return;
        }
    }

    // load mapping: one float4 of Aop and one of X per thread per K step
    const int la_row = t >> 2, la_k = (t & 3) * 4;  // 64 rows x 4 float4
    const int lx_col = t >> 2, lx_k = (t & 3) * 4;  // 64 cols x 4 float4
    const int Kp = (K + 3) & ~3;

    auto load_tiles = [&](int buf, int k0) {
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), x = make_float4(0.f, 0.f, 0.f, 0.f);
        const int gi = m0 + la_row, gk = k0 + la_k;
        if (gi < M && gk < Kp) a = __ldg(reinterpret_cast<const float4*>(Aop + (int64_t)gi * lda + gk));
        if constexpr (SPLIT) {
            float4 a2 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gi < M && gk < Kp) a2 = __ldg(reinterpret_cast<const float4*>(Aop2 + (int64_t)gi * lda + gk));
            As2[buf][la_k + 0][la_row] = a2.x;
            As2[buf][la_k + 1][la_row] = a2.y;
            As2[buf][la_k + 2][la_row] = a2.z;
            As2[buf][la_k + 3][la_row] = a2.w;
        }
        const int gj = n0 + lx_col, gkx = k0 + lx_k;
        if (gj < N && gkx < Kp) x = __ldg(reinterpret_cast<const float4*>(X + (int64_t)gj * ldx + gkx));
        As[buf][la_k + 0][la_row] = a.x;
        As[buf][la_k + 1][la_row] = a.y;
        As[buf][la_k + 2][la_row] = a.z;
        As[buf][la_k + 3][la_row] = a.w;
        Xs[buf][lx_k + 0][lx_col] = x.x;
        Xs[buf][lx_k + 1][lx_col] = x.y;
        Xs[buf][lx_k + 2][lx_col] = x.z;
        Xs[buf][lx_k + 3][lx_col] = x.w;
    };

    // Accumulation: each K tile of 16 products is summed into a fresh FP32
    // partial t, and the partials are merged into acc with Kahan
    // compensation (comp), so the rounding error grows with the number of
    // tiles, not with K.  The low part of a split operand (Aop2) has its own
    // accumulator, added last.
    float acc[4][4], comp[4][4], acc2[SPLIT ? 4 : 1][SPLIT ? 4 : 1];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = comp[a][b] = 0.0f;
    if constexpr (SPLIT) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc2[a][b] = 0.0f;
    }

    int buf = 0;
    load_tiles(0, 0);
    __syncthreads();
    for (int k0 = 0; k0 < Kp; k0 += kBK) {
        if (k0 + kBK < Kp) load_tiles(buf ^ 1, k0 + kBK);
        float t[4][4];
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) t[p][q] = 0.0f;
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            const float4 a = *reinterpret_cast<const float4*>(&As[buf][kk][tr * 4]);
            const float4 x = *reinterpret_cast<const float4*>(&Xs[buf][kk][tc * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w};
            const float xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) t[p][q] = fmaf(av[p], xv[q], t[p][q]);
            if constexpr (SPLIT) {
                const float4 a2 = *reinterpret_cast<const float4*>(&As2[buf][kk][tr * 4]);
                const float av2[4] = {a2.x, a2.y, a2.z, a2.w};
#pragma unroll
                for (int p = 0; p < 4; ++p)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc2[p][q] = fmaf(av2[p], xv[q], acc2[p][q]);
            }
        }
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float yv = t[p][q] - comp[p][q];
                const float sv = acc[p][q] + yv;
                comp[p][q] = (sv - acc[p][q]) - yv;
                acc[p][q] = sv;
            }
        __syncthreads();
        buf ^= 1;
    }
    if constexpr (SPLIT) {
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[p][q] += acc2[p][q] - comp[p][q];
    } else {
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[p][q] -= comp[p][q];
    }

    // epilogue
    double red[4][NR];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < NR; ++r) red[q][r] = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = n0 + tc * 4 + q;
        if (j >= N) continue;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int i = m0 + tr * 4 + p;
            if (i < M) epi(i, j, acc[p][q], red[q]);
        }
    }
    if constexpr (E::NRED > 0) {
        // lanes l and l ^ 16 share a column group (tr differs by one)
        const int warp = t >> 5;
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                double v = red[q][r];
                v += __shfl_xor_sync(0xffffffffu, v, 16);
                red[q][r] = v;
            }
        if ((t & 16) == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int r = 0; r < NR; ++r) red_s[warp][tc * 4 + q][r] = red[q][r];
        }
        __syncthreads();
        if (t < kBN * NR) {
            const int c = t / NR, r = t % NR;
            const int j = n0 + c;
            if (j < N) {
                double s = 0.0;
                for (int w = 0; w < 8; ++w) s += red_s[w][c][r];
                part[((int64_t)blockIdx.y * N + j) * kPartStride + r] = s;
            }
        }
    }
}

// Host-side launcher.  Returns the number of row blocks (the count of
// partials per column the controller must sum), or a negative error code.
// Aop2 (nullable): low part of a split operand, see gemv_kernel.
template <class E>
int launch_sweep(Handle* h, int M, int N, int K, const float* Aop, int64_t lda, const float* X,
                 int64_t ldx, const E& epi, double* part, const int32_t* active,
                 const float* Aop2 = nullptr) {
    cudaStream_t s = h->stream;
    if (N <= 8) {
        const int rows_per_block = kGemvWarps * kGemvRowsPerWarp;
        const int grid = (M + rows_per_block - 1) / rows_per_block;
        switch (N) {
#define L1_GEMV_CASE(nc) \
    case nc: gemv_kernel<nc, E><<<grid, kGemvWarps * 32, 0, s>>>(M, N, K, Aop, Aop2, lda, X, ldx, epi, part); break;
            L1_GEMV_CASE(1) L1_GEMV_CASE(2) L1_GEMV_CASE(3) L1_GEMV_CASE(4)
            L1_GEMV_CASE(5) L1_GEMV_CASE(6) L1_GEMV_CASE(7) L1_GEMV_CASE(8)
#undef L1_GEMV_CASE
            default: return L1_ERR_INVALID_ARG;
        }
        L1_LAUNCH_CHECK(h);
        return grid;
    }
    dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM);
    if (Aop2)
        gemm_simt_kernel<E, true><<<grid, 256, 0, s>>>(M, N, K, Aop, Aop2, lda, X, ldx, epi, part, active);
    else
        gemm_simt_kernel<E, false><<<grid, 256, 0, s>>>(M, N, K, Aop, nullptr, lda, X, ldx, epi, part, active);
    L1_LAUNCH_CHECK(h);
    return (int)grid.y;
}

// number of row blocks launch_sweep will use (for sizing partial buffers)
inline int sweep_row_blocks(int M, int N) {
    if (N <= 8) return (M + kGemvWarps * kGemvRowsPerWarp - 1) / (kGemvWarps * kGemvRowsPerWarp);
    return (M + kBM - 1) / kBM;
}

}  // namespace l1
