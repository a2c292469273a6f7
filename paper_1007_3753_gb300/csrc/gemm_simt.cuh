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

#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.cuh"

namespace l1 {

constexpr int kPartStride = 4;  // doubles per (row block, column) partial

// ------------------------------------------------------ element types of Aop
// Aop may be FP32, BF16 or FP8 e4m3 (one byte, wrapped so that overloads can
// tell it apart); the sweeps convert four consecutive K elements to FP32 as
// they load them and accumulate in FP32.
struct fp8e4m3 {
    uint8_t v;
};

__device__ __forceinline__ float4 load_a4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }

__device__ __forceinline__ float4 load_a4(const __nv_bfloat16* p) {
    // a BF16 value is the high half of the FP32 value with the same bits
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                       __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
}

__device__ __forceinline__ float4 load_a4(const fp8e4m3* p) {
    const unsigned u = __ldg(reinterpret_cast<const unsigned*>(p));
    const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(u & 0xffffu), __NV_E4M3);
    const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(u >> 16), __NV_E4M3);
    const float2 a = __half22float2(__half2(lo)), b = __half22float2(__half2(hi));
    return make_float4(a.x, a.y, b.x, b.y);
}

// Output-row scale of an FP8 operand (Aop(i, k) = scale[i] q(i, k)).
template <class E>
struct EpiRowScale {
    static constexpr int NRED = E::NRED;
    const float* scale;
    E inner;
    __device__ void operator()(int i, int j, float acc, double* red) const { inner(i, j, acc * scale[i], red); }
};

// ------------------------------------------------------------------- GEMV
// N <= NC columns (NC in 1..8): one warp per row, 128-bit loads along K.
// This is the single-right-hand-side path: each element of Aop is read once
// per call, so the kernel is bound by the bandwidth of wherever Aop lives.
constexpr int kGemvWarps = 4;
constexpr int kGemvRowsPerWarp = 1;

// Aop2 (nullable) is the low part of a split operand Aop + Aop2 (same
// layout): its products go to a separate accumulator that is added last, so
// the small terms are not absorbed by the large ones.
template <int NC, class E, class TA>
__global__ void __launch_bounds__(kGemvWarps * 32)
gemv_kernel(int M, int N, int K, const TA* __restrict__ Aop, const TA* __restrict__ Aop2,
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
        const TA* arow = Aop + (int64_t)i * lda;
        const TA* arow2 = Aop2 ? Aop2 + (int64_t)i * lda : nullptr;
        for (int k = lane * 4; k < Kp; k += 128) {
            const float4 a = load_a4(arow + k);
            float4 a2 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (arow2) a2 = load_a4(arow2 + k);
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
constexpr int kBM = 64, kBN = 64, kBK = 32;  // kBK: the deepest K step (split-K chunks are multiples)
constexpr int kKahan = 16;  // products per FP32 partial merged with compensation
// K step of a sweep: 32 for one operand, 16 for a split operand (F_hi, F_lo),
// whose second tile would not fit the static shared-memory budget
template <bool SPLIT>
__host__ __device__ constexpr int bk_of() { return SPLIT ? 16 : 32; }
constexpr int kMaxSplitK = 8;

template <bool SPLIT>
struct SimtSmem {
    static constexpr int BK = bk_of<SPLIT>();
    float As[2][BK][kBM];
    float As2[SPLIT ? 2 : 1][SPLIT ? BK : 1][SPLIT ? kBM : 4];
    float Xs[2][BK][kBN];
};

// true when some column of the tile starting at n0 is still active (all
// threads of the CTA get the same answer)
__device__ __forceinline__ bool tile_has_active(const int32_t* active, int N, int n0, int* flag) {
    if (active == nullptr) return true;
    const int t = threadIdx.x;
    if (t == 0) *flag = 0;
    __syncthreads();
    if (t < kBN && n0 + t < N && active[n0 + t]) *flag = 1;
    __syncthreads();
    return *flag != 0;
}

// Main loop of one 64 x 64 tile over K in [k_begin, k_end) (multiples of 4,
// k_end <= round_up(K, 4)).  Each K tile of 16 products is summed into a
// fresh FP32 partial, and the partials are merged with Kahan compensation, so
// the rounding error grows with the number of K tiles, not with K.  The low
// part of a split operand (Aop2) has its own accumulator, added last.
// out[p][q] is the sum for row m0 + tr*4 + p and column n0 + tc*4 + q.
template <bool SPLIT, class TA>
__device__ __forceinline__ void simt_tile_mainloop(int M, int N, int m0, int n0, int k_begin, int k_end,
                                                   const TA* __restrict__ Aop, const TA* __restrict__ Aop2,
                                                   int64_t lda, const float* __restrict__ X, int64_t ldx,
                                                   SimtSmem<SPLIT>& sm, float (&out)[4][4]) {
    const int t = threadIdx.x;
    const int tc = t & 15, tr = t >> 4;
    // load mapping: BK/16 float4 of Aop and of X per thread per K step
    // (four lanes per row, 64 contiguous bytes each, slices k, k + 16).
    // The transposing stores put row r of K slice k at r ^ swz(k): the four
    // lanes of a row write slices whose swizzles differ in bits 3-4, so a
    // warp's stores hit 32 distinct banks; reads apply the same swizzle to a
    // 4-aligned group.
    const int la_row = t >> 2, la_k = (t & 3) * 4;  // 64 rows x 4 float4 (x 2 halves)
    const int lx_col = t >> 2, lx_k = (t & 3) * 4;  // 64 cols x 4 float4 (x 2 halves)
    auto swz = [](int k) { return ((k >> 2) & 3) << 3; };

    // global -> registers (issued a K step ahead) -> shared memory (stored
    // after the current step's FMAs), so the L2 latency overlaps the math
    constexpr int BK = bk_of<SPLIT>(), NH = BK / 16;
    float4 ra_g[NH], ra2_g[NH], rx_g[NH];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int hf = 0; hf < NH; ++hf) {
            ra_g[hf] = ra2_g[hf] = rx_g[hf] = make_float4(0.f, 0.f, 0.f, 0.f);
            const int gi = m0 + la_row, gk = k0 + la_k + 16 * hf;
            if (gi < M && gk < k_end) {
                ra_g[hf] = load_a4(Aop + (int64_t)gi * lda + gk);
                if constexpr (SPLIT) ra2_g[hf] = load_a4(Aop2 + (int64_t)gi * lda + gk);
            }
            const int gj = n0 + lx_col, gkx = k0 + lx_k + 16 * hf;
            if (gj < N && gkx < k_end) rx_g[hf] = __ldg(reinterpret_cast<const float4*>(X + (int64_t)gj * ldx + gkx));
        }
    };
    auto stash = [&](int buf) {
        const int ra = la_row ^ swz(la_k), rx = lx_col ^ swz(lx_k);
#pragma unroll
        for (int hf = 0; hf < NH; ++hf) {
            const int ka = la_k + 16 * hf, kx = lx_k + 16 * hf;
            if constexpr (SPLIT) {
                sm.As2[buf][ka + 0][ra] = ra2_g[hf].x;
                sm.As2[buf][ka + 1][ra] = ra2_g[hf].y;
                sm.As2[buf][ka + 2][ra] = ra2_g[hf].z;
                sm.As2[buf][ka + 3][ra] = ra2_g[hf].w;
            }
            sm.As[buf][ka + 0][ra] = ra_g[hf].x;
            sm.As[buf][ka + 1][ra] = ra_g[hf].y;
            sm.As[buf][ka + 2][ra] = ra_g[hf].z;
            sm.As[buf][ka + 3][ra] = ra_g[hf].w;
            sm.Xs[buf][kx + 0][rx] = rx_g[hf].x;
            sm.Xs[buf][kx + 1][rx] = rx_g[hf].y;
            sm.Xs[buf][kx + 2][rx] = rx_g[hf].z;
            sm.Xs[buf][kx + 3][rx] = rx_g[hf].w;
        }
    };

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
    fetch(k_begin);
    stash(0);
    __syncthreads();
    for (int k0 = k_begin; k0 < k_end; k0 += BK) {
        const bool more = k0 + BK < k_end;
        if (more) fetch(k0 + BK);
#pragma unroll
        for (int half = 0; half < BK / kKahan; ++half) {
            float tt[4][4];
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) tt[p][q] = 0.0f;
            // fragments of slice kk + 1 are read before the FMAs of slice kk
            const int kb = half * kKahan;
            float4 fa = *reinterpret_cast<const float4*>(&sm.As[buf][kb][(tr * 4) ^ swz(kb)]);
            float4 fx = *reinterpret_cast<const float4*>(&sm.Xs[buf][kb][(tc * 4) ^ swz(kb)]);
            float4 fa2 = make_float4(0.f, 0.f, 0.f, 0.f);
            if constexpr (SPLIT) fa2 = *reinterpret_cast<const float4*>(&sm.As2[buf][kb][(tr * 4) ^ swz(kb)]);
#pragma unroll
            for (int kk = kb; kk < kb + kKahan; ++kk) {
                const float av[4] = {fa.x, fa.y, fa.z, fa.w};
                const float xv[4] = {fx.x, fx.y, fx.z, fx.w};
                const float av2[4] = {fa2.x, fa2.y, fa2.z, fa2.w};
                if (kk + 1 < kb + kKahan) {
                    fa = *reinterpret_cast<const float4*>(&sm.As[buf][kk + 1][(tr * 4) ^ swz(kk + 1)]);
                    fx = *reinterpret_cast<const float4*>(&sm.Xs[buf][kk + 1][(tc * 4) ^ swz(kk + 1)]);
                    if constexpr (SPLIT)
                        fa2 = *reinterpret_cast<const float4*>(&sm.As2[buf][kk + 1][(tr * 4) ^ swz(kk + 1)]);
                }
#pragma unroll
                for (int p = 0; p < 4; ++p)
#pragma unroll
                    for (int q = 0; q < 4; ++q) tt[p][q] = fmaf(av[p], xv[q], tt[p][q]);
                if constexpr (SPLIT) {
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
                    const float yv = tt[p][q] - comp[p][q];
                    const float sv = acc[p][q] + yv;
                    comp[p][q] = (sv - acc[p][q]) - yv;
                    acc[p][q] = sv;
                }
        }
        if (more) stash(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if constexpr (SPLIT) out[p][q] = acc[p][q] + (acc2[p][q] - comp[p][q]);
            else out[p][q] = acc[p][q] - comp[p][q];
        }
}

// Epilogue of one tile: E on every element, then the per-column reduction
// terms of the tile's rows in a fixed order (warp shuffles, shared memory) to
// part[(row_block * N + j) * 4 + r].
template <class E, int NR>
__device__ __forceinline__ void simt_tile_epilogue(int M, int N, int m0, int n0, int row_block,
                                                   const float (&acc)[4][4], const E& epi, double* part,
                                                   double (*red_s)[kBN][NR]) {
    const int t = threadIdx.x;
    const int tc = t & 15, tr = t >> 4;
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
                part[((int64_t)row_block * N + j) * kPartStride + r] = s;
            }
        }
    }
}

// every column of the tile is frozen: nothing to compute, but the partials
// must still be defined for the controller
template <class E>
__device__ __forceinline__ void simt_tile_zero_parts(int N, int n0, int row_block, double* part) {
    if constexpr (E::NRED > 0) {
        const int t = threadIdx.x;
        if (t < kBN && n0 + t < N)
            for (int r = 0; r < E::NRED; ++r) part[((int64_t)row_block * N + n0 + t) * kPartStride + r] = 0.0;
    }
}

template <class E, bool SPLIT, class TA>
__global__ void __launch_bounds__(256)
gemm_simt_kernel(int M, int N, int K, const TA* __restrict__ Aop, const TA* __restrict__ Aop2,
                 int64_t lda, const float* __restrict__ X, int64_t ldx, E epi,
                 double* __restrict__ part, const int32_t* __restrict__ active) {
    constexpr int NR = E::NRED > 0 ? E::NRED : 1;
    // the epilogue's reduction scratch reuses the tiles' shared memory: the
    // main loop ends with a barrier after its last read
    union Smem {
        SimtSmem<SPLIT> tiles;
        double red[8][kBN][NR];
    };
    __shared__ __align__(16) Smem sm;
    __shared__ int any_active;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    if (!tile_has_active(active, N, n0, &any_active)) {
        simt_tile_zero_parts<E>(N, n0, blockIdx.y, part);
        return;
    }
    float acc[4][4];
    simt_tile_mainloop<SPLIT, TA>(M, N, m0, n0, 0, (K + 3) & ~3, Aop, Aop2, lda, X, ldx, sm.tiles, acc);
    simt_tile_epilogue<E, NR>(M, N, m0, n0, blockIdx.y, acc, epi, part, sm.red);
}

// Split-K, for panels too narrow to fill the GPU with output tiles: slice
// blockIdx.z of K (chunk kchunk, a multiple of kBK) writes its tile sum to
// Wk[(z * M + i) * ldw + j] (rows of a slice contiguous over the columns, so
// a thread's four columns move as one float4 and a warp's accesses coalesce;
// ldw = N rounded up to 4).
template <bool SPLIT, class TA>
__global__ void __launch_bounds__(256)
gemm_simt_splitk_kernel(int M, int N, int K, int kchunk, const TA* __restrict__ Aop,
                        const TA* __restrict__ Aop2, int64_t lda, const float* __restrict__ X, int64_t ldx,
                        float* __restrict__ Wk, int64_t ldw, const int32_t* __restrict__ active) {
    __shared__ __align__(16) SimtSmem<SPLIT> sm;
    __shared__ int any_active;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    if (!tile_has_active(active, N, n0, &any_active)) return;
    const int Kp = (K + 3) & ~3;
    const int k_begin = blockIdx.z * kchunk, k_end = min(Kp, k_begin + kchunk);
    float acc[4][4];
    simt_tile_mainloop<SPLIT, TA>(M, N, m0, n0, k_begin, k_end, Aop, Aop2, lda, X, ldx, sm, acc);
    const int t = threadIdx.x, tc = t & 15, tr = t >> 4;
    float* w = Wk + (int64_t)blockIdx.z * M * ldw;
    const int j0 = n0 + tc * 4;
    if (j0 >= N) return;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int i = m0 + tr * 4 + p;
        if (i >= M) continue;
        float* row = w + (int64_t)i * ldw + j0;
        if (j0 + 3 < N) {
            *reinterpret_cast<float4*>(row) = make_float4(acc[p][0], acc[p][1], acc[p][2], acc[p][3]);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (j0 + q < N) row[q] = acc[p][q];
        }
    }
}

// Sums the S slices of every element in slice order with Kahan compensation,
// then runs the epilogue exactly as the single-pass kernel does.
template <class E>
__global__ void __launch_bounds__(256)
splitk_epilogue_kernel(int M, int N, int S, const float* __restrict__ Wk, int64_t ldw, E epi,
                       double* __restrict__ part, const int32_t* __restrict__ active) {
    constexpr int NR = E::NRED > 0 ? E::NRED : 1;
    __shared__ double red_s[8][kBN][NR];
    __shared__ int any_active;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    if (!tile_has_active(active, N, n0, &any_active)) {
        simt_tile_zero_parts<E>(N, n0, blockIdx.y, part);
        return;
    }
    const int t = threadIdx.x, tc = t & 15, tr = t >> 4;
    float acc[4][4];
    const int j0 = n0 + tc * 4;
    const bool vec = j0 + 3 < N;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int i = min(m0 + tr * 4 + p, M - 1);
        float sm[4] = {0.f, 0.f, 0.f, 0.f}, cm[4] = {0.f, 0.f, 0.f, 0.f};
        for (int z = 0; z < S; ++z) {
            const float* row = Wk + ((int64_t)z * M + i) * ldw;
            float v[4];
            if (vec) {
                const float4 f = *reinterpret_cast<const float4*>(row + j0);
                v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = row[min(j0 + q, N - 1)];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float y = v[q] - cm[q];
                const float u = sm[q] + y;
                cm[q] = (u - sm[q]) - y;
                sm[q] = u;
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = sm[q] - cm[q];
    }
    simt_tile_epilogue<E, NR>(M, N, m0, n0, blockIdx.y, acc, epi, part, red_s);
}

// K slices for an M x N sweep: enough CTAs to give every SM two tiles, each
// slice at least 64 deep.
inline int splitk_slices(const Handle* h, int M, int N, int K) {
    const int tiles = ((N + kBN - 1) / kBN) * ((M + kBM - 1) / kBM);
    const int sms = h->sms > 0 ? h->sms : 152;
    if (tiles >= sms || K < 128) return 1;
    int S = (2 * sms + tiles - 1) / tiles;
    S = std::min(S, kMaxSplitK);
    S = std::min(S, std::max(1, K / 64));
    return S;
}

// Host-side launcher.  Returns the number of row blocks (the count of
// partials per column the controller must sum), or a negative error code.
// Aop2 (nullable): low part of a split operand, see gemv_kernel.
template <class E, class TA>
int launch_sweep(Handle* h, int M, int N, int K, const TA* Aop, int64_t lda, const float* X,
                 int64_t ldx, const E& epi, double* part, const int32_t* active,
                 const TA* Aop2 = nullptr) {
    cudaStream_t s = h->stream;
    if (N <= 8) {
        const int rows_per_block = kGemvWarps * kGemvRowsPerWarp;
        const int grid = (M + rows_per_block - 1) / rows_per_block;
        switch (N) {
#define L1_GEMV_CASE(nc) \
    case nc: gemv_kernel<nc, E, TA><<<grid, kGemvWarps * 32, 0, s>>>(M, N, K, Aop, Aop2, lda, X, ldx, epi, part); break;
            L1_GEMV_CASE(1) L1_GEMV_CASE(2) L1_GEMV_CASE(3) L1_GEMV_CASE(4)
            L1_GEMV_CASE(5) L1_GEMV_CASE(6) L1_GEMV_CASE(7) L1_GEMV_CASE(8)
#undef L1_GEMV_CASE
            default: return L1_ERR_INVALID_ARG;
        }
        L1_LAUNCH_CHECK(h);
        return grid;
    }
    dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM);
    int S = splitk_slices(h, M, N, K);
    const int64_t ldw = ((int64_t)N + 3) & ~int64_t(3);
    if (S > 1) {
        const size_t need = (size_t)S * M * ldw;
        if (need > h->splitk_floats) {
            // grows once to the largest narrow sweep this handle has seen; the
            // old scratch stays allocated until the handle is destroyed, since
            // graphs captured earlier may still point at it
            if (h->splitk) cudaStreamSynchronize(s);
            float* p = nullptr;
            if (dev_alloc_t(h, &p, need) != L1_OK) {
                S = 1;  // no room for the slices: single pass
            } else {
                h->splitk = p;
                h->splitk_floats = need;
            }
        }
    }
    if (S > 1) {
        const int Kp = (K + 3) & ~3;
        const int kchunk = ((Kp + S - 1) / S + kBK - 1) / kBK * kBK;
        S = (Kp + kchunk - 1) / kchunk;
        dim3 g3(grid.x, grid.y, S);
        if (Aop2)
            gemm_simt_splitk_kernel<true, TA><<<g3, 256, 0, s>>>(M, N, K, kchunk, Aop, Aop2, lda, X, ldx, h->splitk,
                                                                 ldw, active);
        else
            gemm_simt_splitk_kernel<false, TA><<<g3, 256, 0, s>>>(M, N, K, kchunk, Aop, nullptr, lda, X, ldx,
                                                                  h->splitk, ldw, active);
        L1_LAUNCH_CHECK(h);
        splitk_epilogue_kernel<E><<<grid, 256, 0, s>>>(M, N, S, h->splitk, ldw, epi, part, active);
        L1_LAUNCH_CHECK(h);
        return (int)grid.y;
    }
    if (Aop2)
        gemm_simt_kernel<E, true, TA><<<grid, 256, 0, s>>>(M, N, K, Aop, Aop2, lda, X, ldx, epi, part, active);
    else
        gemm_simt_kernel<E, false, TA><<<grid, 256, 0, s>>>(M, N, K, Aop, nullptr, lda, X, ldx, epi, part, active);
    L1_LAUNCH_CHECK(h);
    return (int)grid.y;
}

// number of row blocks launch_sweep will use (for sizing partial buffers)
inline int sweep_row_blocks(int M, int N) {
    if (N <= 8) return (M + kGemvWarps * kGemvRowsPerWarp - 1) / (kGemvWarps * kGemvRowsPerWarp);
    return (M + kBM - 1) / kBM;
}

}  // namespace l1
