// tcgen05 BF16 sweeps for sm_103a (kind::f16, FP32 accumulation) with the
// fused-epilogue contract of gemm_simt.cuh:
//
//     OUT(M x N) = sum_t  A_{ia(t)} (M x K)  X_{ix(t)} (K x N)
//
// Operand pieces.  An operand is carried as up to three BF16 pieces
// v ~ v_0 + v_1 + v_2 on an aligned grid (split_aligned): three pieces hold
// an FP32 value to 2^-24 of the largest magnitude in its 128-element block.
// A term list picks which piece products are issued: one term (a_0 x_0) is
// the plain BF16 product, six terms (every product of total order <= 2^-16)
// give FP32-level accuracy.  All pieces of one K block are staged once in
// shared memory and every term reads them there.  Layouts: A_p row-major
// (K contiguous, the K-major "A" operand), X_p column-major (K contiguous,
// the K-major "B" operand); both BF16 with leading dimensions that are
// multiples of 8.
//
// One CTA (one per SM) computes a 128 x 128 output tile:
//   warp 0      TMA producer: per K block of 64 elements, NPA tiles of
//               128 x 64 and NPX tiles of 128 x 64 BF16 (128-byte swizzle)
//               into a ring of shared-memory stages
//   warp 1      allocates all 512 TMEM columns (hi[0..1], lo[0..1]); one
//               thread issues every tcgen05.mma; tcgen05.commit frees ring
//               slots and hands each finished 128-K chunk to the epilogue
//   warps 2..9  epilogue: warp w reads TMEM lane quarter w % 4 (32 output
//               rows) and one half of the columns; FP32 sums of the chunks,
//               then either (fused) the functor per element, deterministic
//               per-column reductions (one partial per row block and column)
//               and the aligned pieces of the returned values, or (deferred,
//               and every slice of a split-K launch) the FP32 sums to a
//               scratch for finish_kernel, which runs the same epilogue with
//               one CTA per 128 rows x 8 columns
// Tiles whose columns are all inactive write zero partials and return.
// Every mbarrier wait is bounded; a wait that runs out records an error code
// in *err, the CTA leaves its loops, waits (bounded) for its own copies and
// MMAs, frees TMEM and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "gemm_simt.cuh"
#include "tcgen05.cuh"

namespace l1 {
namespace tc16 {

using tc::mbar_arrive;
using tc::mbar_expect_tx;
using tc::mbar_init;
using tc::mbar_wait;
using tc::mma_commit;
using tc::prefetch_map;
using tc::smem_desc;
using tc::smem_u32;
using tc::tma_load_2d;
using tc::tmem_ld32;

constexpr int kBM = 128;       // output rows per tile = TMEM lanes
#ifndef L1_TC_KB
#define L1_TC_KB 64
#endif
// BF16 elements per K block = one swizzle row (64: 128-byte rows, two
// 96 KB ring stages for three-piece operands; 32: 64-byte rows, four 48 KB
// stages)
constexpr int kKB = L1_TC_KB;
static_assert(kKB == 64 || kKB == 32, "K block");
constexpr int kMmaK = 16;      // K of one kind::f16 MMA
constexpr int kMaxPieces = 3;
constexpr int kMaxTerms = 9;

// codes of a bounded wait that ran out (first one recorded in *err)
enum : int { ERR_NONE = 0, ERR_WAIT_FULL = 11, ERR_WAIT_EMPTY = 12, ERR_WAIT_ACC = 13 };

struct Maps {
    CUtensorMap a[kMaxPieces];
    CUtensorMap x[kMaxPieces];
};

struct Terms {
    int n;
    int ia[kMaxTerms];
    int ix[kMaxTerms];
};

// instruction descriptor: dense, FP32 accumulator, BF16 A and B, both K-major
__host__ __device__ constexpr uint32_t instr_desc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

// BF16 value nearest to x (ties to even), as an FP32; the remainder
// x - bf16_rn(x) is exact in FP32.
__host__ __device__ __forceinline__ float bf16_rn(float x) {
    return __bfloat162float(__float2bfloat16_rn(x));
}

// ------------------------------------------------------------------ kernel
// Exact leading term.  Operand pieces are split on a grid shared by 128
// consecutive K elements (one exponent per row of A and K block of 128, one
// per column of X and K block of 128; see split_aligned): piece p is an
// integer of magnitude <= 256 times 2^(E - 8(p+1)).  The leading product
// a_0 x_0 over one such block is then a sum of 128 integers of magnitude
// <= 2^16 on one common scale, below 2^23 in total, so the tensor core adds
// it without rounding whatever its accumulator does.  It goes to TMEM buffer
// hi[b]; the other terms (2^-8 and smaller) go to lo[b], whose rounding is
// 2^-8 below the result.  After every K block of 128 the epilogue drains
// hi[b] + lo[b] into FP32 register sums (round to nearest: unbiased) while
// the MMA warp fills the other buffer pair (b ^ 1).  Accumulating the whole
// K range in one TMEM accumulator instead rounds every MMA toward zero
// (measured: a relative bias of 3e-7 for one term and 2e-6 for six at
// K = 256), which a slowly converging iteration accumulates.
constexpr int kChunk = 128;            // K elements per drain (= the exponent block)
constexpr int kKBPerChunk = kChunk / kKB;

// Piece sink of an epilogue: the value each element returns is split into
// np aligned BF16 pieces (exponent per column and 128-row block of the tile)
// at p[k][j * ld + i]; np = 0: nothing is written.
struct PieceOut {
    __nv_bfloat16* p[kMaxPieces];
    int np;
    int64_t ld;
};

// Aligned split of v on the grid of a block whose largest magnitude is bmax
// (see above); returns the pieces as floats.
// 2^e as a float from its IEEE bits (normal range, -126 <= e <= 127)
__device__ __forceinline__ float pow2_bits(int e) { return __uint_as_float((uint32_t)(e + 127) << 23); }

__device__ __forceinline__ void split_aligned(float v, float bmax, float& p0, float& p1, float& p2) {
    if (!(bmax > 0.0f)) {
        p0 = p1 = p2 = 0.0f;
        return;
    }
    const int eb = (int)((__float_as_uint(bmax) >> 23) & 0xffu);
    if (eb >= 25 && eb <= 254) {
        // bmax in [2^(eb-127), 2^(eb-126)): bmax < 2^E with E = eb - 126.
        // Every grid step 2^(E - 8(p+1)) and its reciprocal are normal
        // floats here, so dividing by the step and multiplying by the
        // reciprocal give the same (exact) value
        const int E = eb - 126;
        p0 = rintf(v * pow2_bits(8 - E)) * pow2_bits(E - 8);
        const float r1 = v - p0;
        p1 = rintf(r1 * pow2_bits(16 - E)) * pow2_bits(E - 16);
        const float r2 = r1 - p1;
        p2 = rintf(r2 * pow2_bits(24 - E)) * pow2_bits(E - 24);
        return;
    }
    int E;
    frexpf(bmax, &E);  // bmax < 2^E
    const float g0 = ldexpf(1.0f, E - 8), g1 = ldexpf(1.0f, E - 16), g2 = ldexpf(1.0f, E - 24);
    p0 = rintf(v / g0) * g0;
    const float r1 = v - p0;
    p1 = rintf(r1 / g1) * g1;
    const float r2 = r1 - p1;
    p2 = rintf(r2 / g2) * g2;
}

template <int BN, int NPA, int NPX>
struct Cfg {
    static constexpr int kATile = kBM * kKB * 2;  // 16 or 8 KB
    static constexpr int kXTile = BN * kKB * 2;
    static constexpr int kStage = NPA * kATile + NPX * kXTile;
    static constexpr int kStages = (216 * 1024 / kStage) > 6 ? 6 : (216 * 1024 / kStage);
    static_assert(kStages >= 2, "two ring stages must fit");
    static constexpr int kBytes = kStages * kStage + 256 + 1024 /* alignment slack */;
};

constexpr int kEpiWarps = 8;                  // two per TMEM lane quarter
constexpr int kGroupM = 16;                   // row tiles per group of the tile order (4 .. 32: same time)
constexpr int kThreads = 64 + 32 * kEpiWarps;

// The epilogue of one 128 x BN tile whose values are in tile_s (column-
// major [BN][128]): the functor per element (E::load, then E::apply, see
// dalm_tc.cuh) -- its per-column reduction terms
// summed over each warp's 32 rows in FP32 (FP64 arithmetic runs at a small
// fraction of the FP32 rate on this part) into red_s[4][BN][NR] -- then the
// aligned pieces of the values it returns (po).  Run by the kEpiWarps warps
// of a CTA (etid = 0 .. 32 kEpiWarps - 1): warp w covers rows q*32 + lane of
// the tile (q = w mod 4) and the columns cb .. cb + BN/2 - 1.  The warps meet
// at named barrier 1 when pieces are written (an aborted CTA skips the work,
// ok = false, but not the barriers).
template <class E, int BN>
__device__ __forceinline__ void tile_epilogue(const E& epi, const PieceOut& po, bool ok, int i, int M, int N,
                                              int n0, int q, int cb, int lane, int etid, float* tile_s,
                                              double* red_s, float* max_s) {
    constexpr int NR = E::NRED > 0 ? E::NRED : 1;
    constexpr int CPT = BN / 2;
    float* my = tile_s + q * 32 + lane;
    if (ok) {
        // groups of G columns: the state loads of the whole group are issued
        // before any of the group's stores, so that they are in flight at once
        constexpr int G = 8;
        static_assert(CPT % G == 0, "column groups");
        for (int c0 = 0; c0 < CPT; c0 += G) {
            typename E::State st[G];
#pragma unroll
            for (int u = 0; u < G; ++u) {
                const int j = n0 + cb + c0 + u;
                if (i < M && j < N) st[u] = epi.load(i, j);
            }
#pragma unroll
            for (int u = 0; u < G; ++u) {
                const int c = c0 + u, j = n0 + cb + c;
                float rv[NR];
#pragma unroll
                for (int r = 0; r < NR; ++r) rv[r] = 0.0f;
                float ret = 0.0f;
                if (i < M && j < N) ret = epi.apply(i, j, my[(cb + c) * kBM], st[u], rv);
                my[(cb + c) * kBM] = ret;
                if constexpr (E::NRED > 0) {
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        const float sv = warp_sum_f(rv[r]);
                        if (lane == 0) red_s[((q * BN) + cb + c) * NR + r] = (double)sv;
                    }
                }
            }
        }
    }
    if (po.np > 0) {
        // the largest magnitude of each column over the tile's 128 rows sets
        // the grid of its pieces; two threads scan each column
        constexpr int kEpiThreads = 32 * kEpiWarps;
        static_assert(kEpiThreads == 2 * BN, "two threads per column");
        asm volatile("bar.sync 1, %0;" ::"r"(kEpiThreads) : "memory");
        const int col = etid >> 1, half = etid & 1;
        float mx = 0.0f;
        if (ok) {
            const float4* cp = reinterpret_cast<const float4*>(tile_s + col * kBM + half * 64);
#pragma unroll 4
            for (int t = 0; t < 16; ++t) {
                const float4 f = cp[t];
                mx = fmaxf(mx, fmaxf(fmaxf(fabsf(f.x), fabsf(f.y)), fmaxf(fabsf(f.z), fabsf(f.w))));
            }
        }
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
        if (half == 0) max_s[col] = mx;
        asm volatile("bar.sync 1, %0;" ::"r"(kEpiThreads) : "memory");
        if (ok && i < M) {
#pragma unroll 2
            for (int c = 0; c < CPT; ++c) {
                const int j = n0 + cb + c;
                if (j >= N) break;
                float p0, p1, p2;
                split_aligned(my[(cb + c) * kBM], max_s[cb + c], p0, p1, p2);
                const int64_t o = (int64_t)j * po.ld + i;
                po.p[0][o] = __float2bfloat16_rn(p0);
                if (po.np > 1) po.p[1][o] = __float2bfloat16_rn(p1);
                if (po.np > 2) po.p[2][o] = __float2bfloat16_rn(p2);
            }
        }
    }
}

// Sum over the tile's four row quarters of red_s, one partial per (row block,
// column): part[(row_block * N + j) * 4 + r].
template <int BN, int NR>
__device__ __forceinline__ void write_partials(const double* red_s, double* part, int tile_m, int n0, int N) {
    for (int idx = threadIdx.x; idx < BN * NR; idx += blockDim.x) {
        const int c = idx / NR, r = idx % NR;
        const int j = n0 + c;
        if (j < N) {
            double s = 0.0;
            for (int qq = 0; qq < 4; ++qq) s += red_s[((qq * BN) + c) * NR + r];
            part[((int64_t)tile_m * N + j) * kPartStride + r] = s;
        }
    }
}

template <class E, int NPA, int NPX, int BN>
__global__ void __launch_bounds__(kThreads, 1)
sweep_kernel(const __grid_constant__ Maps maps, const Terms tl, int M, int N, int K, E epi, PieceOut po,
             double* __restrict__ part, const int32_t* __restrict__ active, int* __restrict__ err, int ksplit,
             int defer, float* __restrict__ wk) {
    static_assert(BN == 128 || BN == 64, "tile width");
    constexpr int NR = E::NRED > 0 ? E::NRED : 1;
    constexpr int kMmaPerBlock = kKB / kMmaK;  // 4 or 2
    constexpr uint32_t kIdesc = instr_desc_bf16(kBM, BN);
    constexpr uint32_t kTmemCols = 4 * BN;     // hi[0], hi[1], lo[0], lo[1]
    constexpr int CPT = BN / 2;                // columns per epilogue thread
    using S = Cfg<BN, NPA, NPX>;
    constexpr int kStages = S::kStages;

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * S::kStage);
    uint64_t* empty = full + kStages;
    uint64_t* acc_full = empty + kStages;   // [2]
    uint64_t* acc_empty = acc_full + 2;     // [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
    int* flags = reinterpret_cast<int*>(tmem_slot + 1);  // [0]: some column active, [1]: abort
    // after the main loop the ring holds the epilogue's scratch: the tile's
    // values [BN][128] (column-major), the per-column reduction terms
    // [4][BN][NR] doubles and the per-column maxima [BN]
    float* tile_s = reinterpret_cast<float*>(smem);
    double* red_s = reinterpret_cast<double*>(tile_s + BN * kBM);
    float* max_s = reinterpret_cast<float*>(red_s + 4 * BN * NR);
    static_assert((2 * kStages + 4) * 8 + 12 <= 256, "barrier area");
    static_assert(BN * kBM * 4 + 4 * BN * NR * 8 + BN * 4 <= kStages * S::kStage, "epilogue scratch");

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // tile order: groups of kGroupM row tiles, column tiles within a group, so
    // that the CTAs resident at one time share row panels of A and column
    // panels of X in L2 (row-major order streams every column panel once per
    // wave)
    const int tiles_m = (M + kBM - 1) / kBM, tiles_n = (N + BN - 1) / BN;
    // split K (ksplit > 1): CTA z of a tile takes the chunks [c0, c1) and
    // leaves its FP32 sums in wk for finish_kernel; defer (ksplit == 1): the
    // whole K range, the sums to wk, the epilogue to finish_kernel
    const int ntiles = tiles_m * tiles_n;
    const int z = blockIdx.x / ntiles, tid = blockIdx.x - z * ntiles;
    const int per_group = kGroupM * tiles_n;
    const int group = tid / per_group, first_m = group * kGroupM;
    const int gsz = min(kGroupM, tiles_m - first_m);
    const int in_group = tid % per_group;
    const int tile_m = first_m + in_group % gsz, tile_n = in_group / gsz;
    const int m0 = tile_m * kBM, n0 = tile_n * BN;
    const int kblocks = (K + kKB - 1) / kKB;
    const int nchunks = (kblocks + kKBPerChunk - 1) / kKBPerChunk;
    const int cps = (nchunks + ksplit - 1) / ksplit;
    const int c0 = min(nchunks, z * cps), c1 = min(nchunks, c0 + cps);
    const int kb0 = c0 * kKBPerChunk, kb1 = min(kblocks, c1 * kKBPerChunk);
    const bool split = ksplit > 1 || defer != 0;
    const int nterms = tl.n;
    bool has_lo = false;
#pragma unroll
    for (int t = 0; t < kMaxTerms; ++t) has_lo |= t < nterms && (tl.ia[t] | tl.ix[t]) != 0;

    if (threadIdx.x == 0) {
        flags[0] = 0;
        flags[1] = 0;
    }
    __syncthreads();
    if (active != nullptr) {
        for (int c = threadIdx.x; c < BN; c += blockDim.x)
            if (n0 + c < N && active[n0 + c]) flags[0] = 1;
    } else if (threadIdx.x == 0) {
        flags[0] = 1;
    }
    __syncthreads();
    if (!flags[0]) {
        if (split) return;  // finish_kernel writes the partials
        if constexpr (E::NRED > 0) {
            for (int c = threadIdx.x; c < BN; c += blockDim.x)
                if (n0 + c < N)
                    for (int r = 0; r < NR; ++r) part[((int64_t)tile_m * N + n0 + c) * kPartStride + r] = 0.0;
        }
        return;
    }

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], kEpiWarps);  // one arrival per epilogue warp
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------------------------------------------- TMA producer
        if (lane == 0) {
#pragma unroll
            for (int p = 0; p < NPA; ++p) prefetch_map(&maps.a[p]);
#pragma unroll
            for (int p = 0; p < NPX; ++p) prefetch_map(&maps.x[p]);
            int issued = 0;
            for (int lk = 0; lk < kb1 - kb0; ++lk) {
                const int kb = kb0 + lk;
                const int s = lk % kStages;
                const uint32_t ph = (uint32_t)(lk / kStages) & 1u;
                if (!mbar_wait(&empty[s], ph ^ 1u)) {
                    atomicCAS(err, ERR_NONE, ERR_WAIT_EMPTY);
                    atomicExch(&flags[1], 1);
                    break;
                }
                if (*(volatile int*)&flags[1]) break;
                uint8_t* st = smem + s * S::kStage;
                mbar_expect_tx(&full[s], (uint32_t)S::kStage);
#pragma unroll
                for (int p = 0; p < NPA; ++p) tma_load_2d(st + p * S::kATile, &maps.a[p], &full[s], kb * kKB, m0);
#pragma unroll
                for (int p = 0; p < NPX; ++p)
                    tma_load_2d(st + NPA * S::kATile + p * S::kXTile, &maps.x[p], &full[s], kb * kKB, n0);
                issued = lk + 1;
            }
            for (int lk = (issued > kStages ? issued - kStages : 0); lk < issued; ++lk)
                mbar_wait(&full[lk % kStages], (uint32_t)(lk / kStages) & 1u);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issuer
        if (lane == 0) {
            bool ok = true;
            for (int lc = 0; lc < c1 - c0 && ok; ++lc) {
                const int c = c0 + lc, b = lc & 1;
                // the epilogue has drained this buffer pair (chunk c - 2)
                if (!mbar_wait(&acc_empty[b], ((uint32_t)(lc >> 1) & 1u) ^ 1u)) {
                    atomicCAS(err, ERR_NONE, ERR_WAIT_ACC);
                    atomicExch(&flags[1], 1);
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t d_hi = tmem + (uint32_t)(b * BN), d_lo = tmem + (uint32_t)(2 * BN + b * BN);
                bool first_hi = true, first_lo = true;
                const int kb_end = min(kblocks, (c + 1) * kKBPerChunk);
                for (int kb = c * kKBPerChunk; kb < kb_end; ++kb) {
                    const int lk = kb - kb0;
                    const int s = lk % kStages;
                    if (!mbar_wait(&full[s], (uint32_t)(lk / kStages) & 1u)) {
                        atomicCAS(err, ERR_NONE, ERR_WAIT_FULL);
                        atomicExch(&flags[1], 1);
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t st = smem_u32(smem + s * S::kStage);
                    // unrolled over the term slots so that the term list is
                    // read from the kernel parameters, not from a local copy
#pragma unroll
                    for (int t = 0; t < kMaxTerms; ++t) {
                        if (t >= nterms) break;
                        const bool hi = (tl.ia[t] | tl.ix[t]) == 0;
                        const uint32_t a_addr = st + tl.ia[t] * S::kATile;
                        const uint32_t x_addr = st + NPA * S::kATile + tl.ix[t] * S::kXTile;
                        const uint32_t d = hi ? d_hi : d_lo;
                        bool& first = hi ? first_hi : first_lo;
#pragma unroll
                        for (int k = 0; k < kMmaPerBlock; ++k) {
                            const uint64_t ad = smem_desc<kKB * 2>(a_addr + k * kMmaK * 2);
                            const uint64_t bd = smem_desc<kKB * 2>(x_addr + k * kMmaK * 2);
                            mma_bf16(d, ad, bd, kIdesc, first ? 0u : 1u);
                            first = false;
                        }
                    }
                    mma_commit(&empty[s]);
                }
                mma_commit(&acc_full[b]);
            }
            // after an abort, wait until every MMA issued has completed so
            // that none is still writing TMEM when it is freed
            if (!ok) {
                mma_commit(&acc_full[0]);
                mbar_wait(&acc_full[0], 0u);
                mbar_wait(&acc_full[0], 1u);
            }
        }
        __syncwarp();
    } else {
        // -------------------------------------------------------- epilogue
        const int ew = warp - 2;
        const int q = warp & 3;        // TMEM lane quarter this warp may access
        const int cb = (ew >> 2) * CPT;  // first column of this warp's half
        const int i = m0 + q * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
        float sum[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) sum[c] = 0.0f;
        bool ok = true;
        for (int ch = 0; ch < c1 - c0; ++ch) {
            const int b = ch & 1;
            bool ready = true;
            if (lane == 0) ready = mbar_wait(&acc_full[b], (uint32_t)(ch >> 1) & 1u);
            ready = __shfl_sync(0xffffffffu, ready ? 1 : 0, 0) != 0;
            if (!ready || *(volatile int*)&flags[1]) {
                if (lane == 0 && !ready) {
                    atomicCAS(err, ERR_NONE, ERR_WAIT_ACC);
                    atomicExch(&flags[1], 1);
                }
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int c0 = 0; c0 < CPT; c0 += 32) {
                float vh[32], vl[32];
                tmem_ld32(lane_addr + (uint32_t)(b * BN + cb + c0), vh);
                if (has_lo) tmem_ld32(lane_addr + (uint32_t)(2 * BN + b * BN + cb + c0), vl);
#pragma unroll
                for (int cc = 0; cc < 32; ++cc) sum[c0 + cc] += has_lo ? vh[cc] + vl[cc] : vh[cc];
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
        }
        if (split) {
            // this slice's sums; finish_kernel adds the slices in order
            const int64_t Mp = (int64_t)tiles_m * kBM;
            if (ok) {
#pragma unroll
                for (int c = 0; c < CPT; ++c) {
                    const int j = n0 + cb + c;
                    if (j < N) wk[((int64_t)z * N + j) * Mp + i] = sum[c];
                }
            }
        } else if constexpr (BN == 128) {
            // (fused epilogue: 128-wide tiles only; the host defers the
            // epilogue of 64-wide ones)
            // the tile's values go to shared memory (the ring is idle: every
            // MMA, and so every copy it waited for, has completed)
            float* my = tile_s + q * 32 + lane;
            if (ok) {
#pragma unroll
                for (int c = 0; c < CPT; ++c) my[(cb + c) * kBM] = sum[c];
            }
            tile_epilogue<E, BN>(epi, po, ok, i, M, N, n0, q, cb, lane, threadIdx.x - 64, tile_s, red_s, max_s);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if constexpr (E::NRED > 0 && BN == 128) {
        if (!flags[1] && !split) write_partials<BN, NR>(red_s, part, tile_m, n0, N);
    }
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}


// The second half of a split-K or deferred sweep: one CTA of kBM threads
// per (column, kFinRB consecutive 128-row blocks) adds the ksplit slices of
// wk in slice order (FP32) and runs the tile epilogue there: the functor, the
// per-column reduction terms of each row block (FP32 warp sums over 32 rows,
// the four row quarters added in order in FP64, as in the sweep's own
// epilogue) and the aligned BF16 pieces on the grid of the largest magnitude
// of each 128-row block.  A CTA reads each array of its column in runs of up
// to kFinRB x 512 contiguous bytes; rbs (1 .. kFinRB) row blocks per CTA.
#ifndef L1_FIN_RB
#define L1_FIN_RB 2  // measured on the 4096 x 4000 solve: 1 5.13 s, 2 4.94 s, 4 5.02 s, 8 5.24 s
#endif
constexpr int kFinRB = L1_FIN_RB;
static_assert(kFinRB >= 1 && kFinRB <= 8, "row blocks per finish CTA");

// The sums are wk[(z * N + j) * ldw + i] over the slices z < ksplit; with
// colscale they are multiplied by colscale[j] before the epilogue.
template <class E>
__global__ void __launch_bounds__(kBM)
finish_kernel(int M, int N, int ksplit, const float* __restrict__ wk, int64_t ldw, const float* __restrict__ colscale,
              E epi, PieceOut po, double* __restrict__ part, const int32_t* __restrict__ active, int rbs) {
    constexpr int NR = E::NRED > 0 ? E::NRED : 1;
    __shared__ double red_s[4][kFinRB][NR];
    __shared__ float max_s[4][kFinRB];
    const int tiles_m = (M + kBM - 1) / kBM;
    const int groups = (tiles_m + rbs - 1) / rbs;
    const int j = blockIdx.x / groups, rb0 = (blockIdx.x % groups) * rbs;
    const int t = threadIdx.x, q = t >> 5, lane = t & 31;
    const int nrb = min(rbs, tiles_m - rb0);
    if (active != nullptr && !active[j]) {
        if constexpr (E::NRED > 0) {
            if (t < nrb * NR) part[((int64_t)(rb0 + t / NR) * N + j) * kPartStride + t % NR] = 0.0;
        }
        return;
    }
    float v[kFinRB];
    typename E::State st[kFinRB];
    const float cs = colscale ? colscale[j] : 1.0f;
#pragma unroll
    for (int u = 0; u < kFinRB; ++u) {
        const int i = (rb0 + u) * kBM + t;
        v[u] = 0.0f;
        if (u < nrb && i < M) {
            for (int z = 0; z < ksplit; ++z) v[u] += wk[((int64_t)z * N + j) * ldw + i];
            if (colscale) v[u] *= cs;
            st[u] = epi.load(i, j);
        }
    }
#pragma unroll
    for (int u = 0; u < kFinRB; ++u) {
        if (u >= nrb) break;
        const int i = (rb0 + u) * kBM + t;
        float rv[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) rv[r] = 0.0f;
        float ret = 0.0f;
        if (i < M) ret = epi.apply(i, j, v[u], st[u], rv);
        v[u] = ret;
        if constexpr (E::NRED > 0) {
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const float sv = warp_sum_f(rv[r]);
                if (lane == 0) red_s[q][u][r] = (double)sv;
            }
        }
        if (po.np > 0) {
            float mx = fabsf(ret);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) max_s[q][u] = mx;
        }
    }
    __syncthreads();
    if (po.np > 0) {
#pragma unroll
        for (int u = 0; u < kFinRB; ++u) {
            if (u >= nrb) break;
            const int i = (rb0 + u) * kBM + t;
            if (i >= M) break;
            const float mx = fmaxf(fmaxf(max_s[0][u], max_s[1][u]), fmaxf(max_s[2][u], max_s[3][u]));
            float p0, p1, p2;
            split_aligned(v[u], mx, p0, p1, p2);
            const int64_t o = (int64_t)j * po.ld + i;
            po.p[0][o] = __float2bfloat16_rn(p0);
            if (po.np > 1) po.p[1][o] = __float2bfloat16_rn(p1);
            if (po.np > 2) po.p[2][o] = __float2bfloat16_rn(p2);
        }
    }
    if constexpr (E::NRED > 0) {
        if (t < nrb * NR) {
            const int u = t / NR, r = t % NR;
            part[((int64_t)(rb0 + u) * N + j) * kPartStride + r] =
                red_s[0][u][r] + red_s[1][u][r] + red_s[2][u][r] + red_s[3][u][r];
        }
    }
}

}  // namespace tc16
}  // namespace l1
