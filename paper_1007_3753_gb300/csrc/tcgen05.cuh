// tcgen05 tensor-core sweeps for sm_103a with the fused-epilogue contract of
// gemm_simt.cuh:  OUT(M x N) = sum_t  A_{ia(t)} (M x K)  X_{ix(t)} (K x N).
//
// Operand pieces.  A value a is carried as TF32 pieces a = a_0 + a_1 (+ a_2)
// (round-to-nearest splits, see tc.cuh); the product a x is recovered from
// the piece products a_0 x_0 + a_0 x_1 + a_1 x_0 (FP32-level).  All pieces
// of one K block are loaded once into shared memory and every term of the
// list reads them from there, so a three-term product moves each byte from
// L2 once instead of three times.  Layouts are those of the CUDA-core path:
// A_p row-major (K contiguous), X_p column-major (K contiguous).
//
// Accumulation.  Long chains of tcgen05.mma into one TMEM accumulator round
// with a bias (measured on this part) that the DALM iteration accumulates.
// Each (K block, term) product therefore goes to one of kAccBufs TMEM
// buffers, and the epilogue warps drain it into Kahan-compensated FP32
// register sums while the MMA warp fills the next buffer.
//
// One CTA computes a 128 x BN output tile (non-persistent):
//   warp 0      TMA producer: per K block, NPA tiles of 128 x 32 floats and
//               NPX tiles of BN x 32 floats (128-byte swizzle) into a ring
//   warp 1      allocates kAccBufs * BN TMEM columns; one thread issues the
//               tcgen05.mma (kind::tf32) of every term; tcgen05.commit frees
//               ring slots and hands each finished product to the epilogue
//   warps 2..9  epilogue: warp w reads TMEM lane quarter w % 4 (output rows)
//               and half of the columns; compensated sums, then the functor
//               per element and deterministic per-column reductions
// Every mbarrier wait is bounded; a wait that runs out records an error code
// in *err, and the CTA leaves its loops, waits (bounded) for its own copies,
// frees TMEM and returns.
#pragma once

#include <cuda.h>

#include "common.cuh"
#include "gemm_simt.cuh"

namespace l1 {
namespace tc {

constexpr int kMaxPieces = 3;
constexpr int kMaxTerms = 6;
constexpr int kBM = 128;
constexpr int kRowBytes = 128;  // one swizzle-128B row = 32 fp32
constexpr int kElemPerRow = 32;
constexpr int kMmaK = 8;        // K of one kind::tf32 MMA
// epilogue: one warp per (TMEM lane quarter, 32 output columns)
__host__ __device__ constexpr int epi_warps(int bn) { return bn / 8; }
__host__ __device__ constexpr int cta_threads(int bn) { return 64 + 32 * epi_warps(bn); }
constexpr int kAccBufs = 4;     // TMEM accumulator buffers
constexpr uint32_t kSpinLimit = 1u << 26;

enum : int { ERR_NONE = 0, ERR_WAIT_FULL = 1, ERR_WAIT_EMPTY = 2, ERR_WAIT_ACC = 3, ERR_WAIT_DRAIN = 4 };

struct PieceMaps {
    CUtensorMap a[kMaxPieces];
    CUtensorMap x[kMaxPieces];
};

struct TermList {
    int n;
    int ia[kMaxTerms];
    int ix[kMaxTerms];
};

template <int BN, int NPA, int NPX>
struct Smem {
    static constexpr int kATile = kBM * kRowBytes;  // 16 KB
    static constexpr int kXTile = BN * kRowBytes;
    static constexpr int kStage = NPA * kATile + NPX * kXTile;
    // two CTAs per SM for 64-column tiles with up to two pieces per operand
    static constexpr bool kTwoPerSm = BN == 64 && NPA * NPX <= 4;
    static constexpr int kBudget = kTwoPerSm ? 104 * 1024 : 220 * 1024;
    static constexpr int kStages = (kBudget / kStage) > 8 ? 8 : (kBudget / kStage);
    static_assert(kStages >= 2, "stage does not fit twice");
    // barriers and flags after the ring; the epilogue's reduction scratch
    // reuses the ring once the last product has been drained
    static constexpr int kBytes = kStages * kStage + 512 + 1024 /* alignment slack */;
};

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: false when the limit ran out.  try_wait already suspends
// the thread for a short hardware window, so the hot path spins; sleeping
// starts only after 2^16 polls (a stalled pipeline), and the total is capped
// at kSpinLimit polls (seconds).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (uint32_t i = 0; i < kSpinLimit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > (1u << 16)) __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_map(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// tcgen05 shared-memory matrix descriptor: K-major, 128-byte swizzle,
// 8-row core groups 1024 bytes apart (SBO), start address advanced along K
// inside the swizzle row for successive MMAs.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);        // start address
    d |= (uint64_t)1 << 16;                         // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;               // stride byte offset
    d |= (uint64_t)1 << 46;                         // descriptor version
    d |= (uint64_t)2 << 61;                         // SWIZZLE_128B
    return d;
}

// instruction descriptor: dense, FP32 accumulator, TF32 operands, both K-major
__host__ __device__ constexpr uint32_t instr_desc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------------ kernel
template <class E, int BN, int NPA, int NPX>
__global__ void __launch_bounds__(cta_threads(BN), Smem<BN, NPA, NPX>::kTwoPerSm ? 2 : 1)
gemm_tc_kernel(const __grid_constant__ PieceMaps maps, const TermList tl, int M, int N, int K, E epi,
               double* __restrict__ part, const int32_t* __restrict__ active, int* __restrict__ err) {
    constexpr int NR = E::NRED > 0 ? E::NRED : 1;
    constexpr int kMmaPerBlock = kElemPerRow / kMmaK;  // 4
    constexpr uint32_t kIdesc = instr_desc_tf32(kBM, BN);
    constexpr uint32_t kTmemCols = kAccBufs * BN;
    static_assert(BN == 64 || BN == 128, "tile width");
    static_assert(kTmemCols <= 512, "TMEM columns");
    using S = Smem<BN, NPA, NPX>;
    constexpr int kStages = S::kStages;

    extern __shared__ uint8_t smem_raw[];
    // 1024-byte alignment for the 128B-swizzled tiles
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * S::kStage);
    uint64_t* empty = full + kStages;
    uint64_t* acc_full = empty + kStages;       // [kAccBufs] product finished in buffer b
    uint64_t* acc_empty = acc_full + kAccBufs;  // [kAccBufs] buffer b drained
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + kAccBufs);
    int* flags = reinterpret_cast<int*>(tmem_slot + 1);  // [0]: any active column, [1]: abort
    double* red_s = reinterpret_cast<double*>(smem);      // [4][BN][NR], after the last drain
    static_assert(4 * BN * NR * 8 <= kStages * S::kStage, "reduction scratch");

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
    const int kblocks = (K + kElemPerRow - 1) / kElemPerRow;
    const int nterms = tl.n;
    const int nprod = kblocks * nterms;  // products drained one by one

    if (threadIdx.x == 0) {
        flags[0] = 0;
        flags[1] = 0;
    }
    __syncthreads();
    if (active != nullptr) {
        if (threadIdx.x < BN && n0 + threadIdx.x < N && active[n0 + threadIdx.x]) flags[0] = 1;
    } else if (threadIdx.x == 0) {
        flags[0] = 1;
    }
    __syncthreads();
    if (!flags[0]) {
        if constexpr (E::NRED > 0) {
            if (threadIdx.x < BN && n0 + threadIdx.x < N)
                for (int r = 0; r < NR; ++r) part[((int64_t)blockIdx.y * N + n0 + threadIdx.x) * kPartStride + r] = 0.0;
        }
        return;
    }

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < kAccBufs; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], epi_warps(BN));  // one arrival per epilogue warp
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
            for (int kb = 0; kb < kblocks; ++kb) {
                const int s = kb % kStages;
                const uint32_t ph = (uint32_t)(kb / kStages) & 1u;
                if (!mbar_wait(&empty[s], ph ^ 1u)) {
                    atomicCAS(err, ERR_NONE, ERR_WAIT_EMPTY);
                    atomicExch(&flags[1], 1);
                    break;
                }
                if (*(volatile int*)&flags[1]) break;
                uint8_t* st = smem + s * S::kStage;
                mbar_expect_tx(&full[s], (uint32_t)S::kStage);
#pragma unroll
                for (int p = 0; p < NPA; ++p) tma_load_2d(st + p * S::kATile, &maps.a[p], &full[s], kb * kElemPerRow, m0);
#pragma unroll
                for (int p = 0; p < NPX; ++p)
                    tma_load_2d(st + NPA * S::kATile + p * S::kXTile, &maps.x[p], &full[s], kb * kElemPerRow, n0);
                issued = kb + 1;
            }
            // bounded wait for the copies still in flight before leaving
            for (int kb = (issued > kStages ? issued - kStages : 0); kb < issued; ++kb)
                mbar_wait(&full[kb % kStages], (uint32_t)(kb / kStages) & 1u);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int prod = 0;
            bool ok = true;
            for (int kb = 0; kb < kblocks && ok; ++kb) {
                const int s = kb % kStages;
                if (!mbar_wait(&full[s], (uint32_t)(kb / kStages) & 1u)) {
                    atomicCAS(err, ERR_NONE, ERR_WAIT_FULL);
                    atomicExch(&flags[1], 1);
                    break;
                }
                const uint32_t st = smem_u32(smem + s * S::kStage);
                for (int t = 0; t < nterms; ++t, ++prod) {
                    const int b = prod % kAccBufs;
                    if (!mbar_wait(&acc_empty[b], ((uint32_t)(prod / kAccBufs) & 1u) ^ 1u)) {
                        atomicCAS(err, ERR_NONE, ERR_WAIT_DRAIN);
                        atomicExch(&flags[1], 1);
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t a_addr = st + tl.ia[t] * S::kATile;
                    const uint32_t x_addr = st + NPA * S::kATile + tl.ix[t] * S::kXTile;
                    const uint32_t d = tmem + (uint32_t)(b * BN);
#pragma unroll
                    for (int k = 0; k < kMmaPerBlock; ++k) {
                        const uint64_t ad = smem_desc(a_addr + k * kMmaK * 4);
                        const uint64_t bd = smem_desc(x_addr + k * kMmaK * 4);
                        mma_tf32(d, ad, bd, kIdesc, k == 0 ? 0u : 1u);
                    }
                    mma_commit(&acc_full[b]);
                }
                if (ok) mma_commit(&empty[s]);
            }
        }
        __syncwarp();
    } else {
        // -------------------------------------------------------- epilogue
        constexpr int HC = 32;
        const int q = warp & 3;          // TMEM lane quarter this warp may access
        const int h = (warp - 2) >> 2;   // 32-column group
        const int cb = h * HC;
        const int i = m0 + q * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
        float sum[HC], comp[HC];
#pragma unroll
        for (int c = 0; c < HC; ++c) sum[c] = comp[c] = 0.0f;
        bool ok = true;
        for (int prod = 0; prod < nprod && ok; ++prod) {
            const int b = prod % kAccBufs;
            bool ready = true;
            if (lane == 0) ready = mbar_wait(&acc_full[b], (uint32_t)(prod / kAccBufs) & 1u);
            ready = __shfl_sync(0xffffffffu, ready ? 1 : 0, 0) != 0;
            if (!ready) {
                if (lane == 0) {
                    atomicCAS(err, ERR_NONE, ERR_WAIT_ACC);
                    atomicExch(&flags[1], 1);
                }
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int c0 = 0; c0 < HC; c0 += 32) {
                float v[32];
                tmem_ld32(lane_addr + (uint32_t)(b * BN + cb + c0), v);
#pragma unroll
                for (int cc = 0; cc < 32; ++cc) {
                    // Kahan: sum + v with the running compensation
                    const float y = v[cc] - comp[c0 + cc];
                    const float t = sum[c0 + cc] + y;
                    comp[c0 + cc] = (t - sum[c0 + cc]) - y;
                    sum[c0 + cc] = t;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
        }
        if (ok) {
#pragma unroll
            for (int c = 0; c < HC; ++c) {
                const int j = n0 + cb + c;
                double red[NR];
#pragma unroll
                for (int r = 0; r < NR; ++r) red[r] = 0.0;
                if (i < M && j < N) epi(i, j, sum[c] - comp[c], red);
                if constexpr (E::NRED > 0) {
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        const double sv = warp_sum(red[r]);
                        if (lane == 0) red_s[((q * BN) + cb + c) * NR + r] = sv;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if constexpr (E::NRED > 0) {
        if (!flags[1]) {
            for (int idx = threadIdx.x; idx < BN * NR; idx += blockDim.x) {
                const int c = idx / NR, r = idx % NR;
                const int j = n0 + c;
                if (j < N) {
                    double s = 0.0;
                    for (int qq = 0; qq < 4; ++qq) s += red_s[((qq * BN) + c) * NR + r];
                    part[((int64_t)blockIdx.y * N + j) * kPartStride + r] = s;
                }
            }
        }
    }
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

}  // namespace tc
}  // namespace l1
