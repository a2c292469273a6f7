// tcgen05 tensor-core sweeps for sm_103a: OUT(M x N) = sum_t Aop_t(M x K) X_t(K x N)
// with the same fused-epilogue contract as gemm_simt.cuh.
//
// Each term t is a pair of operand "pieces" in the layouts of the SIMT path
// (Aop_t K-major row-major, X_t column-major = K-major).  Summing terms gives
// split-precision products: with TF32 pieces a = a1 + a2 (+ a3) the products
// a1 x1 + a1 x2 + a2 x1 recover FP32-level products on TF32 tensor cores.
//
// Accumulation.  Successive tcgen05.mma into one TMEM accumulator lose about
// four bits over a few hundred steps (measured on this part), which the DALM
// y-step amplifies by cond(B B^T).  The K loop is therefore cut into chunks
// of CHUNK K blocks; each chunk accumulates in one of two TMEM buffers, and
// the epilogue warps drain a finished chunk into Kahan-compensated FP32
// register sums while the MMA warp fills the other buffer.
//
// Structure of one CTA (one 128 x BN output tile, non-persistent):
//   warp 0      TMA producer: for every (term, K block) loads a 128 x 32-float
//               tile of Aop_t and a BN x 32-float tile of X_t (128B swizzle)
//               into a kStages-deep ring ("full" mbarriers)
//   warp 1      allocates 2*BN TMEM columns, issues tcgen05.mma (kind::tf32 or
//               kind::f16) from one thread; tcgen05.commit frees ring slots
//               ("empty") and hands finished chunks to the epilogue
//   warps 2..5  epilogue: tcgen05.ld of each chunk (TMEM lane = output row),
//               compensated sums, then the functor per element and the
//               per-column reductions
// Every mbarrier wait is bounded; a wait that runs out records an error code
// in *err and the CTA leaves its loops, waits (bounded) for its own copies,
// frees TMEM and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "gemm_simt.cuh"

#ifndef L1_TC_KAHAN
#define L1_TC_KAHAN 1
#endif

namespace l1 {
namespace tc {

constexpr int kMaxTerms = 6;
constexpr int kBM = 128;
constexpr int kRowBytes = 128;  // one swizzle-128B row = 32 fp32 or 64 bf16
constexpr int kStages = 4;
constexpr int kThreads = 192;   // 6 warps
constexpr uint32_t kSpinLimit = 1u << 26;

enum : int { ERR_NONE = 0, ERR_WAIT_FULL = 1, ERR_WAIT_EMPTY = 2, ERR_WAIT_ACC = 3, ERR_WAIT_DRAIN = 4 };

struct TermMaps {
    CUtensorMap a[kMaxTerms];
    CUtensorMap x[kMaxTerms];
};

template <int BN>
struct Smem {
    static constexpr int kATile = kBM * kRowBytes;  // 16 KB
    static constexpr int kXTile = BN * kRowBytes;
    static constexpr int kStage = kATile + kXTile;
    // barriers and flags after the ring; the epilogue's reduction scratch
    // reuses the ring once the last chunk has been drained
    static constexpr int kBytes = kStages * kStage + 256 + 1024 /* alignment slack */;
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

// bounded wait: false when the limit ran out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (uint32_t i = 0; i < kSpinLimit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > 64) __nanosleep(32);
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

// instruction descriptor, dense, FP32 accumulator, both operands K-major
// a_fmt/b_fmt: 1 = BF16 (kind::f16), 2 = TF32 (kind::tf32)
__host__ __device__ constexpr uint32_t instr_desc(int fmt, int M, int N) {
    return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

template <bool TF32>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    if constexpr (TF32) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
    }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------------ kernel
template <class E, int BN, bool TF32, int CHUNK>
__global__ void __launch_bounds__(kThreads, 1)
gemm_tc_kernel(const __grid_constant__ TermMaps maps, int terms, int M, int N, int K, E epi,
               double* __restrict__ part, const int32_t* __restrict__ active, int* __restrict__ err) {
    constexpr int NR = E::NRED > 0 ? E::NRED : 1;
    constexpr int kElemPerRow = TF32 ? 32 : 64;           // K elements per 128-byte row
    constexpr int kMmaK = TF32 ? 8 : 16;                   // K per tcgen05.mma
    constexpr int kMmaPerBlock = kElemPerRow / kMmaK;      // 4
    constexpr uint32_t kIdesc = instr_desc(TF32 ? 2 : 1, kBM, BN);
    constexpr uint32_t kTmemCols = 2 * BN;                 // two accumulator buffers
    static_assert(BN == 32 || BN == 64 || BN == 128, "tile width");
    using S = Smem<BN>;

    extern __shared__ uint8_t smem_raw[];
    // 1024-byte alignment for the 128B-swizzled tiles
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * S::kStage);
    uint64_t* empty = full + kStages;
    uint64_t* acc_full = empty + kStages;   // [2] chunk finished in buffer b
    uint64_t* acc_empty = acc_full + 2;     // [2] buffer b drained
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
    int* flags = reinterpret_cast<int*>(tmem_slot + 1);  // [0]: any active column, [1]: abort
    double* red_s = reinterpret_cast<double*>(smem);      // [4][BN][NR], after the last drain
    static_assert(4 * BN * NR * 8 <= kStages * S::kStage, "reduction scratch");

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
    const int kblocks = (K + kElemPerRow - 1) / kElemPerRow;
    const int total = terms * kblocks;
    const int nchunks = (total + CHUNK - 1) / CHUNK;

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
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 4);  // one arrival per epilogue warp
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
            for (int t = 0; t < terms; ++t) {
                prefetch_map(&maps.a[t]);
                prefetch_map(&maps.x[t]);
            }
            int issued = 0;
            for (int it = 0; it < total; ++it) {
                const int s = it % kStages;
                const uint32_t ph = (uint32_t)(it / kStages) & 1u;
                if (!mbar_wait(&empty[s], ph ^ 1u)) {
                    atomicCAS(err, ERR_NONE, ERR_WAIT_EMPTY);
                    atomicExch(&flags[1], 1);
                    break;
                }
                if (*(volatile int*)&flags[1]) break;
                const int t = it / kblocks, kb = it % kblocks;
                uint8_t* a_dst = smem + s * S::kStage;
                uint8_t* x_dst = a_dst + S::kATile;
                mbar_expect_tx(&full[s], (uint32_t)S::kStage);
                tma_load_2d(a_dst, &maps.a[t], &full[s], kb * kElemPerRow, m0);
                tma_load_2d(x_dst, &maps.x[t], &full[s], kb * kElemPerRow, n0);
                issued = it + 1;
            }
            // bounded wait for the copies still in flight before leaving
            for (int it = (issued > kStages ? issued - kStages : 0); it < issued; ++it)
                mbar_wait(&full[it % kStages], (uint32_t)(it / kStages) & 1u);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issuer
        if (lane == 0) {
            for (int it = 0; it < total; ++it) {
                const int s = it % kStages;
                const uint32_t ph = (uint32_t)(it / kStages) & 1u;
                const int chunk = it / CHUNK;
                const int b = chunk & 1;
                const bool first = (it % CHUNK) == 0;
                const bool last = (it % CHUNK) == CHUNK - 1 || it == total - 1;
                if (first && !mbar_wait(&acc_empty[b], ((uint32_t)(chunk >> 1) & 1u) ^ 1u)) {
                    atomicCAS(err, ERR_NONE, ERR_WAIT_DRAIN);
                    atomicExch(&flags[1], 1);
                    break;
                }
                if (!mbar_wait(&full[s], ph)) {
                    atomicCAS(err, ERR_NONE, ERR_WAIT_FULL);
                    atomicExch(&flags[1], 1);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t a_addr = smem_u32(smem + s * S::kStage);
                const uint32_t x_addr = a_addr + S::kATile;
                const uint32_t d = tmem + (uint32_t)(b * BN);
#pragma unroll
                for (int k = 0; k < kMmaPerBlock; ++k) {
                    const uint64_t ad = smem_desc(a_addr + k * kMmaK * (TF32 ? 4 : 2));
                    const uint64_t bd = smem_desc(x_addr + k * kMmaK * (TF32 ? 4 : 2));
                    mma<TF32>(d, ad, bd, kIdesc, (first && k == 0) ? 0u : 1u);
                }
                mma_commit(&empty[s]);
                if (last) mma_commit(&acc_full[b]);
            }
        }
        __syncwarp();
    } else {
        // -------------------------------------------------------- epilogue
        const int q = warp & 3;  // TMEM lane quarter this warp may access
        const int i = m0 + q * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
        float sum[BN], comp[BN];
#pragma unroll
        for (int c = 0; c < BN; ++c) sum[c] = comp[c] = 0.0f;
        bool ok = true;
        for (int chunk = 0; chunk < nchunks && ok; ++chunk) {
            const int b = chunk & 1;
            bool ready = true;
            if (lane == 0) ready = mbar_wait(&acc_full[b], (uint32_t)(chunk >> 1) & 1u);
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
            for (int c0 = 0; c0 < BN; c0 += 16) {
                float v[16];
                tmem_ld16(lane_addr + (uint32_t)(b * BN + c0), v);
#pragma unroll
                for (int cc = 0; cc < 16; ++cc) {
#if L1_TC_KAHAN
                    // Kahan: sum + v with the running compensation
                    const float y = v[cc] - comp[c0 + cc];
                    const float t = sum[c0 + cc] + y;
                    comp[c0 + cc] = (t - sum[c0 + cc]) - y;
                    sum[c0 + cc] = t;
#else
                    sum[c0 + cc] += v[cc];
#endif
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
        }
        if (ok) {
#pragma unroll
            for (int c = 0; c < BN; ++c) {
                const int j = n0 + c;
                double red[NR];
#pragma unroll
                for (int r = 0; r < NR; ++r) red[r] = 0.0;
                if (i < M && j < N) epi(i, j, sum[c] - comp[c], red);
                if constexpr (E::NRED > 0) {
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        const double sv = warp_sum(red[r]);
                        if (lane == 0) red_s[((q * BN) + c) * NR + r] = sv;
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
