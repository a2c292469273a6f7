// Uneven batches of independent (QP_lambda) problems (l1_setup_group): FISTA
// (Eq. 18, §IV-A) for thousands of dictionaries of different sizes in one
// persistent cooperative launch.
//
// Work.  The dictionaries are stored column-major (FP32 or BF16) in one
// allocation.  A work unit is (instance, tile of consecutive columns) sized so
// the tile (padding rows included) fits a 32 KB shared-memory buffer; a tile
// is one contiguous, 16-byte aligned region of the arena.  Each CTA owns a
// contiguous range of the active units of a step and
//   1. streams its tiles from HBM into two shared buffers with 1-D TMA bulk
//      copies (cp.async.bulk + mbarrier), two units in flight,
//   2. on entering an instance loads the rows of its residual r = b - A z
//      (from the previous step's accumulator) that it owns into registers,
//   3. reads each tile from shared memory ONCE into registers (a thread owns
//      16-byte words: 8 BF16 or 4 FP32 rows of up to 8 columns), forms its
//      partial dots of g_J = A_J^T r, and releases the buffer for the next
//      copy; one warp per column sums the partials and updates
//      x_J = soft(z_J + g_J/L, lambda/L), z_J = x_J + mu (x_J - x_J_old),
//   4. adds A_J z_J from the same registers to its rows' accumulator, which
//      goes to global memory (one atomic per row) only when the CTA leaves
//      the instance,
// so every element of every active dictionary is read from HBM once per step
// and from shared memory once.  CTAs are 256 threads with 81 KB of shared
// memory, two per SM, so that one CTA's barriers overlap the other's work.
// After the pass a bounded grid barrier, a per-instance finalisation
// (stopping rule of §VI-C, FISTA momentum), another barrier, and a rebuild
// of the active-instance work list (converged instances drop out:
// compaction).  The same kernel runs the batched power
// iteration for L = ||A_i||_2^2 and the final pass that forms A x for the
// objective.
#include <algorithm>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "common.cuh"

namespace l1 {

enum GroupMode : int { GM_FISTA = 0, GM_POWER_INIT = 1, GM_POWER = 2, GM_FINAL = 3 };

constexpr int kGThreads = 256;                // two CTAs per SM
constexpr int kGWarps = kGThreads / 32;
constexpr int kGMaxM = 4096;               // rows of an instance (RP <= 2 for BF16, 4 for FP32)
constexpr int kGShared = 1024;             // rows of an instance whose rows several threads own (acc_s)
constexpr int kGBufs = 2;                  // tile buffers per CTA (three measured slower, at one and at two CTAs per SM)
constexpr int kGTileBytes = 32 * 1024;     // A tile in shared memory
constexpr int kGPartials = 2048;           // dot partials of one unit (part_s)
constexpr uint32_t kGBarrierSpin = 1u << 26;

struct GroupState {
    int64_t count = 0;
    int prec = L1_A_FP32;
    double lambda = 0.0;
    std::vector<int32_t> hm, hn, hld, hucols;
    std::vector<int64_t> haoff, hboff, hxoff, hnunits;
    int64_t a_elems = 0, sum_m = 0, sum_n = 0;
    // device
    int32_t *m = nullptr, *n = nullptr, *ld = nullptr, *ucols = nullptr;
    int64_t *aoff = nullptr, *boff = nullptr, *xoff = nullptr, *nunits = nullptr;
    void* A = nullptr;
    float *b = nullptr, *x = nullptr, *z = nullptr, *racc[2] = {nullptr, nullptr};
    float *L = nullptr, *mu = nullptr, *cscale = nullptr;
    double *t = nullptr, *d2 = nullptr, *w2 = nullptr, *vv = nullptr, *rho = nullptr, *rel = nullptr;
    double *obj = nullptr, *res2 = nullptr;
    int32_t *active = nullptr, *status = nullptr, *iters = nullptr;
    int32_t *act = nullptr, *nact = nullptr;
    int64_t* upref = nullptr;
    unsigned *bar_count = nullptr, *bar_gen = nullptr;
    int* err = nullptr;
    int grid = 0;
    int smem = 0;
};

struct GArgs {
    int64_t count;
    int bf16;
    const int32_t *m, *n, *ld, *ucols;
    const int64_t *aoff, *boff, *xoff, *nunits;
    const void* A;
    const float* b;
    float *x, *z, *racc0, *racc1;
    float *L, *mu, *cscale;
    double *t, *d2, *w2, *vv, *rho, *rel, *obj, *res2;
    int32_t *active, *status, *iters;
    int32_t *act, *nact;
    int64_t* upref;
    unsigned *bar_count, *bar_gen;
    int* err;
    float lambda;
    double tol;
    int max_steps;
    int mode;
};

__device__ __forceinline__ float soft_g(float v, float a) { return v > a ? v - a : (v < -a ? v + a : 0.0f); }

// Grid-wide barrier for a cooperative launch (all blocks co-resident).  The
// wait is bounded: on expiry it records an error and returns false.
__device__ bool grid_sync(const GArgs& g, volatile int* abort) {
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned* gen = g.bar_gen;
        const unsigned my_gen = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(g.bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            *g.bar_count = 0;
            __threadfence();
            atomicAdd(g.bar_gen, 1u);
        } else {
            uint32_t spins = 0;
            while (*gen == my_gen) {
                if (++spins > kGBarrierSpin || *abort) {
                    atomicCAS(g.err, 0, 1);
                    ok = 0;
                    break;
                }
                if (spins > 1024) __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    if (!ok) *abort = 1;
    return ok != 0;
}

// ----------------------------------------------------------- TMA staging
__device__ __forceinline__ uint32_t g_smem(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 1-D bulk copy global -> shared completing on an mbarrier (both addresses
// 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void g_bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(g_smem(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(g_smem(dst)), "l"(src), "r"(bytes), "r"(g_smem(bar))
                 : "memory");
}

// bounded wait on an mbarrier phase: false when the limit ran out
__device__ __forceinline__ bool g_mbar_wait(uint64_t* bar, uint32_t parity) {
    for (uint32_t i = 0; i < kGBarrierSpin; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(g_smem(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (i > (1u << 16)) __nanosleep(64);
    }
    return false;
}

// Geometry of a work unit: slot k of the active list, instance i, its
// columns col0 .. col0+nc-1, and the instance's n, columns per unit, leading
// dimension and arena offset (so that the next unit needs no memory reads
// unless it starts a new instance).
struct UnitGeom {
    int k, i, col0, nc, n, uc, ld;
    int64_t aoff;
};

__device__ __forceinline__ UnitGeom geom_at(const GArgs& g, int k, int64_t local) {
    UnitGeom r;
    r.k = k;
    r.i = g.act[k];
    r.n = g.n[r.i];
    r.uc = g.ucols[r.i];
    r.ld = g.ld[r.i];
    r.aoff = g.aoff[r.i];
    r.col0 = (int)(local * r.uc);
    r.nc = min(r.uc, r.n - r.col0);
    return r;
}

// unit u: slot k with upref[k] <= u < upref[k+1] (binary search)
__device__ __forceinline__ UnitGeom geom_first(const GArgs& g, int64_t u, int nact) {
    int lo = 0, hi = nact;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (g.upref[mid] <= u) lo = mid;
        else hi = mid;
    }
    return geom_at(g, lo, u - g.upref[lo]);
}

// the unit after p in the active list
__device__ __forceinline__ UnitGeom geom_next(const GArgs& g, const UnitGeom& p) {
    if (p.col0 + p.uc < p.n) {
        UnitGeom r = p;
        r.col0 = p.col0 + p.uc;
        r.nc = min(p.uc, p.n - r.col0);
        return r;
    }
    return geom_at(g, p.k + 1, 0);
}

__device__ __forceinline__ void issue_tile(const GArgs& g, const UnitGeom& q, uint8_t* dst, uint64_t* bar) {
    const int es = g.bf16 ? 2 : 4;
    const int64_t e0 = q.aoff + (int64_t)q.col0 * q.ld;
    g_bulk_load(dst, static_cast<const uint8_t*>(g.A) + e0 * es, (uint32_t)((int64_t)q.nc * q.ld * es), bar);
}

__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }


// ------------------------------------------------------ per-instance thread map
// A column of a unit is RG = ld / E 16-byte words (E = 8 rows for BF16, 4 for
// FP32).  A thread holds up to kGSlots words of a unit in registers: with
// RP = 1 (RG <= 256) the words of row group t % RG in columns
// 8 (t / RG) .. 8 (t / RG) + 7; with RP = 2 or 4 (taller instances, whose
// units have at most 8 / RP columns) the words of row groups t + 256 k
// (k < RP) in every column of the unit.  The thread keeps its rows' residual
// r and its share of the next accumulator A z in registers for as long as the
// CTA stays in the instance, so each tile is read from shared memory once.
constexpr int kGSlots = 8;

struct InstMap {
    int i, m, n, ld, RG, RP;
    int PR;              // dot partials per column (row groups, or threads)
    int p;               // this thread's partial index
    int rg0, col0;       // first row group and column
    int valid;           // the thread owns words of this instance
    int shared_rows;     // several threads own the same rows (acc_s gathers them)
    int64_t bo, xo;
    float Li, mu, cs;
};

__device__ __forceinline__ void map_instance(const GArgs& g, int i, InstMap& im) {
    const int t = threadIdx.x;
    im.i = i;
    im.m = g.m[i];
    im.n = g.n[i];
    im.ld = g.ld[i];
    im.RG = im.ld / (g.bf16 ? 8 : 4);
    im.RP = im.RG <= kGThreads ? 1 : (im.RG <= 2 * kGThreads ? 2 : 4);
    if (im.RP == 1) {
        const int S = (min(g.ucols[i], im.n) + 7) / 8;
        im.rg0 = t % im.RG;
        im.col0 = 8 * (t / im.RG);
        im.valid = t < im.RG * S;
        im.PR = im.RG;
        im.p = im.rg0;
        // rows shared by several slices are gathered in acc_s; the host's
        // unit sizing gives S > 1 only to instances of at most kGShared rows
        // (the guard keeps taller ones on direct global atomics)
        im.shared_rows = S > 1 && im.ld <= kGShared;
    } else {
        im.rg0 = t;
        im.col0 = 0;
        im.valid = 1;
        im.PR = kGThreads;
        im.p = t;
        im.shared_rows = 0;
    }
    im.bo = g.boff[i];
    im.xo = g.xoff[i];
    im.Li = g.mode == GM_FISTA ? 1.0f / g.L[i] : 0.0f;
    im.mu = g.mode == GM_FISTA ? g.mu[i] : 0.0f;
    im.cs = g.mode == GM_POWER ? g.cscale[i] : 0.0f;
}

// Enter an instance: this thread's rows of the residual (FISTA: b - A z from
// the previous step's accumulator; power: A v) and a zero accumulator.
template <bool BF, int RP>
__device__ __forceinline__ void enter_regs(const GArgs& g, const InstMap& im, const float* racc_cur, float* r,
                                           float* acc) {
    constexpr int E = BF ? 8 : 4;
#pragma unroll
    for (int k = 0; k < RP; ++k) {
        const int rg = im.rg0 + kGThreads * k;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int row = rg * E + e;
            float v = 0.0f;
            if (im.valid && rg < im.RG && row < im.m) {
                if (g.mode == GM_FISTA) v = g.b[im.bo + row] - racc_cur[im.bo + row];
                else if (g.mode == GM_POWER) v = racc_cur[im.bo + row];
            }
            r[k * E + e] = v;
            acc[k * E + e] = 0.0f;
        }
    }
}

// Load this thread's words of a staged unit into registers and, in the modes
// that need A^T r, write its partial dot per column to part_s.
template <bool BF, int RP>
__device__ __forceinline__ void load_unit(const InstMap& im, int nc, const uint8_t* tile, bool dots,
                                          const float* r, uint4* a, float* part_s) {
    constexpr int E = BF ? 8 : 4;
    constexpr int CPS = kGSlots / RP;
    const size_t colb = (size_t)im.ld * (BF ? 2 : 4);
#pragma unroll
    for (int k = 0; k < RP; ++k) {
        const int rg = im.rg0 + kGThreads * k;
#pragma unroll
        for (int c = 0; c < CPS; ++c) {
            const int col = im.col0 + c;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (im.valid && rg < im.RG && col < nc)
                v = *reinterpret_cast<const uint4*>(tile + (size_t)col * colb + (size_t)rg * 16);
            a[k * CPS + c] = v;
        }
    }
    if (!dots || !im.valid) return;
#pragma unroll
    for (int c = 0; c < CPS; ++c) {
        float d = 0.0f;
#pragma unroll
        for (int k = 0; k < RP; ++k) {
            const uint4 w = a[k * CPS + c];
            const float* rk = r + k * E;
            if (BF) {
                d = fmaf(bf_lo(w.x), rk[0], d);
                d = fmaf(bf_hi(w.x), rk[1], d);
                d = fmaf(bf_lo(w.y), rk[2], d);
                d = fmaf(bf_hi(w.y), rk[3], d);
                d = fmaf(bf_lo(w.z), rk[4], d);
                d = fmaf(bf_hi(w.z), rk[5], d);
                d = fmaf(bf_lo(w.w), rk[6], d);
                d = fmaf(bf_hi(w.w), rk[7], d);
            } else {
                d = fmaf(__uint_as_float(w.x), rk[0], d);
                d = fmaf(__uint_as_float(w.y), rk[1], d);
                d = fmaf(__uint_as_float(w.z), rk[2], d);
                d = fmaf(__uint_as_float(w.w), rk[3], d);
            }
        }
        const int col = im.col0 + c;
        if (col < nc) part_s[col * im.PR + im.p] = d;
    }
}

// acc(rows) += sum_c A(rows, c) z_c over the thread's words of the unit.
template <bool BF, int RP>
__device__ __forceinline__ void accumulate_unit(const InstMap& im, int nc, const uint4* a, const float* zj_s,
                                                float* acc) {
    constexpr int E = BF ? 8 : 4;
    constexpr int CPS = kGSlots / RP;
    if (!im.valid) return;
#pragma unroll
    for (int c = 0; c < CPS; ++c) {
        const int col = im.col0 + c;
        const float z = col < nc ? zj_s[col] : 0.0f;
#pragma unroll
        for (int k = 0; k < RP; ++k) {
            const uint4 w = a[k * CPS + c];
            float* ak = acc + k * E;
            if (BF) {
                ak[0] = fmaf(bf_lo(w.x), z, ak[0]);
                ak[1] = fmaf(bf_hi(w.x), z, ak[1]);
                ak[2] = fmaf(bf_lo(w.y), z, ak[2]);
                ak[3] = fmaf(bf_hi(w.y), z, ak[3]);
                ak[4] = fmaf(bf_lo(w.z), z, ak[4]);
                ak[5] = fmaf(bf_hi(w.z), z, ak[5]);
                ak[6] = fmaf(bf_lo(w.w), z, ak[6]);
                ak[7] = fmaf(bf_hi(w.w), z, ak[7]);
            } else {
                ak[0] = fmaf(__uint_as_float(w.x), z, ak[0]);
                ak[1] = fmaf(__uint_as_float(w.y), z, ak[1]);
                ak[2] = fmaf(__uint_as_float(w.z), z, ak[2]);
                ak[3] = fmaf(__uint_as_float(w.w), z, ak[3]);
            }
        }
    }
}

// Leave an instance: this thread's share of A z goes to the global
// accumulator, or first to acc_s where several threads own the same rows.
template <bool BF, int RP>
__device__ __forceinline__ void flush_regs(const InstMap& im, const float* acc, float* racc_next, float* acc_s) {
    constexpr int E = BF ? 8 : 4;
    if (!im.valid) return;
#pragma unroll
    for (int k = 0; k < RP; ++k) {
        const int rg = im.rg0 + kGThreads * k;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int row = rg * E + e;
            if (rg < im.RG && row < im.m) {
                if (im.shared_rows) atomicAdd(&acc_s[row], acc[k * E + e]);
                else atomicAdd(&racc_next[im.bo + row], acc[k * E + e]);
            }
        }
    }
}

// The register-held parts are instantiated per (element type, RP); an
// instance's map picks one (instances are at most 4096 rows: RP <= 2 for BF16,
// RP <= 4 for FP32).
#define GROUP_DISPATCH(FN, ...)                                       \
    do {                                                              \
        if (g.bf16) {                                                 \
            if (im.RP == 1) FN<true, 1>(__VA_ARGS__);                 \
            else FN<true, 2>(__VA_ARGS__);                            \
        } else {                                                      \
            if (im.RP == 1) FN<false, 1>(__VA_ARGS__);                \
            else if (im.RP == 2) FN<false, 2>(__VA_ARGS__);           \
            else FN<false, 4>(__VA_ARGS__);                           \
        }                                                             \
    } while (0)

// Per-unit column state, loaded before the tile arrives: x_c, z_c for the
// thread's column c = threadIdx.x < nc.
struct ColState {
    float x, z;
};

__device__ __forceinline__ ColState load_cols(const GArgs& g, const UnitGeom& q) {
    ColState cs{0.0f, 0.0f};
    if ((int)threadIdx.x < q.nc && g.mode != GM_POWER_INIT) {
        const int64_t j = g.xoff[q.i] + q.col0 + threadIdx.x;
        cs.x = g.x[j];
        if (g.mode == GM_FISTA) cs.z = g.z[j];
    }
    return cs;
}

// The columns of a unit, one warp per column: g_c = sum of the column's dot
// partials (A_J^T r), then the per-mode update of x_c, z_c by lane 0, which
// writes z_c to zj_s and adds the column's reduction terms to d2 / w2.
__device__ __forceinline__ void unit_columns(const GArgs& g, const UnitGeom& q, const InstMap& im,
                                             const float* part_s, const ColState* cst_s, float* zj_s, double& d2,
                                             double& w2) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool dots = g.mode == GM_FISTA || g.mode == GM_POWER;
    for (int c = warp; c < q.nc; c += kGWarps) {
        float dot = 0.0f;
        if (dots) {
            const float* pc = part_s + c * im.PR;
            for (int p = lane; p < im.PR; p += 32) dot += pc[p];
            dot = warp_sum_f(dot);
        }
        if (lane == 0) {
            const int64_t j = im.xo + q.col0 + c;
            const ColState cs = cst_s[c];
            float zn;
            if (g.mode == GM_FISTA) {
                // Eq. 18: x = soft(z + A^T(b - A z)/L, lambda/L), z' = x + mu (x - x_old)
                const float xn = soft_g(fmaf(dot, im.Li, cs.z), g.lambda * im.Li);
                zn = fmaf(im.mu, xn - cs.x, xn);
                g.x[j] = xn;
                g.z[j] = zn;
                const float dx = xn - cs.x;
                d2 += (double)dx * dx;
                w2 += (double)cs.x * cs.x;
            } else if (g.mode == GM_POWER) {
                zn = dot * im.cs;  // v' = A^T A v scaled to about unit norm
                g.x[j] = zn;
                d2 += (double)zn * zn;
            } else if (g.mode == GM_POWER_INIT) {
                zn = rsqrtf((float)im.n);
                g.x[j] = zn;
                d2 += (double)zn * zn;
            } else {  // GM_FINAL: A x
                zn = cs.x;
                w2 += fabs((double)zn);
            }
            zj_s[c] = zn;
        }
    }
}

// Leave instance i: gather acc_s into the global accumulator (when rows are
// shared) and add the CTA's reduction terms to the instance's sums.  Ends
// with a block barrier.
__device__ __forceinline__ void flush_instance(const GArgs& g, const InstMap& im, float* racc_next,
                                               const float* acc_s, double* red_s, double& d2, double& w2) {
    if (im.shared_rows) {
        __syncthreads();
        for (int r = threadIdx.x; r < im.m; r += blockDim.x) atomicAdd(&racc_next[im.bo + r], acc_s[r]);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double wd2 = warp_sum(d2), ww2 = warp_sum(w2);
    if (lane == 0) {
        red_s[warp] = wd2;
        red_s[kGWarps + warp] = ww2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s1 = 0.0, s2 = 0.0;
        for (int w = 0; w < kGWarps; ++w) {
            s1 += red_s[w];
            s2 += red_s[kGWarps + w];
        }
        if (g.mode == GM_FISTA) {
            atomicAdd(&g.d2[im.i], s1);
            atomicAdd(&g.w2[im.i], s2);
        } else if (g.mode == GM_FINAL) {
            atomicAdd(&g.w2[im.i], s2);
        } else {
            atomicAdd(&g.vv[im.i], s1);
        }
    }
    d2 = 0.0;
    w2 = 0.0;
    __syncthreads();
}

// rebuild the active-instance list and unit prefix (block 0 only)
__device__ void group_rebuild(const GArgs& g, int64_t* scan_s) {
    if (blockIdx.x != 0) return;
    __shared__ int64_t base_u;
    __shared__ int base_k;
    if (threadIdx.x == 0) {
        base_u = 0;
        base_k = 0;
    }
    __syncthreads();
    for (int64_t c0 = 0; c0 < g.count; c0 += blockDim.x) {
        const int64_t i = c0 + threadIdx.x;
        const int a = (i < g.count && g.active[i]) ? 1 : 0;
        const int64_t u = a ? g.nunits[i] : 0;
        // block-wide inclusive scans of (a, u)
        scan_s[threadIdx.x] = ((int64_t)a << 40) | u;  // u < 2^40, count < 2^23
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {
            const int64_t v = threadIdx.x >= (unsigned)o ? scan_s[threadIdx.x - o] : 0;
            __syncthreads();
            scan_s[threadIdx.x] += v;
            __syncthreads();
        }
        const int64_t incl = scan_s[threadIdx.x];
        const int k_excl = (int)((incl >> 40) - a);
        const int64_t u_excl = (incl & ((int64_t(1) << 40) - 1)) - u;
        if (a) {
            g.act[base_k + k_excl] = (int32_t)i;
            g.upref[base_k + k_excl] = base_u + u_excl;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) {
            base_k += (int)(incl >> 40);
            base_u += incl & ((int64_t(1) << 40) - 1);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        g.upref[base_k] = base_u;
        *g.nact = base_k;
    }
}



__global__ void __launch_bounds__(kGThreads, 2) group_kernel(GArgs g) {
    extern __shared__ __align__(128) uint8_t gsm[];
    uint8_t* tiles[kGBufs];                                                   // kGBufs x kGTileBytes
    for (int k = 0; k < kGBufs; ++k) tiles[k] = gsm + k * kGTileBytes;
    float* acc_s = reinterpret_cast<float*>(gsm + kGBufs * kGTileBytes);      // kGShared floats
    float* part_s = acc_s + kGShared;                                         // kGPartials floats
    float* zj_s = part_s + kGPartials;                                        // 256 floats
    ColState* cst_s = reinterpret_cast<ColState*>(zj_s + 256);                // 256
    double* red_s = reinterpret_cast<double*>(cst_s + 256);                   // 2 * kGWarps
    // the rebuild's scan runs between passes, when part_s is idle
    int64_t* scan_s = reinterpret_cast<int64_t*>(part_s);                     // kGThreads
    uint64_t* bars = reinterpret_cast<uint64_t*>(red_s + 2 * kGWarps);        // kGBufs
    __shared__ UnitGeom geo_s[kGBufs];
    __shared__ int abort_s;
    if (threadIdx.x == 0) {
        abort_s = 0;
        for (int k = 0; k < kGBufs; ++k) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(g_smem(&bars[k])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    volatile int* abort = &abort_s;
    const int nwarps_grid = gridDim.x * kGWarps;
    const int gwarp = blockIdx.x * kGWarps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    uint32_t phase[kGBufs] = {};
    // this thread's rows of the current instance: residual, accumulator
    float r[16], acc[16];
    uint4 a[kGSlots];

    for (int step = 0; step < g.max_steps; ++step) {
        const int cur = step & 1;
        const int nact = *(volatile int32_t*)g.nact;
        if (nact == 0) break;
        const int64_t total = g.upref[nact];
        const bool dots = g.mode == GM_FISTA || g.mode == GM_POWER;
        // ---- pass over this CTA's contiguous range of active units
        {
            const float* racc_cur = cur ? g.racc1 : g.racc0;
            float* racc_next = cur ? g.racc0 : g.racc1;
            const int64_t per = (total + gridDim.x - 1) / gridDim.x;
            const int64_t u0 = min(total, (int64_t)blockIdx.x * per), u1 = min(total, u0 + per);
            // thread 0 keeps kGBufs units in flight: the geometry of the unit
            // in buffer k lives in geo_s[k]; the copy of unit u + kGBufs is
            // issued as soon as every thread has taken unit u's words into
            // registers
            bool pending[kGBufs] = {};
            if (threadIdx.x == 0 && u0 < u1) {
                geo_s[0] = geom_first(g, u0, nact);
                issue_tile(g, geo_s[0], tiles[0], &bars[0]);
                for (int k = 1; k < kGBufs && u0 + k < u1; ++k) {
                    geo_s[k] = geom_next(g, geo_s[k - 1]);
                    issue_tile(g, geo_s[k], tiles[k], &bars[k]);
                }
            }
            for (int k = 0; k < kGBufs; ++k) pending[k] = u0 + k < u1;
            __syncthreads();
            InstMap im;
            im.i = -1;
            double d2 = 0.0, w2 = 0.0;
            bool failed = false;
            // the column state of a unit is loaded one unit ahead (two
            // dependent loads: the instance's offset, then x and z)
            ColState cst_next{0.0f, 0.0f};
            if (u0 < u1) cst_next = load_cols(g, geo_s[0]);
            for (int64_t u = u0; u < u1; ++u) {
                const int b = (int)((u - u0) % kGBufs);
                const UnitGeom q = geo_s[b];
                const ColState cst = cst_next;
                if (u + 1 < u1) cst_next = load_cols(g, geo_s[(b + 1) % kGBufs]);
                if (q.i != im.i) {
                    if (im.i >= 0) {
                        GROUP_DISPATCH(flush_regs, im, acc, racc_next, acc_s);
                        flush_instance(g, im, racc_next, acc_s, red_s, d2, w2);
                    }
                    map_instance(g, q.i, im);
                    if (im.shared_rows)
                        for (int row = threadIdx.x; row < im.ld; row += blockDim.x) acc_s[row] = 0.0f;
                    GROUP_DISPATCH(enter_regs, g, im, racc_cur, r, acc);
                }
                const bool ok = g_mbar_wait(&bars[b], phase[b]);
                if (ok) GROUP_DISPATCH(load_unit, im, q.nc, tiles[b], dots, r, a, part_s);
                if ((int)threadIdx.x < q.nc) cst_s[threadIdx.x] = cst;
                // the block agrees on the copy's outcome; every thread has
                // its words of the unit, so the buffer may be refilled
                if (__syncthreads_or(!ok)) {
                    failed = true;
                    break;
                }
                phase[b] ^= 1u;
                pending[b] = false;
                if (u + kGBufs < u1) {
                    // issued from the last warp, which has a column of the
                    // unit to finish only when the unit has more than
                    // kGWarps - 1 columns (the geometry of a new instance
                    // costs global loads)
                    if (threadIdx.x == kGThreads - 32) {
                        // unit u + kGBufs follows unit u + kGBufs - 1, which
                        // sits in the buffer before this one
                        const UnitGeom q2 = geom_next(g, geo_s[(b + kGBufs - 1) % kGBufs]);
                        geo_s[b] = q2;
                        issue_tile(g, q2, tiles[b], &bars[b]);
                    }
                    pending[b] = true;
                }
                unit_columns(g, q, im, part_s, cst_s, zj_s, d2, w2);
                __syncthreads();
                GROUP_DISPATCH(accumulate_unit, im, q.nc, a, zj_s, acc);
            }
            if (failed) {
                // a copy did not complete in time: record it, give the copies
                // in flight a last bounded wait, and leave
                if (threadIdx.x == 0) atomicCAS(g.err, 0, 2);
                for (int k = 0; k < kGBufs; ++k)
                    if (pending[k]) g_mbar_wait(&bars[k], phase[k]);
                *abort = 1;
                return;
            }
            if (im.i >= 0) {
                GROUP_DISPATCH(flush_regs, im, acc, racc_next, acc_s);
                flush_instance(g, im, racc_next, acc_s, red_s, d2, w2);
            }
        }
        if (!grid_sync(g, abort)) return;
        // ---- per-instance finalisation: one warp per active instance
        float* racc_done = cur ? g.racc1 : g.racc0;   // consumed this step: zero for reuse
        float* racc_new = cur ? g.racc0 : g.racc1;    // accumulated this step
        for (int k = gwarp; k < nact; k += nwarps_grid) {
            const int i = g.act[k];
            const int m = g.m[i];
            const int64_t bo = g.boff[i];
            double s = 0.0;
            if (g.mode == GM_POWER || g.mode == GM_POWER_INIT) {
                for (int r = lane; r < m; r += 32) s += (double)racc_new[bo + r] * racc_new[bo + r];
            } else if (g.mode == GM_FINAL) {
                for (int r = lane; r < m; r += 32) {
                    const double e = (double)g.b[bo + r] - racc_new[bo + r];
                    s += e * e;
                }
            }
            s = warp_sum(s);
            for (int r = lane; r < m; r += 32) racc_done[bo + r] = 0.0f;
            if (lane == 0) {
                if (g.mode == GM_FISTA) {
                    const int it = g.iters[i] + 1;
                    g.iters[i] = it;
                    const double d2 = g.d2[i], w2 = g.w2[i];
                    const double rel = rel_change(sqrt(d2), sqrt(w2));
                    g.rel[i] = rel;
                    g.d2[i] = 0.0;
                    g.w2[i] = 0.0;
                    if (!isfinite(d2) || !isfinite(w2)) { g.status[i] = L1_NONFINITE; g.active[i] = 0; }
                    else if (rel < g.tol) { g.status[i] = L1_CONVERGED; g.active[i] = 0; }
                    else if (it >= g.max_steps) { g.status[i] = L1_MAX_ITER; g.active[i] = 0; }
                    else {
                        const double tt = g.t[i];
                        const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tt * tt));
                        const double tnn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tn * tn));
                        g.t[i] = tn;
                        g.mu[i] = (float)((tn - 1.0) / tnn);
                    }
                } else if (g.mode == GM_FINAL) {
                    const double x1 = g.w2[i];
                    g.res2[i] = s;
                    g.obj[i] = 0.5 * s + (double)g.lambda * x1;
                    g.active[i] = 0;
                } else {
                    // Rayleigh quotient ||A v||^2 / ||v||^2 and the scale that keeps v near unit norm
                    const double vv = g.vv[i];
                    const double rho = vv > 0.0 ? s / vv : 0.0;
                    const double prev = g.rho[i];
                    g.rho[i] = rho;
                    g.vv[i] = 0.0;
                    const int it = g.iters[i] + 1;
                    g.iters[i] = it;
                    g.cscale[i] = (rho > 0.0 && vv > 0.0) ? (float)(1.0 / (rho * sqrt(vv))) : 0.0f;
                    const bool done = (g.mode == GM_POWER && fabs(rho - prev) <= g.tol * rho) || rho == 0.0 ||
                                      it >= g.max_steps;
                    if (done) g.active[i] = 0;
                }
            }
        }
        if (!grid_sync(g, abort)) return;
        if (g.mode == GM_POWER_INIT) g.mode = GM_POWER;  // the first pass only seeds v = 1/sqrt(n)
        group_rebuild(g, scan_s);
        if (!grid_sync(g, abort)) return;
    }
}


// ------------------------------------------------------------------- host
__global__ void quantize_store_kernel(const float* src, int m, int n, int ld, void* dst, int64_t off, int bf16) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)ld * n) return;
    const int64_t j = idx / ld, r = idx % ld;
    const float v = r < m ? src[j * m + r] : 0.0f;
    if (bf16) reinterpret_cast<__nv_bfloat16*>(dst)[off + idx] = __float2bfloat16_rn(v);
    else reinterpret_cast<float*>(dst)[off + idx] = v;
}

// Instances [first, last) take part in the pass; the others stay idle.
__global__ void group_init_kernel(GArgs g, int mode, int64_t first, int64_t last) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.count) return;
    g.active[i] = (i >= first && i < last) ? 1 : 0;
    g.d2[i] = 0.0;
    g.w2[i] = 0.0;
    if (mode == GM_FINAL) return;  // keeps the solve's status, counts and last change
    g.status[i] = L1_MAX_ITER;
    g.iters[i] = 0;
    g.t[i] = 1.0;
    g.mu[i] = 0.0f;
    g.vv[i] = 0.0;
    g.rho[i] = 0.0;
    g.rel[i] = INFINITY;
}

static GArgs make_args(GroupState* G) {
    GArgs a{};
    a.count = G->count;
    a.bf16 = G->prec == L1_A_BF16;
    a.m = G->m; a.n = G->n; a.ld = G->ld; a.ucols = G->ucols;
    a.aoff = G->aoff; a.boff = G->boff; a.xoff = G->xoff; a.nunits = G->nunits;
    a.A = G->A; a.b = G->b; a.x = G->x; a.z = G->z; a.racc0 = G->racc[0]; a.racc1 = G->racc[1];
    a.L = G->L; a.mu = G->mu; a.cscale = G->cscale;
    a.t = G->t; a.d2 = G->d2; a.w2 = G->w2; a.vv = G->vv; a.rho = G->rho; a.rel = G->rel;
    a.obj = G->obj; a.res2 = G->res2;
    a.active = G->active; a.status = G->status; a.iters = G->iters;
    a.act = G->act; a.nact = G->nact; a.upref = G->upref;
    a.bar_count = G->bar_count; a.bar_gen = G->bar_gen; a.err = G->err;
    a.lambda = (float)G->lambda;
    return a;
}

__global__ void rebuild_kernel(GArgs g) {
    __shared__ int64_t scan_s[kGThreads];
    group_rebuild(g, scan_s);
}

static int run_group(Handle* h, int mode, int max_steps, double tol, int64_t first = 0, int64_t last = -1) {
    GroupState* G = h->grp;
    cudaStream_t s = h->stream;
    GArgs a = make_args(G);
    a.mode = mode;
    a.max_steps = max_steps;
    a.tol = tol;
    if (last < 0) last = G->count;
    group_init_kernel<<<(unsigned)((G->count + 255) / 256), 256, 0, s>>>(a, mode, first, last);
    L1_LAUNCH_CHECK(h);
    L1_CUDA_TRY(cudaMemsetAsync(G->racc[0], 0, sizeof(float) * G->sum_m, s));
    L1_CUDA_TRY(cudaMemsetAsync(G->racc[1], 0, sizeof(float) * G->sum_m, s));
    L1_CUDA_TRY(cudaMemsetAsync(G->bar_count, 0, sizeof(unsigned) * 2, s));
    L1_CUDA_TRY(cudaMemsetAsync(G->err, 0, sizeof(int), s));
    rebuild_kernel<<<1, kGThreads, 0, s>>>(a);
    L1_LAUNCH_CHECK(h);
    void* args[] = {&a};
    L1_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)group_kernel, dim3(G->grid), dim3(kGThreads), args,
                                            (size_t)G->smem, s));
    ++h->launches;
    int herr = 0;
    L1_CUDA_TRY(cudaMemcpyAsync(&herr, G->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    L1_CUDA_TRY(cudaStreamSynchronize(s));
    if (herr) {
        set_last_error(herr == 2 ? "group kernel: bounded wait for a tile copy expired"
                                 : "group kernel: bounded grid barrier expired");
        return L1_ERR_TIMEOUT;
    }
    return L1_OK;
}

__global__ void set_L_kernel(GArgs g, double safety, int64_t first, int64_t last) {
    const int64_t i = first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= last) return;
    g.L[i] = (float)(safety * g.rho[i]);
}

static int group_power(Handle* h, int64_t first, int64_t last) {
    // batched power iteration (reading of L in Algorithm 1 step 6 / Eq. 18 as
    // ||A||_2^2): the POWER_INIT pass seeds v = 1/sqrt(n) and u = A v
    L1_TRY(run_group(h, GM_POWER_INIT, 1000, 1e-6, first, last));
    GroupState* G = h->grp;
    GArgs a = make_args(G);
    const int64_t k = last - first;
    set_L_kernel<<<(unsigned)((k + 255) / 256), 256, 0, h->stream>>>(a, 1.01, first, last);
    L1_LAUNCH_CHECK(h);
    return L1_OK;
}

int group_load(Handle* h, int64_t first, int64_t k, const float* const* A) {
    GroupState* G = h->grp;
    if (!G || first < 0 || k <= 0 || first + k > G->count || !A) return L1_ERR_INVALID_ARG;
    int64_t maxmn = 0;
    for (int64_t i = first; i < first + k; ++i) maxmn = std::max<int64_t>(maxmn, (int64_t)G->hm[i] * G->hn[i]);
    float* stage = nullptr;
    if (cudaMalloc(&stage, sizeof(float) * maxmn) != cudaSuccess) {
        cudaGetLastError();
        return L1_ERR_OOM;
    }
    int rc = L1_OK;
    for (int64_t q = 0; q < k && rc == L1_OK; ++q) {
        const int64_t i = first + q;
        if (!A[q]) { rc = L1_ERR_INVALID_ARG; break; }
        const int m = G->hm[i], n = G->hn[i];
        if (cudaMemcpyAsync(stage, A[q], sizeof(float) * (size_t)m * n, cudaMemcpyDefault, h->stream) != cudaSuccess) {
            rc = L1_ERR_CUDA;
            break;
        }
        const int64_t tot = (int64_t)G->hld[i] * n;
        quantize_store_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>(
            stage, m, n, G->hld[i], G->A, G->haoff[i], G->prec == L1_A_BF16);
        ++h->launches;
        if (cudaGetLastError() != cudaSuccess) rc = L1_ERR_CUDA;
    }
    cudaStreamSynchronize(h->stream);
    cudaFree(stage);
    if (rc != L1_OK) return rc;
    if (h->opt.lipschitz > 0.0) {
        std::vector<float> Ls(G->count, (float)h->opt.lipschitz);
        L1_CUDA_TRY(cudaMemcpy(G->L, Ls.data(), sizeof(float) * G->count, cudaMemcpyHostToDevice));
        return L1_OK;
    }
    return group_power(h, first, first + k);
}

int group_setup(Handle* h, const float* const* A, const int64_t* m, const int64_t* n, int64_t count) {
    GroupState* G = new (std::nothrow) GroupState();
    if (!G) return L1_ERR_OOM;
    h->grp = G;
    G->count = count;
    G->prec = h->opt.precision;
    G->lambda = h->opt.lambda;
    const int esize = G->prec == L1_A_BF16 ? 2 : 4;
    G->hm.resize(count); G->hn.resize(count); G->hld.resize(count); G->hucols.resize(count);
    G->haoff.resize(count); G->hboff.resize(count); G->hxoff.resize(count); G->hnunits.resize(count);
    int64_t ao = 0, bo = 0, xo = 0;
    for (int64_t i = 0; i < count; ++i) {
        if (m[i] <= 0 || n[i] <= 0 || m[i] > kGMaxM || n[i] > (1 << 24)) return L1_ERR_INVALID_ARG;
        const int mi = (int)m[i], ni = (int)n[i];
        const int ld = (int)round_up(mi, 8);
        // columns per unit: a full unit is exactly kGThreads register words
        // (a multiple of 8 columns), or 8 / RP columns for taller instances
        const int cap = kGTileBytes / (esize * ld);
        const int rg = ld * esize / 16;
        int uc;
        if (rg <= kGThreads) uc = std::min(256, 8 * (cap / 8));
        else uc = rg <= 2 * kGThreads ? 4 : 2;
        G->hm[i] = mi; G->hn[i] = ni; G->hld[i] = ld; G->hucols[i] = uc;
        G->haoff[i] = ao; G->hboff[i] = bo; G->hxoff[i] = xo;
        G->hnunits[i] = (ni + uc - 1) / uc;
        ao += (int64_t)ld * ni;
        bo += mi;
        xo += ni;
    }
    G->a_elems = ao;
    G->sum_m = bo;
    G->sum_n = xo;
    L1_TRY(dev_alloc(h, &G->A, (size_t)ao * esize));
    L1_TRY(dev_alloc_t(h, &G->m, count)); L1_TRY(dev_alloc_t(h, &G->n, count));
    L1_TRY(dev_alloc_t(h, &G->ld, count)); L1_TRY(dev_alloc_t(h, &G->ucols, count));
    L1_TRY(dev_alloc_t(h, &G->aoff, count)); L1_TRY(dev_alloc_t(h, &G->boff, count));
    L1_TRY(dev_alloc_t(h, &G->xoff, count)); L1_TRY(dev_alloc_t(h, &G->nunits, count));
    L1_TRY(dev_alloc_t(h, &G->b, bo)); L1_TRY(dev_alloc_t(h, &G->x, xo)); L1_TRY(dev_alloc_t(h, &G->z, xo));
    L1_TRY(dev_alloc_t(h, &G->racc[0], bo)); L1_TRY(dev_alloc_t(h, &G->racc[1], bo));
    L1_TRY(dev_alloc_t(h, &G->L, count)); L1_TRY(dev_alloc_t(h, &G->mu, count));
    L1_TRY(dev_alloc_t(h, &G->cscale, count));
    L1_TRY(dev_alloc_t(h, &G->t, count)); L1_TRY(dev_alloc_t(h, &G->d2, count));
    L1_TRY(dev_alloc_t(h, &G->w2, count)); L1_TRY(dev_alloc_t(h, &G->vv, count));
    L1_TRY(dev_alloc_t(h, &G->rho, count)); L1_TRY(dev_alloc_t(h, &G->rel, count));
    L1_TRY(dev_alloc_t(h, &G->obj, count)); L1_TRY(dev_alloc_t(h, &G->res2, count));
    L1_TRY(dev_alloc_t(h, &G->active, count)); L1_TRY(dev_alloc_t(h, &G->status, count));
    L1_TRY(dev_alloc_t(h, &G->iters, count)); L1_TRY(dev_alloc_t(h, &G->act, count));
    L1_TRY(dev_alloc_t(h, &G->nact, 1)); L1_TRY(dev_alloc_t(h, &G->upref, count + 1));
    L1_TRY(dev_alloc_t(h, &G->bar_count, 2));
    G->bar_gen = G->bar_count + 1;
    L1_TRY(dev_alloc_t(h, &G->err, 1));
    L1_CUDA_TRY(cudaMemcpy(G->m, G->hm.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice));
    L1_CUDA_TRY(cudaMemcpy(G->n, G->hn.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice));
    L1_CUDA_TRY(cudaMemcpy(G->ld, G->hld.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice));
    L1_CUDA_TRY(cudaMemcpy(G->ucols, G->hucols.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice));
    L1_CUDA_TRY(cudaMemcpy(G->aoff, G->haoff.data(), sizeof(int64_t) * count, cudaMemcpyHostToDevice));
    L1_CUDA_TRY(cudaMemcpy(G->boff, G->hboff.data(), sizeof(int64_t) * count, cudaMemcpyHostToDevice));
    L1_CUDA_TRY(cudaMemcpy(G->xoff, G->hxoff.data(), sizeof(int64_t) * count, cudaMemcpyHostToDevice));
    L1_CUDA_TRY(cudaMemcpy(G->nunits, G->hnunits.data(), sizeof(int64_t) * count, cudaMemcpyHostToDevice));
    // cooperative grid: every block resident
    static_assert(kGPartials * sizeof(float) >= kGThreads * sizeof(int64_t), "scan scratch inside part_s");
    G->smem = kGBufs * kGTileBytes + (kGShared + kGPartials + 256) * (int)sizeof(float) +
              256 * (int)sizeof(ColState) + 2 * kGWarps * 8 + kGBufs * 8;
    L1_CUDA_TRY(cudaFuncSetAttribute(group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, G->smem));
    int per_sm = 0, sms = 0;
    L1_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, group_kernel, kGThreads, G->smem));
    L1_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    if (per_sm < 1) return L1_ERR_UNSUPPORTED;
    G->grid = per_sm * sms;
    if (A) return group_load(h, 0, count, A);
    return L1_OK;
}

__global__ void group_pack_kernel(GArgs g, l1_result* out, double lam) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.count) return;
    l1_result r;
    r.status = g.status[i];
    r.iters = g.iters[i];
    r.inner_iters = g.iters[i];
    r.label = -1;
    r.sci_label = -1;
    r.reserved = 0;
    r.rel_change = g.rel[i];
    r.primal_obj = g.obj[i];
    r.dual_obj = NAN;
    r.gap = NAN;
    r.resid = sqrt(g.res2[i]);
    r.param = lam / (double)g.L[i];
    out[i] = r;
}

int group_solve(Handle* h, const float* b, int64_t N, double tol, int max_iter, float* x, l1_result* res) {
    GroupState* G = h->grp;
    if (N != G->count) return L1_ERR_INVALID_ARG;
    cudaStream_t s = h->stream;
    L1_CUDA_TRY(cudaMemcpyAsync(G->b, b, sizeof(float) * G->sum_m, cudaMemcpyDefault, s));
    L1_CUDA_TRY(cudaMemsetAsync(G->x, 0, sizeof(float) * G->sum_n, s));
    L1_CUDA_TRY(cudaMemsetAsync(G->z, 0, sizeof(float) * G->sum_n, s));
    L1_TRY(run_group(h, GM_FISTA, max_iter, tol));
    // one more pass forms A x for the objective and the residual
    L1_TRY(run_group(h, GM_FINAL, 1, 0.0));
    GArgs a = make_args(G);
    const unsigned blocks = (unsigned)((G->count + 255) / 256);
    l1_result* rdev = nullptr;
    if (cudaMalloc(&rdev, sizeof(l1_result) * G->count) != cudaSuccess) return L1_ERR_OOM;
    group_pack_kernel<<<blocks, 256, 0, s>>>(a, rdev, G->lambda);
    ++h->launches;
    cudaMemcpyAsync(x, G->x, sizeof(float) * G->sum_n, cudaMemcpyDefault, s);
    cudaMemcpyAsync(res, rdev, sizeof(l1_result) * G->count, cudaMemcpyDefault, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(rdev);
    if (e != cudaSuccess) {
        set_last_error(std::string("group solve: ") + cudaGetErrorString(e));
        return L1_ERR_CUDA;
    }
    return L1_OK;
}

void group_free(Handle* h) {
    delete h->grp;
    h->grp = nullptr;
}

}  // namespace l1
