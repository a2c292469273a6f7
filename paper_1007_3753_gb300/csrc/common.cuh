// Shared definitions of the CUDA library: error plumbing, the handle, device
// helpers.  Everything here is internal; the public surface is include/l1alm.h.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "l1alm.h"

namespace l1 {

// ------------------------------------------------------------------ errors
struct Status {
    int code = L1_OK;
};

void set_last_error(const std::string& msg);

#define L1_CUDA_TRY(expr)                                                                 \
    do {                                                                                  \
        cudaError_t _e = (expr);                                                          \
        if (_e != cudaSuccess) {                                                          \
            ::l1::set_last_error(std::string(#expr) + ": " + cudaGetErrorString(_e));     \
            return _e == cudaErrorMemoryAllocation ? L1_ERR_OOM : L1_ERR_CUDA;            \
        }                                                                                 \
    } while (0)

#define L1_TRY(expr)               \
    do {                           \
        int _rc = (expr);          \
        if (_rc != L1_OK) return _rc; \
    } while (0)

// Every kernel launch in the library goes through this so the handle can count
// its launches and a launch error is reported, not swallowed.
#define L1_LAUNCH_CHECK(h)                                                          \
    do {                                                                            \
        ++(h)->launches;                                                            \
        cudaError_t _e = cudaGetLastError();                                        \
        if (_e != cudaSuccess) {                                                    \
            ::l1::set_last_error(std::string("kernel launch: ") + cudaGetErrorString(_e)); \
            return L1_ERR_CUDA;                                                     \
        }                                                                           \
    } while (0)

inline int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// --------------------------------------------------------- device buffers
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// -------------------------------------------------------------- the handle
// Column phases of the batched PALM state machine.
enum PalmPhase : int32_t { PH_INNER = 0, PH_OUTER = 1, PH_FIRST = 2 };

// Iteration state carried from one sweep to the next, one problem per
// column ("slot"); compaction moves the active slots to the front of the
// other set of the double buffer.
struct PanelSet {
    float* B = nullptr;   // right-hand sides, m x N
    float* Wx = nullptr;  // DALM multiplier x-part / PALM w (current FISTA iterate)
    float* We = nullptr;  // DALM multiplier e-part / PALM e
    float* Ux = nullptr;  // DALM z - w/beta (x-part) / PALM z (FISTA extrapolation)
    float* Ue = nullptr;  // DALM z - w/beta (e-part)
    float* Y = nullptr;   // DALM y / PALM theta
    float* X = nullptr;   // PALM outer x_k
    float* Cc = nullptr;  // PALM c = b - e + theta/xi
    float* colf = nullptr;     // per-slot floats  [8][cap]
    int32_t* coli = nullptr;   // per-slot ints    [16][cap]
    double* cold = nullptr;    // per-slot doubles [8][cap]
};

struct Workspace {
    int64_t cap_N = 0;  // columns the buffers are sized for
    PanelSet ps[2];
    float* R = nullptr;   // DALM right-hand side of Eq. 39 / PALM residual c - A z (scratch)
    // BF16 pieces of the panels the tensor-core sweeps read (scratch)
    __nv_bfloat16* Vh[3] = {nullptr, nullptr, nullptr};  // of V_x (n x N, ld = ldn)
    __nv_bfloat16* Dh[3] = {nullptr, nullptr, nullptr};  // of d (m x N, ld = ldm)
    __nv_bfloat16* Yh[3] = {nullptr, nullptr, nullptr};  // of y (m x N, ld = ldm)
    // results in the caller's column order ("home")
    float* hB = nullptr;
    float* hWx = nullptr;
    float* hWe = nullptr;
    float* hY = nullptr;
    float* hUx = nullptr;  // low-precision A only: z - w/beta at retirement (refinement restart)
    float* hUe = nullptr;
    int32_t* hcoli = nullptr;  // [8][cap]: status, iters, inner, label, sci_label, first-phase iters
    double* hcold = nullptr;   // [10][cap]: rel, param, fin[8] (interleaved per column)
    float* hcolf = nullptr;    // [2][cap]: xi, smax
    double* part = nullptr;    // reduction partials, 2 x [slots][N][4]
    int32_t* newpos = nullptr;
    int32_t* count = nullptr;  // device counter
    int32_t* h_count = nullptr;  // pinned host mirror
    double* resid2 = nullptr;  // classification residuals, [C][N]
    double* classl1 = nullptr; // classification l1 mass, [C][N]
    int32_t* class_off = nullptr;
    size_t part_slots = 0;
};

struct Handle {
    int64_t m = 0, n = 0;
    int64_t ldm = 0, ldn = 0;  // padded leading dimensions (multiples of 32 floats)
    int32_t mode = L1_P1;
    l1_options opt{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int sms = 0;  // multiprocessors of the device
    // split-K slices of the narrow CUDA-core sweeps (grows on demand)
    float* splitk = nullptr;
    size_t splitk_floats = 0;
    // dictionary
    float* A_cm = nullptr;  // column-major m x n, ld = ldm  (rows of A^T contiguous: K-major for A^T y)
    float* A_rm = nullptr;  // row-major m x n, ld = ldn     (K-major for A u)
    float* F = nullptr;     // DALM: (B B^T)^{-1}, m x m symmetric, ld = ldm (high FP32 part)
    float* F_lo = nullptr;  // low FP32 part: F + F_lo = (B B^T)^{-1} to ~48 bits
    // low-precision copies of both layouts of A (l1_options.precision BF16 or
    // FP8 e4m3; same leading dimensions); FP8 carries one FP32 scale per row
    // of each layout: A_rm(i, k) = A_rm_scale[i] q(i, k), A_cm likewise
    void* A_rm_lp = nullptr;
    void* A_cm_lp = nullptr;
    float* A_rm_scale = nullptr;
    float* A_cm_scale = nullptr;
    // tensor-core engine: aligned BF16 pieces of both layouts of A and of
    // (B B^T)^{-1} (same leading dimensions), see gemm_bf16.cuh
    bool use_tc = false;
    __nv_bfloat16* A_rm_h[3] = {nullptr, nullptr, nullptr};
    __nv_bfloat16* A_cm_h[3] = {nullptr, nullptr, nullptr};
    __nv_bfloat16* F_h[3] = {nullptr, nullptr, nullptr};
    // FP32 sums of split-K slices or of deferred-epilogue tiles of the
    // tensor-core sweeps (slices x tiles x 128 x 128 floats)
    float* tc_wk = nullptr;
    size_t tc_wk_elems = 0;
    // autotuned choices of the tensor-core sweeps: (M, K, 128-wide tiles,
    // K slices, deferred epilogue, tile width, microseconds)
    std::vector<std::array<int32_t, 7>> tc_splits;
    int* tc_err = nullptr;  // device: first bounded-wait failure of a tcgen05 sweep
    // encoded TMA tensor maps, keyed by the operand pointers and shapes
    struct MapCacheEntry {
        std::array<uint64_t, 16> key;
        std::vector<CUtensorMap> maps;  // a[0..T), x[0..T)
    };
    std::vector<MapCacheEntry> map_cache;
    double lipschitz = 0.0;
    double setup_ms = 0.0;
    int64_t device_bytes = 0;
    int64_t launches = 0;
    std::vector<int32_t> class_offsets;  // host copy
    Workspace ws;
    std::vector<void*> allocations;     // device buffers owned by the handle
    std::vector<size_t> allocation_bytes;  // their sizes, same order
    // unrolled PALM and its tape (differentiation), see unroll.cu
    bool has_tape = false;
    struct UnrollState* ur = nullptr;
    // uneven batch of independent dictionaries (l1_setup_group), see group.cu
    struct GroupState* grp = nullptr;
    // CUDA graphs of the polling chunks of l1_solve_batch (solve.cu), and the
    // private stream they are captured on
    struct GraphCache* graphs = nullptr;
    cudaStream_t cap_stream = nullptr;
    // sweep profiling (l1_options.profile)
    std::vector<cudaEvent_t> ev_pool;
    int64_t sweep_launches[4] = {0, 0, 0, 0};
    double sweep_ms[4] = {0, 0, 0, 0};
    double sweep_flop[4] = {0, 0, 0, 0};
};

int dev_alloc(Handle* h, void** p, size_t bytes);
// frees a buffer from dev_alloc and takes it off the handle's books
void dev_free(Handle* h, void* p);
template <class T>
inline int dev_alloc_t(Handle* h, T** p, size_t count) {
    return dev_alloc(h, reinterpret_cast<void**>(p), count * sizeof(T));
}

// ----------------------------------------------------------- device helpers
__device__ __forceinline__ float soft_thr(float v, float a) {
    // proximal operator of a*|.| (§IV): sign(v) max(|v| - a, 0), sign(0) = 0
    return v > a ? v - a : (v < -a ? v + a : 0.0f);
}

__device__ __forceinline__ float clamp_unit(float v) {
    // projection onto [-1, 1] (Eq. 38)
    return fminf(1.0f, fmaxf(-1.0f, v));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// relative change with the zero conventions of the stopping rule (§VI-C):
// a zero step is 0, a nonzero step from a zero iterate is +inf.
__host__ __device__ __forceinline__ double rel_change(double diff, double base) {
    if (diff == 0.0) return 0.0;
    if (base == 0.0) return INFINITY;
    return diff / base;
}

}  // namespace l1
