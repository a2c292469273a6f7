// Host side of the tcgen05 sweeps: tensor maps, TF32 operand pieces, launch.
#pragma once

#include "common.cuh"
#include "gemm_tc.cuh"

namespace l1 {
namespace tc {

// Tiled 2-D tensor map over a row-major array of `rows` rows of `inner`
// FP32 elements, row pitch `pitch_bytes`; box = 32 elements (128 bytes) x
// box_rows, 128-byte swizzle.  Returns L1_OK or L1_ERR_CUDA.
int make_map(CUtensorMap* map, const void* base, uint64_t inner, uint64_t rows, uint64_t pitch_bytes,
             uint32_t box_rows);

// TF32 pieces of an FP32 array (see tf32_split3); p3 may be null.
int split_tf32(Handle* h, const float* x, int64_t count, float* p1, float* p2, float* p3);

// the same from FP64 (the DALM factor): p1 + p2 + p3 carries 33 bits
int split_tf32_from_f64(Handle* h, const double* x, int rows, int cols, int64_t ld_src, int64_t ld_dst,
                        float* p1, float* p2, float* p3);

// x rounded to the nearest TF32 value (10 explicit mantissa bits; ties away
// from zero), returned as an FP32 whose low 13 bits are zero.  Rounding to
// nearest makes the remainder x - tf32_rn(x) take either sign, so the product
// term a2 x2 that a three-term split leaves out is not biased (with
// truncation it always has the sign of a x).
__device__ __forceinline__ float tf32_rn(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// pieces of one FP32 value (device side): x == a + b + c exactly
__device__ __forceinline__ void tf32_split3(float x, float& a, float& b, float& c) {
    a = tf32_rn(x);
    const float r = x - a;  // exact (Sterbenz)
    b = tf32_rn(r);
    c = r - b;
}

// Products of TF32 pieces: a x ~ a0 x0 + a0 x1 + a1 x0 (FP32-level), and with
// three pieces each the six terms of total order <= 2^-22.
inline TermList terms_split3() { return TermList{3, {0, 0, 1, 0, 0, 0}, {0, 1, 0, 0, 0, 0}}; }
inline TermList terms_split6() { return TermList{6, {0, 0, 1, 0, 1, 2}, {0, 1, 0, 2, 1, 0}}; }
inline TermList terms_single() { return TermList{1, {0, 0, 0, 0, 0, 0}, {0, 0, 0, 0, 0, 0}}; }

// Tensor maps of a piece set, encoded once per (pointers, shape) and cached
// in the handle (encoding costs host time on every sweep otherwise).
inline int get_maps(Handle* h, int M, int N, int K, const float* const* ap, int npa, const float* const* xp, int npx,
                    int64_t lda, int64_t ldx, int bn, PieceMaps* out) {
    std::array<uint64_t, 16> key{};
    key[0] = (uint64_t)M | ((uint64_t)N << 32);
    key[1] = (uint64_t)K | ((uint64_t)npa << 32) | ((uint64_t)npx << 40) | ((uint64_t)bn << 48);
    key[2] = (uint64_t)lda;
    key[3] = (uint64_t)ldx;
    for (int p = 0; p < npa; ++p) key[4 + p] = reinterpret_cast<uint64_t>(ap[p]);
    for (int p = 0; p < npx; ++p) key[8 + p] = reinterpret_cast<uint64_t>(xp[p]);
    for (const auto& e : h->map_cache) {
        if (e.key == key) {
            for (int p = 0; p < npa; ++p) out->a[p] = e.maps[p];
            for (int p = 0; p < npx; ++p) out->x[p] = e.maps[npa + p];
            return L1_OK;
        }
    }
    std::memset(out, 0, sizeof(*out));
    const uint64_t Kp = (uint64_t)round_up(K, 32);
    for (int p = 0; p < npa; ++p) L1_TRY(make_map(&out->a[p], ap[p], Kp, (uint64_t)M, (uint64_t)lda * 4, kBM));
    for (int p = 0; p < npx; ++p) L1_TRY(make_map(&out->x[p], xp[p], Kp, (uint64_t)N, (uint64_t)ldx * 4, bn));
    Handle::MapCacheEntry e;
    e.key = key;
    for (int p = 0; p < npa; ++p) e.maps.push_back(out->a[p]);
    for (int p = 0; p < npx; ++p) e.maps.push_back(out->x[p]);
    if (h->map_cache.size() > 64) h->map_cache.erase(h->map_cache.begin());
    h->map_cache.push_back(std::move(e));
    return L1_OK;
}

template <class E, int BN, int NPA, int NPX>
int launch_inst(Handle* h, const PieceMaps& maps, const TermList& tl, int M, int N, int K, const E& epi,
                double* part, const int32_t* active) {
    using S = Smem<BN, NPA, NPX>;
    static bool attr_set = false;
    if (!attr_set) {
        L1_CUDA_TRY(cudaFuncSetAttribute(gemm_tc_kernel<E, BN, NPA, NPX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         S::kBytes));
        attr_set = true;
    }
    dim3 grid((N + BN - 1) / BN, (M + kBM - 1) / kBM);
    gemm_tc_kernel<E, BN, NPA, NPX><<<grid, cta_threads(BN), S::kBytes, h->stream>>>(maps, tl, M, N, K, epi, part,
                                                                                     active, h->tc_err);
    L1_LAUNCH_CHECK(h);
    return (int)grid.y;
}

// Launch one tensor-core sweep sum_t a_{ia(t)} x_{ix(t)} with epilogue epi:
// npa (npx) pieces of the K-major A (X) operand.  Returns the number of row
// blocks (partials per column) or a negative error code.
template <class E>
int launch(Handle* h, int M, int N, int K, const float* const* ap, int npa, const float* const* xp, int npx,
           const TermList& tl, int64_t lda, int64_t ldx, const E& epi, double* part, const int32_t* active) {
    // 64-column tiles: at the batched sizes of interest (M ~ 1e3, N ~ 1e3)
    // they keep every SM busy; 128-column tiles halve the L2 traffic but leave
    // half of the SMs idle and measured slower
    const int bn = 64;
    PieceMaps maps;
    L1_TRY(get_maps(h, M, N, K, ap, npa, xp, npx, lda, ldx, bn, &maps));
    const int sel = npa * 10 + npx;
    if (bn == 128) {
        if (sel == 22) return launch_inst<E, 128, 2, 2>(h, maps, tl, M, N, K, epi, part, active);
        if (sel == 11) return launch_inst<E, 128, 1, 1>(h, maps, tl, M, N, K, epi, part, active);
        if (sel == 33) return launch_inst<E, 128, 3, 3>(h, maps, tl, M, N, K, epi, part, active);
    } else {
        if (sel == 22) return launch_inst<E, 64, 2, 2>(h, maps, tl, M, N, K, epi, part, active);
        if (sel == 11) return launch_inst<E, 64, 1, 1>(h, maps, tl, M, N, K, epi, part, active);
        if (sel == 33) return launch_inst<E, 64, 3, 3>(h, maps, tl, M, N, K, epi, part, active);
    }
    return L1_ERR_INVALID_ARG;
}

inline int row_blocks(int M) { return (M + kBM - 1) / kBM; }

}  // namespace tc
}  // namespace l1
