// Host side of the tcgen05 sweeps: tensor maps, TF32 operand pieces, launch.
#pragma once

#include "common.cuh"
#include "gemm_tc.cuh"

namespace l1 {
namespace tc {

// Tiled 2-D tensor map over a row-major array of `rows` rows of `inner`
// elements (FP32 or BF16), row pitch `pitch_bytes`; box = 128 bytes along
// the row x box_rows, 128-byte swizzle.  Returns L1_OK or L1_ERR_CUDA.
int make_map(CUtensorMap* map, const void* base, int elem_bytes, uint64_t inner, uint64_t rows,
             uint64_t pitch_bytes, uint32_t box_rows);

// TF32 pieces of an FP32 array: p1 = x with the low 13 mantissa bits
// cleared, p2 the same for x - p1, p3 = x - p1 - p2 (exact: 24 = 11 + 11 + 2
// significant bits), so p1 + p2 + p3 == x and tcgen05 kind::tf32 reads each
// piece without truncation.  count elements; p3 may be null.
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

struct Term {
    const float* a;  // K-major M x K (row pitch lda floats)
    const float* x;  // column-major K x N (column pitch ldx floats)
};

constexpr int kBN = 64;
// K blocks (of 32 TF32 elements, 4 MMAs) accumulated in TMEM before the
// epilogue drains them into compensated register sums
#ifndef L1_TC_CHUNK
#define L1_TC_CHUNK 1
#endif
constexpr int kDrainChunk = L1_TC_CHUNK;

// Tensor maps of a term list, encoded once per (pointers, shape) and cached
// in the handle (encoding costs host time on every sweep otherwise).
inline int get_maps(Handle* h, int M, int N, int K, const Term* terms, int nterms, int64_t lda, int64_t ldx,
                    TermMaps* out) {
    std::array<uint64_t, 16> key{};
    key[0] = (uint64_t)M | ((uint64_t)N << 32);
    key[1] = (uint64_t)K | ((uint64_t)nterms << 32);
    key[2] = (uint64_t)lda;
    key[3] = (uint64_t)ldx;
    for (int t = 0; t < nterms; ++t) {
        key[4 + 2 * t] = reinterpret_cast<uint64_t>(terms[t].a);
        key[5 + 2 * t] = reinterpret_cast<uint64_t>(terms[t].x);
    }
    for (const auto& e : h->map_cache) {
        if (e.key == key) {
            for (int t = 0; t < nterms; ++t) {
                out->a[t] = e.maps[t];
                out->x[t] = e.maps[nterms + t];
            }
            return L1_OK;
        }
    }
    std::memset(out, 0, sizeof(*out));
    const uint64_t Kp = (uint64_t)round_up(K, 32);
    for (int t = 0; t < nterms; ++t) {
        L1_TRY(make_map(&out->a[t], terms[t].a, 4, Kp, (uint64_t)M, (uint64_t)lda * 4, kBM));
        L1_TRY(make_map(&out->x[t], terms[t].x, 4, Kp, (uint64_t)N, (uint64_t)ldx * 4, kBN));
    }
    Handle::MapCacheEntry e;
    e.key = key;
    for (int t = 0; t < nterms; ++t) e.maps.push_back(out->a[t]);
    for (int t = 0; t < nterms; ++t) e.maps.push_back(out->x[t]);
    if (h->map_cache.size() > 64) h->map_cache.erase(h->map_cache.begin());
    h->map_cache.push_back(std::move(e));
    return L1_OK;
}

// Launch one split-TF32 sweep sum_t a_t x_t with epilogue epi.  Returns the
// number of row blocks (partials per column) or a negative error code.
template <class E>
int launch(Handle* h, int M, int N, int K, const Term* terms, int nterms, int64_t lda, int64_t ldx,
           const E& epi, double* part, const int32_t* active) {
    constexpr int BN = kBN;
    if (nterms < 1 || nterms > kMaxTerms) return L1_ERR_INVALID_ARG;
    TermMaps maps;
    L1_TRY(get_maps(h, M, N, K, terms, nterms, lda, ldx, &maps));
    using S = Smem<BN>;
    constexpr int CHUNK = kDrainChunk;
    static bool attr_set = false;
    if (!attr_set) {
        L1_CUDA_TRY(cudaFuncSetAttribute(gemm_tc_kernel<E, BN, true, CHUNK>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes));
        attr_set = true;
    }
    dim3 grid((N + BN - 1) / BN, (M + kBM - 1) / kBM);
    gemm_tc_kernel<E, BN, true, CHUNK><<<grid, kThreads, S::kBytes, h->stream>>>(maps, nterms, M, N, K, epi, part,
                                                                                 active, h->tc_err);
    L1_LAUNCH_CHECK(h);
    return (int)grid.y;
}

inline int row_blocks(int M) { return (M + kBM - 1) / kBM; }

}  // namespace tc
}  // namespace l1
