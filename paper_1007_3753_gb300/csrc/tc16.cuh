// Host side of the BF16 tcgen05 sweeps (gemm_bf16.cuh): tensor maps of the
// BF16 operand pieces, cached per handle, and the launch.
#pragma once

#include "common.cuh"
#include "gemm_bf16.cuh"
#include "tc.cuh"
#include "tcgen05.cuh"

namespace l1 {
namespace tc16 {

// BF16 operand pieces of one sweep: K-major A pieces (row pitch lda
// elements), K-major X pieces (column pitch ldx elements).
struct Operands {
    const __nv_bfloat16* a[kMaxPieces];
    int npa;
    const __nv_bfloat16* x[kMaxPieces];
    int npx;
    int64_t lda, ldx;
};

// Term lists: which piece products a sweep issues (i-th term a_{ia} x_{ix}).
inline Terms terms_1x1() { return Terms{1, {0}, {0}}; }
// x split in two or three pieces, a single (BF16) A: a0 x0 + a0 x1 (+ a0 x2)
inline Terms terms_1xN(int npx) {
    Terms t{npx, {0, 0, 0}, {0, 1, 2}};
    return t;
}
// 16-bit products: a0 x0 + a0 x1 + a1 x0
inline Terms terms_2x2() { return Terms{3, {0, 0, 1}, {0, 1, 0}}; }
// FP32-level products of three-piece operands: every term of order <= 2^-16
inline Terms terms_3x3() { return Terms{6, {0, 0, 1, 0, 1, 2}, {0, 1, 0, 2, 1, 0}}; }
// three-piece A, two-piece x: a0 x0 + a0 x1 + a1 x0 + a1 x1 + a2 x0
inline Terms terms_3x2() { return Terms{5, {0, 0, 1, 1, 2}, {0, 1, 0, 1, 0}}; }

inline int get_maps(Handle* h, int M, int N, int K, const Operands& op, int bn, Maps* out) {
    std::array<uint64_t, 16> key{};
    key[0] = (uint64_t)M | ((uint64_t)N << 32);
    key[1] = (uint64_t)K | ((uint64_t)op.npa << 32) | ((uint64_t)op.npx << 40) | ((uint64_t)bn << 48) |
             (uint64_t)0xB0ull << 56;  // BF16 maps
    key[2] = (uint64_t)op.lda;
    key[3] = (uint64_t)op.ldx;
    for (int p = 0; p < op.npa; ++p) key[4 + p] = reinterpret_cast<uint64_t>(op.a[p]);
    for (int p = 0; p < op.npx; ++p) key[8 + p] = reinterpret_cast<uint64_t>(op.x[p]);
    for (const auto& e : h->map_cache) {
        if (e.key == key) {
            for (int p = 0; p < op.npa; ++p) out->a[p] = e.maps[p];
            for (int p = 0; p < op.npx; ++p) out->x[p] = e.maps[op.npa + p];
            return L1_OK;
        }
    }
    std::memset(out, 0, sizeof(*out));
    for (int p = 0; p < op.npa; ++p)
        L1_TRY(tc::make_map_bf16(&out->a[p], op.a[p], (uint64_t)K, (uint64_t)M, (uint64_t)op.lda * 2, kKB, kBM));
    for (int p = 0; p < op.npx; ++p)
        L1_TRY(tc::make_map_bf16(&out->x[p], op.x[p], (uint64_t)K, (uint64_t)N, (uint64_t)op.ldx * 2, kKB, bn));
    Handle::MapCacheEntry e;
    e.key = key;
    for (int p = 0; p < op.npa; ++p) e.maps.push_back(out->a[p]);
    for (int p = 0; p < op.npx; ++p) e.maps.push_back(out->x[p]);
    if (h->map_cache.size() > 64) h->map_cache.erase(h->map_cache.begin());
    h->map_cache.push_back(std::move(e));
    return L1_OK;
}

// Row blocks per finish-kernel CTA: long contiguous runs of a column when
// the batch is wide, one block per CTA (more CTAs) when it is narrow.
inline int fin_row_blocks(int tiles_m, int N) {
    const int sms = 152;
    return (int64_t)N * tiles_m >= 8LL * sms * kFinRB ? kFinRB : 1;
}

// How a sweep's output tiles are produced: their width bn (128, or 64 for
// narrow batches: half the MMA work per CTA, three ring stages), K slices
// (ks > 1: split-K, the slices' FP32 sums added in slice order by
// finish_kernel, deterministic for a given batch width) and whether the tile
// epilogue runs in the sweep (fused; 128-wide tiles only) or in
// finish_kernel from the tile's FP32 sums (deferred; always with ks > 1 or
// bn = 64).  The scratch holds ks x tiles x 128 x bn floats.
struct Split {
    int ks, defer, bn;
};

// split-K slices may fill up to this many waves of one CTA per SM
constexpr int kSplitWaves = 4;

inline Split normalise(const Handle* h, Split want, int M, int N, int K) {
    const int chunks = (K + kChunk - 1) / kChunk;
    const int bn = want.bn == 64 ? 64 : 128;
    int ks = std::max(1, std::min(std::min(want.ks, chunks), 16));
    const int cps = (chunks + ks - 1) / ks;
    ks = (chunks + cps - 1) / cps;  // no empty slice
    Split r{ks, (ks > 1 || want.defer || bn == 64) ? 1 : 0, bn};
    const size_t tiles = (size_t)((M + kBM - 1) / kBM) * ((N + bn - 1) / bn);
    if (r.defer && (size_t)r.ks * tiles * kBM * bn > h->tc_wk_elems) r = Split{1, 0, 128};
    return r;
}

// The autotuner's choice for (M, K) at the batch's count of 128-wide tiles
// (tune_splits): the entry of that count, else of the nearest smaller one
// (its slice count capped so that the CTAs fill no more waves of one CTA per
// SM than the entry's did).  Without one (tuning off, or a
// shape it did not time): 128-wide tiles, the epilogue deferred, and enough
// K slices to give every SM a CTA when a quarter of them has a tile.
inline Split split_choice(const Handle* h, int M, int N, int K) {
    const int sms = h->sms > 0 ? h->sms : 152;
    if (!h->tc_wk) return Split{1, 0, 128};
    const int tm = (M + kBM - 1) / kBM, tiles = tm * ((N + 127) / 128);
    const std::array<int32_t, 7>* near = nullptr;
    for (const auto& e : h->tc_splits)
        if (e[0] == M && e[1] == K && e[2] <= tiles && (!near || e[2] > (*near)[2])) near = &e;
    if (near) {
        const int bn = (*near)[5];
        const int tb = tm * ((N + bn - 1) / bn);
        const int tb_e = (*near)[2] * (128 / bn);  // the entry's tiles of width bn
        const int waves = std::max(1, ((*near)[3] * tb_e + sms - 1) / sms);
        return normalise(h, Split{std::min((*near)[3], std::max(1, waves * sms / tb)), (*near)[4], bn}, M, N, K);
    }
    const int chunks = (K + kChunk - 1) / kChunk;
    if (4 * tiles > sms || chunks < 4) return normalise(h, Split{1, 1, 128}, M, N, K);
    return normalise(h, Split{std::min(sms / tiles, 16), 1, 128}, M, N, K);
}

// Time the tile strategies of each tensor-core sweep shape of the handle (A u,
// the y-step, A^T y): fused, deferred and split-K with every useful slice
// count, at tile counts from one column tile up to 4096 columns, on scratch
// panels; record the fastest in h->tc_splits.  Skipped (fixed rule) when the
// scratch cannot be allocated.
int tune_splits(Handle* h);

// One BF16 tensor-core sweep sum_t a_{ia(t)} x_{ix(t)} with epilogue epi
// (gemm_bf16.cuh), tiles and slices as sp says (resolved by launch):
// operands split on the aligned grid of 128-element K blocks, exactly one
// leading term (0, 0); the functor returns the value that goes to the piece
// sink po (po.np = 0: none).  Returns the number of row blocks (partials per
// column) or a negative error code.
template <class E, int NPA, int NPX, int BN>
int launch_inst(Handle* h, const Maps& maps, const Terms& tl, int M, int N, int K, const E& epi,
                const PieceOut& po, double* part, const int32_t* active, Split sp) {
    using S = Cfg<BN, NPA, NPX>;
    static bool attr_set = false;
    if (!attr_set) {
        L1_CUDA_TRY(cudaFuncSetAttribute(sweep_kernel<E, NPA, NPX, BN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes));
        attr_set = true;
    }
    const int tiles_m = (M + kBM - 1) / kBM, tiles = tiles_m * ((N + BN - 1) / BN);
    const int ks = sp.ks;
    sweep_kernel<E, NPA, NPX, BN><<<tiles * ks, kThreads, S::kBytes, h->stream>>>(
        maps, tl, M, N, K, epi, po, part, active, h->tc_err, ks, sp.defer, h->tc_wk);
    L1_LAUNCH_CHECK(h);
    if (sp.defer) {
        const int rbs = fin_row_blocks(tiles_m, N);
        finish_kernel<E><<<N * ((tiles_m + rbs - 1) / rbs), kBM, 0, h->stream>>>(
            M, N, ks, h->tc_wk, (int64_t)tiles_m * kBM, nullptr, epi, po, part, active, rbs);
        L1_LAUNCH_CHECK(h);
    }
    return tiles_m;
}

// finish_kernel on sums that are not a sweep's: S(i, j) = sum over z <
// ksplit of src[(z * N + j) * lds + i], times colscale[j] when given.
// Returns the number of row blocks.
template <class E>
int finish(Handle* h, int M, int N, int ksplit, const float* src, int64_t lds, const float* colscale, const E& epi,
           const PieceOut& po, double* part, const int32_t* active) {
    const int tiles_m = (M + kBM - 1) / kBM;
    const int rbs = fin_row_blocks(tiles_m, N);
    finish_kernel<E><<<N * ((tiles_m + rbs - 1) / rbs), kBM, 0, h->stream>>>(M, N, ksplit, src, lds, colscale, epi,
                                                                           po, part, active, rbs);
    L1_LAUNCH_CHECK(h);
    return tiles_m;
}

// Piece counts (npa, npx) a launch may use: square splits of two or three
// pieces, and one-piece A with a two- or three-piece panel; 64-wide tiles
// for the three-piece square split.  force.ks > 0 overrides the tile choice.
template <class E>
int launch(Handle* h, int M, int N, int K, const Operands& op, const Terms& tl, const E& epi, const PieceOut& po,
           double* part, const int32_t* active, Split force = Split{0, 0, 128}) {
    if (tl.n < 1 || tl.n > kMaxTerms) return L1_ERR_INVALID_ARG;
    int nhi = 0;
    for (int t = 0; t < tl.n; ++t) {
        if (tl.ia[t] < 0 || tl.ia[t] >= op.npa || tl.ix[t] < 0 || tl.ix[t] >= op.npx) return L1_ERR_INVALID_ARG;
        nhi += (tl.ia[t] | tl.ix[t]) == 0;
    }
    if (nhi != 1) return L1_ERR_INVALID_ARG;  // exactly one leading term a_0 x_0
    if ((op.lda & 7) || (op.ldx & 7) || po.np < 0 || po.np > kMaxPieces || (po.np > 0 && (po.ld < M)))
        return L1_ERR_INVALID_ARG;
    const int cfg = op.npa * 10 + op.npx;
    Split sp = force.ks > 0 ? normalise(h, force, M, N, K) : split_choice(h, M, N, K);
    if (sp.bn == 64 && cfg != 33) sp = normalise(h, Split{sp.ks, 1, 128}, M, N, K);
    Maps maps;
    L1_TRY(get_maps(h, M, N, K, op, sp.bn, &maps));
    switch (cfg) {
        case 12: return launch_inst<E, 1, 2, 128>(h, maps, tl, M, N, K, epi, po, part, active, sp);
        case 13: return launch_inst<E, 1, 3, 128>(h, maps, tl, M, N, K, epi, po, part, active, sp);
        case 22: return launch_inst<E, 2, 2, 128>(h, maps, tl, M, N, K, epi, po, part, active, sp);
        case 33:
            if (sp.bn == 64) return launch_inst<E, 3, 3, 64>(h, maps, tl, M, N, K, epi, po, part, active, sp);
            return launch_inst<E, 3, 3, 128>(h, maps, tl, M, N, K, epi, po, part, active, sp);
        default: return L1_ERR_UNSUPPORTED;
    }
}

inline int row_blocks(int M) { return (M + kBM - 1) / kBM; }

// Aligned pieces (split_aligned, 128-element blocks along K) of `lines`
// lines of K elements, `ld` apart: the value is hi (+ lo, an FP32 pair,
// nullable); p[0 .. np) receive the pieces with the same layout.
int split_aligned_lines(Handle* h, const float* hi, const float* lo, int64_t lines, int K, int64_t ld,
                        __nv_bfloat16* const* p, int np);

// Three pieces of both layouts of A (h->A_rm_h, h->A_cm_h) and of
// (B B^T)^{-1} = F + F_lo (h->F_h).
int make_dictionary_pieces(Handle* h);
int make_factor_pieces(Handle* h);

}  // namespace tc16
}  // namespace l1
