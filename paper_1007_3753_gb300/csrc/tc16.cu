// Aligned BF16 pieces of the operands of the tensor-core sweeps (see
// gemm_bf16.cuh): the dictionary's two layouts and (B B^T)^{-1} once at
// setup, the carried panel after a compaction.
#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "tc16.cuh"

namespace l1 {
namespace tc16 {

// One warp per (line, 128-element block of K): the block's largest magnitude
// sets the grid, then each element is split into np pieces (split_aligned).
// hi (+ lo, nullable) is the value (lo: the low part of an FP32 pair);
// lines are `ld` elements apart; pieces are written with the same layout.
__global__ void split_aligned_kernel(const float* __restrict__ hi, const float* __restrict__ lo, int64_t lines,
                                     int K, int64_t ld, __nv_bfloat16* __restrict__ p0,
                                     __nv_bfloat16* __restrict__ p1, __nv_bfloat16* __restrict__ p2, int np) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nblk = (K + kChunk - 1) / kChunk;
    if (gw >= lines * nblk) return;
    const int64_t line = gw / nblk;
    const int k0 = (int)(gw % nblk) * kChunk;
    float v[kChunk / 32];
    float mx = 0.0f;
#pragma unroll
    for (int t = 0; t < kChunk / 32; ++t) {
        const int k = k0 + t * 32 + lane;
        float x = 0.0f;
        if (k < K) {
            const int64_t o = line * ld + k;
            // an FP32 pair hi + lo is rounded once, to the nearest FP32 value
            // of the FP64 sum (its exact value is below the pieces' grid)
            x = lo ? (float)((double)hi[o] + (double)lo[o]) : hi[o];
        }
        v[t] = x;
        mx = fmaxf(mx, fabsf(x));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
#pragma unroll
    for (int t = 0; t < kChunk / 32; ++t) {
        const int k = k0 + t * 32 + lane;
        if (k >= K) continue;
        float a, b, c;
        split_aligned(v[t], mx, a, b, c);
        const int64_t o = line * ld + k;
        p0[o] = __float2bfloat16_rn(a);
        if (np > 1) p1[o] = __float2bfloat16_rn(b);
        if (np > 2) p2[o] = __float2bfloat16_rn(c);
    }
}

int split_aligned_lines(Handle* h, const float* hi, const float* lo, int64_t lines, int K, int64_t ld,
                        __nv_bfloat16* const* p, int np) {
    if (lines <= 0 || K <= 0) return L1_OK;
    const int nblk = (K + kChunk - 1) / kChunk;
    const int64_t warps = lines * nblk;
    const int64_t blocks = (warps * 32 + 255) / 256;
    split_aligned_kernel<<<(unsigned)blocks, 256, 0, h->stream>>>(hi, lo, lines, K, ld, p[0], np > 1 ? p[1] : nullptr,
                                                                   np > 2 ? p[2] : nullptr, np);
    L1_LAUNCH_CHECK(h);
    return L1_OK;
}

int make_dictionary_pieces(Handle* h) {
    const int m = (int)h->m, n = (int)h->n;
    for (int p = 0; p < kMaxPieces; ++p) {
        L1_TRY(dev_alloc_t(h, &h->A_rm_h[p], (size_t)h->ldn * m));
        L1_TRY(dev_alloc_t(h, &h->A_cm_h[p], (size_t)h->ldm * n));
    }
    const int sms = h->sms > 0 ? h->sms : 152;
    L1_TRY(dev_alloc_t(h, &h->tc_wk, (size_t)kSplitWaves * sms * 128 * 128));
    h->tc_wk_elems = (size_t)kSplitWaves * sms * 128 * 128;
    // A u: K = n along the rows of A; A^T y: K = m along the columns of A
    L1_TRY(split_aligned_lines(h, h->A_rm, nullptr, m, n, h->ldn, h->A_rm_h, kMaxPieces));
    L1_TRY(split_aligned_lines(h, h->A_cm, nullptr, n, m, h->ldm, h->A_cm_h, kMaxPieces));
    return L1_OK;
}

int make_factor_pieces(Handle* h) {
    const int m = (int)h->m;
    for (int p = 0; p < kMaxPieces; ++p) L1_TRY(dev_alloc_t(h, &h->F_h[p], (size_t)h->ldm * m));
    // F is symmetric: its columns are its rows, K-major as the A operand
    L1_TRY(split_aligned_lines(h, h->F, h->F_lo, m, m, h->ldm, h->F_h, kMaxPieces));
    return L1_OK;
}

// --------------------------------------------------------------- autotuner
namespace {

// Epilogue of the timing launches: the traffic of the heaviest real one (the
// y-step's, EpiTcY for CAB): three floats read and four written per output
// element, besides the BF16 pieces.
struct EpiTune {
    static constexpr int NRED = 0;
    struct State {
        float a, b, c;
        int act;
    };
    float* S;  // four planes of ld x N
    int64_t ld, plane;
    __device__ State load(int i, int j) const {
        const int64_t o = (int64_t)j * ld + i;
        return State{S[o], S[plane + o], S[2 * plane + o], 1};
    }
    __device__ float apply(int i, int j, float acc, const State& st, float*) const {
        const int64_t o = (int64_t)j * ld + i;
        const float y = fmaf(st.a, 0.5f, acc);
        S[o] = y;
        S[plane + o] = fmaf(st.b, 0.5f, y);
        S[2 * plane + o] = fmaf(st.c, 0.5f, y);
        S[3 * plane + o] = y - st.c;
        return y;
    }
};

// scratch panel pieces: BF16 values of magnitude below 1 (piece p scaled by
// 2^-8p) from an integer hash, so the timed products are not of zeros
__global__ void tune_fill_kernel(__nv_bfloat16* x, int64_t count, int p) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    uint32_t v = (uint32_t)i * 2654435761u + 0x9e3779b9u * (uint32_t)(p + 1);
    v ^= v >> 15;
    v *= 2246822519u;
    v ^= v >> 13;
    const float f = ((float)(v & 0xffffu) / 32768.0f - 1.0f) * ldexpf(1.0f, -8 * p);
    x[i] = __float2bfloat16_rn(f);
}

}  // namespace

int tune_splits(Handle* h) {
    h->tc_splits.clear();
    const int sms = h->sms > 0 ? h->sms : 152;
    const int m = (int)h->m, n = (int)h->n;
    struct Shape {
        int M, K;
        __nv_bfloat16* const* a;
        int64_t lda;
    };
    const Shape shapes[3] = {{m, n, h->A_rm_h, h->ldn}, {m, m, h->F_h, h->ldm}, {n, m, h->A_cm_h, h->ldm}};
    const int nshapes = h->F_h[0] ? 3 : 2;  // no factor pieces: A u and A^T y only
    // column-tile counts timed (batch widths up to 4096); a width between two
    // of them takes the smaller one's choice
    static const int kTileCols[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32};
    constexpr int kMaxTilesN = 32;
    if (!h->tc_wk) return L1_OK;
    const int Nt = kMaxTilesN * 128;
    const int64_t Kp = round_up(std::max(m, n), 8), Mp = round_up(std::max(m, n), 128);
    const size_t xbytes = (size_t)kMaxPieces * Kp * Nt * 2, sbytes = (size_t)4 * Mp * Nt * 4,
                 pbytes = (size_t)kMaxPieces * Mp * Nt * 2, wbytes = (size_t)Mp * Nt * 4;
    uint8_t* scratch = nullptr;
    if (xbytes + sbytes + pbytes + wbytes > ((size_t)3 << 30) ||
        cudaMalloc(&scratch, xbytes + sbytes + pbytes + wbytes) != cudaSuccess) {
        cudaGetLastError();
        return L1_OK;  // keep the fixed rule
    }
    __nv_bfloat16* X[kMaxPieces];
    __nv_bfloat16* P[kMaxPieces];
    for (int p = 0; p < kMaxPieces; ++p) {
        X[p] = reinterpret_cast<__nv_bfloat16*>(scratch) + (size_t)p * Kp * Nt;
        P[p] = reinterpret_cast<__nv_bfloat16*>(scratch + xbytes + sbytes) + (size_t)p * Mp * Nt;
    }
    float* S = reinterpret_cast<float*>(scratch + xbytes);
    // the timing launches use a scratch of their own for the deferred and
    // split sums (the handle's may be smaller)
    float* const wk_keep = h->tc_wk;
    const size_t wk_keep_elems = h->tc_wk_elems;
    h->tc_wk = reinterpret_cast<float*>(scratch + xbytes + sbytes + pbytes);
    h->tc_wk_elems = (size_t)Mp * Nt;
    cudaStream_t s = h->stream;
    int rc = L1_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    do {
        if (cudaMemsetAsync(S, 0, sbytes, s) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
            cudaEventCreate(&e1) != cudaSuccess) {
            rc = L1_ERR_CUDA;
            break;
        }
        const int64_t cnt = Kp * Nt;
        for (int p = 0; p < kMaxPieces; ++p) {
            tune_fill_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(X[p], cnt, p);
            ++h->launches;
        }
        const Terms tl = terms_3x3();
        for (int si = 0; si < 3; ++si) {
            if (nshapes == 2 && si == 1) continue;
            const Shape& sh = shapes[si];
            const int tm = (sh.M + kBM - 1) / kBM;
            const int chunks = (sh.K + kChunk - 1) / kChunk;
            for (int tn : kTileCols) {
                if (rc != L1_OK) break;
                const int tiles = tm * tn, N = tn * 128;
                Operands op{{sh.a[0], sh.a[1], sh.a[2]}, 3, {X[0], X[1], X[2]}, 3, sh.lda, Kp};
                const EpiTune epi{S, Mp, (int64_t)Mp * Nt};
                const PieceOut po{{P[0], P[1], P[2]}, 3, Mp};
                // candidates: 128-wide tiles fused, deferred, and split-K with
                // each distinct slice count up to four waves of one CTA per SM
                // (a narrow batch of 32 row tiles fills 128 of 152 SMs with
                // four slices; nine slices run 288 CTAs in two waves);
                // 64-wide tiles deferred and split the same way
                std::vector<Split> cands = {Split{1, 0, 128}, Split{1, 1, 128}};
                for (int bn : {128, 64}) {
                    const int tb = tm * ((N + bn - 1) / bn);
                    if (bn == 64) cands.push_back(Split{1, 1, 64});
                    int last = 1;
                    for (int ks = 2; ks <= std::min(16, chunks) && ks * tb <= kSplitWaves * sms; ++ks) {
                        const Split c = normalise(h, Split{ks, 1, bn}, sh.M, N, sh.K);
                        if (c.ks > 1 && c.bn == bn && c.ks != last) {
                            cands.push_back(c);
                            last = c.ks;
                        }
                    }
                }
                std::vector<float> times;
                for (const Split& c : cands) {
                    constexpr int kReps = 3;
                    for (int r = 0; r <= kReps && rc == L1_OK; ++r) {
                        if (r == 1) cudaEventRecord(e0, s);
                        const int q = launch<EpiTune>(h, sh.M, N, sh.K, op, tl, epi, po, nullptr, nullptr, c);
                        if (q < 0) rc = q;
                    }
                    if (rc) break;
                    cudaEventRecord(e1, s);
                    if (cudaEventSynchronize(e1) != cudaSuccess) {
                        rc = L1_ERR_CUDA;
                        break;
                    }
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    times.push_back(1e3f * ms / kReps);
                }
                if (rc) break;
                // the first candidate (128-wide fused, deferred, fewer
                // slices, then 64-wide) within 2 % of the fastest
                float fastest = 1e30f;
                for (float t : times) fastest = std::min(fastest, t);
                size_t best = 0;
                while (times[best] > 1.02f * fastest) ++best;
                h->tc_splits.push_back({sh.M, sh.K, tiles, cands[best].ks, cands[best].defer, cands[best].bn,
                                        (int32_t)std::lround(times[best])});
            }
            if (rc) break;
        }
    } while (false);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    h->tc_wk = wk_keep;
    h->tc_wk_elems = wk_keep_elems;
    if (rc == L1_OK) {
        int herr = 0;
        if (cudaMemcpy(&herr, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = L1_ERR_CUDA;
        else if (herr != 0) {
            // a bounded wait inside a timing launch ran out
            set_last_error("split-K autotuner: tcgen05 sweep wait expired (code " + std::to_string(herr) + ")");
            cudaMemset(h->tc_err, 0, sizeof(int));
            rc = L1_ERR_TIMEOUT;
        }
    }
    cudaFree(scratch);
    h->map_cache.clear();  // drop the scratch panels' tensor maps
    if (rc != L1_OK) {
        h->tc_splits.clear();
        if (rc == L1_ERR_CUDA)
            set_last_error(std::string("split-K autotuner: ") + cudaGetErrorString(cudaGetLastError()));
    }
    return rc;
}

}  // namespace tc16
}  // namespace l1
