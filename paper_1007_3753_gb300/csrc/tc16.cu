// Aligned BF16 pieces of the operands of the tensor-core sweeps (see
// gemm_bf16.cuh): the dictionary's two layouts and (B B^T)^{-1} once at
// setup, the carried panel after a compaction.
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
    L1_TRY(dev_alloc_t(h, &h->tc_wk, (size_t)sms * 128 * 128));
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

}  // namespace tc16
}  // namespace l1
