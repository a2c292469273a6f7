// Host side of the tcgen05 sweeps (see tc.cuh).
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "tc.cuh"

namespace l1 {
namespace tc {

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

int make_map(CUtensorMap* map, const void* base, uint64_t inner, uint64_t rows, uint64_t pitch_bytes,
             uint32_t box_rows) {
    auto fn = encode_fn();
    if (!fn) {
        set_last_error("cuTensorMapEncodeTiled unavailable");
        return L1_ERR_CUDA;
    }
    // TMA rules: 16-byte aligned base and pitch; the box's inner extent is
    // 128 bytes (32 floats) and every x coordinate used is a multiple of 32
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (pitch_bytes & 15)) return L1_ERR_INVALID_ARG;
    const cuuint64_t dims[2] = {inner, rows};
    const cuuint64_t strides[1] = {pitch_bytes};
    const cuuint32_t box[2] = {32, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_last_error("cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
        return L1_ERR_CUDA;
    }
    return L1_OK;
}

__global__ void split_tf32_kernel(const float* x, int64_t count, float* p1, float* p2, float* p3) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float a, b, c;
    tf32_split3(x[i], a, b, c);
    p1[i] = a;
    p2[i] = b;
    if (p3) p3[i] = c;
}

__global__ void split_tf32_f64_kernel(const double* x, int rows, int cols, int64_t ld_src, int64_t ld_dst,
                                      float* p1, float* p2, float* p3) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)ld_dst * cols) return;
    const int64_t c = idx / ld_dst, r = idx % ld_dst;
    const double v = r < rows ? x[c * ld_src + r] : 0.0;
    const float a = tf32_rn((float)v);
    const double r1 = v - (double)a;
    const float b = tf32_rn((float)r1);
    const float cc = (float)(r1 - (double)b);
    p1[idx] = a;
    p2[idx] = b;
    if (p3) p3[idx] = cc;
}

int split_tf32(Handle* h, const float* x, int64_t count, float* p1, float* p2, float* p3) {
    split_tf32_kernel<<<(unsigned)((count + 255) / 256), 256, 0, h->stream>>>(x, count, p1, p2, p3);
    L1_LAUNCH_CHECK(h);
    return L1_OK;
}

int split_tf32_from_f64(Handle* h, const double* x, int rows, int cols, int64_t ld_src, int64_t ld_dst,
                        float* p1, float* p2, float* p3) {
    const int64_t total = ld_dst * cols;
    split_tf32_f64_kernel<<<(unsigned)((total + 255) / 256), 256, 0, h->stream>>>(x, rows, cols, ld_src, ld_dst,
                                                                                  p1, p2, p3);
    L1_LAUNCH_CHECK(h);
    return L1_OK;
}

}  // namespace tc
}  // namespace l1
