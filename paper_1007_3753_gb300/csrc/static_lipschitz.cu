// l1_lipschitz_static: power-iteration estimate of ||A||_2^2 that allocates
// no memory.  Everything else in this library allocates device memory in
// l1_setup (and cudaFree's it in l1_destroy); this entry point is for callers
// that cannot do that: a process whose device memory is all handed to its own
// pool allocator (cudaMalloc would fail or fragment the pool), or a loop that
// must not stall the device (cudaMalloc and cudaFree can synchronise it).
//
// Its scratch lives in one file-scope device array of fixed size, so every
// GPU that loads this library holds those bytes until the process exits.
// Host code cannot pass the array's name to a kernel (on the host the name
// stands for a host-side shadow, not a device address); the device address
// comes from cudaGetSymbolAddress, looked up once per device, with that
// device current, on the first call made there.
//
// The kernels are a variant of the handle's power iteration (same start
// vector, same Rayleigh quotient, same stopping rule) that reads A in the
// caller's column-major layout instead of the handle's two copies of A.
#include <math.h>

#include <mutex>
#include <string>

#include "common.cuh"

namespace l1 {
namespace {

// Limits of the static scratch.
constexpr int kStaticMaxM = 8192;    // rows of A
constexpr int kStaticMaxN = 65536;   // columns of A
constexpr int kChunks = 32;          // column chunks of the A v sweep
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// Layout of the scratch, in doubles (floats take half a double each).
constexpr int kOffState = 0;                                   // rho, scale, it, done
constexpr int kOffQ = 32;                                      // [kStaticMaxM / 256] partial ||u||^2
constexpr int kOffR = kOffQ + kStaticMaxM / kThreads;          // [kStaticMaxN / 8]  partial ||v||^2
constexpr int kOffU = kOffR + kStaticMaxN / (kThreads / 32);   // u = A v, kStaticMaxM floats
constexpr int kOffV = kOffU + kStaticMaxM / 2;                 // v, kStaticMaxN floats
constexpr int kOffP = kOffV + kStaticMaxN / 2;                 // [kChunks][m] floats, partial A v
constexpr int kScratchDoubles = kOffP + kChunks * kStaticMaxM / 2;  // 176,192 doubles = 1.34 MiB
static_assert(kScratchDoubles == 176192, "scratch layout");

static __device__ __align__(256) double g_static_scratch[kScratchDoubles];

struct Carve {
    double* state;
    double* q;
    double* r;
    float* u;
    float* v;
    float* p;
};

__device__ __forceinline__ Carve carve(double* base) {
    return Carve{base + kOffState, base + kOffQ, base + kOffR, reinterpret_cast<float*>(base + kOffU),
                 reinterpret_cast<float*>(base + kOffV), reinterpret_cast<float*>(base + kOffP)};
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
    return s;  // valid on thread 0
}

// v = 1/sqrt(n) and a cleared state; every call starts from here, whatever
// the previous call left in the scratch.
__global__ void static_init_kernel(double* base, int n, float v0) {
    Carve c = carve(base);
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) c.v[j] = v0;
    if (j == 0) {
        c.state[0] = 0.0;  // rho
        c.state[1] = 1.0;  // scale of v
        c.state[2] = 0.0;  // iterations done
        c.state[3] = 0.0;  // done flag
    }
}

// P[chunk][i] = sum over the chunk's columns j of A(i, j) v(j)
__global__ void static_av_kernel(double* base, const float* __restrict__ A, int64_t lda, int m, int n,
                                 int cw) {
    Carve c = carve(base);
    if (c.state[3] != 0.0) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int j0 = blockIdx.y * cw, j1 = min(n, j0 + cw);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    int j = j0;
    for (; j + 4 <= j1; j += 4) {
        a0 = fmaf(A[(int64_t)j * lda + i], c.v[j], a0);
        a1 = fmaf(A[(int64_t)(j + 1) * lda + i], c.v[j + 1], a1);
        a2 = fmaf(A[(int64_t)(j + 2) * lda + i], c.v[j + 2], a2);
        a3 = fmaf(A[(int64_t)(j + 3) * lda + i], c.v[j + 3], a3);
    }
    for (; j < j1; ++j) a0 = fmaf(A[(int64_t)j * lda + i], c.v[j], a0);
    c.p[(int64_t)blockIdx.y * m + i] = ((a0 + a1) + (a2 + a3)) * (float)c.state[1];
}

// u = sum of the chunk partials; Q[block] = partial ||u||^2
__global__ void static_u_kernel(double* base, int m, int chunks) {
    __shared__ double sh[kThreads / 32];
    Carve c = carve(base);
    if (c.state[3] != 0.0) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double sq = 0.0;
    if (i < m) {
        float s = 0.f;
        for (int k = 0; k < chunks; ++k) s += c.p[(int64_t)k * m + i];
        c.u[i] = s;
        sq = (double)s * s;
    }
    sq = block_sum(sq, sh);
    if (threadIdx.x == 0) c.q[blockIdx.x] = sq;
}

// v(j) = A(:, j)^T u, one warp per column; R[block] = partial ||v||^2
__global__ void static_atu_kernel(double* base, const float* __restrict__ A, int64_t lda, int m, int n) {
    __shared__ double sh[kThreads / 32];
    Carve c = carve(base);
    if (c.state[3] != 0.0) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + w;
    double sq = 0.0;
    if (j < n) {
        const float* col = A + (int64_t)j * lda;
        float s = 0.f;
        for (int i = lane; i < m; i += 32) s = fmaf(col[i], c.u[i], s);
        s = warp_sum_f(s);
        if (lane == 0) {
            c.v[j] = s;
            sq = (double)s * s;
        }
    }
    sq = block_sum(sq, sh);
    if (threadIdx.x == 0) c.r[blockIdx.x] = sq;
}

// rho = ||A v||^2 (Rayleigh quotient of A^T A at the unit vector v); stop when
// it changes by at most rtol relative, or when A^T A v = 0.
__global__ void static_finish_kernel(double* base, int nq, int nr, double rtol) {
    __shared__ double sh[kThreads / 32];
    Carve c = carve(base);
    if (c.state[3] != 0.0) return;
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < nq; k += blockDim.x) a += c.q[k];
    for (int k = threadIdx.x; k < nr; k += blockDim.x) b += c.r[k];
    a = block_sum(a, sh);
    __syncthreads();
    b = block_sum(b, sh);
    if (threadIdx.x == 0) {
        const double rho_new = a, it = c.state[2] + 1.0;
        const bool done = (it > 1.0 && fabs(rho_new - c.state[0]) <= rtol * rho_new) || b == 0.0;
        c.state[0] = rho_new;
        c.state[1] = b > 0.0 ? 1.0 / sqrt(b) : 0.0;
        c.state[2] = it;
        c.state[3] = done ? 1.0 : 0.0;
    }
}

std::mutex g_addr_mu;
double* g_addr[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up once).
int static_scratch(int dev, double** out) {
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            set_last_error(std::string("l1_lipschitz_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return L1_ERR_CUDA;
        }
        g_addr[dev] = static_cast<double*>(p);
    }
    *out = g_addr[dev];
    return L1_OK;
}

}  // namespace
}  // namespace l1

extern "C" {

L1_API int l1_lipschitz_static(const float* A, int64_t m, int64_t n, int64_t lda, int32_t max_iter, double rtol,
                               void* stream, double* rho_out, int32_t* status_out, int32_t* iters_out) {
    using namespace l1;
    if (!A || !rho_out || m <= 0 || n <= 0 || lda < m || max_iter <= 0 || !(rtol >= 0.0))
        return L1_ERR_INVALID_ARG;
    if (m > kStaticMaxM || n > kStaticMaxN) {
        set_last_error("l1_lipschitz_static: A is " + std::to_string(m) + " x " + std::to_string(n) +
                       "; the static scratch holds at most " + std::to_string(kStaticMaxM) + " x " +
                       std::to_string(kStaticMaxN));
        return L1_ERR_INVALID_ARG;
    }
    int dev = 0;
    L1_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_last_error("l1_lipschitz_static: device ordinal out of range");
        return L1_ERR_INVALID_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        // the call copies the state to pageable host memory and synchronises
        // its stream, neither of which a stream capture allows
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        L1_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
        if (cs != cudaStreamCaptureStatusNone) {
            set_last_error("l1_lipschitz_static: the stream is being captured; the call synchronises it");
            return L1_ERR_INVALID_ARG;
        }
    }
    cudaPointerAttributes attr{};
    L1_CUDA_TRY(cudaPointerGetAttributes(&attr, A));
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) {
        set_last_error("l1_lipschitz_static: A must be device (or managed) memory");
        return L1_ERR_INVALID_ARG;
    }
    if (attr.type == cudaMemoryTypeDevice && attr.device != dev) {
        // a pointer into another GPU's memory would be dereferenced as a peer
        // address by the kernels below; refuse it instead
        set_last_error("l1_lipschitz_static: A lives on device " + std::to_string(attr.device) +
                       " but device " + std::to_string(dev) + " is current");
        return L1_ERR_INVALID_ARG;
    }
    double* base = nullptr;
    L1_TRY(static_scratch(dev, &base));

    const int mi = (int)m, ni = (int)n;
    const int cw = (ni + kChunks - 1) / kChunks;
    const int chunks = (ni + cw - 1) / cw;
    const int nq = (mi + kThreads - 1) / kThreads;
    const int nr = (ni + (kThreads / 32) - 1) / (kThreads / 32);
    static_init_kernel<<<(ni + kThreads - 1) / kThreads, kThreads, 0, s>>>(base, ni,
                                                                          (float)(1.0 / sqrt((double)ni)));
    L1_CUDA_TRY(cudaGetLastError());
    // iterations are enqueued in batches; once the device-side rule fires the
    // remaining launches of a batch return at once
    constexpr int kBatch = 8;
    double state[4] = {0.0, 0.0, 0.0, 0.0};
    for (int it = 0; it < max_iter; it += kBatch) {
        const int k = max_iter - it < kBatch ? max_iter - it : kBatch;
        for (int t = 0; t < k; ++t) {
            static_av_kernel<<<dim3(nq, chunks), kThreads, 0, s>>>(base, A, lda, mi, ni, cw);
            static_u_kernel<<<nq, kThreads, 0, s>>>(base, mi, chunks);
            static_atu_kernel<<<nr, kThreads, 0, s>>>(base, A, lda, mi, ni);
            static_finish_kernel<<<1, kThreads, 0, s>>>(base, nq, nr, rtol);
        }
        L1_CUDA_TRY(cudaGetLastError());
        L1_CUDA_TRY(cudaMemcpyAsync(state, base + kOffState, sizeof(state), cudaMemcpyDeviceToHost, s));
        L1_CUDA_TRY(cudaStreamSynchronize(s));
        if (state[3] != 0.0) break;
    }
    *rho_out = state[0];
    if (status_out) *status_out = state[3] != 0.0 ? L1_CONVERGED : L1_MAX_ITER;
    if (iters_out) *iters_out = (int32_t)state[2];
    return L1_OK;
}

}  // extern "C"
