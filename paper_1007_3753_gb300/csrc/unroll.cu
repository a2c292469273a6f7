// Unrolled PALM in P1 mode with a checkpointed tape, and its adjoint.
//
// Forward (reading R11 of Algorithm 1 for differentiation): x = 0, theta = 0;
// K inner FISTA steps in total (Eq. 18 applied to the augmented Lagrangian of
// Eq. 33), split into outer blocks of J steps; every block restarts FISTA from
// z = w = x with t = 1 and ends with x = w and the multiplier step
// theta += xi (b - A x).  xi (per column) and L are constants, so no gradient
// flows through them.  One inner step, per column:
//   r = b + theta/xi - A z;  v = z + A^T r / L;  w' = soft(v, 1/(xi L));
//   z' = w' + mu (w' - w),  mu = (t - 1)/t',  t' = (1 + sqrt(1 + 4 t^2))/2.
//
// Tape: (z, w, theta) every ckpt_every steps, and x at the end of every outer
// block.  The backward pass recomputes one segment of ckpt_every steps from
// its checkpoint (recording z, r and v of each step), then runs reverse-mode
// differentiation of exactly the statements above through that segment:
//   vbar = [|v| > 1/(xi L)] (wbar + (1 + mu) zbar),  wbar <- -mu zbar,
//   q = A vbar,  zbar <- vbar - A^T q / L,  cbar += q / L,
//   grad_A += (r vbar^T - q z^T) / L,
// and at the block boundaries
//   theta step:  grad_b += xi tbar,  xbar -= xi A^T tbar,  grad_A -= xi tbar x^T,
//   block start: xbar = wbar + zbar,  grad_b += cbar,  tbar += cbar / xi.
// The grad_A terms of a segment are summed as two rank-(N x steps) products
// (one kernel each) once the segment is reversed.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "gemm_simt.cuh"
#include "setup.cuh"

namespace l1 {

struct UnrollState {
    int N = 0, K = 0, J = 0, C = 0, n_outer = 0, nseg = 0;
    float* B = nullptr;    // copy of b (m x N)
    float* xi = nullptr;   // per column xi
    float* thr = nullptr;  // per column 1 / (xi L)
    float *Z = nullptr, *W = nullptr, *TH = nullptr, *R = nullptr;  // forward state
    float *ckZ = nullptr, *ckW = nullptr, *ckTH = nullptr;          // [nseg][N][ld]
    float* Xo = nullptr;                                            // [n_outer][N][ldn]
    float *sZ = nullptr, *sV = nullptr, *sVb = nullptr;             // [C][N][ldn]
    float *sR = nullptr, *sQ = nullptr;                             // [C][N][ldm]
    float *Xb = nullptr, *Wb = nullptr, *Zb = nullptr;              // n x N adjoints
    float *Tb = nullptr, *Cb = nullptr, *P = nullptr, *gB = nullptr;  // m x N adjoints
    float* gA = nullptr;                                            // m x n, ld = ldm
    double* part = nullptr;
    double* fin = nullptr;  // [N][2]: ||b - A x||^2, ||x||_1
    std::vector<double> mu;  // mu of every step
    bool has_tape = false;
    std::vector<void*> allocs;
    int64_t bytes = 0;
};

namespace {

// ------------------------------------------------------------ epilogues
// r = b + theta / xi - A z
struct EpiUrR {
    static constexpr int NRED = 0;
    float* R;
    const float* B;
    const float* TH;
    const float* xi;
    int64_t ldm;
    __device__ void operator()(int i, int j, float acc, double*) const {
        const int64_t o = (int64_t)j * ldm + i;
        R[o] = (B[o] + TH[o] / xi[j]) - acc;
    }
};

// v = z + g / L, w' = soft(v, 1/(xi L)), z' = w' + mu (w' - w);  g = A^T r.
// Zin may alias W (first step of a block, z = w).
struct EpiUrStep {
    static constexpr int NRED = 0;
    const float* Zin;
    float* Z;
    float* W;
    float* Vtape;  // nullable
    float* Ztape;  // nullable
    const float* thr;
    float Linv, mu;
    int64_t ldn;
    __device__ void operator()(int i, int j, float acc, double*) const {
        const int64_t o = (int64_t)j * ldn + i;
        const float z = Zin[o], w = W[o];
        const float v = fmaf(acc, Linv, z);
        const float wn = soft_thr(v, thr[j]);
        if (Ztape) Ztape[o] = z;
        if (Vtape) Vtape[o] = v;
        W[o] = wn;
        Z[o] = fmaf(mu, wn - w, wn);
    }
};

// theta += xi (b - A x)
struct EpiUrTheta {
    static constexpr int NRED = 0;
    float* TH;
    const float* B;
    const float* xi;
    int64_t ldm;
    __device__ void operator()(int i, int j, float acc, double*) const {
        const int64_t o = (int64_t)j * ldm + i;
        TH[o] = fmaf(xi[j], B[o] - acc, TH[o]);
    }
};

// red[0] = ||b - A x||^2
struct EpiUrResid {
    static constexpr int NRED = 1;
    const float* B;
    int64_t ldm;
    __device__ void operator()(int i, int j, float acc, double* red) const {
        const double d = (double)B[(int64_t)j * ldm + i] - (double)acc;
        red[0] += d * d;
    }
};

// q = A vbar;  cbar += q / L
struct EpiUrQ {
    static constexpr int NRED = 0;
    float* Q;
    float* Cb;
    float Linv;
    int64_t ldm;
    __device__ void operator()(int i, int j, float acc, double*) const {
        const int64_t o = (int64_t)j * ldm + i;
        Q[o] = acc;
        Cb[o] = fmaf(acc, Linv, Cb[o]);
    }
};

// zbar = vbar - A^T q / L
struct EpiUrZb {
    static constexpr int NRED = 0;
    float* Zb;
    const float* Vb;
    float Linv;
    int64_t ldn;
    __device__ void operator()(int i, int j, float acc, double*) const {
        const int64_t o = (int64_t)j * ldn + i;
        Zb[o] = fmaf(-acc, Linv, Vb[o]);
    }
};

// xbar -= xi A^T tbar
struct EpiUrXbTheta {
    static constexpr int NRED = 0;
    float* Xb;
    const float* xi;
    int64_t ldn;
    __device__ void operator()(int i, int j, float acc, double*) const {
        const int64_t o = (int64_t)j * ldn + i;
        Xb[o] = fmaf(-xi[j], acc, Xb[o]);
    }
};

// ------------------------------------------------------- elementwise steps
__global__ void ur_xi_kernel(const float* B, int64_t ldm, int m, int N, double xi0, double L, float* xi,
                             float* thr) {
    __shared__ double sh[4];
    const int j = blockIdx.x;
    if (j >= N) return;
    double s = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) s += fabs((double)B[(int64_t)j * ldm + i]);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        const double b1 = sh[0] + sh[1] + sh[2] + sh[3];
        // R3 start value 2m/||b||_1 (held constant); b = 0 keeps every iterate 0
        const double x = xi0 > 0.0 ? xi0 : (b1 > 0.0 ? 2.0 * m / b1 : 1.0);
        xi[j] = (float)x;
        thr[j] = (float)(1.0 / (x * L));
    }
}

// vbar = [|v| > thr] (wbar + (1 + mu) zbar);  wbar = -mu zbar
__global__ void ur_vbar_kernel(int n, int N, int64_t ldn, const float* V, const float* thr, float mu,
                               float* Wb, const float* Zb, float* Vb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= n || j >= N) return;
    const int64_t o = (int64_t)j * ldn + i;
    const float zb = Zb[o];
    const float wn_bar = fmaf(1.0f + mu, zb, Wb[o]);
    Vb[o] = fabsf(V[o]) > thr[j] ? wn_bar : 0.0f;
    Wb[o] = -mu * zb;
}

// block start: xbar = wbar + zbar
__global__ void ur_xbar_kernel(int n, int N, int64_t ldn, const float* Wb, const float* Zb, float* Xb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= n || j >= N) return;
    const int64_t o = (int64_t)j * ldn + i;
    Xb[o] = Wb[o] + Zb[o];
}

// block start: grad_b += cbar;  tbar += cbar / xi
__global__ void ur_cbar_kernel(int m, int N, int64_t ldm, const float* Cb, const float* xi, float* gB,
                               float* Tb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= m || j >= N) return;
    const int64_t o = (int64_t)j * ldm + i;
    const float cb = Cb[o];
    gB[o] += cb;
    Tb[o] += cb / xi[j];
}

// theta step of a block that has a successor: P = xi tbar;  grad_b += P
__global__ void ur_theta_bar_kernel(int m, int N, int64_t ldm, const float* Tb, const float* xi, float* P,
                                    float* gB) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= m || j >= N) return;
    const int64_t o = (int64_t)j * ldm + i;
    const float p = xi[j] * Tb[o];
    P[o] = p;
    gB[o] += p;
}

// block end (reverse entry): wbar = xbar, zbar = 0 (n part); cbar = 0 (m part)
__global__ void ur_block_enter_kernel(int n, int m, int N, int64_t ldn, int64_t ldm, const float* Xb,
                                      float* Wb, float* Zb, float* Cb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (j >= N) return;
    if (i < n) {
        const int64_t o = (int64_t)j * ldn + i;
        Wb[o] = Xb[o];
        Zb[o] = 0.0f;
    }
    if (i < m) Cb[(int64_t)j * ldm + i] = 0.0f;
}

__global__ void ur_final_kernel(const double* part, int np, int N, const float* W, int64_t ldn, int n,
                                double* fin) {
    __shared__ double sh[4];
    const int j = blockIdx.x;
    double r = 0.0, x1 = 0.0;
    for (int p = threadIdx.x; p < np; p += blockDim.x) r += part[((int64_t)p * N + j) * kPartStride];
    for (int i = threadIdx.x; i < n; i += blockDim.x) x1 += fabs((double)W[(int64_t)j * ldn + i]);
    r = warp_sum(r);
    x1 = warp_sum(x1);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) sh[w] = r;
    __syncthreads();
    double rs = 0.0;
    if (threadIdx.x == 0) rs = sh[0] + sh[1] + sh[2] + sh[3];
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[w] = x1;
    __syncthreads();
    if (threadIdx.x == 0) {
        fin[2 * j] = rs;
        fin[2 * j + 1] = sh[0] + sh[1] + sh[2] + sh[3];
    }
}

// --------------------------------------------------- rank-K update (NT GEMM)
// C(M x Nn, col-major, ldc) += alpha * sum_k P(i, k) Q(j, k), with P M x K and
// Q Nn x K column-major (ldp, ldq multiples of 4 floats).  64 x 64 tile per
// 256-thread CTA, 4 x 4 per thread, K step 16 through double-buffered shared
// memory; every K tile's 16 products go to a fresh partial merged with Kahan
// compensation.  One CTA owns each tile of C, so the update is deterministic.
constexpr int kRT = 64, kRK = 16;

__global__ void __launch_bounds__(256)
rank_update_kernel(int M, int Nn, int K, const float* __restrict__ P, int64_t ldp, const float* __restrict__ Q,
                   int64_t ldq, float alpha, float* __restrict__ Cm, int64_t ldc) {
    __shared__ __align__(16) float Ps[2][kRK][kRT];
    __shared__ __align__(16) float Qs[2][kRK][kRT];
    const int t = threadIdx.x;
    const int tc = t & 15, tr = t >> 4;
    const int m0 = blockIdx.y * kRT, n0 = blockIdx.x * kRT;
    const int l_k = t >> 4, l_i = (t & 15) * 4;  // 16 k x 16 float4
    auto load = [&](int buf, int k0) {
        float4 p = make_float4(0.f, 0.f, 0.f, 0.f), q = make_float4(0.f, 0.f, 0.f, 0.f);
        const int k = k0 + l_k;
        if (k < K) {
            if (m0 + l_i < M) p = __ldg(reinterpret_cast<const float4*>(P + (int64_t)k * ldp + m0 + l_i));
            if (n0 + l_i < Nn) q = __ldg(reinterpret_cast<const float4*>(Q + (int64_t)k * ldq + n0 + l_i));
        }
        *reinterpret_cast<float4*>(&Ps[buf][l_k][l_i]) = p;
        *reinterpret_cast<float4*>(&Qs[buf][l_k][l_i]) = q;
    };
    float acc[4][4], comp[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = comp[a][b] = 0.0f;
    int buf = 0;
    load(0, 0);
    __syncthreads();
    for (int k0 = 0; k0 < K; k0 += kRK) {
        if (k0 + kRK < K) load(buf ^ 1, k0 + kRK);
        float tt[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) tt[a][b] = 0.0f;
#pragma unroll
        for (int kk = 0; kk < kRK; ++kk) {
            const float4 a4 = *reinterpret_cast<const float4*>(&Ps[buf][kk][tr * 4]);
            const float4 b4 = *reinterpret_cast<const float4*>(&Qs[buf][kk][tc * 4]);
            const float av[4] = {a4.x, a4.y, a4.z, a4.w};
            const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) tt[a][b] = fmaf(av[a], bv[b], tt[a][b]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const float y = tt[a][b] - comp[a][b];
                const float s = acc[a][b] + y;
                comp[a][b] = (s - acc[a][b]) - y;
                acc[a][b] = s;
            }
        __syncthreads();
        buf ^= 1;
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int j = n0 + tc * 4 + b;
        if (j >= Nn) continue;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int i = m0 + tr * 4 + a;
            if (i < M) {
                float* c = Cm + (int64_t)j * ldc + i;
                *c = fmaf(alpha, acc[a][b] - comp[a][b], *c);
            }
        }
    }
}

int rank_update(Handle* h, int M, int Nn, int K, const float* P, int64_t ldp, const float* Q, int64_t ldq,
                float alpha, float* Cm, int64_t ldc) {
    if (K <= 0) return L1_OK;
    dim3 grid((Nn + kRT - 1) / kRT, (M + kRT - 1) / kRT);
    rank_update_kernel<<<grid, 256, 0, h->stream>>>(M, Nn, K, P, ldp, Q, ldq, alpha, Cm, ldc);
    L1_LAUNCH_CHECK(h);
    return L1_OK;
}

// ------------------------------------------------------------- buffers
void ur_release(UnrollState* u) {
    for (void* p : u->allocs) cudaFree(p);
    u->allocs.clear();
    u->bytes = 0;
}

template <class T>
int ur_alloc(Handle* h, UnrollState* u, T** p, size_t count) {
    void* q = nullptr;
    const size_t bytes = std::max<size_t>(16, count * sizeof(T));
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_last_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
        return L1_ERR_OOM;
    }
    if (cudaMemsetAsync(q, 0, bytes, h->stream) != cudaSuccess) {
        cudaFree(q);
        return L1_ERR_CUDA;
    }
    u->allocs.push_back(q);
    u->bytes += (int64_t)bytes;
    *p = static_cast<T*>(q);
    return L1_OK;
}

int ur_prepare(Handle* h, int N) {
    UnrollState* u = h->ur;
    if (!u) {
        u = new (std::nothrow) UnrollState();
        if (!u) return L1_ERR_OOM;
        h->ur = u;
    }
    const int K = h->opt.unroll_K, J = h->opt.unroll_J, C = h->opt.ckpt_every;
    if (u->N == N && u->K == K && !u->allocs.empty()) return L1_OK;
    cudaStreamSynchronize(h->stream);
    h->device_bytes -= u->bytes;
    ur_release(u);
    u->N = N;
    u->K = K;
    u->J = J;
    u->C = C;
    u->n_outer = (K + J - 1) / J;
    u->nseg = (K + C - 1) / C;
    u->has_tape = false;
    const size_t mN = (size_t)h->ldm * N, nN = (size_t)h->ldn * N;
    const int steps = std::min(C, K);
    L1_TRY(ur_alloc(h, u, &u->B, mN));
    L1_TRY(ur_alloc(h, u, &u->xi, N));
    L1_TRY(ur_alloc(h, u, &u->thr, N));
    L1_TRY(ur_alloc(h, u, &u->Z, nN));
    L1_TRY(ur_alloc(h, u, &u->W, nN));
    L1_TRY(ur_alloc(h, u, &u->TH, mN));
    L1_TRY(ur_alloc(h, u, &u->R, mN));
    L1_TRY(ur_alloc(h, u, &u->ckZ, nN * u->nseg));
    L1_TRY(ur_alloc(h, u, &u->ckW, nN * u->nseg));
    L1_TRY(ur_alloc(h, u, &u->ckTH, mN * u->nseg));
    L1_TRY(ur_alloc(h, u, &u->Xo, nN * u->n_outer));
    L1_TRY(ur_alloc(h, u, &u->sZ, nN * steps));
    L1_TRY(ur_alloc(h, u, &u->sV, nN * steps));
    L1_TRY(ur_alloc(h, u, &u->sVb, nN * steps));
    L1_TRY(ur_alloc(h, u, &u->sR, mN * steps));
    L1_TRY(ur_alloc(h, u, &u->sQ, mN * steps));
    L1_TRY(ur_alloc(h, u, &u->Xb, nN));
    L1_TRY(ur_alloc(h, u, &u->Wb, nN));
    L1_TRY(ur_alloc(h, u, &u->Zb, nN));
    L1_TRY(ur_alloc(h, u, &u->Tb, mN));
    L1_TRY(ur_alloc(h, u, &u->Cb, mN));
    L1_TRY(ur_alloc(h, u, &u->P, mN));
    L1_TRY(ur_alloc(h, u, &u->gB, mN));
    L1_TRY(ur_alloc(h, u, &u->gA, (size_t)h->ldm * h->n));
    L1_TRY(ur_alloc(h, u, &u->part, (size_t)sweep_row_blocks((int)h->m, N) * N * kPartStride));
    L1_TRY(ur_alloc(h, u, &u->fin, (size_t)2 * N));
    h->device_bytes += u->bytes;
    // FISTA momentum of every step (t restarts at 1 in every block)
    u->mu.assign(K, 0.0);
    double t = 1.0;
    for (int s = 0; s < K; ++s) {
        if (s % J == 0) t = 1.0;
        const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
        u->mu[s] = (t - 1.0) / tn;
        t = tn;
    }
    return L1_OK;
}

inline bool block_end(const UnrollState* u, int s) { return (s % u->J) == u->J - 1 || s == u->K - 1; }

// One forward inner step s.  With a tape slot (>= 0) the step records z, r
// and v there and r lives in the slot.
int ur_step(Handle* h, UnrollState* u, int s, int slot) {
    const int m = (int)h->m, n = (int)h->n, N = u->N;
    const int64_t ldm = h->ldm, ldn = h->ldn;
    const float Linv = (float)(1.0 / h->lipschitz);
    const bool first = (s % u->J) == 0;
    const float* zin = first ? u->W : u->Z;
    float* R = slot >= 0 ? u->sR + (size_t)slot * N * ldm : u->R;
    int np = launch_sweep(h, m, N, n, h->A_rm, ldn, zin, ldn, EpiUrR{R, u->B, u->TH, u->xi, ldm}, nullptr,
                          nullptr);
    if (np < 0) return np;
    EpiUrStep st{zin, u->Z, u->W, nullptr, nullptr, u->thr, Linv, (float)u->mu[s], ldn};
    if (slot >= 0) {
        st.Vtape = u->sV + (size_t)slot * N * ldn;
        st.Ztape = u->sZ + (size_t)slot * N * ldn;
    }
    np = launch_sweep(h, n, N, m, h->A_cm, ldm, R, ldm, st, nullptr, nullptr);
    return np < 0 ? np : L1_OK;
}

// theta += xi (b - A x) at the end of block s / J (x = w)
int ur_theta(Handle* h, UnrollState* u) {
    const int np = launch_sweep(h, (int)h->m, u->N, (int)h->n, h->A_rm, h->ldn, u->W, h->ldn,
                                EpiUrTheta{u->TH, u->B, u->xi, h->ldm}, nullptr, nullptr);
    return np < 0 ? np : L1_OK;
}

}  // namespace

void unroll_free(Handle* h) {
    if (!h->ur) return;
    ur_release(h->ur);
    delete h->ur;
    h->ur = nullptr;
}

int unroll_forward(Handle* h, const float* b, int64_t ldb, int N, float* x, int64_t ldx, l1_result* res) {
    L1_TRY(ur_prepare(h, N));
    UnrollState* u = h->ur;
    cudaStream_t st = h->stream;
    const int m = (int)h->m, n = (int)h->n;
    const int64_t ldm = h->ldm, ldn = h->ldn;
    const size_t nN = (size_t)ldn * N, mN = (size_t)ldm * N;
    u->has_tape = false;
    h->has_tape = false;
    L1_CUDA_TRY(cudaMemcpy2DAsync(u->B, ldm * sizeof(float), b, ldb * sizeof(float), m * sizeof(float), N,
                                  cudaMemcpyDefault, st));
    L1_CUDA_TRY(cudaMemsetAsync(u->Z, 0, nN * sizeof(float), st));
    L1_CUDA_TRY(cudaMemsetAsync(u->W, 0, nN * sizeof(float), st));
    L1_CUDA_TRY(cudaMemsetAsync(u->TH, 0, mN * sizeof(float), st));
    ur_xi_kernel<<<N, 128, 0, st>>>(u->B, ldm, m, N, h->opt.xi0, h->lipschitz, u->xi, u->thr);
    L1_LAUNCH_CHECK(h);
    for (int s = 0; s < u->K; ++s) {
        if (s % u->C == 0) {
            const int k = s / u->C;
            L1_CUDA_TRY(cudaMemcpyAsync(u->ckZ + k * nN, u->Z, nN * sizeof(float), cudaMemcpyDeviceToDevice, st));
            L1_CUDA_TRY(cudaMemcpyAsync(u->ckW + k * nN, u->W, nN * sizeof(float), cudaMemcpyDeviceToDevice, st));
            L1_CUDA_TRY(cudaMemcpyAsync(u->ckTH + k * mN, u->TH, mN * sizeof(float), cudaMemcpyDeviceToDevice, st));
        }
        L1_TRY(ur_step(h, u, s, -1));
        if (block_end(u, s)) {
            const int o = s / u->J;
            L1_CUDA_TRY(cudaMemcpyAsync(u->Xo + o * nN, u->W, nN * sizeof(float), cudaMemcpyDeviceToDevice, st));
            if (o < u->n_outer - 1) L1_TRY(ur_theta(h, u));
        }
    }
    // outputs: x = w, and per column ||b - A x|| and ||x||_1
    const int np = launch_sweep(h, m, N, n, h->A_rm, ldn, u->W, ldn, EpiUrResid{u->B, ldm}, u->part, nullptr);
    if (np < 0) return np;
    ur_final_kernel<<<N, 128, 0, st>>>(u->part, np, N, u->W, ldn, n, u->fin);
    L1_LAUNCH_CHECK(h);
    L1_CUDA_TRY(cudaMemcpy2DAsync(x, ldx * sizeof(float), u->W, ldn * sizeof(float), n * sizeof(float), N,
                                  cudaMemcpyDefault, st));
    std::vector<double> fin(2 * (size_t)N);
    std::vector<float> xi(N);
    L1_CUDA_TRY(cudaMemcpyAsync(fin.data(), u->fin, sizeof(double) * 2 * N, cudaMemcpyDeviceToHost, st));
    L1_CUDA_TRY(cudaMemcpyAsync(xi.data(), u->xi, sizeof(float) * N, cudaMemcpyDeviceToHost, st));
    L1_CUDA_TRY(cudaStreamSynchronize(st));
    for (int j = 0; j < N; ++j) {
        l1_result& r = res[j];
        r = l1_result{};
        const bool finite = std::isfinite(fin[2 * j]) && std::isfinite(fin[2 * j + 1]);
        r.status = finite ? L1_MAX_ITER : L1_NONFINITE;
        r.iters = u->n_outer;
        r.inner_iters = u->K;
        r.label = -1;
        r.sci_label = -1;
        r.rel_change = NAN;
        r.primal_obj = fin[2 * j + 1];
        r.dual_obj = NAN;
        r.gap = NAN;
        r.resid = std::sqrt(fin[2 * j]);
        r.param = xi[j];
    }
    u->has_tape = true;
    h->has_tape = true;
    return L1_OK;
}

int unroll_backward(Handle* h, const float* grad_x, int N, float* grad_b, float* grad_A) {
    UnrollState* u = h->ur;
    if (!u || !u->has_tape) return L1_ERR_NO_TAPE;
    if (N != u->N) return L1_ERR_INVALID_ARG;
    cudaStream_t st = h->stream;
    const int m = (int)h->m, n = (int)h->n;
    const int64_t ldm = h->ldm, ldn = h->ldn;
    const size_t nN = (size_t)ldn * N, mN = (size_t)ldm * N;
    const float Linv = (float)(1.0 / h->lipschitz);
    const dim3 gn((n + 255) / 256, N), gm((m + 255) / 256, N), gmn((std::max(m, n) + 255) / 256, N);

    L1_CUDA_TRY(cudaMemsetAsync(u->Xb, 0, nN * sizeof(float), st));
    L1_CUDA_TRY(cudaMemcpy2DAsync(u->Xb, ldn * sizeof(float), grad_x, (size_t)n * sizeof(float), n * sizeof(float),
                                  N, cudaMemcpyDefault, st));
    L1_CUDA_TRY(cudaMemsetAsync(u->Tb, 0, mN * sizeof(float), st));
    L1_CUDA_TRY(cudaMemsetAsync(u->gB, 0, mN * sizeof(float), st));
    L1_CUDA_TRY(cudaMemsetAsync(u->gA, 0, (size_t)ldm * n * sizeof(float), st));

    for (int seg = u->nseg - 1; seg >= 0; --seg) {
        const int s0 = seg * u->C, s1 = std::min(u->K, s0 + u->C);
        // recompute the segment from its checkpoint, recording the tape
        L1_CUDA_TRY(cudaMemcpyAsync(u->Z, u->ckZ + seg * nN, nN * sizeof(float), cudaMemcpyDeviceToDevice, st));
        L1_CUDA_TRY(cudaMemcpyAsync(u->W, u->ckW + seg * nN, nN * sizeof(float), cudaMemcpyDeviceToDevice, st));
        L1_CUDA_TRY(cudaMemcpyAsync(u->TH, u->ckTH + seg * mN, mN * sizeof(float), cudaMemcpyDeviceToDevice, st));
        for (int s = s0; s < s1; ++s) {
            L1_TRY(ur_step(h, u, s, s - s0));
            if (block_end(u, s) && s + 1 < s1) L1_TRY(ur_theta(h, u));
        }
        // reverse through it
        for (int s = s1 - 1; s >= s0; --s) {
            const int slot = s - s0, o = s / u->J;
            const float mu = (float)u->mu[s];
            float* Vb = u->sVb + (size_t)slot * nN;
            float* Q = u->sQ + (size_t)slot * mN;
            if (block_end(u, s)) {
                if (o < u->n_outer - 1) {
                    // theta_{o+1} = theta_o + xi (b - A x_o)
                    ur_theta_bar_kernel<<<gm, 256, 0, st>>>(m, N, ldm, u->Tb, u->xi, u->P, u->gB);
                    L1_LAUNCH_CHECK(h);
                    const int np = launch_sweep(h, n, N, m, h->A_cm, ldm, u->Tb, ldm,
                                                EpiUrXbTheta{u->Xb, u->xi, ldn}, nullptr, nullptr);
                    if (np < 0) return np;
                    L1_TRY(rank_update(h, m, n, N, u->P, ldm, u->Xo + (size_t)o * nN, ldn, -1.0f, u->gA, ldm));
                }
                ur_block_enter_kernel<<<gmn, 256, 0, st>>>(n, m, N, ldn, ldm, u->Xb, u->Wb, u->Zb, u->Cb);
                L1_LAUNCH_CHECK(h);
            }
            ur_vbar_kernel<<<gn, 256, 0, st>>>(n, N, ldn, u->sV + (size_t)slot * nN, u->thr, mu, u->Wb, u->Zb, Vb);
            L1_LAUNCH_CHECK(h);
            int np = launch_sweep(h, m, N, n, h->A_rm, ldn, Vb, ldn, EpiUrQ{Q, u->Cb, Linv, ldm}, nullptr, nullptr);
            if (np < 0) return np;
            np = launch_sweep(h, n, N, m, h->A_cm, ldm, Q, ldm, EpiUrZb{u->Zb, Vb, Linv, ldn}, nullptr, nullptr);
            if (np < 0) return np;
            if (s % u->J == 0) {
                ur_xbar_kernel<<<gn, 256, 0, st>>>(n, N, ldn, u->Wb, u->Zb, u->Xb);
                L1_LAUNCH_CHECK(h);
                ur_cbar_kernel<<<gm, 256, 0, st>>>(m, N, ldm, u->Cb, u->xi, u->gB, u->Tb);
                L1_LAUNCH_CHECK(h);
            }
        }
        // grad_A += (sum over the segment of r vbar^T - q z^T) / L
        const int Kseg = (s1 - s0) * N;
        L1_TRY(rank_update(h, m, n, Kseg, u->sR, ldm, u->sVb, ldn, Linv, u->gA, ldm));
        L1_TRY(rank_update(h, m, n, Kseg, u->sQ, ldm, u->sZ, ldn, -Linv, u->gA, ldm));
    }
    if (grad_b)
        L1_CUDA_TRY(cudaMemcpy2DAsync(grad_b, (size_t)m * sizeof(float), u->gB, ldm * sizeof(float),
                                      m * sizeof(float), N, cudaMemcpyDefault, st));
    if (grad_A)
        L1_CUDA_TRY(cudaMemcpy2DAsync(grad_A, (size_t)m * sizeof(float), u->gA, ldm * sizeof(float),
                                      m * sizeof(float), n, cudaMemcpyDefault, st));
    L1_CUDA_TRY(cudaStreamSynchronize(st));
    return L1_OK;
}

}  // namespace l1
