// Uneven batches of independent (QP_lambda) problems (l1_setup_group): FISTA
// (Eq. 18, §IV-A) for thousands of dictionaries of different sizes in one
// persistent cooperative launch.
//
// Work.  The dictionaries are stored column-major (FP32 or BF16) in one
// allocation.  A work unit is (instance, tile of consecutive columns) sized so
// the tile fits in shared memory (<= 64 KB).  One FISTA step over a unit
//   1. stages r = b - A z (the instance's residual, from the accumulator of
//      the previous step) in shared memory,
//   2. reads its A tile from HBM once into shared memory while forming
//      g_J = A_J^T r (one warp per column),
//   3. updates x_J = soft(z_J + g_J/L, lambda/L), z_J = x_J + mu (x_J - x_J_old)
//      and the per-instance sums ||dx||^2, ||x_old||^2,
//   4. adds A_J z_J to the next step's accumulator from the tile in shared
//      memory (red.global.add),
// so every element of every active dictionary is read from HBM once per step.
// After the pass a bounded grid barrier, a per-instance finalisation (stopping
// rule of §VI-C, FISTA momentum), another barrier, and a rebuild of the
// active-instance work list (converged instances drop out: compaction).
// The same kernel runs the batched power iteration for L = ||A_i||_2^2 and
// the final pass that forms A x for the objective.
#include <algorithm>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "common.cuh"

namespace l1 {

enum GroupMode : int { GM_FISTA = 0, GM_POWER_INIT = 1, GM_POWER = 2, GM_FINAL = 3 };

constexpr int kGThreads = 256;
constexpr int kGWarps = kGThreads / 32;
constexpr int kGMaxM = 8192;               // rows of r staged in shared memory
constexpr int kGTileBytes = 64 * 1024;     // A tile in shared memory
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

__device__ __forceinline__ float load_a(const GArgs& g, int64_t idx) {
    if (g.bf16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(g.A)[idx]);
    return reinterpret_cast<const float*>(g.A)[idx];
}

// one work unit: columns col0 .. col0+nc-1 of instance i
__device__ void group_unit(const GArgs& g, int i, int col0, int nc, int cur, float* r_s, uint8_t* tile_raw,
                           float* zj_s, double* red_s) {
    const int m = g.m[i], ld = g.ld[i];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float* racc_cur = cur ? g.racc1 : g.racc0;
    float* racc_next = cur ? g.racc0 : g.racc1;
    const int64_t bo = g.boff[i], xo = g.xoff[i] + col0;
    const int64_t a0 = g.aoff[i] + (int64_t)col0 * ld;
    const bool dots = g.mode == GM_FISTA || g.mode == GM_POWER;
    float* tile_f = reinterpret_cast<float*>(tile_raw);
    __nv_bfloat16* tile_h = reinterpret_cast<__nv_bfloat16*>(tile_raw);

    // 1. residual (FISTA: b - A z) or u = A v (power) into shared memory
    if (dots) {
        for (int r = threadIdx.x; r < m; r += blockDim.x) {
            const float acc = racc_cur[bo + r];
            r_s[r] = g.mode == GM_FISTA ? g.b[bo + r] - acc : acc;
        }
    }
    __syncthreads();
    // 2-3. stage the tile; per column the dot product and the update
    double d2 = 0.0, w2 = 0.0;
    for (int c = warp; c < nc; c += kGWarps) {
        const int64_t colbase = a0 + (int64_t)c * ld;
        float dot = 0.0f;
        if (g.bf16) {
            for (int r = lane; r < m; r += 32) {
                const __nv_bfloat16 v = reinterpret_cast<const __nv_bfloat16*>(g.A)[colbase + r];
                tile_h[c * m + r] = v;
                if (dots) dot = fmaf(__bfloat162float(v), r_s[r], dot);
            }
        } else {
            for (int r = lane; r < m; r += 32) {
                const float v = reinterpret_cast<const float*>(g.A)[colbase + r];
                tile_f[c * m + r] = v;
                if (dots) dot = fmaf(v, r_s[r], dot);
            }
        }
        dot = warp_sum_f(dot);
        if (lane == 0) {
            const int64_t j = xo + c;
            float zn;
            if (g.mode == GM_FISTA) {
                // Eq. 18: x = soft(z + A^T(b - A z)/L, lambda/L), z' = x + mu (x - x_old)
                const float Li = 1.0f / g.L[i];
                const float xo_ = g.x[j];
                const float xn = soft_g(fmaf(dot, Li, g.z[j]), g.lambda * Li);
                zn = fmaf(g.mu[i], xn - xo_, xn);
                g.x[j] = xn;
                g.z[j] = zn;
                const float dx = xn - xo_;
                d2 += (double)dx * dx;
                w2 += (double)xo_ * xo_;
            } else if (g.mode == GM_POWER) {
                zn = dot * g.cscale[i];  // v' = A^T A v scaled to about unit norm
                g.x[j] = zn;
                d2 += (double)zn * zn;
            } else if (g.mode == GM_POWER_INIT) {
                zn = rsqrtf((float)g.n[i]);
                g.x[j] = zn;
                d2 += (double)zn * zn;
            } else {  // GM_FINAL: A x
                zn = g.x[j];
                w2 += fabs((double)zn);
            }
            zj_s[c] = zn;
        }
    }
    __syncthreads();
    // 4. partial product A_J z_J into the next accumulator
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
        float acc = 0.0f;
        if (g.bf16) {
            for (int c = 0; c < nc; ++c) acc = fmaf(__bfloat162float(tile_h[c * m + r]), zj_s[c], acc);
        } else {
            for (int c = 0; c < nc; ++c) acc = fmaf(tile_f[c * m + r], zj_s[c], acc);
        }
        atomicAdd(&racc_next[bo + r], acc);
    }
    // per-instance sums (lane 0 of each warp holds its columns' terms)
    if (lane == 0) {
        red_s[warp] = d2;
        red_s[kGWarps + warp] = w2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s1 = 0.0, s2 = 0.0;
        for (int w = 0; w < kGWarps; ++w) {
            s1 += red_s[w];
            s2 += red_s[kGWarps + w];
        }
        if (g.mode == GM_FISTA) {
            atomicAdd(&g.d2[i], s1);
            atomicAdd(&g.w2[i], s2);
        } else if (g.mode == GM_FINAL) {
            atomicAdd(&g.w2[i], s2);
        } else {
            atomicAdd(&g.vv[i], s1);
        }
    }
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

__global__ void __launch_bounds__(kGThreads) group_kernel(GArgs g) {
    extern __shared__ __align__(16) uint8_t gsm[];
    float* r_s = reinterpret_cast<float*>(gsm);                                   // kGMaxM floats
    uint8_t* tile = gsm + kGMaxM * sizeof(float);                                  // kGTileBytes
    float* zj_s = reinterpret_cast<float*>(tile + kGTileBytes);                    // 256 floats
    double* red_s = reinterpret_cast<double*>(zj_s + 256);                         // 2 * kGWarps
    int64_t* scan_s = reinterpret_cast<int64_t*>(red_s + 2 * kGWarps);             // kGThreads
    __shared__ int abort_s;
    if (threadIdx.x == 0) abort_s = 0;
    __syncthreads();
    volatile int* abort = &abort_s;
    const int nwarps_grid = gridDim.x * kGWarps;
    const int gwarp = blockIdx.x * kGWarps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;

    for (int step = 0; step < g.max_steps; ++step) {
        const int cur = step & 1;
        const int nact = *(volatile int32_t*)g.nact;
        if (nact == 0) break;
        const int64_t total = g.upref[nact];
        // ---- pass over the active units
        for (int64_t u = blockIdx.x; u < total; u += gridDim.x) {
            int lo = 0, hi = nact;  // last k with upref[k] <= u
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (g.upref[mid] <= u) lo = mid;
                else hi = mid;
            }
            const int i = g.act[lo];
            const int64_t local = u - g.upref[lo];
            const int col0 = (int)(local * g.ucols[i]);
            const int nc = min(g.ucols[i], g.n[i] - col0);
            group_unit(g, i, col0, nc, cur, r_s, tile, zj_s, red_s);
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

__global__ void group_init_kernel(GArgs g, int mode) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.count) return;
    g.active[i] = 1;
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

static int run_group(Handle* h, int mode, int max_steps, double tol) {
    GroupState* G = h->grp;
    cudaStream_t s = h->stream;
    GArgs a = make_args(G);
    a.mode = mode;
    a.max_steps = max_steps;
    a.tol = tol;
    group_init_kernel<<<(unsigned)((G->count + 255) / 256), 256, 0, s>>>(a, mode);
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
        set_last_error("group kernel: bounded grid barrier expired");
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
    L1_TRY(run_group(h, GM_POWER_INIT, 1000, 1e-6));
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
    return group_power(h, 0, G->count);
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
        int uc = kGTileBytes / (esize * mi);
        uc = std::max(1, std::min(uc, 256));
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
    G->smem = kGMaxM * (int)sizeof(float) + kGTileBytes + 256 * (int)sizeof(float) + 2 * kGWarps * 8 +
              kGThreads * 8;
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
