// Host driver of l1_solve_batch: per-column state, the PALM / DALM / FISTA
// sweep sequences, finalisation and classification.
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "gemm_simt.cuh"
#include "setup.cuh"
#include "solver_kernels.cuh"

namespace l1 {

namespace {

// l1_result as written by the device (identical layout)
static_assert(sizeof(l1_result) == 6 * 4 + 6 * 8, "l1_result layout");

__global__ void init_cols_kernel(Cols c, const float* B, int64_t ldm, int m, int mode, int solver,
                                 double beta_opt, double xi0_opt, double xi_max, double lambda) {
    __shared__ double sh[4];
    const int j = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) s += fabs((double)B[(int64_t)j * ldm + i]);
    s = block_sum_128(s, sh);
    if (threadIdx.x != 0) return;
    c.b1[j] = s;
    // DALM: beta = ||b||_1 / m unless given (reading of the unspecified beta of §V-B)
    const double beta = beta_opt > 0.0 ? beta_opt : (s > 0.0 ? s / m : 1.0);
    c.beta[j] = (float)beta;
    c.binv[j] = (float)(1.0 / beta);
    // PALM: xi_0 = 2m / ||b||_1 (§V-A); FISTA for QP uses xi = 1/lambda so that
    // the threshold 1/(xi L) is lambda / L (Eq. 18)
    double xi0;
    if (mode == L1_QP_LAMBDA) xi0 = 1.0 / lambda;
    else xi0 = xi0_opt > 0.0 ? xi0_opt : (s > 0.0 ? 2.0 * m / s : 1.0);
    c.xi[j] = (float)xi0;
    c.xicap[j] = (float)(xi0 * xi_max);
    c.mu[j] = 0.0f;
    c.t[j] = 1.0;
    c.active[j] = 1;
    c.status[j] = L1_MAX_ITER;
    c.iters[j] = 0;
    c.inner[j] = 0;
    c.phase[j] = PH_FIRST;
    c.l[j] = 0;
    c.label[j] = -1;
    c.sci_label[j] = -1;
    c.rel[j] = INFINITY;
    c.de2[j] = 0.0;
    c.e2[j] = 0.0;
    c.smax[j] = 0.0f;
    (void)solver;
}

__global__ void pack_results_kernel(Cols c, l1_result* out, int solver, int mode, double Linv,
                                    double lambda) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= c.N) return;
    l1_result r;
    r.status = c.status[j];
    r.iters = c.iters[j];
    r.inner_iters = c.inner[j];
    r.label = c.label[j];
    r.sci_label = c.sci_label[j];
    r.reserved = 0;
    r.rel_change = c.rel[j];
    const double* f = c.fin + (int64_t)j * 8;
    r.primal_obj = f[0];
    r.dual_obj = f[1];
    r.gap = f[2];
    r.resid = f[3];
    if (mode == L1_QP_LAMBDA) r.param = lambda * Linv;
    else if (solver == L1_DALM) r.param = c.beta[j];
    else r.param = 0.0;  // filled from xi0 below
    out[j] = r;
}

__global__ void store_xi0_kernel(Cols c, l1_result* out, const float* xi0) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < c.N) out[j].param = xi0[j];
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// CUDA-event timing of each sweep (l1_options.profile): the events of one
// polling chunk are read back after the chunk's host synchronisation.
struct SweepProf {
    Handle* h;
    bool on;
    int used = 0;
    std::vector<int> kind;
    std::vector<double> flop;
    int reserve(int launches) {
        if (!on) return L1_OK;
        while ((int)h->ev_pool.size() < 2 * launches) {
            cudaEvent_t e;
            L1_CUDA_TRY(cudaEventCreate(&e));
            h->ev_pool.push_back(e);
        }
        return L1_OK;
    }
    void start(int k, double f) {
        if (!on) return;
        cudaEventRecord(h->ev_pool[2 * used], h->stream);
        kind.push_back(k);
        flop.push_back(f);
    }
    void stop() {
        if (!on) return;
        cudaEventRecord(h->ev_pool[2 * used + 1], h->stream);
        ++used;
    }
    void collect() {  // after a synchronisation of h->stream
        for (int i = 0; i < used; ++i) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, h->ev_pool[2 * i], h->ev_pool[2 * i + 1]) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            h->sweep_ms[kind[i]] += ms;
            h->sweep_flop[kind[i]] += flop[i];
            h->sweep_launches[kind[i]] += 1;
        }
        used = 0;
        kind.clear();
        flop.clear();
    }
};

static int ensure_workspace(Handle* h, int N) {
    Workspace& w = h->ws;
    if (w.cap_N >= N) return L1_OK;
    // release the old panels (they are recorded in h->allocations)
    auto release = [&](void* p) {
        if (!p) return;
        cudaFree(p);
        auto it = std::find(h->allocations.begin(), h->allocations.end(), p);
        if (it != h->allocations.end()) h->allocations.erase(it);
    };
    release(w.B); release(w.Wx); release(w.We); release(w.Ux); release(w.Ue); release(w.R);
    release(w.Y); release(w.X); release(w.Cc); release(w.part); release(w.colstat);
    release(w.colf); release(w.coli); release(w.active_count); release(w.resid2);
    release(w.classl1); release(w.class_off);
    if (w.h_active) { cudaFreeHost(w.h_active); w.h_active = nullptr; }
    w = Workspace{};
    const int64_t ldm = h->ldm, ldn = h->ldn;
    const int m = (int)h->m, n = (int)h->n;
    L1_TRY(dev_alloc_t(h, &w.B, ldm * N));
    L1_TRY(dev_alloc_t(h, &w.Wx, ldn * N));
    L1_TRY(dev_alloc_t(h, &w.We, ldm * N));
    L1_TRY(dev_alloc_t(h, &w.Ux, ldn * N));
    L1_TRY(dev_alloc_t(h, &w.Ue, ldm * N));
    L1_TRY(dev_alloc_t(h, &w.R, ldm * N));
    L1_TRY(dev_alloc_t(h, &w.Y, ldm * N));
    L1_TRY(dev_alloc_t(h, &w.X, ldn * N));
    L1_TRY(dev_alloc_t(h, &w.Cc, ldm * N));
    const int np = std::max(std::max(sweep_row_blocks(m, N), sweep_row_blocks(n, N)),
                            std::max(sweep_row_blocks(m, 1), sweep_row_blocks(n, 1)));
    w.part_slots = (size_t)np;
    // two partial buffers: one for sweeps over the m rows, one over the n rows
    L1_TRY(dev_alloc_t(h, &w.part, 2 * (size_t)np * N * kPartStride));
    L1_TRY(dev_alloc_t(h, &w.colstat, (size_t)N * 16));
    L1_TRY(dev_alloc_t(h, &w.colf, (size_t)N * 8));
    L1_TRY(dev_alloc_t(h, &w.coli, (size_t)N * 16));
    L1_TRY(dev_alloc_t(h, &w.active_count, 1));
    if (cudaMallocHost(&w.h_active, sizeof(int32_t)) != cudaSuccess) return L1_ERR_OOM;
    const int C = (int)h->class_offsets.size() - 1;
    if (C > 0) {
        L1_TRY(dev_alloc_t(h, &w.resid2, (size_t)C * N));
        L1_TRY(dev_alloc_t(h, &w.classl1, (size_t)C * N));
        L1_TRY(dev_alloc_t(h, &w.class_off, (size_t)C + 1));
        L1_CUDA_TRY(cudaMemcpy(w.class_off, h->class_offsets.data(), sizeof(int32_t) * (C + 1),
                               cudaMemcpyHostToDevice));
    }
    w.cap_N = N;
    return L1_OK;
}

static Cols make_cols(Handle* h, int N) {
    Workspace& w = h->ws;
    Cols c{};
    c.N = N;
    const int64_t cap = w.cap_N;
    c.beta = w.colf + 0 * cap;
    c.binv = w.colf + 1 * cap;
    c.xi = w.colf + 2 * cap;
    c.xicap = w.colf + 3 * cap;
    c.mu = w.colf + 4 * cap;
    c.smax = w.colf + 5 * cap;
    c.active = w.coli + 0 * cap;
    c.status = w.coli + 1 * cap;
    c.iters = w.coli + 2 * cap;
    c.inner = w.coli + 3 * cap;
    c.phase = w.coli + 4 * cap;
    c.l = w.coli + 5 * cap;
    c.label = w.coli + 6 * cap;
    c.sci_label = w.coli + 7 * cap;
    c.t = w.colstat + 0 * cap;
    c.rel = w.colstat + 1 * cap;
    c.de2 = w.colstat + 2 * cap;
    c.e2 = w.colstat + 3 * cap;
    c.b1 = w.colstat + 4 * cap;
    c.fin = w.colstat + 8 * cap;  // [N][8]
    return c;
}

int solve_batch(Handle* h, const float* b, int64_t ldb, int N, double tol, int max_iter,
                float* x, int64_t ldx, float* y, int64_t ldy, l1_result* res) {
    L1_TRY(ensure_workspace(h, N));
    Workspace& w = h->ws;
    cudaStream_t s = h->stream;
    const int m = (int)h->m, n = (int)h->n;
    const int64_t ldm = h->ldm, ldn = h->ldn;
    const int mode = h->mode;
    const int solver = (mode == L1_QP_LAMBDA) ? L1_PALM : h->opt.solver;
    const bool cab = mode == L1_CAB;
    const l1_options& o = h->opt;
    Cols c = make_cols(h, N);
    double* part_m = w.part;
    double* part_n = w.part + w.part_slots * (size_t)N * kPartStride;

    // ---- inputs and initial state
    L1_CUDA_TRY(cudaMemcpy2DAsync(w.B, ldm * sizeof(float), b, ldb * sizeof(float), m * sizeof(float),
                                  N, cudaMemcpyDefault, s));
    const size_t pm = sizeof(float) * ldm * N, pn = sizeof(float) * ldn * N;
    L1_CUDA_TRY(cudaMemsetAsync(w.Wx, 0, pn, s));
    L1_CUDA_TRY(cudaMemsetAsync(w.Ux, 0, pn, s));
    L1_CUDA_TRY(cudaMemsetAsync(w.X, 0, pn, s));
    L1_CUDA_TRY(cudaMemsetAsync(w.Ue, 0, pm, s));
    L1_CUDA_TRY(cudaMemsetAsync(w.Y, 0, pm, s));
    L1_CUDA_TRY(cudaMemsetAsync(w.R, 0, pm, s));
    L1_CUDA_TRY(cudaMemsetAsync(w.Cc, 0, pm, s));
    if (solver == L1_PALM && cab) {
        // Algorithm 1 input: e_1 = b
        L1_CUDA_TRY(cudaMemcpyAsync(w.We, w.B, pm, cudaMemcpyDeviceToDevice, s));
    } else {
        L1_CUDA_TRY(cudaMemsetAsync(w.We, 0, pm, s));
    }
    const double xi_max = o.xi_max > 0.0 ? o.xi_max : 1e4;
    init_cols_kernel<<<N, 128, 0, s>>>(c, w.B, ldm, m, mode, solver, o.beta, o.xi0, xi_max, o.lambda);
    L1_LAUNCH_CHECK(h);

    const int check_every = o.check_every > 0 ? o.check_every : 16;
    int done_iters = 0;
    SweepProf prof{h, o.profile != 0};
    L1_TRY(prof.reserve(3 * check_every));
    double n_act = N;  // columns active at the last poll (algorithmic FLOP count)
    if (solver == L1_DALM) {
        // Algorithm 2: three sweeps per iteration
        while (true) {
            for (int r = 0; r < check_every; ++r) {
                prof.start(0, 2.0 * m * n * n_act);
                int rc = launch_sweep(h, m, N, n, h->A_rm, ldn, w.Ux, ldn,
                                      EpiDalmRhs{w.R, w.Ue, w.B, c.binv, c.active, ldm, cab ? 1 : 0},
                                      part_m, c.active);
                prof.stop();
                if (rc < 0) return rc;
                prof.start(1, 2.0 * m * m * n_act);
                const int np_e = launch_sweep(h, m, N, m, h->F, ldm, w.R, ldm,
                                              EpiDalmY{w.Y, w.We, w.Ue, c.beta, c.binv, c.active, ldm, cab ? 1 : 0},
                                              part_m, c.active);
                prof.stop();
                if (np_e < 0) return np_e;
                prof.start(2, 2.0 * m * n * n_act);
                const int np_x = launch_sweep(h, n, N, m, h->A_cm, ldm, w.Y, ldm,
                                              EpiDalmS{w.Wx, w.Ux, c.beta, c.binv, c.active, ldn}, part_n,
                                              c.active);
                prof.stop();
                if (np_x < 0) return np_x;
                ctrl_dalm_kernel<<<N, 128, 0, s>>>(c, cab ? part_m : nullptr, np_e, part_n, np_x, tol, max_iter);
                L1_LAUNCH_CHECK(h);
            }
            done_iters += check_every;
            count_active_kernel<<<1, 1024, 0, s>>>(c.active, N, w.active_count);
            L1_LAUNCH_CHECK(h);
            L1_CUDA_TRY(cudaMemcpyAsync(w.h_active, w.active_count, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            L1_CUDA_TRY(cudaStreamSynchronize(s));
            prof.collect();
            n_act = *w.h_active;
            if (*w.h_active == 0 || done_iters >= max_iter) break;
        }
    } else {
        // Algorithm 1 / Eq. 18: two sweeps per inner FISTA step
        PalmParams p;
        p.mode = mode;
        p.growth = (mode == L1_CAB || mode == L1_QP_LAMBDA) ? 1.0f
                   : (float)(o.xi_growth > 0.0 ? o.xi_growth : 1.2);
        p.Linv = (float)(1.0 / h->lipschitz);
        const int inner_max = o.inner_max > 0 ? o.inner_max : 50;
        const double inner_tol = o.inner_tol > 0.0 ? o.inner_tol : 0.1 * tol;
        const int64_t step_cap = (mode == L1_QP_LAMBDA) ? (int64_t)max_iter : (int64_t)max_iter * inner_max;
        int64_t steps = 0;
        while (true) {
            for (int r = 0; r < check_every; ++r) {
                prof.start(0, 2.0 * m * n * n_act);
                const int np_A = launch_sweep(h, m, N, n, h->A_rm, ldn, w.Ux, ldn,
                                              EpiPalmA{w.R, w.Cc, w.We, w.Y, w.B, c, p, ldm}, part_m, c.active);
                prof.stop();
                if (np_A < 0) return np_A;
                prof.start(2, 2.0 * m * n * n_act);
                const int np_At = launch_sweep(h, n, N, m, h->A_cm, ldm, w.R, ldm,
                                               EpiPalmAt{w.Wx, w.Ux, w.X, c, p, ldn}, part_n, c.active);
                prof.stop();
                if (np_At < 0) return np_At;
                ctrl_palm_kernel<<<N, 128, 0, s>>>(c, p, part_m, np_A, part_n, np_At, w.Wx, w.X, w.Ux, ldn, n,
                                                   tol, inner_tol, inner_max, max_iter);
                L1_LAUNCH_CHECK(h);
            }
            steps += check_every;
            count_active_kernel<<<1, 1024, 0, s>>>(c.active, N, w.active_count);
            L1_LAUNCH_CHECK(h);
            L1_CUDA_TRY(cudaMemcpyAsync(w.h_active, w.active_count, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            L1_CUDA_TRY(cudaStreamSynchronize(s));
            prof.collect();
            n_act = *w.h_active;
            if (*w.h_active == 0 || steps >= step_cap) break;
        }
    }
    (void)done_iters;

    // ---- finalisation: objective, dual point, gap, residual
    L1_CUDA_TRY(cudaMemsetAsync(c.smax, 0, sizeof(float) * N, s));
    const float* E = (cab || mode == L1_P1_2) ? w.We : nullptr;
    const float* xi_fin = (solver == L1_PALM && mode != L1_QP_LAMBDA) ? c.xi : nullptr;
    const int np_F1 = launch_sweep(h, m, N, n, h->A_rm, ldn, w.Wx, ldn,
                                   EpiFinalA{w.R, w.Y, E, w.B, xi_fin, c.smax, ldm, mode}, part_m, nullptr);
    if (np_F1 < 0) return np_F1;
    const int np_F2 = launch_sweep(h, n, N, m, h->A_cm, ldm, (mode == L1_QP_LAMBDA) ? w.R : w.Y, ldm,
                                   EpiFinalAt{w.Wx, c.smax, ldn}, part_n, nullptr);
    if (np_F2 < 0) return np_F2;
    final_metrics_kernel<<<N, 128, 0, s>>>(c, part_m, np_F1, part_n, np_F2, mode, o.lambda);
    L1_LAUNCH_CHECK(h);

    // ---- classification (CAB with classes)
    const int C = (int)h->class_offsets.size() - 1;
    if (cab && C > 0) {
        classify_resid_kernel<<<dim3(C, N), 128, 0, s>>>(h->A_rm, ldn, m, w.class_off, w.B, w.We, w.Wx, ldm,
                                                          ldn, N, w.resid2, w.classl1);
        L1_LAUNCH_CHECK(h);
        classify_argmin_kernel<<<(N + 127) / 128, 128, 0, s>>>(w.resid2, w.classl1, C, N, c.label, c.sci_label);
        L1_LAUNCH_CHECK(h);
    }

    // ---- outputs
    l1_result* res_dev = reinterpret_cast<l1_result*>(w.R);  // R is free now; N*72 B <= ldm*N*4
    static_assert(sizeof(l1_result) <= 128, "result size");
    if ((size_t)N * sizeof(l1_result) > sizeof(float) * (size_t)ldm * N) return L1_ERR_INVALID_ARG;
    pack_results_kernel<<<(N + 127) / 128, 128, 0, s>>>(c, res_dev, solver, mode, 1.0 / h->lipschitz, o.lambda);
    L1_LAUNCH_CHECK(h);
    if (solver == L1_PALM && mode != L1_QP_LAMBDA) {
        // report xi_0 (the first outer step's penalty); xicap / xi_max = xi_0
        // is recomputed on the device to avoid keeping another array
        store_xi0_kernel<<<(N + 127) / 128, 128, 0, s>>>(c, res_dev, c.xicap);
        L1_LAUNCH_CHECK(h);
    }
    L1_CUDA_TRY(cudaMemcpy2DAsync(x, ldx * sizeof(float), w.Wx, ldn * sizeof(float), n * sizeof(float), N,
                                  cudaMemcpyDefault, s));
    if (cab) {
        L1_CUDA_TRY(cudaMemcpy2DAsync(x + n, ldx * sizeof(float), w.We, ldm * sizeof(float), m * sizeof(float),
                                      N, cudaMemcpyDefault, s));
    }
    if (y) {
        L1_CUDA_TRY(cudaMemcpy2DAsync(y, ldy * sizeof(float), w.Y, ldm * sizeof(float), m * sizeof(float), N,
                                      cudaMemcpyDefault, s));
    }
    L1_CUDA_TRY(cudaMemcpyAsync(res, res_dev, sizeof(l1_result) * N, cudaMemcpyDefault, s));
    L1_CUDA_TRY(cudaStreamSynchronize(s));
    if (solver == L1_PALM && mode != L1_QP_LAMBDA)
        for (int j = 0; j < N; ++j) res[j].param /= xi_max;
    return L1_OK;
}

}  // namespace l1
