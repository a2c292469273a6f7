// Host driver of l1_solve_batch: per-column state, the PALM / DALM / FISTA
// sweep sequences, convergence masking and compaction, finalisation and
// classification.
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "gemm_simt.cuh"
#include "setup.cuh"
#include "solver_kernels.cuh"
#include "tc16.cuh"

namespace l1 {

namespace {

static_assert(sizeof(l1_result) == 6 * 4 + 6 * 8, "l1_result layout");

__global__ void init_cols_kernel(Cols c, const float* B, int64_t ldm, int m, int mode,
                                 double beta_opt, double xi0_opt, double xi_max, double lambda,
                                 double lambda0) {
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
    // the threshold 1/(xi L) is lambda / L (Eq. 18); with continuation (R17)
    // xi starts at 1/lambda_0 and grows to its cap 1/lambda
    double xi0;
    if (mode == L1_QP_LAMBDA) xi0 = 1.0 / (lambda0 > lambda ? lambda0 : lambda);
    else xi0 = xi0_opt > 0.0 ? xi0_opt : (s > 0.0 ? 2.0 * m / s : 1.0);
    c.xi[j] = (float)xi0;
    c.xicap[j] = mode == L1_QP_LAMBDA ? (float)(1.0 / lambda) : (float)(xi0 * xi_max);
    c.mu[j] = 0.0f;
    c.t[j] = 1.0;
    c.active[j] = 1;
    c.status[j] = L1_MAX_ITER;
    c.iters[j] = 0;
    c.inner[j] = 0;
    c.phase[j] = PH_FIRST;
    c.l[j] = 0;
    c.rel[j] = INFINITY;
    c.de2[j] = 0.0;
    c.e2[j] = 0.0;
    c.orig[j] = j;
}

struct HomeRes {
    int32_t* status;
    int32_t* iters;
    int32_t* inner;
    int32_t* label;
    int32_t* sci_label;
    double* rel;
    double* param;
    double* fin;  // [N][8]
    float* xi;
    float* smax;
};

__global__ void pack_results_kernel(HomeRes hr, int N, l1_result* out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    l1_result r;
    r.status = hr.status[j];
    r.iters = hr.iters[j];
    r.inner_iters = hr.inner[j];
    r.label = hr.label[j];
    r.sci_label = hr.sci_label[j];
    r.reserved = 0;
    r.rel_change = hr.rel[j];
    const double* f = hr.fin + (int64_t)j * 8;
    r.primal_obj = f[0];
    r.dual_obj = f[1];
    r.gap = f[2];
    r.resid = f[3];
    r.param = hr.param[j];
    out[j] = r;
}

__global__ void fill_i32_kernel(int32_t* p, int n, int32_t v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// Refinement restart: keep the first phase's iteration count apart, and leave
// columns that went non-finite retired.
__global__ void refine_restart_kernel(Cols c, const int32_t* home_status, const int32_t* home_iters,
                                      int32_t* iters1, int N) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    iters1[j] = home_iters[j];
    if (home_status[j] == L1_NONFINITE) {
        c.active[j] = 0;
        c.status[j] = L1_NONFINITE;
    }
}

__global__ void add_iters_kernel(int32_t* iters, int32_t* inner, const int32_t* iters1, int N) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    iters[j] += iters1[j];
    inner[j] += iters1[j];
}

__global__ void set_param_kernel(double* param, int n, double v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) param[i] = v;
}

// CUDA-event timing of each sweep (l1_options.profile): the events of one
// polling chunk are read back after the chunk's host synchronisation.
struct SweepProf {
    Handle* h;
    bool on;
    bool capturing = false;  // the chunk is being captured into a graph
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
    // Inside a capture, external records become event nodes of the graph (a
    // plain record there only marks a dependency); outside, plain records.
    void record(cudaEvent_t e) {
        if (capturing) cudaEventRecordWithFlags(e, h->stream, cudaEventRecordExternal);
        else cudaEventRecord(e, h->stream);
    }
    void start(int k, double f) {
        if (!on) return;
        record(h->ev_pool[2 * used]);
        kind.push_back(k);
        flop.push_back(f);
    }
    void stop() {
        if (!on) return;
        record(h->ev_pool[2 * used + 1]);
        ++used;
    }
    // a replayed graph records the events of the chunk it was captured from
    void adopt(const std::vector<int>& k, const std::vector<double>& f) {
        if (!on) return;
        kind = k;
        flop = f;
        used = (int)k.size();
    }
    void reset() {
        used = 0;
        kind.clear();
        flop.clear();
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

}  // namespace

// CUDA graphs of the polling chunks: the launches of check_every iterations
// depend only on the panel set, the number of slots, the phase and the
// stopping parameters, so each such chunk is captured once and replayed.
struct GraphEntry {
    int q, N, phase, solver, max_iter;
    double tol;
    cudaGraphExec_t exec;
    int64_t nlaunch;
    std::vector<int> kinds;
    std::vector<double> flops;
};

struct GraphCache {
    std::vector<GraphEntry> entries;
};

void graph_cache_clear(Handle* h) {
    if (!h->graphs) return;
    for (GraphEntry& e : h->graphs->entries) cudaGraphExecDestroy(e.exec);
    delete h->graphs;
    h->graphs = nullptr;
}

static GraphEntry* graph_find(Handle* h, int q, int N, int phase, int solver, double tol, int max_iter) {
    if (!h->graphs) return nullptr;
    for (GraphEntry& e : h->graphs->entries)
        if (e.q == q && e.N == N && e.phase == phase && e.solver == solver && e.tol == tol && e.max_iter == max_iter)
            return &e;
    return nullptr;
}

// largest split-K scratch a sweep of this handle needs for up to N columns
static size_t splitk_need(const Handle* h, int N) {
    const int m = (int)h->m, n = (int)h->n;
    const int shapes[3][2] = {{m, n}, {m, m}, {n, m}};  // (M, K) of A u, F r, A^T y
    size_t need = 0;
    for (const auto& sh : shapes)
        for (int Nn = 9; Nn <= N; ++Nn) {
            const int S = splitk_slices(h, sh[0], Nn, sh[1]);
            if (S > 1) need = std::max(need, (size_t)S * sh[0] * (size_t)(((int64_t)Nn + 3) & ~int64_t(3)));
        }
    return need;
}

// A u (rm) or A^T y (cm) sweep on the low-precision copy of A
template <class E>
static int sweep_lowp(Handle* h, bool rm, int M, int N, int K, const float* X, int64_t ldx, const E& e,
                      double* part, const int32_t* active) {
    const int64_t lda = rm ? h->ldn : h->ldm;
    const void* A = rm ? h->A_rm_lp : h->A_cm_lp;
    if (h->opt.precision == L1_A_BF16)
        return launch_sweep(h, M, N, K, static_cast<const __nv_bfloat16*>(A), lda, X, ldx, e, part, active);
    const float* sc = rm ? h->A_rm_scale : h->A_cm_scale;
    return launch_sweep(h, M, N, K, static_cast<const fp8e4m3*>(A), lda, X, ldx, EpiRowScale<E>{sc, e}, part,
                        active);
}

static int ensure_workspace(Handle* h, int N) {
    Workspace& w = h->ws;
    if (w.cap_N >= N) return L1_OK;
    // release the old buffers (recorded in h->allocations)
    std::vector<void*> old;
    for (int q = 0; q < 2; ++q) {
        PanelSet& p = w.ps[q];
        old.insert(old.end(), {p.B, p.Wx, p.We, p.Ux, p.Ue, p.Y, p.X, p.Cc, p.colf, p.coli, p.cold});
    }
    old.insert(old.end(), {w.R, w.hB, w.hWx, w.hWe, w.hY, w.hUx, w.hUe, w.hcoli, w.hcold, w.hcolf, w.part, w.newpos,
                           w.count, w.resid2, w.classl1, w.class_off});
    for (int k = 0; k < 3; ++k) old.insert(old.end(), {w.Vh[k], w.Dh[k], w.Yh[k]});
    for (void* p : old) dev_free(h, p);
    if (w.h_count) cudaFreeHost(w.h_count);
    w = Workspace{};
    graph_cache_clear(h);  // the captured launches point into the old buffers
    const int64_t ldm = h->ldm, ldn = h->ldn;
    const int m = (int)h->m, n = (int)h->n;
    for (int q = 0; q < 2; ++q) {
        PanelSet& p = w.ps[q];
        L1_TRY(dev_alloc_t(h, &p.B, ldm * N));
        L1_TRY(dev_alloc_t(h, &p.Wx, ldn * N));
        L1_TRY(dev_alloc_t(h, &p.We, ldm * N));
        L1_TRY(dev_alloc_t(h, &p.Ux, ldn * N));
        L1_TRY(dev_alloc_t(h, &p.Ue, ldm * N));
        L1_TRY(dev_alloc_t(h, &p.Y, ldm * N));
        L1_TRY(dev_alloc_t(h, &p.X, ldn * N));
        L1_TRY(dev_alloc_t(h, &p.Cc, ldm * N));
        L1_TRY(dev_alloc_t(h, &p.colf, (size_t)8 * N));
        L1_TRY(dev_alloc_t(h, &p.coli, (size_t)16 * N));
        L1_TRY(dev_alloc_t(h, &p.cold, (size_t)8 * N));
    }
    L1_TRY(dev_alloc_t(h, &w.R, ldm * N));
    if (h->use_tc) {
        for (int k = 0; k < 3; ++k) {
            L1_TRY(dev_alloc_t(h, &w.Vh[k], ldn * N));
            L1_TRY(dev_alloc_t(h, &w.Dh[k], ldm * N));
            L1_TRY(dev_alloc_t(h, &w.Yh[k], ldm * N));
        }
    }
    L1_TRY(dev_alloc_t(h, &w.hB, ldm * N));
    L1_TRY(dev_alloc_t(h, &w.hWx, ldn * N));
    L1_TRY(dev_alloc_t(h, &w.hWe, ldm * N));
    L1_TRY(dev_alloc_t(h, &w.hY, ldm * N));
    if (h->opt.precision != L1_A_FP32 || h->use_tc) {
        L1_TRY(dev_alloc_t(h, &w.hUx, ldn * N));
        L1_TRY(dev_alloc_t(h, &w.hUe, ldm * N));
    }
    L1_TRY(dev_alloc_t(h, &w.hcoli, (size_t)8 * N));
    L1_TRY(dev_alloc_t(h, &w.hcold, (size_t)10 * N));
    L1_TRY(dev_alloc_t(h, &w.hcolf, (size_t)2 * N));
    const int np = std::max(std::max(sweep_row_blocks(m, N), sweep_row_blocks(n, N)),
                            std::max(sweep_row_blocks(m, 1), sweep_row_blocks(n, 1)));
    w.part_slots = (size_t)np;
    L1_TRY(dev_alloc_t(h, &w.part, 2 * (size_t)np * N * kPartStride));
    {
        // sized now so that no sweep allocates while a chunk is captured
        const size_t need = splitk_need(h, N);
        if (need > h->splitk_floats) {
            // the graphs that could point at the old scratch are gone (above)
            dev_free(h, h->splitk);
            h->splitk = nullptr;
            h->splitk_floats = 0;
            L1_TRY(dev_alloc_t(h, &h->splitk, need));
            h->splitk_floats = need;
        }
    }
    if (h->use_tc && h->tc_wk) {
        // the tensor-core sweeps' FP32 tile sums (split-K slices, deferred
        // epilogues): every output tile of the widest sweep at this width
        const size_t tm = (size_t)(std::max(m, n) + 127) / 128, tn = (size_t)(N + 127) / 128;
        const size_t need = std::max((size_t)tc16::kSplitWaves * (h->sms > 0 ? h->sms : 152), tm * tn) * 128 * 128;
        if (need > h->tc_wk_elems) {
            dev_free(h, h->tc_wk);
            h->tc_wk = nullptr;
            h->tc_wk_elems = 0;
            L1_TRY(dev_alloc_t(h, &h->tc_wk, need));
            h->tc_wk_elems = need;
        }
    }
    L1_TRY(dev_alloc_t(h, &w.newpos, (size_t)N));
    L1_TRY(dev_alloc_t(h, &w.count, 1));
    if (cudaMallocHost(&w.h_count, 2 * sizeof(int32_t)) != cudaSuccess) return L1_ERR_OOM;
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

static Cols make_cols(Handle* h, int q, int N) {
    PanelSet& p = h->ws.ps[q];
    const int64_t cap = h->ws.cap_N;
    Cols c{};
    c.N = N;
    c.beta = p.colf + 0 * cap;
    c.binv = p.colf + 1 * cap;
    c.xi = p.colf + 2 * cap;
    c.xicap = p.colf + 3 * cap;
    c.mu = p.colf + 4 * cap;
    c.active = p.coli + 0 * cap;
    c.status = p.coli + 1 * cap;
    c.iters = p.coli + 2 * cap;
    c.inner = p.coli + 3 * cap;
    c.phase = p.coli + 4 * cap;
    c.l = p.coli + 5 * cap;
    c.orig = p.coli + 6 * cap;
    c.t = p.cold + 0 * cap;
    c.rel = p.cold + 1 * cap;
    c.de2 = p.cold + 2 * cap;
    c.e2 = p.cold + 3 * cap;
    c.b1 = p.cold + 4 * cap;
    return c;
}

static HomeRes make_home_res(Handle* h) {
    Workspace& w = h->ws;
    const int64_t cap = w.cap_N;
    HomeRes r{};
    r.status = w.hcoli + 0 * cap;
    r.iters = w.hcoli + 1 * cap;
    r.inner = w.hcoli + 2 * cap;
    r.label = w.hcoli + 3 * cap;
    r.sci_label = w.hcoli + 4 * cap;
    r.rel = w.hcold + 0 * cap;
    r.param = w.hcold + 1 * cap;
    r.fin = w.hcold + 2 * cap;  // [cap][8]
    r.xi = w.hcolf + 0 * cap;
    r.smax = w.hcolf + 1 * cap;
    return r;
}

static Home make_home(Handle* h) {
    Workspace& w = h->ws;
    HomeRes r = make_home_res(h);
    Home hm{};
    hm.N = (int)w.cap_N;
    hm.Wx = w.hWx;
    hm.We = w.hWe;
    hm.Y = w.hY;
    hm.status = r.status;
    hm.iters = r.iters;
    hm.inner = r.inner;
    hm.rel = r.rel;
    hm.param = r.param;
    hm.xi = r.xi;
    return hm;
}

// Move the active slots of set q to the front of set q^1 and write the
// results of the others home; *n_out = number of active slots.
static int compact(Handle* h, int q, int N_cur, int solver, double xi_max, int* n_out) {
    Workspace& w = h->ws;
    cudaStream_t s = h->stream;
    Cols src = make_cols(h, q, N_cur), dst = make_cols(h, q ^ 1, N_cur);
    Home hm = make_home(h);
    compact_scan_kernel<<<1, 1024, 0, s>>>(src.active, N_cur, w.newpos, w.count);
    L1_LAUNCH_CHECK(h);
    const PanelSet &a = w.ps[q], &b = w.ps[q ^ 1];
    struct P {
        const float* src;
        float* dst;
        float* home;
        int64_t ld;
        int rows;
    };
    const int m = (int)h->m, n = (int)h->n;
    const P panels[] = {{a.B, b.B, nullptr, h->ldm, m},  {a.Wx, b.Wx, w.hWx, h->ldn, n},
                        {a.We, b.We, w.hWe, h->ldm, m},  {a.Ux, b.Ux, w.hUx, h->ldn, n},
                        {a.Ue, b.Ue, w.hUe, h->ldm, m}, {a.Y, b.Y, w.hY, h->ldm, m},
                        {a.X, b.X, nullptr, h->ldn, n},   {a.Cc, b.Cc, nullptr, h->ldm, m}};
    for (const P& p : panels) {
        dim3 grid((unsigned)std::min(8, (p.rows + 255) / 256), (unsigned)N_cur);
        compact_panel_kernel<<<grid, 256, 0, s>>>(p.src, p.dst, p.home, p.ld, p.rows, N_cur, w.newpos, src.orig);
        L1_LAUNCH_CHECK(h);
    }
    compact_cols_kernel<<<(N_cur + 255) / 256, 256, 0, s>>>(src, dst, hm, N_cur, w.newpos, solver, xi_max);
    L1_LAUNCH_CHECK(h);
    L1_CUDA_TRY(cudaMemcpyAsync(w.h_count, w.count, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    L1_CUDA_TRY(cudaStreamSynchronize(s));
    *n_out = *w.h_count;
    return L1_OK;
}

// Tensor-core sweeps: the term list of a p x p split (p pieces of each operand)
static tc16::Terms terms_square(int p) {
    return p >= 3 ? tc16::terms_3x3() : (p == 2 ? tc16::terms_2x2() : tc16::terms_1x1());
}

// Retiring slots of a tensor-core set carry (V, Z); their home copies must
// hold the CUDA-core state U = Z - W/beta (the refinement restarts from it).
// inactive_only: convert the retiring slots (before a compaction), else the
// active ones (when the set continues on the CUDA-core sweeps).
static int tc_to_simt(Handle* h, const PanelSet& P, const Cols& c, int N_cur, bool cab, bool inactive_only) {
    const int m = (int)h->m, n = (int)h->n;
    dim3 gx((unsigned)std::min(8, (n + 255) / 256), (unsigned)N_cur), ge((unsigned)std::min(8, (m + 255) / 256),
                                                                          (unsigned)N_cur);
    tc_state_to_simt_kernel<<<gx, 256, 0, h->stream>>>(P.Ux, P.X, P.Wx, c.binv, c.active, h->ldn, n,
                                                        inactive_only ? 1 : 0);
    L1_LAUNCH_CHECK(h);
    if (cab) {
        tc_state_to_simt_kernel<<<ge, 256, 0, h->stream>>>(P.Ue, P.Cc, P.We, c.binv, c.active, h->ldm, m,
                                                            inactive_only ? 1 : 0);
        L1_LAUNCH_CHECK(h);
    }
    return L1_OK;
}

// DALM state of the active slots from (w, y): z = clamp(B^T y + w/beta) and
// U = z - w/beta, or with have_u the given U; for the tensor-core engine
// (tc) also Z = z and V = z - B^T y - w/beta, and the BF16 pieces of V_x.
// One A^T y sweep on the FP32 dictionary gives B^T y (its identity block is y).
static int dalm_restart(Handle* h, const PanelSet& P, const Cols& c, int N_cur, bool cab, bool have_u, bool tc,
                        double* part_n, int pieces) {
    const int m = (int)h->m, n = (int)h->n;
    const int rc = launch_sweep(h, n, N_cur, m, h->A_cm, h->ldm, P.Y, h->ldm,
                                EpiDalmRestart{P.Ux, P.X, P.Wx, c.binv, c.active, h->ldn, have_u ? 1 : 0, tc ? 1 : 0},
                                part_n, c.active);
    if (rc < 0) return rc;
    if (cab) {
        dim3 ge((unsigned)std::min(8, (m + 255) / 256), (unsigned)N_cur);
        dalm_restart_e_kernel<<<ge, 256, 0, h->stream>>>(P.Ue, P.Cc, P.We, P.Y, c.binv, c.active, h->ldm, m,
                                                          have_u ? 1 : 0, tc ? 1 : 0);
        L1_LAUNCH_CHECK(h);
    }
    if (tc) L1_TRY(tc16::split_aligned_lines(h, P.Ux, nullptr, N_cur, n, h->ldn, h->ws.Vh, pieces));
    return L1_OK;
}

int solve_batch(Handle* h, const float* b, int64_t ldb, int N, double tol, int max_iter,
                float* x, int64_t ldx, float* y, int64_t ldy, l1_result* res,
                const float* x_init, int64_t ldxi, const float* y_init, int64_t ldyi) {
    L1_TRY(ensure_workspace(h, N));
    Workspace& w = h->ws;
    cudaStream_t s = h->stream;
    const int m = (int)h->m, n = (int)h->n;
    const int64_t ldm = h->ldm, ldn = h->ldn;
    const int mode = h->mode;
    const int solver = (mode == L1_QP_LAMBDA) ? L1_PALM : h->opt.solver;
    const bool cab = mode == L1_CAB;
    const l1_options& o = h->opt;
    const double xi_max = o.xi_max > 0.0 ? o.xi_max : 1e4;
    double* part_m = w.part;
    double* part_n = w.part + w.part_slots * (size_t)w.cap_N * kPartStride;

    // ---- inputs and initial state (set 0, slot j = column j)
    int q = 0;
    PanelSet* P = &w.ps[0];
    L1_CUDA_TRY(cudaMemcpy2DAsync(w.hB, ldm * sizeof(float), b, ldb * sizeof(float), m * sizeof(float),
                                  N, cudaMemcpyDefault, s));
    const size_t pm = sizeof(float) * ldm * N, pn = sizeof(float) * ldn * N;
    L1_CUDA_TRY(cudaMemcpyAsync(P->B, w.hB, pm, cudaMemcpyDeviceToDevice, s));
    L1_CUDA_TRY(cudaMemsetAsync(P->Wx, 0, pn, s));
    L1_CUDA_TRY(cudaMemsetAsync(P->Ux, 0, pn, s));
    L1_CUDA_TRY(cudaMemsetAsync(P->X, 0, pn, s));
    L1_CUDA_TRY(cudaMemsetAsync(P->Ue, 0, pm, s));
    L1_CUDA_TRY(cudaMemsetAsync(P->Y, 0, pm, s));
    L1_CUDA_TRY(cudaMemsetAsync(P->Cc, 0, pm, s));
    if (solver == L1_PALM && cab) {
        // Algorithm 1 input: e_1 = b
        L1_CUDA_TRY(cudaMemcpyAsync(P->We, P->B, pm, cudaMemcpyDeviceToDevice, s));
    } else {
        L1_CUDA_TRY(cudaMemsetAsync(P->We, 0, pm, s));
    }
    // AMP (R18): z_0 = b (in Y) and x_0 = 0 unless y_init / x_init give them
    if (solver == L1_AMP) L1_CUDA_TRY(cudaMemcpyAsync(P->Y, P->B, pm, cudaMemcpyDeviceToDevice, s));
    // warm start: x_init = w_0 ([x; e] for CAB), y_init = y_0 (DALM) or
    // theta_0 (PALM); PALM and FISTA start their first inner loop at z = x_0
    if (x_init) {
        L1_CUDA_TRY(cudaMemcpy2DAsync(P->Wx, ldn * sizeof(float), x_init, ldxi * sizeof(float), n * sizeof(float),
                                      N, cudaMemcpyDefault, s));
        if (solver == L1_PALM) {
            L1_CUDA_TRY(cudaMemcpyAsync(P->X, P->Wx, pn, cudaMemcpyDeviceToDevice, s));
            L1_CUDA_TRY(cudaMemcpyAsync(P->Ux, P->Wx, pn, cudaMemcpyDeviceToDevice, s));
        }
        if (cab)
            L1_CUDA_TRY(cudaMemcpy2DAsync(P->We, ldm * sizeof(float), x_init + n, ldxi * sizeof(float),
                                          m * sizeof(float), N, cudaMemcpyDefault, s));
    }
    if (y_init)
        L1_CUDA_TRY(cudaMemcpy2DAsync(P->Y, ldm * sizeof(float), y_init, ldyi * sizeof(float), m * sizeof(float), N,
                                      cudaMemcpyDefault, s));
    Cols c = make_cols(h, 0, N);
    init_cols_kernel<<<N, 128, 0, s>>>(c, P->B, ldm, m, mode, o.beta, o.xi0, xi_max, o.lambda,
                                       o.lambda0);
    L1_LAUNCH_CHECK(h);
    if (solver == L1_AMP) {
        // tau_0: the given value, else 1.5 ||b||_2 / sqrt(m) per column (R18)
        amp_init_kernel<<<N, 128, 0, s>>>(c, P->B, ldm, m, o.tau0);
        L1_LAUNCH_CHECK(h);
    }

    const int check_every = o.check_every > 0 ? o.check_every : 16;
    SweepProf prof{h, o.profile != 0};
    L1_TRY(prof.reserve(3 * check_every));
    int N_cur = N;  // slots in the current set; every active slot is < N_cur
    PalmParams pp;
    pp.mode = mode;
    pp.growth = (mode == L1_CAB || mode == L1_QP_LAMBDA) ? 1.0f : (float)(o.xi_growth > 0.0 ? o.xi_growth : 1.2);
    // FISTA with continuation (R17): lambda_{k+1} = max(rho lambda_k, lambda)
    if (mode == L1_QP_LAMBDA && o.lambda0 > o.lambda)
        pp.growth = (float)(1.0 / (o.cont_rho > 0.0 ? o.cont_rho : 0.95));
    pp.Linv = h->lipschitz > 0.0 ? (float)(1.0 / h->lipschitz) : 0.0f;
    const int inner_max = o.inner_max > 0 ? o.inner_max : 50;
    const double inner_tol = o.inner_tol > 0.0 ? o.inner_tol : 0.1 * tol;
    // host budget of sweep rounds: every column has stopped by then (max_iter)
    const int64_t round_cap = (solver != L1_PALM || mode == L1_QP_LAMBDA) ? (int64_t)max_iter
                                                                          : (int64_t)max_iter * inner_max;
    int64_t rounds = 0;
    // low-precision A: phase 1 sweeps the BF16 / FP8 copy, phase 2 (refinement)
    // resumes every column on the FP32 A
    const bool lowp = o.precision != L1_A_FP32;
    int phase = 1;
    int32_t* iters1 = w.hcoli + 5 * w.cap_N;
    // tensor-core engine (batched DALM): BF16 pieces of A and the panels
    // DALM with a CG y-step: tensor cores only, to the last column
    const bool cg = o.cg_steps > 0;
    const int tc_min = cg ? 1 : (o.tc_min_cols > 0 ? o.tc_min_cols : 1);
    const int tcp = o.tc_pieces > 0 ? std::min(o.tc_pieces, 3) : 3;      // A sweeps
    const int tcy = o.tc_pieces_y > 0 ? std::min(o.tc_pieces_y, 3) : 3;  // y-step
    bool tc_mode = h->use_tc && solver != L1_PALM && N_cur >= tc_min;
    // AMP on the tensor cores: the A^T z sweep reads the BF16 pieces of z_0
    if (solver == L1_AMP && tc_mode) L1_TRY(tc16::split_aligned_lines(h, P->Y, nullptr, N_cur, m, ldm, w.Yh, tcp));
    if (solver == L1_DALM && (x_init || y_init || tc_mode)) {
        // the state z_1 (and V_1) of the first iteration from (w_0, y_0); a
        // cold start is all zeros either way, but the pieces of V are written
        if (x_init || y_init) L1_TRY(dalm_restart(h, *P, c, N_cur, cab, false, tc_mode, part_n, tcp));
        else L1_TRY(tc16::split_aligned_lines(h, P->Ux, nullptr, N_cur, n, ldn, w.Vh, tcp));
    }
    while (true) {
        P = &w.ps[q];
        c = make_cols(h, q, N_cur);
        const bool lowp_now = lowp && phase == 1;
        const double na = N_cur;
        auto run_chunk = [&](cudaStream_t s) -> int {
        for (int r = 0; r < check_every; ++r) {
            if (solver == L1_DALM && tc_mode && cg) {
                // Algorithm 2 with one conjugate-gradient y-step (§V-B,
                // reading R15) on the tensor cores: d = B V + b/beta and
                // ||d||^2; ||A^T d||^2; alpha = ||d||^2 / ||B^T d||^2;
                // y += alpha d with the CAB e-part (EpiTcY on alpha d); A^T y
                // with the x-part (EpiTcS)
                const tc16::Terms ta = terms_square(tcp);
                tc16::Operands o1{{h->A_rm_h[0], h->A_rm_h[1], h->A_rm_h[2]}, tcp,
                                  {w.Vh[0], w.Vh[1], w.Vh[2]}, tcp, ldn, ldn};
                tc16::PieceOut po1{{w.Dh[0], w.Dh[1], w.Dh[2]}, tcp, ldm};
                prof.start(0, 2.0 * m * n * na);
                const int np_d = tc_sweep(h, m, N_cur, n, o1, ta,
                                          EpiCgD{w.R, P->Ue, P->B, c.binv, c.active, ldm, cab ? 1 : 0}, po1, part_m,
                                          c.active);
                prof.stop();
                if (np_d < 0) return np_d;
                tc16::Operands o2{{h->A_cm_h[0], h->A_cm_h[1], h->A_cm_h[2]}, tcp,
                                  {w.Dh[0], w.Dh[1], w.Dh[2]}, tcp, ldm, ldm};
                tc16::PieceOut po0{{nullptr, nullptr, nullptr}, 0, ldn};
                prof.start(1, 2.0 * m * n * na);
                const int np_q = tc_sweep(h, n, N_cur, m, o2, ta, EpiCgQ{c.active}, po0, part_n, c.active);
                prof.stop();
                if (np_q < 0) return np_q;
                float* alpha = P->colf + 5 * w.cap_N;
                cg_alpha_kernel<<<N_cur, 128, 0, s>>>(c, part_m, np_d, part_n, np_q, cab ? 1 : 0, alpha);
                L1_LAUNCH_CHECK(h);
                tc16::PieceOut po2{{w.Yh[0], w.Yh[1], w.Yh[2]}, tcp, ldm};
                const int np_e = tc_scaled_y(
                    h, m, N_cur, w.R, ldm, alpha,
                    EpiTcY{P->Y, P->We, P->Cc, P->Ue, c.beta, c.binv, c.active, ldm, cab ? 1 : 0}, po2, part_m,
                    c.active);
                if (np_e < 0) return np_e;
                tc16::Operands o3{{h->A_cm_h[0], h->A_cm_h[1], h->A_cm_h[2]}, tcp,
                                  {w.Yh[0], w.Yh[1], w.Yh[2]}, tcp, ldm, ldm};
                tc16::PieceOut po3{{w.Vh[0], w.Vh[1], w.Vh[2]}, tcp, ldn};
                prof.start(2, 2.0 * m * n * na);
                const int np_x = tc_sweep(h, n, N_cur, m, o3, ta,
                                          EpiTcS{P->Wx, P->X, P->Ux, c.beta, c.binv, c.active, ldn}, po3, part_n,
                                          c.active);
                prof.stop();
                if (np_x < 0) return np_x;
                ctrl_dalm_kernel<<<(N_cur + kCtrlCols - 1) / kCtrlCols, 128, 0, s>>>(c, cab ? part_m : nullptr, np_e,
                                                                                     part_n, np_x, tol, max_iter);
                L1_LAUNCH_CHECK(h);
            } else if (solver == L1_DALM && tc_mode) {
                // Algorithm 2 on the BF16 tensor cores, the y-step as a
                // correction (EpiTcD / EpiTcY / EpiTcS): pa pieces of A (one,
                // the BF16 A itself, in the first phase of a BF16 solve), tcp
                // pieces of the panels V_x and y, tcy of F and d
                const int pa = lowp_now ? 1 : tcp;
                const tc16::Terms ta = lowp_now ? tc16::terms_1xN(tcp) : terms_square(tcp);
                tc16::Operands o1{{h->A_rm_h[0], h->A_rm_h[1], h->A_rm_h[2]}, pa,
                                  {w.Vh[0], w.Vh[1], w.Vh[2]}, tcp, ldn, ldn};
                tc16::PieceOut po1{{w.Dh[0], w.Dh[1], w.Dh[2]}, tcy, ldm};
                prof.start(0, 2.0 * m * n * na);
                int rc = tc_sweep(h, m, N_cur, n, o1, ta, EpiTcD{P->Ue, P->B, c.binv, c.active, ldm, cab ? 1 : 0},
                                      po1, nullptr, c.active);
                prof.stop();
                if (rc < 0) return rc;
                tc16::Operands o2{{h->F_h[0], h->F_h[1], h->F_h[2]}, tcy, {w.Dh[0], w.Dh[1], w.Dh[2]}, tcy, ldm, ldm};
                tc16::PieceOut po2{{w.Yh[0], w.Yh[1], w.Yh[2]}, tcp, ldm};
                prof.start(1, 2.0 * m * m * na);
                const int np_e = tc_sweep(
                    h, m, N_cur, m, o2, terms_square(tcy),
                    EpiTcY{P->Y, P->We, P->Cc, P->Ue, c.beta, c.binv, c.active, ldm, cab ? 1 : 0}, po2, part_m,
                    c.active);
                prof.stop();
                if (np_e < 0) return np_e;
                tc16::Operands o3{{h->A_cm_h[0], h->A_cm_h[1], h->A_cm_h[2]}, pa,
                                  {w.Yh[0], w.Yh[1], w.Yh[2]}, tcp, ldm, ldm};
                tc16::PieceOut po3{{w.Vh[0], w.Vh[1], w.Vh[2]}, tcp, ldn};
                prof.start(2, 2.0 * m * n * na);
                const int np_x = tc_sweep(h, n, N_cur, m, o3, ta,
                                              EpiTcS{P->Wx, P->X, P->Ux, c.beta, c.binv, c.active, ldn}, po3, part_n,
                                              c.active);
                prof.stop();
                if (np_x < 0) return np_x;
                ctrl_dalm_kernel<<<(N_cur + kCtrlCols - 1) / kCtrlCols, 128, 0, s>>>(c, cab ? part_m : nullptr, np_e,
                                                                                     part_n, np_x, tol, max_iter);
                L1_LAUNCH_CHECK(h);
            } else if (solver == L1_DALM) {
                // Algorithm 2: three sweeps per iteration on the CUDA cores
                const EpiDalmRhs e1{w.R, P->Ue, P->B, c.binv, c.active, ldm, cab ? 1 : 0};
                const EpiDalmY e2{P->Y, P->We, P->Ue, c.beta, c.binv, c.active, ldm, cab ? 1 : 0};
                const EpiDalmS e3{P->Wx, P->Ux, c.beta, c.binv, c.active, ldn};
                prof.start(0, 2.0 * m * n * na);
                int rc;
                if (lowp_now) rc = sweep_lowp(h, true, m, N_cur, n, P->Ux, ldn, e1, part_m, c.active);
                else rc = launch_sweep(h, m, N_cur, n, h->A_rm, ldn, P->Ux, ldn, e1, part_m, c.active);
                prof.stop();
                if (rc < 0) return rc;
                prof.start(1, 2.0 * m * m * na);  // algorithmic: one m x m product per column
                const int np_e = launch_sweep(h, m, N_cur, m, h->F, ldm, w.R, ldm, e2, part_m, c.active, h->F_lo);
                prof.stop();
                if (np_e < 0) return np_e;
                prof.start(2, 2.0 * m * n * na);
                int np_x;
                if (lowp_now) np_x = sweep_lowp(h, false, n, N_cur, m, P->Y, ldm, e3, part_n, c.active);
                else np_x = launch_sweep(h, n, N_cur, m, h->A_cm, ldm, P->Y, ldm, e3, part_n, c.active);
                prof.stop();
                if (np_x < 0) return np_x;
                ctrl_dalm_kernel<<<(N_cur + kCtrlCols - 1) / kCtrlCols, 128, 0, s>>>(c, cab ? part_m : nullptr, np_e,
                                                                                     part_n, np_x, tol, max_iter);
                L1_LAUNCH_CHECK(h);
            } else if (solver == L1_AMP && tc_mode) {
                // AMP (§IV) on the tensor cores: x-step on A^T z (reads the
                // pieces of z, writes those of x), the controller, z-step on
                // A x (reads the pieces of x, writes those of z)
                const tc16::Terms ta = terms_square(tcp);
                tc16::Operands o1{{h->A_cm_h[0], h->A_cm_h[1], h->A_cm_h[2]}, tcp,
                                  {w.Yh[0], w.Yh[1], w.Yh[2]}, tcp, ldm, ldm};
                tc16::PieceOut po1{{w.Vh[0], w.Vh[1], w.Vh[2]}, tcp, ldn};
                prof.start(2, 2.0 * m * n * na);
                const int np_x = tc_sweep(h, n, N_cur, m, o1, ta, EpiTcAmpX{P->Wx, c.xi, c.active, ldn}, po1, part_n,
                                          c.active);
                prof.stop();
                if (np_x < 0) return np_x;
                ctrl_amp_kernel<<<(N_cur + kCtrlCols - 1) / kCtrlCols, 128, 0, s>>>(c, part_n, np_x, m, tol,
                                                                                    max_iter);
                L1_LAUNCH_CHECK(h);
                tc16::Operands o2{{h->A_rm_h[0], h->A_rm_h[1], h->A_rm_h[2]}, tcp,
                                  {w.Vh[0], w.Vh[1], w.Vh[2]}, tcp, ldn, ldn};
                tc16::PieceOut po2{{w.Yh[0], w.Yh[1], w.Yh[2]}, tcp, ldm};
                prof.start(0, 2.0 * m * n * na);
                const int rc = tc_sweep(h, m, N_cur, n, o2, ta, EpiTcAmpZ{P->Y, P->B, c.mu, c.active, ldm}, po2,
                                        nullptr, c.active);
                prof.stop();
                if (rc < 0) return rc;
            } else if (solver == L1_AMP) {
                // AMP (§IV): the x-step on A^T z, the controller (stopping
                // rule, eta, tau), the z-step on A x
                prof.start(2, 2.0 * m * n * na);
                const int np_x = launch_sweep(h, n, N_cur, m, h->A_cm, ldm, P->Y, ldm,
                                              EpiAmpX{P->Wx, c.xi, c.active, ldn}, part_n, c.active);
                prof.stop();
                if (np_x < 0) return np_x;
                ctrl_amp_kernel<<<(N_cur + kCtrlCols - 1) / kCtrlCols, 128, 0, s>>>(c, part_n, np_x, m, tol,
                                                                                    max_iter);
                L1_LAUNCH_CHECK(h);
                prof.start(0, 2.0 * m * n * na);
                const int np_z = launch_sweep(h, m, N_cur, n, h->A_rm, ldn, P->Wx, ldn,
                                              EpiAmpZ{P->Y, P->B, c.mu, c.active, ldm}, part_m, c.active);
                prof.stop();
                if (np_z < 0) return np_z;
            } else {
                // Algorithm 1 / Eq. 18: two sweeps per inner FISTA step
                prof.start(0, 2.0 * m * n * na);
                const int np_A = launch_sweep(h, m, N_cur, n, h->A_rm, ldn, P->Ux, ldn,
                                              EpiPalmA{w.R, P->Cc, P->We, P->Y, P->B, c, pp, ldm}, part_m, c.active);
                prof.stop();
                if (np_A < 0) return np_A;
                if (mode == L1_P1_2) {
                    p12_fixup_kernel<<<N_cur, 128, 0, s>>>(c, part_m, np_A, P->We, P->Cc, w.R, ldm, m, o.epsilon);
                    L1_LAUNCH_CHECK(h);
                }
                prof.start(2, 2.0 * m * n * na);
                const int np_At = launch_sweep(h, n, N_cur, m, h->A_cm, ldm, w.R, ldm,
                                               EpiPalmAt{P->Wx, P->Ux, P->X, c, pp, ldn}, part_n, c.active);
                prof.stop();
                if (np_At < 0) return np_At;
                ctrl_palm_kernel<<<N_cur, 128, 0, s>>>(c, pp, part_m, np_A, part_n, np_At, P->Wx, P->X, P->Ux, ldn, n,
                                                       tol, inner_tol, inner_max, max_iter);
                L1_LAUNCH_CHECK(h);
            }
        }
        return L1_OK;
        };
        if (tc_mode) {
            // the tensor-core sweeps run directly (a chunk of them takes
            // milliseconds; launch overhead does not matter)
            L1_TRY(run_chunk(s));
        } else {
            // capture the chunk once (on the private stream, so that the
            // caller's stream may be the legacy default stream) and replay it
            GraphEntry* ge = graph_find(h, q, N_cur, phase, solver, tol, max_iter);
            if (!ge) {
                if (!h->cap_stream) L1_CUDA_TRY(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
                const int64_t l0 = h->launches;
                prof.reset();
                h->stream = h->cap_stream;
                cudaError_t ce = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
                prof.capturing = true;
                int crc = ce == cudaSuccess ? run_chunk(h->cap_stream) : L1_ERR_CUDA;
                prof.capturing = false;
                cudaGraph_t graph = nullptr;
                const cudaError_t ee = ce == cudaSuccess ? cudaStreamEndCapture(h->cap_stream, &graph) : ce;
                h->stream = s;
                if (crc == L1_OK && ee != cudaSuccess) {
                    set_last_error(std::string("chunk capture: ") + cudaGetErrorString(ee));
                    crc = L1_ERR_CUDA;
                }
                cudaGraphExec_t exec = nullptr;
                if (crc == L1_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
                    set_last_error("chunk graph: instantiation failed");
                    crc = L1_ERR_CUDA;
                }
                if (graph) cudaGraphDestroy(graph);
                if (crc != L1_OK) {
                    cudaGetLastError();
                    return crc;
                }
                if (!h->graphs) h->graphs = new GraphCache();
                if (h->graphs->entries.size() >= 512) {
                    for (GraphEntry& e : h->graphs->entries) cudaGraphExecDestroy(e.exec);
                    h->graphs->entries.clear();
                }
                h->graphs->entries.push_back(
                    GraphEntry{q, N_cur, phase, solver, max_iter, tol, exec, h->launches - l0, prof.kind, prof.flop});
                ge = &h->graphs->entries.back();
                h->launches = l0;
                prof.reset();
            }
            L1_CUDA_TRY(cudaGraphLaunch(ge->exec, s));
            h->launches += ge->nlaunch;
            prof.adopt(ge->kinds, ge->flops);
        }
        rounds += check_every;
        count_active_kernel<<<1, 1024, 0, s>>>(c.active, N_cur, w.count);
        L1_LAUNCH_CHECK(h);
        L1_CUDA_TRY(cudaMemcpyAsync(w.h_count, w.count, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        if (h->tc_err) L1_CUDA_TRY(cudaMemcpyAsync(w.h_count + 1, h->tc_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        L1_CUDA_TRY(cudaStreamSynchronize(s));
        prof.collect();
        if (h->tc_err && w.h_count[1] != 0) {
            // a bounded wait inside a tensor-core sweep ran out: report it and
            // leave the context usable
            set_last_error("tcgen05 sweep: bounded wait expired (code " + std::to_string(w.h_count[1]) + ")");
            L1_CUDA_TRY(cudaMemsetAsync(h->tc_err, 0, sizeof(int), s));
            return L1_ERR_TIMEOUT;
        }
        const int n_act = *w.h_count;
        const bool done = n_act == 0 || rounds >= round_cap;
        auto tiles = [](int v) { return (v + kBN - 1) / kBN; };
        const bool shrink = n_act < N_cur && (tiles(n_act) < tiles(N_cur) || (n_act <= 8 && N_cur > 8));
        if (done || shrink) {
            if (done) {
                // retire every slot
                fill_i32_kernel<<<(N_cur + 255) / 256, 256, 0, s>>>(c.active, N_cur, 0);
                L1_LAUNCH_CHECK(h);
            }
            // retiring slots of a tensor-core DALM set go home in the CUDA-core
            // form (the AMP state x, z is the same in both)
            if (tc_mode && solver == L1_DALM) L1_TRY(tc_to_simt(h, *P, c, N_cur, cab, true));
            int cnt = 0;
            L1_TRY(compact(h, q, N_cur, solver, xi_max, &cnt));
            q ^= 1;
            N_cur = cnt;
            if (tc_mode && !done && N_cur > 0) {
                const PanelSet& Pn = w.ps[q];
                if (N_cur < tc_min) {
                    // too narrow for the tensor-core tiles: continue on the
                    // CUDA-core sweeps from the equivalent state
                    if (solver == L1_DALM) L1_TRY(tc_to_simt(h, Pn, make_cols(h, q, N_cur), N_cur, cab, false));
                    tc_mode = false;
                } else if (solver == L1_AMP) {
                    L1_TRY(tc16::split_aligned_lines(h, Pn.Y, nullptr, N_cur, m, ldm, w.Yh, tcp));
                } else {
                    L1_TRY(tc16::split_aligned_lines(h, Pn.Ux, nullptr, N_cur, n, ldn, w.Vh, tcp));
                }
            }
        }
        if (done && lowp && phase == 1 && o.refine >= 0) {
            // refinement: reload every column's state (w, z - w/beta, y) from
            // home and continue the same iteration on the FP32 operator
            HomeRes hr1 = make_home_res(h);
            phase = 2;
            rounds = 0;
            q = 0;
            P = &w.ps[0];
            L1_CUDA_TRY(cudaMemcpyAsync(P->B, w.hB, pm, cudaMemcpyDeviceToDevice, s));
            L1_CUDA_TRY(cudaMemcpyAsync(P->Wx, w.hWx, pn, cudaMemcpyDeviceToDevice, s));
            L1_CUDA_TRY(cudaMemcpyAsync(P->Ux, w.hUx, pn, cudaMemcpyDeviceToDevice, s));
            L1_CUDA_TRY(cudaMemcpyAsync(P->We, w.hWe, pm, cudaMemcpyDeviceToDevice, s));
            L1_CUDA_TRY(cudaMemcpyAsync(P->Ue, w.hUe, pm, cudaMemcpyDeviceToDevice, s));
            L1_CUDA_TRY(cudaMemcpyAsync(P->Y, w.hY, pm, cudaMemcpyDeviceToDevice, s));
            c = make_cols(h, 0, N);
            init_cols_kernel<<<N, 128, 0, s>>>(c, P->B, ldm, m, mode, o.beta, o.xi0, xi_max, o.lambda,
                                       o.lambda0);
            L1_LAUNCH_CHECK(h);
            refine_restart_kernel<<<(N + 255) / 256, 256, 0, s>>>(c, hr1.status, hr1.iters, iters1, N);
            L1_LAUNCH_CHECK(h);
            N_cur = N;
            tc_mode = h->use_tc && solver == L1_DALM && N_cur >= tc_min;
            if (tc_mode) L1_TRY(dalm_restart(h, *P, c, N_cur, cab, true, true, part_n, tcp));
            continue;
        }
        if (done) break;
    }
    if (phase == 2) {
        HomeRes hr2 = make_home_res(h);
        add_iters_kernel<<<(N + 255) / 256, 256, 0, s>>>(hr2.iters, hr2.inner, iters1, N);
        L1_LAUNCH_CHECK(h);
    }

    // ---- finalisation on the home panels: objective, dual point, gap, residual
    HomeRes hr = make_home_res(h);
    if (mode == L1_QP_LAMBDA) {
        set_param_kernel<<<(N + 255) / 256, 256, 0, s>>>(hr.param, N, o.lambda / h->lipschitz);
        L1_LAUNCH_CHECK(h);
    }
    L1_CUDA_TRY(cudaMemsetAsync(hr.smax, 0, sizeof(float) * N, s));
    const float* E = (cab || mode == L1_P1_2) ? w.hWe : nullptr;
    const float* xi_fin = (solver == L1_PALM && mode != L1_QP_LAMBDA) ? hr.xi : nullptr;
    const int np_F1 = launch_sweep(h, m, N, n, h->A_rm, ldn, w.hWx, ldn,
                                   EpiFinalA{w.R, w.hY, E, w.hB, xi_fin, hr.smax, ldm, mode}, part_m, nullptr);
    if (np_F1 < 0) return np_F1;
    const int np_F2 = launch_sweep(h, n, N, m, h->A_cm, ldm, (mode == L1_QP_LAMBDA) ? w.R : w.hY, ldm,
                                   EpiFinalAt{w.hWx, hr.smax, ldn}, part_n, nullptr);
    if (np_F2 < 0) return np_F2;
    final_metrics_kernel<<<N, 128, 0, s>>>(N, hr.smax, hr.fin, part_m, np_F1, part_n, np_F2, mode,
                                           mode == L1_P1_2 ? o.epsilon : o.lambda);
    L1_LAUNCH_CHECK(h);

    // ---- classification (CAB with classes)
    const int C = (int)h->class_offsets.size() - 1;
    if (cab && C > 0) {
        int csz_max = 0;
        for (int c = 0; c < C; ++c) csz_max = std::max(csz_max, h->class_offsets[c + 1] - h->class_offsets[c]);
        constexpr int kClassSmem = 160 * 1024;
        if ((size_t)csz_max * 32 * sizeof(float) <= kClassSmem) {
            const int sm = csz_max * 32 * (int)sizeof(float);
            L1_CUDA_TRY(cudaFuncSetAttribute(classify_tile_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kClassSmem));
            classify_tile_kernel<32><<<dim3(C, (N + 31) / 32), 256, sm, s>>>(
                h->A_cm, ldm, m, w.class_off, w.hB, w.hWe, w.hWx, ldn, N, w.resid2, w.classl1);
        } else if ((size_t)csz_max * 4 * sizeof(float) <= kClassSmem) {
            const int sm = csz_max * 4 * (int)sizeof(float);
            L1_CUDA_TRY(cudaFuncSetAttribute(classify_tile_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kClassSmem));
            classify_tile_kernel<4><<<dim3(C, (N + 3) / 4), 256, sm, s>>>(
                h->A_cm, ldm, m, w.class_off, w.hB, w.hWe, w.hWx, ldn, N, w.resid2, w.classl1);
        } else {
            classify_resid_kernel<<<dim3(C, N), 128, 0, s>>>(h->A_rm, ldn, m, w.class_off, w.hB, w.hWe, w.hWx,
                                                              ldm, ldn, N, w.resid2, w.classl1);
        }
        L1_LAUNCH_CHECK(h);
        classify_argmin_kernel<<<(N + 127) / 128, 128, 0, s>>>(w.resid2, w.classl1, C, N, hr.label, hr.sci_label);
        L1_LAUNCH_CHECK(h);
    } else {
        fill_i32_kernel<<<(N + 255) / 256, 256, 0, s>>>(hr.label, N, -1);
        L1_LAUNCH_CHECK(h);
        fill_i32_kernel<<<(N + 255) / 256, 256, 0, s>>>(hr.sci_label, N, -1);
        L1_LAUNCH_CHECK(h);
    }

    // ---- outputs
    l1_result* res_dev = reinterpret_cast<l1_result*>(w.R);  // R is free now
    if ((size_t)N * sizeof(l1_result) > sizeof(float) * (size_t)ldm * N) return L1_ERR_INVALID_ARG;
    pack_results_kernel<<<(N + 127) / 128, 128, 0, s>>>(hr, N, res_dev);
    L1_LAUNCH_CHECK(h);
    L1_CUDA_TRY(cudaMemcpy2DAsync(x, ldx * sizeof(float), w.hWx, ldn * sizeof(float), n * sizeof(float), N,
                                  cudaMemcpyDefault, s));
    if (cab) {
        L1_CUDA_TRY(cudaMemcpy2DAsync(x + n, ldx * sizeof(float), w.hWe, ldm * sizeof(float), m * sizeof(float),
                                      N, cudaMemcpyDefault, s));
    }
    if (y) {
        L1_CUDA_TRY(cudaMemcpy2DAsync(y, ldy * sizeof(float), w.hY, ldm * sizeof(float), m * sizeof(float), N,
                                      cudaMemcpyDefault, s));
    }
    L1_CUDA_TRY(cudaMemcpyAsync(res, res_dev, sizeof(l1_result) * N, cudaMemcpyDefault, s));
    L1_CUDA_TRY(cudaStreamSynchronize(s));
    return L1_OK;
}

}  // namespace l1
