// The C ABI of include/l1alm.h: argument checks, handle lifetime, setup.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>

#include "common.cuh"
#include "setup.cuh"
#include "tc16.cuh"

namespace l1 {

static thread_local std::string g_last_error;

void set_last_error(const std::string& msg) { g_last_error = msg; }

int dev_alloc(Handle* h, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_last_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
        *p = nullptr;
        return L1_ERR_OOM;
    }
    e = cudaMemsetAsync(*p, 0, bytes, h->stream);
    if (e != cudaSuccess) {
        cudaFree(*p);
        *p = nullptr;
        set_last_error(std::string("cudaMemset: ") + cudaGetErrorString(e));
        return L1_ERR_CUDA;
    }
    h->allocations.push_back(*p);
    h->allocation_bytes.push_back(bytes);
    h->device_bytes += (int64_t)bytes;
    return L1_OK;
}

void dev_free(Handle* h, void* p) {
    if (!p) return;
    cudaFree(p);
    for (size_t i = 0; i < h->allocations.size(); ++i) {
        if (h->allocations[i] != p) continue;
        h->device_bytes -= (int64_t)h->allocation_bytes[i];
        h->allocations.erase(h->allocations.begin() + (std::ptrdiff_t)i);
        h->allocation_bytes.erase(h->allocation_bytes.begin() + (std::ptrdiff_t)i);
        break;
    }
}

static void free_all(Handle* h) {
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    graph_cache_clear(h);
    if (h->cap_stream) {
        cudaStreamDestroy(h->cap_stream);
        h->cap_stream = nullptr;
    }
    for (void* p : h->allocations) cudaFree(p);
    h->allocations.clear();
    h->allocation_bytes.clear();
    if (h->ws.h_count) cudaFreeHost(h->ws.h_count);
    h->ws = Workspace{};
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    h->ev_pool.clear();
}

}  // namespace l1

using namespace l1;

extern "C" {

void l1_options_init(l1_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->solver = L1_DALM;
    opt->precision = L1_A_FP32;
    opt->engine = L1_ENGINE_AUTO;
    opt->inner_max = 50;
    opt->xi_growth = 1.2;
    opt->xi_max = 1e4;
    opt->check_every = 16;
    opt->unroll_J = 10;
    opt->ckpt_every = 20;
}

const char* l1_status_string(int code) {
    switch (code) {
        case L1_OK: return "L1_OK / L1_CONVERGED";
        case L1_MAX_ITER: return "L1_MAX_ITER";
        case L1_NONFINITE: return "L1_NONFINITE";
        case L1_ERR_INVALID_ARG: return "L1_ERR_INVALID_ARG";
        case L1_ERR_NOT_SPD: return "L1_ERR_NOT_SPD";
        case L1_ERR_OOM: return "L1_ERR_OOM";
        case L1_ERR_CUDA: return "L1_ERR_CUDA";
        case L1_ERR_TIMEOUT: return "L1_ERR_TIMEOUT";
        case L1_ERR_NO_TAPE: return "L1_ERR_NO_TAPE";
        case L1_ERR_UNSUPPORTED: return "L1_ERR_UNSUPPORTED";
        default: return "unknown l1 code";
    }
}

const char* l1_last_error(void) { return g_last_error.c_str(); }

int l1_setup(const float* A, int64_t m, int64_t n, int64_t lda, int32_t mode, const l1_options* opt,
             l1_handle* out) {
    if (!out) return L1_ERR_INVALID_ARG;
    *out = nullptr;
    if (!A || m <= 0 || n <= 0 || lda < m || m > (1 << 20) || n > (1 << 24)) return L1_ERR_INVALID_ARG;
    if (mode < L1_P1 || mode > L1_CAB) return L1_ERR_INVALID_ARG;
    l1_options o;
    if (opt) o = *opt;
    else l1_options_init(&o);
    if (o.solver != L1_PALM && o.solver != L1_DALM && o.solver != L1_AMP) return L1_ERR_INVALID_ARG;
    if (o.precision < L1_A_FP32 || o.precision > L1_A_FP8E4M3) return L1_ERR_INVALID_ARG;
    if (o.engine < L1_ENGINE_AUTO || o.engine > L1_ENGINE_TC) return L1_ERR_INVALID_ARG;
    if (mode == L1_QP_LAMBDA && !(o.lambda > 0.0)) return L1_ERR_INVALID_ARG;
    if (mode == L1_P1_2 && !(o.epsilon > 0.0)) return L1_ERR_INVALID_ARG;
    if (o.class_count < 0 || (o.class_count > 0 && !o.class_offsets)) return L1_ERR_INVALID_ARG;
    if (o.class_count > 0) {
        if (o.class_offsets[0] != 0 || o.class_offsets[o.class_count] != n) return L1_ERR_INVALID_ARG;
        for (int c = 0; c < o.class_count; ++c)
            if (o.class_offsets[c + 1] <= o.class_offsets[c]) return L1_ERR_INVALID_ARG;
    }
    // requests the library does not implement
    if (mode == L1_P1_2 && o.solver != L1_PALM) return L1_ERR_UNSUPPORTED;  // R10 is a PALM
    // low-precision A: batched DALM with refinement (BF16 on either engine,
    // FP8 on the CUDA-core sweeps)
    if (o.precision != L1_A_FP32 && (o.solver != L1_DALM || mode == L1_QP_LAMBDA || o.unroll_K > 0))
        return L1_ERR_UNSUPPORTED;
    if (o.precision == L1_A_FP8E4M3 && o.engine == L1_ENGINE_TC) return L1_ERR_UNSUPPORTED;
    if (o.tc_pieces < 0 || o.tc_pieces > 3 || o.tc_pieces_y < 0 || o.tc_pieces_y > 3 || o.tc_min_cols < 0)
        return L1_ERR_INVALID_ARG;
    if (o.tc_pieces == 1 || o.tc_pieces_y == 1) return L1_ERR_UNSUPPORTED;  // a one-piece panel cannot converge
    if (o.engine == L1_ENGINE_TC && (o.solver == L1_PALM || mode == L1_QP_LAMBDA)) return L1_ERR_UNSUPPORTED;
    if (o.cg_steps < 0) return L1_ERR_INVALID_ARG;
    // FISTA with continuation (R17): batched (QP_lambda) only
    if (o.lambda0 < 0.0 || o.cont_rho < 0.0 || o.cont_rho > 1.0) return L1_ERR_INVALID_ARG;
    if (o.lambda0 > 0.0 && (mode != L1_QP_LAMBDA || o.unroll_K > 0)) return L1_ERR_UNSUPPORTED;
    // DALM with a CG y-step (R15): one step, FP32 dictionary, tensor-core sweeps
    if (o.cg_steps > 0 && (o.cg_steps != 1 || o.solver != L1_DALM || mode == L1_QP_LAMBDA ||
                           o.precision != L1_A_FP32 || o.engine == L1_ENGINE_SIMT || o.unroll_K > 0))
        return L1_ERR_UNSUPPORTED;
    // AMP (R18): P1 with an FP32 dictionary, none of the other options
    if (o.tau0 < 0.0) return L1_ERR_INVALID_ARG;
    if (o.tau0 > 0.0 && o.solver != L1_AMP) return L1_ERR_UNSUPPORTED;
    if (o.solver == L1_AMP && (mode != L1_P1 || o.precision != L1_A_FP32 || o.unroll_K > 0 || o.cg_steps > 0))
        return L1_ERR_UNSUPPORTED;
    if (o.unroll_K < 0 || o.unroll_J < 0 || o.ckpt_every < 0) return L1_ERR_INVALID_ARG;
    if (o.unroll_K > 0) {
        // R11: unrolled PALM in P1 mode on the CUDA cores
        if (mode != L1_P1 || o.solver != L1_PALM || o.engine == L1_ENGINE_TC) return L1_ERR_UNSUPPORTED;
        if (o.unroll_J == 0) o.unroll_J = 10;
        if (o.ckpt_every == 0) o.ckpt_every = 20;
    }

    Handle* h = new (std::nothrow) Handle();
    if (!h) return L1_ERR_OOM;
    h->m = m;
    h->n = n;
    h->ldm = round_up(m, 32);
    h->ldn = round_up(n, 32);
    h->mode = mode;
    h->opt = o;
    h->opt.class_offsets = nullptr;
    h->stream = static_cast<cudaStream_t>(o.stream);
    cudaGetDevice(&h->device);
    cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
    if (o.class_count > 0) h->class_offsets.assign(o.class_offsets, o.class_offsets + o.class_count + 1);

    int rc = L1_OK;
    float* stage = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    do {
        if (cudaEventCreate(&ev0) != cudaSuccess || cudaEventCreate(&ev1) != cudaSuccess) { rc = L1_ERR_CUDA; break; }
        cudaEventRecord(ev0, h->stream);
        rc = dev_alloc_t(h, &h->A_cm, (size_t)h->ldm * n);
        if (rc) break;
        rc = dev_alloc_t(h, &h->A_rm, (size_t)h->ldn * m);
        if (rc) break;
        if (cudaMalloc(&stage, sizeof(float) * (size_t)m * n) != cudaSuccess) { rc = L1_ERR_OOM; break; }
        if (cudaMemcpy2DAsync(stage, m * sizeof(float), A, lda * sizeof(float), m * sizeof(float), n,
                              cudaMemcpyDefault, h->stream) != cudaSuccess) {
            set_last_error("l1_setup: copy of A failed");
            rc = L1_ERR_CUDA;
            break;
        }
        rc = make_layouts(h, stage, m);
        if (rc) break;
        if (o.precision != L1_A_FP32) {
            rc = make_lowp(h);
            if (rc) break;
        }
        // tensor-core engine (batched DALM): aligned BF16 pieces of both
        // layouts of A (those of (B B^T)^{-1} follow the factor below)
        // (the automatic choice for DALM: its products track the FP64
        // iteration more closely than the CUDA-core FP32 sweeps and run faster
        // at width; FP8 dictionaries stay on the CUDA cores)
        h->use_tc = (o.engine == L1_ENGINE_TC || (o.engine == L1_ENGINE_AUTO && o.precision != L1_A_FP8E4M3)) &&
                    o.solver != L1_PALM && mode != L1_QP_LAMBDA && o.unroll_K == 0;
        if (h->use_tc) {
            rc = dev_alloc_t(h, &h->tc_err, 1);
            if (!rc) rc = tc16::make_dictionary_pieces(h);
            if (rc) break;
        }
        const bool needs_L = (mode == L1_QP_LAMBDA) || (o.solver == L1_PALM);
        if (o.lipschitz > 0.0) {
            h->lipschitz = o.lipschitz;
        } else if (needs_L) {
            double rho = 0.0;
            rc = power_iteration(h, 1000, 1e-6, &rho);
            if (rc) break;
            h->lipschitz = 1.01 * rho;
            if (!(h->lipschitz > 0.0)) { rc = L1_ERR_INVALID_ARG; break; }  // A == 0
        }
        if (o.solver == L1_AMP) {
            // AMP sweeps A x and A^T z only: no factor
            if (h->use_tc && o.tune >= 0) {
                rc = tc16::tune_splits(h);
                if (rc) break;
            }
        } else if (o.solver == L1_DALM && mode != L1_QP_LAMBDA && o.cg_steps > 0) {
            // the CG y-step needs no factor of B B^T
            if (h->use_tc && o.tune >= 0) {
                rc = tc16::tune_splits(h);
                if (rc) break;
            }
        } else if (o.solver == L1_DALM && mode != L1_QP_LAMBDA) {
            rc = dev_alloc_t(h, &h->F, (size_t)h->ldm * m);
            if (rc) break;
            rc = dev_alloc_t(h, &h->F_lo, (size_t)h->ldm * m);
            if (rc) break;
            rc = dalm_factor(h, mode == L1_CAB ? 1.0 : 0.0);
            if (rc) break;
            if (h->use_tc) {
                rc = tc16::make_factor_pieces(h);
                if (rc) break;
                if (o.tune >= 0) {
                    rc = tc16::tune_splits(h);
                    if (rc) break;
                }
            }
        }
        cudaEventRecord(ev1, h->stream);
        if (cudaEventSynchronize(ev1) != cudaSuccess) { rc = L1_ERR_CUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        h->setup_ms = ms;
    } while (false);
    if (stage) {
        cudaStreamSynchronize(h->stream);
        cudaFree(stage);
    }
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (rc == L1_OK) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_last_error(std::string("l1_setup: ") + cudaGetErrorString(e));
            rc = L1_ERR_CUDA;
        }
    }
    if (rc != L1_OK) {
        free_all(h);
        delete h;
        return rc;
    }
    *out = reinterpret_cast<l1_handle>(h);
    return L1_OK;
}

int l1_setup_group(const float* const* A, const int64_t* m, const int64_t* n, int64_t count, int32_t mode,
                   const l1_options* opt, l1_handle* out) {
    if (!out) return L1_ERR_INVALID_ARG;
    *out = nullptr;
    if (!m || !n || count <= 0 || count > (1 << 22) || mode != L1_QP_LAMBDA) return L1_ERR_INVALID_ARG;
    l1_options o;
    if (opt) o = *opt;
    else l1_options_init(&o);
    if (!(o.lambda > 0.0)) return L1_ERR_INVALID_ARG;
    if (o.precision != L1_A_FP32 && o.precision != L1_A_BF16) return L1_ERR_UNSUPPORTED;
    if (o.lambda0 != 0.0) return L1_ERR_UNSUPPORTED;  // continuation: l1_setup batches only
    if (o.solver == L1_AMP || o.tau0 != 0.0) return L1_ERR_UNSUPPORTED;  // AMP solves P1
    for (int64_t i = 0; i < count; ++i)
        if (m[i] <= 0 || n[i] <= 0) return L1_ERR_INVALID_ARG;
    Handle* h = new (std::nothrow) Handle();
    if (!h) return L1_ERR_OOM;
    h->mode = mode;
    h->opt = o;
    h->opt.class_offsets = nullptr;
    h->opt.solver = L1_PALM;
    h->stream = static_cast<cudaStream_t>(o.stream);
    cudaGetDevice(&h->device);
    int rc = group_setup(h, A, m, n, count);
    if (rc == L1_OK) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) {
            set_last_error(std::string("l1_setup_group: ") + cudaGetErrorString(e));
            rc = L1_ERR_CUDA;
        }
    }
    if (rc != L1_OK) {
        free_all(h);
        group_free(h);
        delete h;
        return rc;
    }
    *out = reinterpret_cast<l1_handle>(h);
    return L1_OK;
}

int l1_group_load(l1_handle hh, int64_t first, int64_t k, const float* const* A) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !h->grp || !A) return L1_ERR_INVALID_ARG;
    return group_load(h, first, k, A);
}

int l1_solve_batch(l1_handle hh, const float* b, int64_t ldb, int64_t N, double tol, int32_t max_iter, float* x,
                   int64_t ldx, float* y, int64_t ldy, l1_result* res, const float* x_init, int64_t ldxi,
                   const float* y_init, int64_t ldyi) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (h && h->grp) {
        if (!b || !x || !res || y || x_init || y_init || max_iter <= 0 || !(tol >= 0.0)) return L1_ERR_INVALID_ARG;
        return group_solve(h, b, N, tol, max_iter, x, res);
    }
    if (!h || !b || !x || !res || N <= 0 || N > 65535 || max_iter <= 0 || !(tol >= 0.0)) return L1_ERR_INVALID_ARG;
    if (ldb < h->m) return L1_ERR_INVALID_ARG;
    const int64_t nx = (h->mode == L1_CAB) ? h->n + h->m : h->n;
    if (ldx < nx) return L1_ERR_INVALID_ARG;
    if (y && ldy < h->m) return L1_ERR_INVALID_ARG;
    if (x_init && ldxi < nx) return L1_ERR_INVALID_ARG;
    if (y_init && ldyi < h->m) return L1_ERR_INVALID_ARG;
    if (h->opt.unroll_K > 0 && (y || x_init || y_init)) return L1_ERR_INVALID_ARG;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != h->device) cudaSetDevice(h->device);
    int rc = h->opt.unroll_K > 0
                 ? unroll_forward(h, b, ldb, (int)N, x, ldx, res)
                 : solve_batch(h, b, ldb, (int)N, tol, max_iter, x, ldx, y, ldy, res, x_init, ldxi, y_init, ldyi);
    if (dev != h->device) cudaSetDevice(dev);
    return rc;
}

int l1_backward(l1_handle hh, const float* grad_x, int64_t N, float* grad_b, float* grad_A) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !grad_x || N <= 0 || N > 65535) return L1_ERR_INVALID_ARG;
    if (!h->has_tape || !h->ur) return L1_ERR_NO_TAPE;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != h->device) cudaSetDevice(h->device);
    int rc = unroll_backward(h, grad_x, (int)N, grad_b, grad_A);
    if (dev != h->device) cudaSetDevice(dev);
    return rc;
}

int l1_set_stream(l1_handle hh, void* stream) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return L1_ERR_INVALID_ARG;
    h->stream = static_cast<cudaStream_t>(stream);
    return L1_OK;
}

int l1_get_info(l1_handle hh, l1_info* info) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !info) return L1_ERR_INVALID_ARG;
    info->m = h->m;
    info->n = h->n;
    info->mode = h->mode;
    info->solver = h->opt.solver;
    info->precision = h->opt.precision;
    info->engine = h->opt.engine;
    info->lipschitz = h->lipschitz;
    info->setup_ms = h->setup_ms;
    info->device_bytes = h->device_bytes;
    info->gpu_launches = h->launches;
    for (int k = 0; k < 4; ++k) {
        info->sweep_launches[k] = h->sweep_launches[k];
        info->sweep_ms[k] = h->sweep_ms[k];
        info->sweep_flop[k] = h->sweep_flop[k];
    }
    return L1_OK;
}

int l1_tuning(l1_handle hh, int32_t* out, int32_t cap) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || cap < 0 || (cap > 0 && !out)) return L1_ERR_INVALID_ARG;
    const int k = (int)std::min<size_t>(h->tc_splits.size(), (size_t)cap);
    for (int e = 0; e < k; ++e)
        for (int f = 0; f < 7; ++f) out[7 * e + f] = h->tc_splits[e][f];
    return k;
}

int l1_destroy(l1_handle hh) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return L1_OK;
    free_all(h);
    group_free(h);
    unroll_free(h);
    delete h;
    return L1_OK;
}

}  // extern "C"
