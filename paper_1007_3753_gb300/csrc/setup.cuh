// One-time setup steps (definitions in setup.cu).
#pragma once

#include "common.cuh"

namespace l1 {

// A_cm / A_rm from a device column-major copy of A
int make_layouts(Handle* h, const float* A_dev, int64_t lda);

// BF16 / FP8 copies of both layouts of A (l1_options.precision)
int make_lowp(Handle* h);

// Rayleigh-quotient estimate of ||A||_2^2 by power iteration on A^T A
int power_iteration(Handle* h, int max_iter, double rtol, double* L_out);

// h->F = (A A^T + diag_add I)^{-1} in FP32 via an FP64 Cholesky factor;
// L1_ERR_NOT_SPD when a pivot is not positive beyond rounding
int dalm_factor(Handle* h, double diag_add);

// uneven groups of independent dictionaries (group.cu)
int group_setup(Handle* h, const float* const* A, const int64_t* m, const int64_t* n, int64_t count);
int group_load(Handle* h, int64_t first, int64_t k, const float* const* A);
int group_solve(Handle* h, const float* b, int64_t N, double tol, int max_iter, float* x, l1_result* res);
void group_free(Handle* h);

// unrolled PALM with a checkpointed tape and its adjoint (unroll.cu)
int unroll_forward(Handle* h, const float* b, int64_t ldb, int N, float* x, int64_t ldx, l1_result* res);
int unroll_backward(Handle* h, const float* grad_x, int N, float* grad_b, float* grad_A);
void unroll_free(Handle* h);

// release the cached CUDA graphs of solve_batch (solve.cu)
void graph_cache_clear(Handle* h);

// batched solve (solve.cu)
int solve_batch(Handle* h, const float* b_dev, int64_t ldb, int N, double tol, int max_iter,
                float* x_dev, int64_t ldx, float* y_dev, int64_t ldy, l1_result* res,
                const float* x_init, int64_t ldxi, const float* y_init, int64_t ldyi);

}  // namespace l1
