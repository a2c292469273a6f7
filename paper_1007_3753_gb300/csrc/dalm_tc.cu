// Instantiations of the tensor-core DALM and AMP sweeps (see dalm_tc.cuh).
#include "dalm_tc.cuh"

namespace l1 {

int tc_sweep(Handle* h, int M, int N, int K, const tc16::Operands& op, const tc16::Terms& tl, const EpiTcD& epi,
             const tc16::PieceOut& po, double* part, const int32_t* active) {
    return tc16::launch(h, M, N, K, op, tl, epi, po, part, active);
}

int tc_sweep(Handle* h, int M, int N, int K, const tc16::Operands& op, const tc16::Terms& tl, const EpiTcY& epi,
             const tc16::PieceOut& po, double* part, const int32_t* active) {
    return tc16::launch(h, M, N, K, op, tl, epi, po, part, active);
}

int tc_sweep(Handle* h, int M, int N, int K, const tc16::Operands& op, const tc16::Terms& tl, const EpiTcS& epi,
             const tc16::PieceOut& po, double* part, const int32_t* active) {
    return tc16::launch(h, M, N, K, op, tl, epi, po, part, active);
}

int tc_sweep(Handle* h, int M, int N, int K, const tc16::Operands& op, const tc16::Terms& tl, const EpiCgD& epi,
             const tc16::PieceOut& po, double* part, const int32_t* active) {
    return tc16::launch(h, M, N, K, op, tl, epi, po, part, active);
}

int tc_sweep(Handle* h, int M, int N, int K, const tc16::Operands& op, const tc16::Terms& tl, const EpiCgQ& epi,
             const tc16::PieceOut& po, double* part, const int32_t* active) {
    return tc16::launch(h, M, N, K, op, tl, epi, po, part, active);
}

int tc_sweep(Handle* h, int M, int N, int K, const tc16::Operands& op, const tc16::Terms& tl, const EpiTcAmpX& epi,
             const tc16::PieceOut& po, double* part, const int32_t* active) {
    return tc16::launch(h, M, N, K, op, tl, epi, po, part, active);
}

int tc_sweep(Handle* h, int M, int N, int K, const tc16::Operands& op, const tc16::Terms& tl, const EpiTcAmpZ& epi,
             const tc16::PieceOut& po, double* part, const int32_t* active) {
    return tc16::launch(h, M, N, K, op, tl, epi, po, part, active);
}

int tc_scaled_y(Handle* h, int M, int N, const float* S, int64_t lds, const float* alpha, const EpiTcY& epi,
                const tc16::PieceOut& po, double* part, const int32_t* active) {
    return tc16::finish(h, M, N, 1, S, lds, alpha, epi, po, part, active);
}

}  // namespace l1
