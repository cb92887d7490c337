// Exact-digit (near-FP64) tcgen05 GEMM: host-side interface inside the library.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "omm_internal.cuh"

namespace omm {
namespace tc {

constexpr int kExactMaxDigits = 8;
constexpr int kExactMaxPairs = kExactMaxDigits * (kExactMaxDigits + 1) / 2;

// C_z = alpha 2^(eA_i + eB_j) sum_{t+u <= s+1} 2^-(7(t+u)-2) A_t B_u^T + beta Cin_z
// with A, B the digit planes of rows scaled by 2^-eA / 2^-eB (see tc_exact.cu).
struct ExactArgs {
    int M, N, K;
    int npairs;
    uint8_t pa[kExactMaxPairs], pb[kExactMaxPairs];   // level-major pair order
    int a_row0, b_row0, a_row_step, b_row_step;
    double alpha, beta;
    const double *Cin;
    int64_t ldcin, cin_step;
    double *C;         // FP64 output, or nullptr when C32 is set
    float *C32;        // FP32 output (the result is rounded once, after the FP64 combination)
    int64_t ldc, c_step;
    const int *eA;     // row exponents of A (indexed by output row)
    const int *eB;     // row exponents of B (indexed by output column)
    int64_t eA_step, eB_step;   // per batch z
    const DevState *state;
    int *err;
};

void exact_pairs(int s, ExactArgs &a);
// Digits of the K-major operand rows of the FP64 column-major matrix X (rows x cols, ld):
// k_along_rows: operand row r = column r of X, K = rows; else operand row r = row r of X, K = cols.
// Writes the row exponents e[] and planes dst[t * plane + r * ldk + k].
int exact_pack(bool k_along_rows, int64_t rows, int64_t cols, const double *X, int64_t ld, int *e,
               __nv_bfloat16 *dst, int64_t ldk, int64_t plane, int s, const DevState *state, cudaStream_t st);
int exact_gemm(const CUtensorMap &mapA, const CUtensorMap &mapB, const ExactArgs &a, int nbatch, cudaStream_t st);

}  // namespace tc
}  // namespace omm
