// Cholesky reduction pieces (chol.cu).
#pragma once

#include "omm_internal.cuh"

namespace omm {
namespace chol {

// In place: lower triangle of A (column-major m x m, ld m) <- L with A = L L^T;
// strict upper triangle zeroed; state->status = OMM_ERR_NOT_SPD on a bad pivot.
int cholesky(double *A, int64_t m, DevState *state, cudaStream_t st);
// B (m x nrhs, ld ldb) <- L^-1 B
int trsm_ll(const double *L, int64_t m, double *B, int64_t ldb, int64_t nrhs, cudaStream_t st);
// Hs <- L^-1 Hs L^-T (symmetrised), S <- I, L <- Cholesky factor of S (m x m each)
int reduce_standard(double *Hs, double *S, double *L, int64_t m, DevState *state, cudaStream_t st);
// B <- L^-T B
int trsm_llt(const double *L, int64_t m, double *B, int64_t ldb, int64_t nrhs, cudaStream_t st);

}  // namespace chol
}  // namespace omm
