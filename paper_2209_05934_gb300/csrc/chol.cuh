// Cholesky reduction pieces (chol.cu).
#pragma once

#include "omm_internal.cuh"

namespace omm {
namespace chol {

constexpr int kChunkK = 512;  // K chunk of the W transforms

// Device workspace of one handle: the digit planes of the exact-digit GEMMs
// (bytes) and Y = L^-1 (Linv, m x m column-major, zero above the diagonal).
struct Work {
    void *ws = nullptr;
    int64_t bytes = 0;
    int s = 7;               // digits of the exact-digit GEMM
    double *Linv = nullptr;
};

int64_t work_bytes(int64_t m, int64_t n, int s);
int64_t linv_elems(int64_t m);

// In place: lower triangle of A (column-major m x m, ld m) <- L with A = L L^T;
// strict upper triangle zeroed; w.Linv <- L^-1; state->status = OMM_ERR_NOT_SPD
// on a non-positive pivot.
int cholesky(double *A, int64_t m, const Work &w, DevState *state, cudaStream_t st);
// Wt (m x n, ld m) <- T^T W for a lower-triangular T: W~ = L^T W with T = L,
// W = L^-T W~ with T = L^-1
int lt_times(const double *T, int64_t m, const double *W, double *Wt, int64_t n, const Work &w, cudaStream_t st);
// L <- Cholesky factor of S, w.Linv <- L^-1 (m x m each)
int factor(const double *S, double *L, int64_t m, const Work &w, DevState *state, cudaStream_t st);
// Hs <- L^-1 Hs L^-T (symmetrised) with L^-1 from factor(); T (m x m scratch) <- I
int transform(double *Hs, double *T, int64_t m, const Work &w, cudaStream_t st);
// Kinetic-energy preconditioner (Eq. 6): P <- (S + T / tau)^-1 = Y^T Y with
// Y = L^-1 of the Cholesky factor of S + T / tau (symmetrised; w.Linv <- Y);
// state->status = OMM_ERR_NOT_SPD when S + T / tau is not positive definite.
int precon(const double *S, const double *T, double tau, double *P, int64_t m, const Work &w, DevState *state,
           cudaStream_t st);

}  // namespace chol
}  // namespace omm
