// Cholesky-reduced variant of the dense form (section "Overview of OMM
// approaches": the generalised problem H C = S C Lambda is reduced to the
// standard one through the Cholesky factorisation of S).
//
//   S = L L^T,   H~ = L^-1 H' L^-T,   W~ = L^T W,   W = L^-T W~.
//
// Blocked FP64 algorithms on column-major m x m arrays, panel width NB:
//   cholesky      right-looking: factor the NB x NB diagonal block in one CTA,
//                 solve the panel below it row by row, update the trailing
//                 matrix with the FP64 GEMM;
//   trsm_ll       B <- L^-1 B    (forward block substitution, GEMM updates);
//   trsm_llt      B <- L^-T B    (backward block substitution, GEMM updates).
// A non-positive pivot sets state->status = OMM_ERR_NOT_SPD.
#include <math.h>

#include "chol.cuh"
#include "omm_internal.cuh"

namespace omm {
namespace chol {
namespace {

constexpr int NB = 64;

// In-place Cholesky of the nb x nb diagonal block at A + k0 (1 + lda): lower
// triangle gets L_kk, the strict upper triangle is zeroed.
__global__ void potrf_diag_kernel(double *A, int64_t lda, int64_t k0, int nb, DevState *state) {
    __shared__ double a[NB][NB + 1];
    const int t = threadIdx.x;   // NB threads
    for (int j = 0; j < nb; ++j)
        a[t][j] = (t < nb) ? A[(k0 + t) + (k0 + j) * lda] : 0.0;
    __syncthreads();
    __shared__ int bad;
    if (t == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (t == 0) {
            const double d = a[j][j];
            if (!(d > 0.0)) bad = 1;
            a[j][j] = d > 0.0 ? sqrt(d) : 1.0;
        }
        __syncthreads();
        if (t > j && t < nb) a[t][j] /= a[j][j];
        __syncthreads();
        // rank-1 update of the trailing part of the block, column by column
        for (int c = j + 1; c < nb; ++c)
            if (t >= c && t < nb) a[t][c] -= a[t][j] * a[c][j];
        __syncthreads();
    }
    if (t < nb)
        for (int j = 0; j < nb; ++j) A[(k0 + t) + (k0 + j) * lda] = (j <= t) ? a[t][j] : 0.0;
    if (t == 0 && bad) state->status = OMM_ERR_NOT_SPD;
}

// Rows k0+nb .. m-1 of the panel: x L_kk^T = a  (forward substitution per row).
__global__ void trsm_panel_kernel(double *A, int64_t lda, int64_t k0, int nb, int64_t m) {
    __shared__ double l[NB][NB + 1];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int r = e % nb, c = e / nb;
        l[r][c] = A[(k0 + r) + (k0 + c) * lda];
    }
    __syncthreads();
    for (int64_t row = k0 + nb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < m;
         row += (int64_t)gridDim.x * blockDim.x) {
        double x[NB];
        for (int j = 0; j < nb; ++j) {
            double v = A[row + (k0 + j) * lda];
            for (int q = 0; q < j; ++q) v -= x[q] * l[j][q];
            x[j] = v / l[j][j];
        }
        for (int j = 0; j < nb; ++j) A[row + (k0 + j) * lda] = x[j];
    }
}

// Zero the strict upper triangle (the factor is read as a lower triangle).
__global__ void zero_upper_kernel(double *A, int64_t lda, int64_t m) {
    for (int64_t j = blockIdx.y; j < m; j += gridDim.y)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < j; i += (int64_t)gridDim.x * blockDim.x)
            A[i + j * lda] = 0.0;
}

// Diagonal-block solves of the triangular solves with nrhs right-hand sides:
// lower: X_i = L_ii^-1 B_i (forward); transposed: X_i = L_ii^-T B_i (backward).
template <bool TRANS>
__global__ void trsm_diag_kernel(const double *L, int64_t ldl, int64_t k0, int nb, double *B, int64_t ldb,
                                 int64_t nrhs) {
    __shared__ double l[NB][NB + 1];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int r = e % nb, c = e / nb;
        l[r][c] = L[(k0 + r) + (k0 + c) * ldl];
    }
    __syncthreads();
    for (int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; col < nrhs;
         col += (int64_t)gridDim.x * blockDim.x) {
        double x[NB];
        double *b = B + k0 + col * ldb;
        if (!TRANS) {
            for (int i = 0; i < nb; ++i) {
                double v = b[i];
                for (int q = 0; q < i; ++q) v -= l[i][q] * x[q];
                x[i] = v / l[i][i];
            }
        } else {
            for (int i = nb - 1; i >= 0; --i) {
                double v = b[i];
                for (int q = i + 1; q < nb; ++q) v -= l[q][i] * x[q];
                x[i] = v / l[i][i];
            }
        }
        for (int i = 0; i < nb; ++i) b[i] = x[i];
    }
}

// dst = src^T (m x m, column-major), 32 x 32 shared-memory tiles
__global__ void transpose_kernel(const double *src, double *dst, int64_t m) {
    __shared__ double t[32][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
    for (int r = ly; r < 32; r += 8)
        if (i0 + lx < m && j0 + r < m) t[r][lx] = src[(i0 + lx) + (j0 + r) * m];
    __syncthreads();
    for (int r = ly; r < 32; r += 8)
        if (j0 + lx < m && i0 + r < m) dst[(j0 + lx) + (i0 + r) * m] = t[lx][r];
}

// dst = (a + a^T) / 2, read from a (a is left unchanged)
__global__ void symmetrize_identity_kernel(double *a, double *dst, int64_t m) {
    __shared__ double t[32][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
    for (int r = ly; r < 32; r += 8)
        if (j0 + lx < m && i0 + r < m) t[r][lx] = a[(j0 + lx) + (i0 + r) * m];   // block (j, i)
    __syncthreads();
    for (int r = ly; r < 32; r += 8) {
        const int64_t i = i0 + lx, j = j0 + r;
        if (i < m && j < m) dst[i + j * m] = 0.5 * (a[i + j * m] + t[lx][r]);
    }
}

__global__ void identity_kernel(double *a, int64_t m) {
    for (int64_t j = blockIdx.y; j < m; j += gridDim.y)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
            a[i + j * m] = (i == j) ? 1.0 : 0.0;
}

int blocks(int64_t n, int per) {
    int64_t b = ceil_div(n, per);
    if (b > 152 * 8) b = 152 * 8;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

int cholesky(double *A, int64_t m, DevState *state, cudaStream_t st) {
    for (int64_t k0 = 0; k0 < m; k0 += NB) {
        const int nb = (int)(m - k0 < NB ? m - k0 : NB);
        potrf_diag_kernel<<<1, NB, 0, st>>>(A, m, k0, nb, state);
        count_launch();
        OMM_CUDA_TRY(cudaGetLastError());
        const int64_t rest = m - k0 - nb;
        if (rest <= 0) break;
        trsm_panel_kernel<<<blocks(rest, 128), 128, 0, st>>>(A, m, k0, nb, m);
        count_launch();
        OMM_CUDA_TRY(cudaGetLastError());
        // A22 -= L21 L21^T
        GemmBatch b{};
        b.A[0] = A + (k0 + nb) + k0 * m;
        b.B[0] = A + (k0 + nb) + k0 * m;
        b.Cin[0] = A + (k0 + nb) + (k0 + nb) * m;
        b.C[0] = A + (k0 + nb) + (k0 + nb) * m;
        const int rc = dgemm_batched(false, true, rest, rest, nb, -1.0, b, 1, m, m, 1.0, m, m, nullptr, st);
        if (rc != OMM_OK) return rc;
    }
    dim3 g((unsigned)blocks(m, 256), (unsigned)(m < 4096 ? m : 4096));
    zero_upper_kernel<<<g, 256, 0, st>>>(A, m, m);
    count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

int reduce_standard(double *Hs, double *S, double *L, int64_t m, DevState *state, cudaStream_t st) {
    OMM_CUDA_TRY(cudaMemcpyAsync(L, S, m * m * sizeof(double), cudaMemcpyDeviceToDevice, st));
    int rc = cholesky(L, m, state, st);
    if (rc != OMM_OK) return rc;
    if ((rc = trsm_ll(L, m, Hs, m, m, st))) return rc;                 // X = L^-1 H'
    dim3 g((unsigned)ceil_div(m, 32), (unsigned)ceil_div(m, 32));
    transpose_kernel<<<g, 256, 0, st>>>(Hs, S, m);                       // S slot <- X^T = H' L^-T
    count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    if ((rc = trsm_ll(L, m, S, m, m, st))) return rc;                   // L^-1 H' L^-T
    symmetrize_identity_kernel<<<g, 256, 0, st>>>(S, Hs, m);             // H slot <- symmetric part
    count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    dim3 gi((unsigned)blocks(m, 256), (unsigned)(m < 4096 ? m : 4096));
    identity_kernel<<<gi, 256, 0, st>>>(S, m);                           // S slot <- I
    count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

int trsm_ll(const double *L, int64_t m, double *B, int64_t ldb, int64_t nrhs, cudaStream_t st) {
    for (int64_t k0 = 0; k0 < m; k0 += NB) {
        const int nb = (int)(m - k0 < NB ? m - k0 : NB);
        trsm_diag_kernel<false><<<blocks(nrhs, 128), 128, 0, st>>>(L, m, k0, nb, B, ldb, nrhs);
        count_launch();
        OMM_CUDA_TRY(cudaGetLastError());
        const int64_t rest = m - k0 - nb;
        if (rest <= 0) break;
        // B2 -= L21 X1
        GemmBatch b{};
        b.A[0] = L + (k0 + nb) + k0 * m;
        b.B[0] = B + k0;
        b.Cin[0] = B + k0 + nb;
        b.C[0] = B + k0 + nb;
        const int rc = dgemm_batched(false, false, rest, nrhs, nb, -1.0, b, 1, m, ldb, 1.0, ldb, ldb, nullptr, st);
        if (rc != OMM_OK) return rc;
    }
    return OMM_OK;
}

int trsm_llt(const double *L, int64_t m, double *B, int64_t ldb, int64_t nrhs, cudaStream_t st) {
    const int64_t nblk = ceil_div(m, NB);
    for (int64_t bi = nblk - 1; bi >= 0; --bi) {
        const int64_t k0 = bi * NB;
        const int nb = (int)(m - k0 < NB ? m - k0 : NB);
        trsm_diag_kernel<true><<<blocks(nrhs, 128), 128, 0, st>>>(L, m, k0, nb, B, ldb, nrhs);
        count_launch();
        OMM_CUDA_TRY(cudaGetLastError());
        if (k0 == 0) break;
        // B_top -= L_(k, 0:k)^T X_k
        GemmBatch b{};
        b.A[0] = L + k0;            // rows k0.., columns 0..k0-1 ; used transposed
        b.B[0] = B + k0;
        b.Cin[0] = B;
        b.C[0] = B;
        const int rc = dgemm_batched(true, false, k0, nrhs, nb, -1.0, b, 1, m, ldb, 1.0, ldb, ldb, nullptr, st);
        if (rc != OMM_OK) return rc;
    }
    return OMM_OK;
}

}  // namespace chol
}  // namespace omm
