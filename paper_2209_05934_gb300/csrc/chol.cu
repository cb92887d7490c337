// Cholesky-reduced variant of the dense form (section "Overview of OMM
// approaches": the generalised problem H C = S C Lambda is reduced to the
// standard one through the Cholesky factorisation of S).
//
//   S = L L^T,   Y = L^-1,   H~ = Y H' Y^T,   W~ = L^T W,   W = Y^T W~.
//
// FP64-accurate throughout; the O(m^3) work runs on the tensor cores through
// the exact-digit GEMM (row-scaled base-128 digits, exact integer-valued FP32
// partial sums, FP64 combination), because the FP64 CUDA-core rate of this part
// is a small fraction of the tensor rate.
//
// L and Y come from one recursive factor-and-invert on halves: with
// S = [A11 A21^T; A21 A22],
//   L11, Y11 <- recursion on A11;  L21 = A21 Y11^T;  A22 -= L21 L21^T;
//   L22, Y22 <- recursion on A22;  Y21 = -Y22 (L21 Y11),
// so every GEMM at the top has K = m/2.  The 64 x 64 leaves are factored and
// inverted by one CTA in shared memory.  Inverting the diagonal blocks adds an
// error of order cond(L) eps, immaterial for the well-conditioned overlaps of
// localised basis sets.  The triangular products skip the zero triangle by
// chunking K.  A non-positive pivot sets state->status = OMM_ERR_NOT_SPD.
#include <math.h>

#include "chol.cuh"
#include "omm_internal.cuh"

namespace omm {
namespace chol {
namespace {

constexpr int kLeaf = 64;       // leaf size of the recursion
constexpr int kLeafThreads = 256;
constexpr int kRowBlock = 512;  // row / column blocks of the triangular products
constexpr int kLeafSmem = (2 * kLeaf * (kLeaf + 1) + 4 * kLeaf) * (int)sizeof(double);

// Cholesky factor and inverse of the s x s diagonal block at (n0, n0), s <= 64:
// lower triangles of A and Y get L_kk and L_kk^-1, their strict upper
// triangles inside the block are zeroed.
__global__ void __launch_bounds__(kLeafThreads) chol_leaf_kernel(double *A, double *Y, int64_t m, int64_t n0, int s,
                                                                 DevState *state) {
    extern __shared__ double sm[];
    double(*a)[kLeaf + 1] = (double(*)[kLeaf + 1])sm;
    double(*y)[kLeaf + 1] = (double(*)[kLeaf + 1])(sm + kLeaf * (kLeaf + 1));
    double(*part)[kLeaf] = (double(*)[kLeaf])(sm + 2 * kLeaf * (kLeaf + 1));
    __shared__ int bad;
    __shared__ double rdiag[kLeaf];   // 1 / l(j, j): one division per pivot (FP64 division is slow here)
    const int tid = threadIdx.x;
    for (int e = tid; e < s * s; e += kLeafThreads) {
        const int r = e % s, c = e / s;
        a[r][c] = A[(n0 + r) + (n0 + c) * m];
    }
    if (tid == 0) bad = 0;
    __syncthreads();
    // right-looking factorisation, element-parallel trailing updates
    for (int j = 0; j < s; ++j) {
        if (tid == 0) {
            double d = a[j][j];
            if (!(d > 0.0)) {
                bad = 1;
                d = 1.0;
            }
            a[j][j] = sqrt(d);
            rdiag[j] = 1.0 / a[j][j];
        }
        __syncthreads();
        const double rjj = rdiag[j];
        for (int r = j + 1 + tid; r < s; r += kLeafThreads) a[r][j] *= rjj;
        __syncthreads();
        // lanes along rows, the 8 warps along columns (no integer division)
        for (int c = j + 1 + (tid >> 5); c < s; c += kLeafThreads / 32) {
            const double acj = a[c][j];
            for (int r = c + (tid & 31); r < s; r += 32) a[r][c] -= a[r][j] * acj;
        }
        __syncthreads();
    }
    // Y = L^-1 row by row: y(i, j) = (delta_ij - sum_{j <= q < i} l(i, q) y(q, j)) / l(i, i),
    // columns j across 64 threads, the q-sum in 4 interleaved slices
    const int j = tid % kLeaf, g = tid / kLeaf;
    for (int i = 0; i < s; ++i) {
        double v = 0.0;
        if (j < i)
            for (int q = j + g; q < i; q += 4) v += a[i][q] * y[q][j];
        part[g][j] = v;
        __syncthreads();
        if (g == 0 && j < s) {
            const double sum = part[0][j] + part[1][j] + part[2][j] + part[3][j];
            y[i][j] = (j < i) ? -sum * rdiag[i] : (j == i ? rdiag[i] : 0.0);
        }
        __syncthreads();
    }
    for (int e = tid; e < s * s; e += kLeafThreads) {
        const int r = e % s, c = e / s;
        A[(n0 + r) + (n0 + c) * m] = (c <= r) ? a[r][c] : 0.0;
        Y[(n0 + r) + (n0 + c) * m] = (c <= r) ? y[r][c] : 0.0;
    }
    if (tid == 0 && bad) state->status = OMM_ERR_NOT_SPD;
}

// Zero the strict upper triangle (the factor is read as a lower triangle).
__global__ void zero_upper_kernel(double *A, int64_t lda, int64_t m) {
    for (int64_t j = blockIdx.y; j < m; j += gridDim.y)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < j; i += (int64_t)gridDim.x * blockDim.x)
            A[i + j * lda] = 0.0;
}

// a <- (a + a^T) / 2 in place; the CTA for tile pair (bx, by), bx >= by,
// rewrites both tiles
__global__ void symmetrize_kernel(double *a, int64_t m) {
    if (blockIdx.x < blockIdx.y) return;
    __shared__ double t1[32][33], t2[32][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
    for (int r = ly; r < 32; r += 8) {
        t1[r][lx] = (i0 + lx < m && j0 + r < m) ? a[(i0 + lx) + (j0 + r) * m] : 0.0;   // (i0 + lx, j0 + r)
        t2[r][lx] = (j0 + lx < m && i0 + r < m) ? a[(j0 + lx) + (i0 + r) * m] : 0.0;   // (j0 + lx, i0 + r)
    }
    __syncthreads();
    for (int r = ly; r < 32; r += 8) {
        if (i0 + lx < m && j0 + r < m) a[(i0 + lx) + (j0 + r) * m] = 0.5 * (t1[r][lx] + t2[lx][r]);
        if (j0 + lx < m && i0 + r < m) a[(j0 + lx) + (i0 + r) * m] = 0.5 * (t2[r][lx] + t1[lx][r]);
    }
}

__global__ void identity_kernel(double *a, int64_t m) {
    for (int64_t j = blockIdx.y; j < m; j += gridDim.y)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
            a[i + j * m] = (i == j) ? 1.0 : 0.0;
}

// M = S + T / tau, elementwise (the division as written, not a reciprocal product)
__global__ void spd_sum_kernel(const double *__restrict__ S, const double *__restrict__ T, double tau, double *M,
                               int64_t count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        M[i] = S[i] + T[i] / tau;
}

int blocks(int64_t n, int per) {
    int64_t b = ceil_div(n, per);
    if (b > 152 * 8) b = 152 * 8;
    return (int)(b < 1 ? 1 : b);
}

int xmm(bool tA, bool tB, int64_t M, int64_t N, int64_t K, double alpha, const double *A, int64_t lda,
        const double *B, int64_t ldb, double beta, double *C, int64_t ldc, const Work &w, cudaStream_t st) {
    if (M <= 0 || N <= 0 || K <= 0) return OMM_OK;
    return omm_op_exact_gemm(tA, tB, M, N, K, w.s, alpha, A, lda, B, ldb, beta, beta != 0.0 ? C : nullptr, ldc, C,
                             ldc, w.ws, w.bytes, st);
}

int64_t xbytes(int64_t M, int64_t N, int64_t K, int s) { return omm_op_exact_gemm_workspace_bytes(M, N, K, s); }

// split of a node of size s: the first half rounded up to a multiple of the leaf
int64_t split(int64_t s) { return ceil_div(ceil_div(s, 2), kLeaf) * kLeaf; }

int chol_inv(double *A, double *Y, int64_t m, int64_t n0, int64_t s, const Work &w, DevState *state,
             cudaStream_t st) {
    if (s <= kLeaf) {
        chol_leaf_kernel<<<1, kLeafThreads, kLeafSmem, st>>>(A, Y, m, n0, (int)s, state);
        count_launch();
        OMM_CUDA_TRY(cudaGetLastError());
        return OMM_OK;
    }
    const int64_t h = split(s), r = s - h;
    int rc = chol_inv(A, Y, m, n0, h, w, state, st);
    if (rc != OMM_OK) return rc;
    double *A21 = A + (n0 + h) + n0 * m;
    double *A22 = A + (n0 + h) + (n0 + h) * m;
    const double *Y11 = Y + n0 + n0 * m;
    double *Y21 = Y + (n0 + h) + n0 * m;
    const double *Y22 = Y + (n0 + h) + (n0 + h) * m;
    // L21 = A21 Y11^T (in place: operands are packed before the GEMM runs)
    if ((rc = xmm(false, true, r, h, h, 1.0, A21, m, Y11, m, 0.0, A21, m, w, st))) return rc;
    // A22 -= L21 L21^T
    if ((rc = xmm(false, true, r, r, h, -1.0, A21, m, A21, m, 1.0, A22, m, w, st))) return rc;
    if ((rc = chol_inv(A, Y, m, n0 + h, r, w, state, st))) return rc;
    // Y21 = -Y22 (L21 Y11), the inner product parked in Y21
    if ((rc = xmm(false, false, r, h, h, 1.0, A21, m, Y11, m, 0.0, Y21, m, w, st))) return rc;
    return xmm(false, false, r, h, r, -1.0, Y22, m, Y21, m, 0.0, Y21, m, w, st);
}

}  // namespace

int64_t work_bytes(int64_t m, int64_t n, int s) {
    int64_t b = xbytes(kRowBlock < m ? kRowBlock : m, m, m, s);               // triangular products
    const int64_t h = split(m), r = m - h;
    if (m > kLeaf) {
        // top node of the recursion (the largest): (r, h, h), (r, r, h), (r, h, r)
        const int64_t t0 = xbytes(r, h, h, s), t1 = xbytes(r, r, h, s), t2 = xbytes(r, h, r, s);
        b = b > t0 ? b : t0;
        b = b > t1 ? b : t1;
        b = b > t2 ? b : t2;
    }
    const int64_t t3 = xbytes(m, n, kChunkK < m ? kChunkK : m, s);             // W transforms
    return b > t3 ? b : t3;
}

int64_t linv_elems(int64_t m) { return m * m; }

int cholesky(double *A, int64_t m, const Work &w, DevState *state, cudaStream_t st) {
    static int attr = 0;
    if (attr < kLeafSmem) {
        OMM_CUDA_TRY(cudaFuncSetAttribute(chol_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kLeafSmem));
        attr = kLeafSmem;
    }
    OMM_CUDA_TRY(cudaMemsetAsync(w.Linv, 0, (size_t)(m * m) * sizeof(double), st));
    int rc = chol_inv(A, w.Linv, m, 0, m, w, state, st);
    if (rc != OMM_OK) return rc;
    dim3 g((unsigned)blocks(m, 256), (unsigned)(m < 4096 ? m : 4096));
    zero_upper_kernel<<<g, 256, 0, st>>>(A, m, m);
    count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

// Wt = T^T W for a lower-triangular T (L, or Y), in K chunks of rows of T, last
// chunk first: rows [kc, kc+kw) of T touch output rows [0, kc+kw) only, and the
// first chunk taken (the last rows) covers every output row.
int lt_times(const double *T, int64_t m, const double *W, double *Wt, int64_t n, const Work &w, cudaStream_t st) {
    const int64_t nchunk = ceil_div(m, kChunkK);
    for (int64_t c = nchunk - 1; c >= 0; --c) {
        const int64_t kc = c * kChunkK;
        const int64_t kw = m - kc < kChunkK ? m - kc : kChunkK;
        const int rc = xmm(true, false, kc + kw, n, kw, 1.0, T + kc, m, W + kc, m, c == nchunk - 1 ? 0.0 : 1.0, Wt, m,
                           w, st);
        if (rc != OMM_OK) return rc;
    }
    return OMM_OK;
}

int factor(const double *S, double *L, int64_t m, const Work &w, DevState *state, cudaStream_t st) {
    OMM_CUDA_TRY(cudaMemcpyAsync(L, S, m * m * sizeof(double), cudaMemcpyDeviceToDevice, st));
    return cholesky(L, m, w, state, st);
}

int transform(double *Hs, double *T, int64_t m, const Work &w, cudaStream_t st) {
    const double *Y = w.Linv;
    int rc;
    // T = Y H': rows [r0, r0 + rr) of Y have nonzeros in columns < r0 + rr only
    for (int64_t r0 = 0; r0 < m; r0 += kRowBlock) {
        const int64_t rr = m - r0 < kRowBlock ? m - r0 : kRowBlock;
        if ((rc = xmm(false, false, rr, m, r0 + rr, 1.0, Y + r0, m, Hs, m, 0.0, T + r0, m, w, st))) return rc;
    }
    // H~ = T Y^T: columns [c0, c0 + cc) of Y^T have nonzeros in rows < c0 + cc only
    for (int64_t c0 = 0; c0 < m; c0 += kRowBlock) {
        const int64_t cc = m - c0 < kRowBlock ? m - c0 : kRowBlock;
        if ((rc = xmm(false, true, m, cc, c0 + cc, 1.0, T, m, Y + c0, m, 0.0, Hs + c0 * m, m, w, st))) return rc;
    }
    dim3 g((unsigned)ceil_div(m, 32), (unsigned)ceil_div(m, 32));
    symmetrize_kernel<<<g, 256, 0, st>>>(Hs, m);
    count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    dim3 gi((unsigned)blocks(m, 256), (unsigned)(m < 4096 ? m : 4096));
    identity_kernel<<<gi, 256, 0, st>>>(T, m);
    count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

int precon(const double *S, const double *T, double tau, double *P, int64_t m, const Work &w, DevState *state,
           cudaStream_t st) {
    spd_sum_kernel<<<blocks(m * m, 256), 256, 0, st>>>(S, T, tau, P, m * m);
    count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    int rc = cholesky(P, m, w, state, st);
    if (rc != OMM_OK) return rc;
    // P = Y^T Y by row blocks: rows [r0, r0 + rr) of P take columns [r0, r0 + rr)
    // of Y, which are zero above row r0, so the K range is [r0, m)
    const double *Y = w.Linv;
    for (int64_t r0 = 0; r0 < m; r0 += kRowBlock) {
        const int64_t rr = m - r0 < kRowBlock ? m - r0 : kRowBlock;
        if ((rc = xmm(true, false, rr, m, m - r0, 1.0, Y + r0 + r0 * m, m, Y + r0, m, 0.0, P + r0, m, w, st)))
            return rc;
    }
    dim3 g((unsigned)ceil_div(m, 32), (unsigned)ceil_div(m, 32));
    symmetrize_kernel<<<g, 256, 0, st>>>(P, m);
    count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

}  // namespace chol
}  // namespace omm
