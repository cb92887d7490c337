// FP64 GEMM for the plain double-precision form of the OMM CG step.
//
// GB300 executes FP64 on its CUDA cores only (no FP64 tensor-core kind in
// tcgen05), at a small fraction of the BF16 tensor rate, so this kernel is
// DFMA-bound: a 64x64 output tile per 256-thread block, a 4x4 register tile
// per thread, K staged through shared memory 16 at a time with a two-slot
// double buffer.  Operands are column-major with optional transposes.
#include "omm_internal.cuh"

namespace omm {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <bool TA, bool TB>
__global__ void __launch_bounds__(NT) dgemm_kernel(int64_t M, int64_t N, int64_t K, double alpha,
                                                    GemmBatch bt, int64_t lda, int64_t ldb,
                                                    double beta, int64_t ldcin, int64_t ldc,
                                                    const DevState *state) {
    if (state != nullptr && *((volatile const int *)&state->done)) return;
    const int b = blockIdx.z;
    const double *__restrict__ A = bt.A[b];
    const double *__restrict__ B = bt.B[b];
    const double *Cin = bt.Cin[b];
    double *C = bt.C[b];

    __shared__ double As[2][BK][BM + 1];
    __shared__ double Bs[2][BK][BN + 1];

    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int64_t i0 = (int64_t)blockIdx.x * BM;
    const int64_t j0 = (int64_t)blockIdx.y * BN;

    double acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;

    double ra[4], rb[4];
    auto load_regs = [&](int64_t k0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + NT * q;
            int ii, kk;
            if (!TA) { ii = e % BM; kk = e / BM; } else { ii = e / BK; kk = e % BK; }
            const int64_t gi = i0 + ii, gk = k0 + kk;
            double v = 0.0;
            if (gi < M && gk < K) v = TA ? A[gk + gi * lda] : A[gi + gk * lda];
            ra[q] = v;
            int jj;
            if (!TB) { kk = e % BK; jj = e / BK; } else { jj = e % BN; kk = e / BN; }
            const int64_t gj = j0 + jj;
            const int64_t gk2 = k0 + kk;
            double w = 0.0;
            if (gj < N && gk2 < K) w = TB ? B[gj + gk2 * ldb] : B[gk2 + gj * ldb];
            rb[q] = w;
        }
    };
    auto store_smem = [&](int slot) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + NT * q;
            int ii, kk;
            if (!TA) { ii = e % BM; kk = e / BM; } else { ii = e / BK; kk = e % BK; }
            As[slot][kk][ii] = ra[q];
            int jj;
            if (!TB) { kk = e % BK; jj = e / BK; } else { jj = e % BN; kk = e / BN; }
            Bs[slot][kk][jj] = rb[q];
        }
    };

    const int64_t nk = ceil_div(K, BK);
    if (nk > 0) {
        load_regs(0);
        store_smem(0);
    }
    __syncthreads();
    for (int64_t t = 0; t < nk; ++t) {
        const int slot = (int)(t & 1);
        if (t + 1 < nk) load_regs((t + 1) * BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[4], bb[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[slot][kk][ty + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; ++c) bb[c] = Bs[slot][kk][tx + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], bb[c], acc[r][c]);
        }
        if (t + 1 < nk) store_smem(slot ^ 1);
        __syncthreads();
    }

#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t gi = i0 + ty + 16 * r;
        if (gi >= M) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t gj = j0 + tx + 16 * c;
            if (gj >= N) continue;
            double v = alpha * acc[r][c];
            if (beta != 0.0) v = fma(beta, Cin[gi + gj * ldcin], v);
            C[gi + gj * ldc] = v;
        }
    }
}

}  // namespace

int dgemm_batched(bool tA, bool tB, int64_t M, int64_t N, int64_t K, double alpha,
                  const GemmBatch &bt, int nbatch, int64_t lda, int64_t ldb, double beta,
                  int64_t ldcin, int64_t ldc, const DevState *state, cudaStream_t st) {
    if (M < 0 || N < 0 || K < 0 || nbatch < 1 || nbatch > 4) return OMM_ERR_ARG;
    if (M == 0 || N == 0) return OMM_OK;
    dim3 grid((unsigned)ceil_div(M, BM), (unsigned)ceil_div(N, BN), (unsigned)nbatch);
    if (grid.x > 2147483647u || grid.y > 65535u) return OMM_ERR_ARG;
    if (!tA && !tB)
        dgemm_kernel<false, false><<<grid, NT, 0, st>>>(M, N, K, alpha, bt, lda, ldb, beta, ldcin, ldc, state);
    else if (tA && !tB)
        dgemm_kernel<true, false><<<grid, NT, 0, st>>>(M, N, K, alpha, bt, lda, ldb, beta, ldcin, ldc, state);
    else if (!tA && tB)
        dgemm_kernel<false, true><<<grid, NT, 0, st>>>(M, N, K, alpha, bt, lda, ldb, beta, ldcin, ldc, state);
    else
        dgemm_kernel<true, true><<<grid, NT, 0, st>>>(M, N, K, alpha, bt, lda, ldb, beta, ldcin, ldc, state);
    omm::count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

}  // namespace omm

extern "C" int omm_op_dgemm(int32_t transA, int32_t transB, int64_t M, int64_t N, int64_t K,
                            double alpha, const double *A, int64_t lda, const double *B,
                            int64_t ldb, double beta, const double *Cin, int64_t ldcin,
                            double *C, int64_t ldc, void *stream) {
    if (M < 0 || N < 0 || K < 0) return OMM_ERR_ARG;
    if (M == 0 || N == 0) return OMM_OK;
    if (C == nullptr || ldc < M) return OMM_ERR_ARG;
    if (K > 0 && (A == nullptr || B == nullptr)) return OMM_ERR_ARG;
    if (K > 0 && lda < (transA ? K : M)) return OMM_ERR_ARG;
    if (K > 0 && ldb < (transB ? N : K)) return OMM_ERR_ARG;
    if (beta != 0.0 && (Cin == nullptr || ldcin < M)) return OMM_ERR_ARG;
    omm::GemmBatch bt{};
    bt.A[0] = A;
    bt.B[0] = B;
    bt.Cin[0] = Cin;
    bt.C[0] = C;
    return omm::dgemm_batched(transA != 0, transB != 0, M, N, K, alpha, bt, 1, lda, ldb, beta,
                              beta != 0.0 ? ldcin : ldc, ldc, nullptr, (cudaStream_t)stream);
}
