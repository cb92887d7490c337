// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/omm.h"

namespace omm {

// process-wide count of kernels launched by the library (host side)
int64_t launch_count();
void count_launch(int64_t k = 1);

// thread-local description of the last failure (omm_last_error)
void set_error(const char *fmt, ...);

#define OMM_CUDA_TRY(expr)                                                              \
    do {                                                                                \
        cudaError_t e_ = (expr);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            ::omm::set_error("%s:%d: %s -> %s", __FILE__, __LINE__, #expr,              \
                             cudaGetErrorString(e_));                                   \
            return OMM_ERR_CUDA;                                                        \
        }                                                                               \
    } while (0)

// Device-resident CG state of one solve.  Kernels of an iteration read `done`
// first and return at once when it is set, so a launched chunk of iterations
// finishes as no-ops after convergence.
struct DevState {
    int k;              // CG steps taken
    int done;           // 1 once converged or failed
    int status;         // OMM_OK or OMM_ERR_*
    int max_iter;
    int n;
    int restart;        // D = -G at the next direction update
    double tol, orth_tol, eta;
    double E, E_prev, rel;       // E_k, E_{k-1}, last relative change
    double x;                    // current step length
    double c[5];                 // quartic coefficients
    double gg, gg_prev, ggp, gd; // <G,G>, <Gp,Gp>, <G,Gp>, <G,D_old>
    double beta;
    double trh0, sh, orth2;      // tr h0, <s0,h0>, ||s0 - I||_F^2
    double charge;
    int wait_timeout;            // set by a tensor-core kernel whose bounded wait gave up
    double gD;                   // <G, D> of the current direction (= c1 / 2)
    double E_next;               // energy at the line minimum, from the quartic
    double e_shift;              // constant of the reported energy: 2 eta n_occ
    float x_f, beta_f;           // x and beta rounded once for the FP32 kernels
    int done_upd;                // done as the mixed form's line minimum left it: the m x n update
                                 // reads this copy, since the n x n update (run beside it) may set
                                 // done when the step converges
};

// -------- FP64 GEMM (dense_fp64.cu)
struct GemmBatch {
    const double *A[4];
    const double *B[4];
    const double *Cin[4];
    double *C[4];
};

// C_b = alpha op(A_b) op(B_b) + beta Cin_b for b < nbatch; column-major.
// If `state` is non-null the kernel returns at once when state->done is set.
int dgemm_batched(bool tA, bool tB, int64_t M, int64_t N, int64_t K, double alpha,
                  const GemmBatch &bt, int nbatch, int64_t lda, int64_t ldb, double beta,
                  int64_t ldcin, int64_t ldc, const DevState *state, cudaStream_t st);

// K for the density matrices (omm_get_density): 2I - S_W, or H'_W + eta (2I - S_W)
int launch_density_K(int64_t n, const double *h0s0, double eta, int mode, double *K, cudaStream_t st);

// -------- reductions and CG updates (cg_kernels.cu)
constexpr int kRedBlocksMax = 512;
constexpr int kRedSlots = 16;

int64_t red_scratch_bytes();

// coefficients + line minimum into state (x, c, status/done on failure)
int launch_coeffs_linemin(int n, const double *h0, const double *s0, int64_t ldh, const double *Z,
                          int64_t ldz, double *scratch, unsigned int *counter, DevState *state,
                          double *coeffs_out, cudaStream_t st, bool do_linemin);

// Optional BF16 digit output of an elementwise kernel: planes of `plane`
// elements, digit row stride `ld`; ptr == nullptr disables it.
struct DigitOut {
    void *ptr;
    int64_t ld;
    int64_t plane;
    int nd = 3;   // planes written (the consumer's digit count, 2 or 3)
};

// W += x D, HW += x HD, SW += x SD  (three m x n arrays, ld = m), optionally
// writing the digits of W (columns) and of the rows of [SW | HW]
int launch_update(int64_t m, int64_t n, double *W, const double *D, double *HW, const double *HD, double *SW,
                  const double *SD, const DevState *state, DigitOut wd, DigitOut swhw, cudaStream_t st);

// h0 += x (X + X^T) + x^2 sym(h2); s0 likewise; then energy, orthonormality,
// convergence test (mode 0), or initial symmetrisation + energy (mode 1).
int launch_nn_update_energy(int n, double *h0, double *s0, int64_t ldh, const double *Z,
                            int64_t ldz, double *scratch, unsigned int *counter, DevState *state,
                            int mode, cudaStream_t st, DigitOut hsw = DigitOut{nullptr, 0, 0});

// <Z,G>, <Z,Gp>, <G,D> then beta (PR+) and the restart decision; Z = P G is the
// preconditioned gradient (Z = G without preconditioning)
int launch_dots_beta(int64_t mn, const double *G, const double *Zg, const double *Gp, const double *D,
                     double *scratch, unsigned int *counter, DevState *state, int first,
                     cudaStream_t st);

// D = -Z + beta D (or -Z on restart); Gp = G; optionally the digits of D (columns)
int launch_direction(int64_t m, int64_t n, const double *G, const double *Zg, double *Gp, double *D,
                     const DevState *state, cudaStream_t st, DigitOut dd = DigitOut{nullptr, 0, 0});

// MD-step guess: Wd block b <- W1 block i1[b], or 2 W1[i1[b]] - W2[i2[b]] with
// W2 given (a negative index reads zero; i1[b] < 0 makes the block zero).
// Blocks of blk doubles; i1 = i2 = nullptr means the identity map.
int launch_md_guess(int64_t nblk, int blk, double *Wd, const double *W1, const int64_t *i1, const double *W2,
                    const int64_t *i2, cudaStream_t st);

// H' = H - eta S (dense, m x m), eta read from state
int launch_shift(int64_t mm, const double *H, const double *S, double *Hs, const DevState *state,
                 cudaStream_t st);

// Gershgorin bound into state->eta (dense, column-major m x m, symmetric)
int launch_gershgorin(int64_t m, const double *H, const double *S, double *scratch,
                      unsigned int *counter, DevState *state, cudaStream_t st);

// -------- FP32-glue kernels of the mixed form (mixed_kernels.cu).  The FP64
// state (W, H'W, SW, H_W, S_W) is updated from FP32 increments; the search
// direction, gradient and products are FP32 (see mixed_kernels.cu).
// slope / nslope: the per-block parts of <G, D> left by mx_direction (round1),
// summed for c1; nslope = 0 takes state->gD from the dots kernel
int mx_coeffs_linemin(int n, const double *h0, const double *s0, int64_t ldh, const float *Z, int64_t ldz,
                      double *scratch, unsigned int *counter, DevState *state, const double *slope, int nslope,
                      cudaStream_t st);
int mx_update(int64_t m, int64_t n, double *W, const float *D, double *HW, const float *HD, double *SW,
              const float *SD, const DevState *state, DigitOut wd, DigitOut swhw, cudaStream_t st);
int mx_nn_update(int n, double *h0, double *s0, int64_t ldh, const float *Z, int64_t ldz, double *scratch,
                 unsigned int *counter, DevState *state, DigitOut hsw, cudaStream_t st);
// Zg: the preconditioned gradient P G, or nullptr (Z = G)
int mx_dots_beta(int64_t mn, const float *G, const float *Zg, const float *Gp, const float *D, double *scratch,
                 unsigned int *counter, DevState *state, int first, cudaStream_t st);
// Df: the CG recurrence's direction, updated in place.  round1: D receives Df
// rounded to one BF16 digit (the search direction; its digits to dd) and each
// block's part of <G, D> goes to slope[block] (*slope_blocks of them, at most
// kRedBlocksMax), for mx_coeffs_linemin; otherwise D is ignored, Df is the
// search direction and *slope_blocks = 0.
int mx_direction(int64_t m, int64_t n, const float *G, const float *Zg, float *Gp, float *Df, float *D,
                 DevState *state, DigitOut dd, bool round1, double *slope, int *slope_blocks, cudaStream_t st);
// mx_dots_beta and mx_direction in one cooperative launch with a grid barrier
// (m % 4 == 0, 16-byte aligned arrays): the same dots, beta, restart test and
// direction.  bar: two zeroed words kept for the handle (arrival count and
// generation of the grid barrier).  OMM_ERR_UNSUPPORTED when the form does not
// apply (the caller then launches the two kernels).
int mx_dots_direction(int64_t m, int64_t n, const float *G, const float *Zg, float *Gp, float *Df, float *D,
                      DevState *state, DigitOut dd, bool round1, double *slope, int *slope_blocks, double *scratch,
                      unsigned int *bar, int first, cudaStream_t st);
// digits of an FP32 m x n column-major array: column j -> row j of the planes
int mx_digits(int64_t m, int64_t n, const float *A, const DevState *state, DigitOut dd, cudaStream_t st);
int mx_round(int64_t count, const double *src, float *dst, const DevState *state, cudaStream_t st);

__device__ __host__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace omm
