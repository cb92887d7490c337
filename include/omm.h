/*
 * omm.h -- C ABI of the GB300 orbital-minimization (OMM) library.
 *
 * The library minimises the Ordejon-Mauri energy functional
 *     E~(W) = 2 Tr[(2 I - W^T S W) W^T H W]                  (Eq. 4)
 * over the m x n coefficient matrix W (the paper's C) by conjugate gradients
 * with an exact quartic line search (Introduction; section "Solver library").
 * H is the m x m Hamiltonian, S the m x m overlap matrix (both symmetric, S
 * positive definite), n the number of occupied orbitals.  Two forms exist:
 * dense (cubic scaling) and block sparse with a localisation pattern fixed
 * on W (linear scaling, section "Solver library": the gradient is kept on
 * the sparsity pattern of the initial W).
 *
 * Conventions for every entry point:
 *   - dense matrices are column-major; W is m x n with leading dimension m
 *     (orbital j occupies W[j*m .. j*m+m-1], i.e. the paper's C^dagger in
 *     row-major order);
 *   - block-sparse values are stored block after block in the pattern's CSR
 *     order, each block row-major;
 *   - every function returns an int status: OMM_OK (0) or a negative OMM_ERR_*
 *     code; no function aborts the process; on error, outputs are left
 *     untouched unless the description says otherwise;
 *   - the caller owns every pointer it passes; the library copies what it
 *     keeps and never frees caller memory;
 *   - "stream" arguments are cudaStream_t values passed as void*; NULL means
 *     the legacy default stream for op-level calls and a library-owned stream
 *     for handles.  A library-owned stream is non-blocking: device inputs must
 *     be complete before a call that reads them (synchronize the stream that
 *     produced them, or pass that stream in omm_options.stream).
 * A handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef OMM_GB300_H
#define OMM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
enum {
    OMM_OK = 0,
    OMM_ERR_ARG = -1,          /* invalid argument (sizes, NULL pointer, layout) */
    OMM_ERR_NOMEM = -2,        /* device or pinned host allocation failed */
    OMM_ERR_CUDA = -3,         /* a CUDA runtime call failed */
    OMM_ERR_NOT_SPD = -4,      /* S is not positive definite (Cholesky pivot <= 0,
                                  or no Gershgorin lower bound for eta_auto) */
    OMM_ERR_LINESEARCH = -5,   /* the quartic along the search line has no minimum
                                  (section "Recommendations for OMM solver use") */
    OMM_ERR_MAXITER = -6,      /* max_iter CG steps without meeting the tolerance;
                                  W, E and iters still describe the last iterate */
    OMM_ERR_PATTERN = -7,      /* sparsity pattern malformed or inconsistent */
    OMM_ERR_NONFINITE = -8,    /* NaN or Inf in the energy or line-search data */
    OMM_ERR_TIMEOUT = -9,      /* a bounded device-side wait gave up */
    OMM_ERR_STATE = -10,       /* call out of order (e.g. solve before set_HS) */
    OMM_ERR_UNSUPPORTED = -11  /* option combination not available */
};

/* arithmetic of the solve */
enum {
    OMM_PREC_FP64 = 0,   /* every product in FP64 */
    OMM_PREC_MIXED = 1   /* BF16-split tensor-core products for the bulk of the
                            CG, FP64 state, then an accurate refinement sweep */
};

typedef struct omm_handle omm_handle;

/*
 * Block-sparse pattern for the linear-scaling form.  H and S share one
 * pattern of bm x bm blocks; W uses bm x bn blocks (basis atom x orbitals of
 * one host atom).  Block rows index basis atoms; nbr = m / bm; W has nbc =
 * n / bn block columns.  Column indices must be sorted and unique within
 * each block row.  Arrays are host memory, read during omm_create only.
 */
typedef struct {
    int32_t bm, bn;
    int64_t nbr, nbc;
    const int64_t *H_rowptr;   /* nbr + 1 */
    const int32_t *H_col;      /* H_rowptr[nbr] */
    const int64_t *W_rowptr;   /* nbr + 1 */
    const int32_t *W_col;      /* W_rowptr[nbr], values in [0, nbc) */
} omm_pattern;

typedef struct {
    double eta;            /* Kim shift H' = H - eta S (n' = n); used when eta_auto == 0 */
    int32_t eta_auto;      /* 1 (default): eta = Gershgorin upper bound of the spectrum,
                              which makes every line-search quartic bounded below */
    int32_t precision;     /* OMM_PREC_FP64 (default) or OMM_PREC_MIXED (dense only) */
    int32_t cholesky;      /* 1: Cholesky-reduced variant (dense only, either precision):
                              S = L L^T, the CG runs on W~ = L^T W with H~ = L^-1 H' L^-T and
                              overlap I; W_out (and OMM_ARRAY_W after omm_solve_end) is
                              mapped back with W = L^-T W~; the other arrays describe the
                              reduced problem */
    int32_t max_iter;      /* CG step limit, default 10000 */
    double orth_tol;       /* > 0: also require ||W^T S W - I||_F < orth_tol to stop */
    double filter_eps;     /* block filtering threshold, default 1e-8 (sparse form): an
                              input block pair is dropped from the stored H/S pattern
                              when both ||H_b||_F < eps and ||S_b||_F < eps (squares summed
                              in row-major element order, strict comparison) */
    void *stream;          /* cudaStream_t for all work of the handle, NULL = own stream */
    int32_t refine;        /* arithmetic of the mixed form's refinement sweep (re-anchoring
                              and gradient): OMM_REFINE_EXACT (default) or OMM_REFINE_FP64 */
    int32_t exact_digits;  /* digits per operand of the exact-digit products, 1..8, default 7 */
    int32_t split_digits;  /* BF16 digits per operand of the mixed form's split products (the
                              CG increments H'D, SD, the contractions and the first phase's
                              gradient), 2 or 3 (3 digit pairs or 6), default 2: the first
                              phase then stops at RelTol 1e-7 (its increments carry ~1e-5
                              relative error) and the refinement, re-anchored exactly and with
                              an exact-digit gradient, reaches tol; 3 runs the first phase to
                              max(0.1 tol, 1e-12) */
    int32_t graphs;        /* 1 (default): after one eager chunk of CG steps per phase, replay
                              the chunk as a captured CUDA graph (needs a stream other than
                              the legacy default stream; off while profiling); 0: launch
                              every kernel from the host */
    int32_t n_occupied;    /* Kim functional (section "Overview of OMM approaches", steps
                              (1)-(3)): with 0 < n_occupied < n the handle's n columns are
                              n' > n_occupied trial orbitals, the reported energy is
                              E~_eta + 2 eta n_occupied, and eta must be given inside the gap
                              (eta_auto = 0; the Gershgorin bound lies above the spectrum).
                              Start from small coefficients (the functional is unbounded
                              along unoccupied directions beyond a barrier near unit norm) and
                              leave orth_tol at 0: S_W converges to diag(I, 0).  With the
                              mixed form take split_digits = 3: two-digit increments (~1e-5
                              relative error) can carry an iterate across that barrier, after
                              which the solve ends in OMM_ERR_NONFINITE.  0 (default):
                              n_occupied = n */
    int32_t precon;        /* kinetic-energy preconditioning (Eq. 6; dense handles only, not
                              with the Cholesky variant): the CG gradient G is multiplied by
                              P = (S + T / tau_T)^-1 before it forms the search direction and
                              the Polak-Ribiere ratio.  0 (default): off; k > 0: applied in the
                              first k solves after each omm_set_T (the OMM.Precon count of
                              Table 1, counted in solves); < 0: applied in every solve.  T is
                              given with omm_set_T */
    double tau_T;          /* kinetic-energy scale of P, in the energy unit of H; default
                              10 Ry = 136.0569 eV (Table 1, OMM.TPreconScale) */
    double screen_eps;     /* norm-based screening of the block products of the sparse form
                              (the filtered block multiply of the DBCSR library the paper's
                              linear-scaling solver runs on, section "Solver library"): a
                              block product A_ik B_kj of H'W, SW, H'D, SD, W^T(H'W), W^T(SW),
                              W^T(H'D), W^T(SD), D^T(H'D), D^T(SD), (SW) H_W or (H'W) S_W is
                              skipped when ||A_ik||_F ||B_kj||_F < screen_eps (compared as
                              squared norms against screen_eps^2).  Each skipped product
                              changes its output block by less than screen_eps in Frobenius
                              norm; stored patterns never change.  The squared norms of every
                              operand block are kept on the device (about 8 doubles per
                              block of H, W, H'W and W^T H W).  0 (default): off; must be
                              finite and >= 0 (OMM_ERR_ARG); ignored by dense handles */
    int32_t gemm_pair;     /* mixed form: 1 (default) runs the two-digit split products on CTA
                              pairs (tcgen05.mma.cta_group::2: 256 x 256 tiles, each SM of a
                              pair holding half of the B tile); 0: one CTA per 128 x 256 tile.
                              Three-digit products always take one CTA per tile */
    int32_t gemm_persistent; /* mixed form, 1: the step's split products (H'D and SD, the
                              contractions, the first phase's gradient) run as persistent
                              launches over a tile list (152 CTAs, or 76 pairs, each taking
                              every 152nd tile; the next tile's operands load while the last
                              one's results are written); 0 (default): one CTA (or pair) per
                              tile.  The results are the same bits either way */
    int32_t dir_digits;    /* mixed form: BF16 digits of the search direction D.  1
                              (default): the line search and the update run along D
                              rounded to one BF16 digit (8 significant bits), so the split
                              products H'D and SD take one digit of D exactly (2 digit
                              pairs per product in place of 3, or 3 in place of 6 with
                              split_digits = 3) and the D^T rows of the contraction one
                              digit plane; the slope <G, D> of the quartic is taken of the
                              rounded D, and the CG recurrence (beta, the restart test, the
                              next direction) keeps the unrounded direction in a separate
                              FP32 array (4 m n bytes more).  The state W, H'W, SW, H_W, S_W
                              stays consistent to the split products' accuracy and the
                              converged result is held to the same bars.  0: D keeps
                              split_digits digits */
} omm_options;

enum {
    OMM_REFINE_EXACT = 0,  /* exact-digit BF16 tensor-core products (omm_op_exact_gemm) */
    OMM_REFINE_FP64 = 1    /* FP64 CUDA-core products (omm_op_dgemm) */
};

typedef struct {
    double E;              /* energy of the final iterate: E~_eta + 2 eta n, where E~_eta
                              is Eq. 4 with H' (equals E~ with H at the dense minimum) */
    double E_rel_change;   /* last |2 (E_k - E_{k-1}) / (E_k + E_{k-1})| (Table 1, RelTol) */
    double orth;           /* ||W^T S W - I||_F at the final iterate */
    double charge;         /* 2 Tr[(2 I - S_W) S_W] (Listing 1) */
    double eta;            /* shift actually used */
    int32_t iters;         /* CG steps taken in the last solve */
    int32_t status;        /* status of the last solve */
    int32_t iters_mixed;   /* steps taken with split-precision products */
    int32_t iters_refine;  /* steps taken in the accurate refinement sweep */
    double t_setup_ms;     /* device time of the last omm_set_HS */
    double t_solve_ms;     /* device time of the last omm_solve */
    int64_t nnzb_H;        /* stored blocks of H/S after filtering (sparse) */
    int64_t nnzb_W;        /* blocks of W's pattern (sparse) */
    int64_t nnzb_HW;       /* blocks of the structural pattern of H W (sparse) */
    int64_t nnzb_N;        /* blocks of the structural pattern of W^T H W (sparse) */
} omm_diag;

/* Fill *opt with the defaults listed above. */
void omm_default_options(omm_options *opt);

/*
 * Create a solver for an m x n problem.  block_size is the basis block size
 * bm (atom block of H and S); for the dense form it only has to divide
 * nothing and may be 0.  pattern == NULL selects the dense form; otherwise
 * the pattern is validated (OMM_ERR_PATTERN) and copied.  opt == NULL takes
 * the defaults.  All device memory of the handle is allocated here
 * (OMM_ERR_NOMEM on failure).  *out receives the handle on OMM_OK.
 */
int omm_create(int64_t m, int64_t n, int32_t block_size, const omm_pattern *pattern,
               const omm_options *opt, omm_handle **out);

/*
 * Load H and S (section "Solver input and output": H and S are the solver's
 * input at every SCF step).  Dense: column-major m x m arrays (symmetric, so
 * row-major is the same).  Sparse: block values in the pattern's order.
 * on_device != 0: H and S are device pointers; else host pointers.
 * Runs the per-(H,S) setup on the device: the shift H' = H - eta S (with the
 * Gershgorin eta when eta_auto), block filtering (sparse), Cholesky reduction
 * (when selected).  The previous solution W stays resident for warm starts.
 */
int omm_set_HS(omm_handle *h, const double *H, const double *S, int32_t on_device);

/*
 * Replace H only (dense handles): the overlap of the last successful
 * omm_set_HS is kept, and with the Cholesky variant so are its factor L and
 * L^-1, so only the shift, H~ = L^-1 H' L^-T and the packing run.  This is the
 * SCF case where the basis, hence S, is fixed and the Hamiltonian changes
 * between solves.  The result equals omm_set_HS(h, H, S_previous) bit for bit.
 * Returns OMM_ERR_STATE before a successful omm_set_HS or while a solve is in
 * flight, OMM_ERR_UNSUPPORTED for sparse handles.
 */
int omm_set_H(omm_handle *h, const double *H, int32_t on_device);

/*
 * Kinetic-energy matrix T (m x m column-major FP64, symmetric, host or device
 * memory; copied into the handle) of the preconditioner P = (S + T/tau_T)^-1
 * of Eq. 6 (section "Overview of OMM approaches").  P is formed on the GPU at
 * the first preconditioned solve after omm_set_T or a new S (omm_set_HS):
 * Cholesky factor of S + T/tau_T, its inverse Y = L^-1 and P = Y^T Y, with
 * exact-digit tensor-core products; omm_set_H keeps it.  Each CG step then
 * adds one m x m by m x n product Z = P G (FP64 form: FP64 product; mixed
 * form: split product on the FP32 gradient).  Resets the count of
 * preconditioned solves (omm_options.precon > 0).  Returns
 * OMM_ERR_UNSUPPORTED for sparse handles and handles created with precon = 0,
 * OMM_ERR_STATE while a solve is in flight.  A solve with precon != 0 and no T
 * returns OMM_ERR_STATE; S + T/tau_T that is not positive definite makes that
 * solve return OMM_ERR_NOT_SPD.
 */
int omm_set_T(omm_handle *h, const double *T, int32_t on_device);

/*
 * Initial guess of a new MD step (section "C† matrix initialization and
 * update"): the resident W of dst (the warm start of its next solve with
 * W0 == NULL) <- the resident W of prev, the previous MD step's solution,
 * carried onto dst's localisation pattern, or with prev2 != NULL (the step
 * before) the linear extrapolation 2 W_prev - W_prev2 (Table 1,
 * OMM.Extrapolate).  Sparse handles: a W block of dst's pattern that prev does
 * not hold (its atoms came within R_C) is zero; blocks of prev outside dst's
 * pattern (atoms moved apart) are dropped; a block prev2 lacks counts as zero
 * in the extrapolation.  The block maps are merged on the host from the three
 * handles' patterns and the values gathered on the GPU on dst's stream.  Dense
 * handles: W elementwise; the Cholesky variant reads and writes W in the
 * original basis.  dst may be prev or prev2 (dense, or an identical pattern).
 * Synchronous.  OMM_ERR_ARG: NULL dst or prev, or handles of different form,
 * sizes or block shapes; OMM_ERR_STATE: a source without a solution, or a
 * handle with a solve in flight.
 */
int omm_md_guess(omm_handle *dst, omm_handle *prev, omm_handle *prev2);

/*
 * Minimise from W0 (m x n column-major; sparse: 8x2-style block values in the
 * W pattern's order) to the RelTol criterion of Table 1:
 *     |2 (E_k - E_{k-1}) / (E_k + E_{k-1})| < tol   at k >= 1,
 * plus ||S_W - I||_F < orth_tol when orth_tol > 0.  W0 == NULL warm-starts from
 * the resident W of the previous solve (OMM_ERR_STATE if there is none).
 * W_out (nullable) receives the final W in the layout of W0; E_out and
 * iters_out (nullable) receive the energy and the number of CG steps.  On
 * OMM_ERR_MAXITER the outputs describe the last iterate.
 */
int omm_solve(omm_handle *h, const double *W0, int32_t W0_on_device, double tol,
              double *W_out, int32_t W_out_on_device, double *E_out, int32_t *iters_out);

/*
 * The same solve in three non-blocking steps, for drivers that keep several
 * handles busy at once (batched and serving use).  omm_solve_begin enqueues
 * the start-up and a first chunk of CG steps on the handle's stream and
 * returns.  omm_solve_progress checks the chunk (blocking != 0: waits for it);
 * when it has finished it enqueues the next chunk or the next phase
 * (split-precision -> refinement), and sets *done = 1 once the solve is over.
 * omm_solve_end copies W out (as omm_solve) and returns the solve's status.
 * omm_solve(h, ...) is begin + progress(blocking) until done + end.
 */
int omm_solve_begin(omm_handle *h, const double *W0, int32_t W0_on_device, double tol);
int omm_solve_progress(omm_handle *h, int32_t blocking, int32_t *done);
int omm_solve_end(omm_handle *h, double *W_out, int32_t W_out_on_device, double *E_out,
                  int32_t *iters_out);

/*
 * Batched solves: `count` distinct handles (any sizes, forms and options, each
 * after its omm_set_HS) minimised together, each on its own stream so their
 * kernels overlap on the device (independent k-points, spins or systems,
 * section "Recommendations for OMM solver use": spin channels are solved in
 * sequence by the paper; here they run at once).  W0[i] as in omm_solve (W0
 * == NULL or W0[i] == NULL warm-starts); the solutions stay in the handles
 * (omm_get_array).  E_out, iters_out, status_out: arrays of count entries,
 * nullable.  Returns OMM_OK or the first non-OK per-handle status.  Results
 * do not depend on what runs beside them: every reduction has a fixed order.
 */
int omm_batch_solve(omm_handle **handles, int32_t count, const double *const *W0, int32_t W0_on_device,
                    double tol, double *E_out, int32_t *iters_out, int32_t *status_out);

/*
 * The same batch as omm_batch_solve, run as one group (independent systems such
 * as spins, k-points or the uneven systems of a batch; section "Recommendations
 * for OMM solver use").  The first, split-precision phase of every system runs in
 * lock step: each CG step's three split products (H'D and SD, the contractions,
 * the gradient) are each ONE persistent grouped tensor-core launch over the tile
 * lists of all systems (longest K first), while each system's line minimum,
 * updates and direction run on its own stream in between; a chunk of 8 such steps
 * is captured once as a CUDA graph and replayed until every system has left the
 * first phase.  The refinement then runs per system as in omm_batch_solve.
 * tile_mode: 0 one CTA per 128 x 256 tile, 1 CTA pairs (256 x 256 tiles,
 * tcgen05.mma.cta_group::2), -1 autotune: the first call for a group of this
 * shape (the systems' (m, n) in order) times both modes on each of the three
 * products and keeps the faster per product for every later call of the same
 * shape (omm_batch_last_tuning reports the choice).  Every result equals the same
 * solve run alone with omm_solve, bit for bit, whatever the mode.
 * Requirements: dense handles of the mixed form with split_digits = 2, no
 * Cholesky variant, no preconditioning, profiling off, each on its own stream
 * other than the legacy default stream (OMM_ERR_UNSUPPORTED otherwise).
 * Arguments and results as omm_batch_solve; synchronous.
 */
int omm_batch_solve_grouped(omm_handle **handles, int32_t count, const double *const *W0, int32_t W0_on_device,
                            double tol, int32_t tile_mode, double *E_out, int32_t *iters_out, int32_t *status_out);

/*
 * Tile modes of the last omm_batch_solve_grouped call: modes[3] for the products,
 * the contractions and the gradient (0 single CTA, 1 CTA pair); ms[6] (nullable):
 * the autotuner's timed milliseconds per product and mode, 0 when the mode was
 * given or taken from an earlier call.
 */
int omm_batch_last_tuning(int32_t *modes, float *ms);

/* Diagnostics of the last set_HS / solve. */
int omm_get_diag(omm_handle *h, omm_diag *d);

/*
 * Copy one internal m x n or n x n FP64 array of the handle (for inspection
 * and tests).  which: 0 W, 1 H'W, 2 S W, 3 G, 4 D, 5 H_W (n x n), 6 S_W (n x n).
 * dst is host memory unless on_device.  With the Cholesky variant, 0 is W in
 * the original basis (after omm_solve_end) and 1..6 belong to the reduced
 * problem (H~, I, W~).  Sparse handles return the block values of the
 * corresponding patterns.
 */
int omm_get_array(omm_handle *h, int32_t which, double *dst, int32_t on_device);

/*
 * Density matrix (Eq. 5) or energy density (defined with Eq. 6) of the last
 * solve, as an SCF step and the forces consume them:
 *   OMM_DENSITY_RHO    rho   = 2 W (2I - S_W) W^T
 *   OMM_DENSITY_RHO_E  rho_E = 2 W H'_W W^T + eta rho
 * with H' = H - eta S the matrix the functional was minimised for (the Kim
 * construction's step (3); at S_W = I this is 2 W H_W W^T of the unshifted H).
 * W is the solution in the original basis (also for the Cholesky variant);
 * S_W and H'_W are formed afresh from it.  dst: m x m column-major, host
 * unless on_device.  Every product runs as an exact-digit tensor-core GEMM
 * (FP64-accurate).  The first call allocates the handle's workspace for it
 * (about 14 (m + n) m bytes with 7 digits, plus m^2 doubles for host output).
 * Linear-scaling form: rho / rho_E only on the pattern of S (section "Solver
 * library"), i.e. every block of the P_H given to omm_create, as nnzb(P_H)
 * blocks of bm x bm, row-major within a block, in P_H's CSR order; FP64 block
 * kernels over gather lists built at the first request.  OMM_ERR_STATE unless
 * omm_solve / omm_solve_end returned since the last omm_set_HS / omm_set_H.
 */
#define OMM_DENSITY_RHO 0
#define OMM_DENSITY_RHO_E 1
int omm_get_density(omm_handle *h, int32_t which, double *dst, int32_t on_device);

void omm_destroy(omm_handle *h);
const char *omm_status_str(int status);

/*
 * Block patterns of a linear-scaling handle (host block-CSR arrays; rowptr
 * receives nrows + 1 entries, col the entries counted by omm_get_diag's nnzb_*):
 *   OMM_PATTERN_H   stored pattern of H and S after the block filtering of the
 *                   last omm_set_HS (nbr rows);
 *   OMM_PATTERN_W   localisation pattern of W (nbr rows);
 *   OMM_PATTERN_HW  structural pattern of H W, the union over K in row I of H
 *                   of the W rows K (nbr rows) -- where H'W, SW, H'D, SD live;
 *   OMM_PATTERN_N   structural pattern of W^T H W on n x n blocks of bn x bn
 *                   (nbc rows) -- where H_W, S_W and the contractions live.
 * The product patterns follow the pattern given at omm_create; blocks that the
 * filter drops are stored as zeros.
 */
enum { OMM_PATTERN_H = 0, OMM_PATTERN_W = 1, OMM_PATTERN_HW = 2, OMM_PATTERN_N = 3 };
int omm_get_pattern(omm_handle *h, int32_t which, int64_t *rowptr, int32_t *col);

/* Human-readable detail of the last failure on the calling thread (which
 * CUDA call failed and why); empty when none.  Owned by the library. */
const char *omm_last_error(void);

/*
 * Per-stage device timing of a handle.  While profiling is on, the library
 * records CUDA events on the handle's stream around each stage of every CG
 * step; omm_get_stage_times returns the summed milliseconds and the number of
 * timed launches per stage (arrays of nstages entries, nullable), optionally
 * resetting them.  Stages: products H'D, SD (0); n x n contractions (1);
 * line-search coefficients and minimum (2); W/H'W/SW and H_W/S_W update with
 * energy test (3); gradient (4); CG direction (5); per-(H,S) setup (6);
 * solve start-up (7); split-precision operand packing (8); refinement
 * re-anchoring (9); kinetic-energy preconditioner product P G (10).
 */
enum {
    OMM_STAGE_PRODUCTS = 0, OMM_STAGE_CONTRACT = 1, OMM_STAGE_LINESEARCH = 2,
    OMM_STAGE_UPDATE = 3, OMM_STAGE_GRADIENT = 4, OMM_STAGE_DIRECTION = 5,
    OMM_STAGE_SETUP = 6, OMM_STAGE_START = 7, OMM_STAGE_PACK = 8, OMM_STAGE_ANCHOR = 9,
    OMM_STAGE_PRECON = 10, OMM_NSTAGES = 11
};
int omm_set_profiling(omm_handle *h, int32_t on);
int omm_get_stage_times(omm_handle *h, double *ms, int64_t *launches, int32_t nstages,
                        int32_t reset);

/* Total number of CUDA kernels this library has launched in the process. */
int64_t omm_kernel_launches(void);

/*
 * Self-test of the bounded waits.  Every mbarrier wait in the tensor-core
 * kernels gives up at a deadline, records the timeout and unwinds, so that a
 * lost signal ends in OMM_ERR_TIMEOUT from the solve instead of a hung GPU.
 * This call runs one such wait on a barrier that nothing completes, limited
 * to limit_ns (1e3 .. 1e10 ns), on `stream`, and waits for it:
 * *status_out = OMM_ERR_TIMEOUT when the wait gave up (the expected outcome),
 * OMM_OK if the barrier completed.  The CUDA context stays usable.
 * Returns OMM_ERR_ARG for a limit out of range or a NULL status_out.
 */
int omm_selftest_bounded_wait(int64_t limit_ns, int32_t *status_out, void *stream);

/* ------------------------------------------------------------------------
 * Op-level entry points: single steps of the hot path on caller-owned device
 * memory, enqueued on `stream`, asynchronous.  They allocate nothing.
 * ---------------------------------------------------------------------- */

/*
 * FP64 GEMM  C = alpha op(A) op(B) + beta Cin  (the products H D, S D, W^T H D,
 * S W H_W + H W S_W of the CG step, section "Solver library").  Column-major;
 * op(X) = X or X^T (trans != 0); M, N, K >= 0; leading dimensions >= the
 * stored row counts.  Cin may equal C; beta == 0 ignores Cin.
 */
int omm_op_dgemm(int32_t transA, int32_t transB, int64_t M, int64_t N, int64_t K,
                 double alpha, const double *A, int64_t lda, const double *B, int64_t ldb,
                 double beta, const double *Cin, int64_t ldcin, double *C, int64_t ldc,
                 void *stream);

/*
 * Coefficients c[0..4] of the line-search quartic E~_eta(W + x D) (Introduction:
 * the quartic's parameters are computed analytically), from the n x n blocks
 *   h0 = W^T H' W, s0 = W^T S W, X = W^T H' D, Y = W^T S D, h2 = D^T H' D, s2 = D^T S D:
 *   c0 = 2 [2 tr h0 - <s0,h0>]
 *   c1 = 2 [4 tr X - 2 <s0,X> - 2 <Y,h0>]
 *   c2 = 2 [2 tr h2 - <s0,h2> - 2 <Y,X> - 2 <Y,X^T> - <s2,h0>]
 *   c3 = 2 [-2 <Y,h2> - 2 <s2,X>]
 *   c4 = -2 <s2,h2>
 * (<A,B> = sum_ij A_ij B_ij; h0, s0, h2, s2 symmetric).  All six inputs are
 * device n x n column-major arrays with leading dimensions ld_h (h0, s0) and
 * ld_z (X, Y, h2, s2).  coeffs: 5 doubles of device memory.  scratch: device
 * memory of at least omm_op_quartic_coeffs_scratch_bytes(n) bytes, 16-byte
 * aligned, holding per-block partial sums and a completion counter that must
 * be zero on entry (cudaMemset once; the kernel leaves it zero again).
 * Reduction order is fixed: equal inputs give bitwise equal coefficients.
 */
int64_t omm_op_quartic_coeffs_scratch_bytes(int64_t n);
int omm_op_quartic_coeffs(int64_t n, const double *h0, const double *s0, int64_t ld_h,
                          const double *X, const double *Y, const double *h2,
                          const double *s2, int64_t ld_z, double *coeffs, void *scratch,
                          int64_t scratch_bytes, void *stream);

/*
 * omm_op_quartic_coeffs without caller-provided scratch, for callers that
 * cannot allocate device memory (the paper has no counterpart: libOMM runs on
 * CPUs).  Same inputs, output and reduction order as omm_op_quartic_coeffs;
 * the scratch is a static device array of omm_op_quartic_coeffs_static_max_bytes()
 * bytes (53,504) held by every GPU that loads the library until the process
 * exits.  The kernel never launches more blocks than that array has partial
 * slots for, so every n in [0, 2^31 - 1] fits; n outside that range, a NULL
 * input or output, or ld_h, ld_z < n is rejected with OMM_ERR_ARG and a
 * message in omm_last_error().  Every call looks up the array's device address
 * with the current device; the first call on a device (and the first after a
 * device reset moved the array) also zeroes its completion counter and
 * synchronises the device, so make that first call before any stream capture.
 * All calls share the one array
 * and the kernel leaves the counter at zero for the next call: calls that may
 * overlap on the GPU (different streams, other host threads) race and must be
 * serialised by the caller.  Allocates nothing.
 */
int64_t omm_op_quartic_coeffs_static_max_bytes(void);
int omm_op_quartic_coeffs_static(int64_t n, const double *h0, const double *s0, int64_t ld_h,
                                 const double *X, const double *Y, const double *h2,
                                 const double *s2, int64_t ld_z, double *coeffs, void *stream);

/*
 * Minimiser x of c0 + c1 x + ... + c4 x^4 (device coeffs, 5 doubles) into
 * *x_out (device double) and a status (device int32: OMM_OK, OMM_ERR_LINESEARCH
 * when the quartic has no minimum, OMM_ERR_NONFINITE).  Candidates are the
 * real roots of the derivative with positive curvature; the lowest value
 * wins, ties go to the smaller |x|, then to x > 0.
 */
int omm_op_line_min(const double *coeffs, double *x_out, int32_t *status_out, void *stream);

/*
 * The integer-pipe conversions the solve's kernels inline (FP64 conversions
 * issue on the narrow FP64 unit of this part), element by element over device
 * arrays, so that each can be compared with the hardware conversion.  The
 * paper has no counterpart; this is a self-test of the arithmetic of the mixed
 * form.  op:
 *   0  in double[n] -> out float[n]: round to nearest even; |x| < 2^-126 gives a
 *      signed zero, overflow an infinity, NaN a quiet NaN;
 *   1  in float[n] -> out double[n]: exact (subnormals included);
 *   2  in int64[n], e int32[n] -> out double[n] = in * 2^e rounded to nearest
 *      even (the caller keeps the result normal);
 *   3  in double[n], e int32[n] -> out double[n] = in * 2^e (exact when the
 *      result is normal; otherwise as ldexp).
 * Asynchronous on `stream`; OMM_ERR_ARG for op outside 0..3, n < 0 or a NULL
 * array (e is read only by ops 2 and 3).
 */
int omm_op_convert(int32_t op, int64_t n, const void *in, const int32_t *e, void *out, void *stream);

/*
 * Split-precision tensor-core GEMM  C = alpha op(A) op(B) + beta Cin  (FP64 in
 * and out, column-major, op as in omm_op_dgemm).  Each operand is split into
 * ndigits BF16 digits (x = d1 + d2 + d3 + rest, d1 = bf16(x), d2 = bf16(x - d1),
 * ...), the digit products with p + q <= ndigits + 1 run on the tcgen05 tensor
 * cores with FP32 accumulation, and the epilogue forms the FP64 result.
 * ndigits = 3 gives FP32-level accuracy (about 1e-7 of |A| |B|), 2 about
 * 1e-5, 1 plain BF16.  This is the arithmetic of the bulk CG products of the
 * mixed-precision form.  workspace: device memory of at least
 * omm_op_split_gemm_workspace_bytes(M, N, K, ndigits) bytes (digit planes).
 */
int64_t omm_op_split_gemm_workspace_bytes(int64_t M, int64_t N, int64_t K, int32_t ndigits);
int omm_op_split_gemm(int32_t transA, int32_t transB, int64_t M, int64_t N, int64_t K,
                      int32_t ndigits, double alpha, const double *A, int64_t lda,
                      const double *B, int64_t ldb, double beta, const double *Cin,
                      int64_t ldcin, double *C, int64_t ldc, void *workspace,
                      int64_t workspace_bytes, void *stream);

/*
 * Exact-digit tensor-core GEMM  C = alpha op(A) op(B) + beta Cin  (FP64 in and
 * out, column-major, op as in omm_op_dgemm), accurate to about 2^-(7 ndigits - 6)
 * of (max_k |op(A)_ik|)(max_k |op(B)_kj|) sqrt(K).  Each row of op(A) and column of
 * op(B) is scaled by a power of two into (-1, 1) and cut into ndigits
 * fixed-point digits of at most 64 in magnitude (error-free splitting after
 * Ozaki, Ogita, Oishi & Rump 2012); every digit-pair product is accumulated
 * exactly in FP32 on the tcgen05 tensor cores over K chunks of <= 4096, summed
 * exactly in integers per weight level and combined in FP64.  It gives the
 * mixed-precision form its accurate re-anchoring and refinement gradient.
 * ndigits 1..8 (7 in the solver: 28 digit pairs).  workspace: device memory of
 * at least omm_op_exact_gemm_workspace_bytes(M, N, K, ndigits) bytes.
 */
int64_t omm_op_exact_gemm_workspace_bytes(int64_t M, int64_t N, int64_t K, int32_t ndigits);
int omm_op_exact_gemm(int32_t transA, int32_t transB, int64_t M, int64_t N, int64_t K,
                      int32_t ndigits, double alpha, const double *A, int64_t lda,
                      const double *B, int64_t ldb, double beta, const double *Cin,
                      int64_t ldcin, double *C, int64_t ldc, void *workspace,
                      int64_t workspace_bytes, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* OMM_GB300_H */
