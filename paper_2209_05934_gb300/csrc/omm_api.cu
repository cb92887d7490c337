// Solver handle of the C ABI: device memory, the per-(H,S) setup and the
// device-resident CG loop of the dense form.
//
// Layout in HBM (all column-major FP64, m basis functions, n orbitals):
//   HS   m x 2m   [H' | S]         (shifted Hamiltonian next to the overlap)
//   WD   m x 2n   [W  | D]         (iterate and search direction side by side)
//   HDSD m x 2n   [H'D | S D]
//   SWHW m x 2n   [S W | H'W]
//   h0s0 2n x n   [H_W ; S_W]      (stacked, ld 2n)
//   Z    2n x 2n  [W D]^T [H'D S D] = [[X, Y], [h2, s2]]
//   G, Gp m x n
// The side-by-side layouts turn each step into one GEMM: the two products
// H'D and SD share D; the four n x n contractions are [W D]^T [H'D SD]; the
// gradient is 4 H'W - 2 [SW H'W] [H_W ; S_W].
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <mutex>
#include <vector>

#include "chol.cuh"
#include "omm_internal.cuh"
#include "sparse.cuh"
#include "tc_exact.cuh"
#include "tc_gemm.cuh"

// Mixed-precision buffers: BF16 digit planes (three digits, K-major) of the
// operands of the split tensor-core products, and their TMA descriptors.
//   HSd   [3][2m][ldm]   columns of [H' | S] (= rows, symmetric)   A of H'D, SD
//   WDd   [3][2n][ldm]   columns of [W | D]                         A of Z; B of H'D, SD
//   HDSDd [3][2n][ldm]   columns of [H'D | SD]                      B of Z
//   SWHWd [3][m][ld2n]   rows of [SW | H'W]                         A of the gradient
//   HSWd  [3][n][ld2n]   columns of [H_W ; S_W]                     B of the gradient
// FP32 increments of the mixed form (column-major): HDSD32 = [H'D | SD] (m x 2n),
// Z32 = [[X, Y], [h2, s2]] (2n x 2n), G32, Gp32, D32 (m x n).
// Kinetic-energy preconditioning: Pd [3][m][ldm] columns of P (= rows) as the A
// operand and Gd [3][n][ldm] columns of G as the B operand of P G -> PG32 (m x n).
struct MixedBufs {
    int64_t ldm = 0, ld2n = 0;
    int bk = 32;   // K-block width of the split products: 64 (128-byte swizzle) with two digits, else 32
    __nv_bfloat16 *HSd = nullptr, *WDd = nullptr, *HDSDd = nullptr, *SWHWd = nullptr, *HSWd = nullptr;
    CUtensorMap mapHS_A, mapWD_A, mapWD_B, mapHDSD_B, mapSWHW_A, mapHSW_B;
    // the B operands again with 128-row boxes: half of a 256-wide tile per CTA of a pair
    CUtensorMap mapHDSD_H, mapHSW_H, mapG_H;
    float *HDSD32 = nullptr, *Z32 = nullptr, *G32 = nullptr, *Gp32 = nullptr, *D32 = nullptr;
    float *Df32 = nullptr;   // unrounded CG direction (dir_digits = 1; D32 is its one-digit rounding)
    __nv_bfloat16 *Pd = nullptr, *Gd = nullptr;
    CUtensorMap mapP_A, mapG_B;
    float *PG32 = nullptr;
};

// Exact-digit operands of the refinement sweep (s digits, row-scaled), each
// with its per-row exponents:
//   HSx   [s][2m][ldm]  columns of [H' | S]     A of the anchor H'W, SW
//   Wx    [s][n][ldm]   columns of W            B of the anchor; A of H_W, S_W
//   HWSWx [s][2n][ldm]  columns of [H'W | SW]   B of H_W, S_W
//   SWHWx [s][m][ld2n]  rows of [SW | H'W]      A of the gradient
//   HSWx  [s][n][ld2n]  columns of [H_W ; S_W]  B of the gradient
struct ExactBufs {
    int s = 0;
    __nv_bfloat16 *HSx = nullptr, *Wx = nullptr, *HWSWx = nullptr, *SWHWx = nullptr, *HSWx = nullptr;
    int *e = nullptr;   // exponents: [2m HS | n W | 2n HWSW | m SWHW | n HSW]
    int *eHS = nullptr, *eW = nullptr, *eHWSW = nullptr, *eSWHW = nullptr, *eHSW = nullptr;
    CUtensorMap mapHS_A, mapW, mapHWSW_B, mapSWHW_A, mapHSW_B;
};

// Device copy of a persistent tile list (one problem) of a handle's split product.
struct HandleList {
    omm::tc::TileProblem *probs = nullptr;
    omm::tc::TileRef *tiles = nullptr;
    int ntiles = 0;
};

struct omm_handle {
    int64_t m = 0, n = 0;
    int32_t bm = 0;
    bool sparse = false;
    omm_options opt{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    double *HS = nullptr, *WD = nullptr, *HDSD = nullptr, *SWHW = nullptr;
    double *h0s0 = nullptr, *Z = nullptr, *G = nullptr, *Gp = nullptr;
    double *scratch = nullptr;
    unsigned int *counters = nullptr;
    omm::DevState *dstate = nullptr;
    omm::DevState *hstate = nullptr;   // pinned
    bool have_HS = false, have_W = false;
    bool have_S = false;      // a successful dense setup left S (and the Cholesky factor) in place
    bool solved = false;      // omm_solve_end has returned a solution for the current H, S
    // density matrices (omm_get_density): K (n x n), T = W K (m x n), the
    // exact-digit GEMM workspace and, for host output, an m x m staging array
    double *dK = nullptr, *dT = nullptr, *dOut = nullptr;
    void *dWs = nullptr;
    int64_t dWs_bytes = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    omm_diag diag{};
    int chunk = 8;
    int cur_dig = 3;          // digits of the split products of the current phase
    int slope_blocks = 0;     // per-block slope parts the last mixed direction left in slot 3
    // one CUDA graph per phase for the chunk of CG steps, captured after one
    // eager chunk of that phase (modules loaded, kernel attributes set)
    static constexpr int kPhases = 7;
    cudaGraphExec_t graph[kPhases] = {};
    int64_t graph_kernels[kPhases] = {};
    int graph_eager[kPhases] = {};
    MixedBufs mx;
    ExactBufs ex;
    HandleList lists[3];      // persistent tile lists of the step's split products (gemm_persistent)
    double *L = nullptr;      // Cholesky variant: factor of S (m x m)
    double *Wsave = nullptr;  // Cholesky variant: W in the original basis (m x n)
    double *S0 = nullptr;     // Cholesky variant: the original S (its slot holds I)
    omm::chol::Work cw;       // Cholesky variant and preconditioner: GEMM workspace and L^-1
    // kinetic-energy preconditioning (Eq. 6): T as given, P = (S + T/tau)^-1 and
    // the preconditioned gradient P G (m x n)
    double *Tk = nullptr, *P = nullptr, *PG = nullptr;
    bool have_T = false;      // omm_set_T has run
    bool p_ready = false;     // P matches the current S and T
    bool precon_on = false;   // the current solve applies P
    bool graph_precon = false;  // precon_on of the captured chunk graphs
    int precon_left = 0;      // preconditioned solves left (omm_options.precon > 0)
    int phase = 0;            // PH_* of the asynchronous driver
    int k_mixed = 0;          // CG steps of the split-precision phase
    int status = OMM_OK;      // status of the finished solve
    double tol_target = 0.0;
    cudaEvent_t ev_poll = nullptr;
    // second stream of the mixed form: H_W, S_W updates run beside the m x n updates
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool grouped = false;     // inside omm_batch_solve_grouped's lock-step phase
    omm::sp::Host sh;   // linear-scaling form: patterns and gather lists (host)
    omm::sp::Dev sd;    // linear-scaling form: device arrays
    // optional per-stage device timing (omm_set_profiling)
    bool profiling = false;
    static constexpr int kMaxEv = 2048;
    cudaEvent_t evs[kMaxEv] = {};
    int ev_stage[kMaxEv / 2] = {};
    int nev = 0;
    double stage_ms[OMM_NSTAGES] = {};
    int64_t stage_launches[OMM_NSTAGES] = {};
};

namespace {

template <class T>
int dalloc(T **p, size_t count) {
    if (count == 0) count = 1;
    if (cudaMalloc((void **)p, count * sizeof(T)) != cudaSuccess) {
        *p = nullptr;
        return OMM_ERR_NOMEM;
    }
    return OMM_OK;
}

void free_handle(omm_handle *h) {
    if (h == nullptr) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (int i = 0; i < omm_handle::kPhases; ++i)
        if (h->graph[i]) cudaGraphExecDestroy(h->graph[i]);
    for (int i = 0; i < omm_handle::kMaxEv; ++i)
        if (h->evs[i]) cudaEventDestroy(h->evs[i]);
    cudaFree(h->HS);
    cudaFree(h->WD);
    cudaFree(h->HDSD);
    cudaFree(h->SWHW);
    cudaFree(h->h0s0);
    cudaFree(h->Z);
    cudaFree(h->G);
    cudaFree(h->Gp);
    cudaFree(h->scratch);
    cudaFree(h->counters);
    cudaFree(h->dstate);
    cudaFree(h->mx.HSd);
    cudaFree(h->mx.WDd);
    cudaFree(h->mx.HDSDd);
    cudaFree(h->mx.SWHWd);
    cudaFree(h->mx.HSWd);
    cudaFree(h->mx.HDSD32);
    cudaFree(h->mx.Z32);
    cudaFree(h->mx.G32);
    cudaFree(h->mx.Gp32);
    cudaFree(h->mx.D32);
    cudaFree(h->mx.Df32);
    cudaFree(h->ex.HSx);
    cudaFree(h->ex.Wx);
    cudaFree(h->ex.HWSWx);
    cudaFree(h->ex.SWHWx);
    cudaFree(h->ex.HSWx);
    cudaFree(h->ex.e);
    cudaFree(h->L);
    cudaFree(h->Wsave);
    cudaFree(h->S0);
    cudaFree(h->cw.ws);
    cudaFree(h->cw.Linv);
    cudaFree(h->dK);
    cudaFree(h->dT);
    cudaFree(h->dOut);
    cudaFree(h->dWs);
    cudaFree(h->Tk);
    cudaFree(h->P);
    cudaFree(h->PG);
    cudaFree(h->mx.Pd);
    cudaFree(h->mx.Gd);
    cudaFree(h->mx.PG32);
    for (auto &L : h->lists) {
        cudaFree(L.probs);
        cudaFree(L.tiles);
    }
    omm::sp::release(h->sd);
    if (h->hstate) cudaFreeHost(h->hstate);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->ev_poll) cudaEventDestroy(h->ev_poll);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->aux) cudaStreamDestroy(h->aux);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

#define TRY(expr)                       \
    do {                                \
        int rc_ = (expr);               \
        if (rc_ != OMM_OK) return rc_;  \
    } while (0)

// Stage timing: events around each stage launch while profiling is on;
// harvested (summed per stage) at every host synchronisation point.
struct StageTimer {
    omm_handle *h;
    int stage;
    int slot = -1;
    StageTimer(omm_handle *h_, int stage_) : h(h_), stage(stage_) {
        if (!h->profiling || h->nev + 2 > omm_handle::kMaxEv) return;
        // a CG-step stage enqueued after the solve finished (the rest of a chunk)
        // returns at once on the device: it is neither timed nor counted, so the
        // per-launch averages hold real launches only (profiling waits on the
        // stream here; its stage times are device events)
        if (stage <= OMM_STAGE_DIRECTION || stage == OMM_STAGE_PRECON) {
            int dn = 0;
            if (cudaMemcpyAsync(&dn, &h->dstate->done, sizeof(int), cudaMemcpyDeviceToHost, h->stream) ==
                    cudaSuccess &&
                cudaStreamSynchronize(h->stream) == cudaSuccess && dn != 0)
                return;
        }
        slot = h->nev;
        h->nev += 2;
        for (int i = 0; i < 2; ++i)
            if (!h->evs[slot + i]) cudaEventCreate(&h->evs[slot + i]);
        h->ev_stage[slot / 2] = stage;
        cudaEventRecord(h->evs[slot], h->stream);
    }
    ~StageTimer() {
        if (slot >= 0) cudaEventRecord(h->evs[slot + 1], h->stream);
    }
};

void harvest_stage_times(omm_handle *h) {
    for (int e = 0; e + 1 < h->nev; e += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->evs[e], h->evs[e + 1]) == cudaSuccess) {
            h->stage_ms[h->ev_stage[e / 2]] += ms;
            h->stage_launches[h->ev_stage[e / 2]] += 1;
        }
    }
    h->nev = 0;
}

// counters: 0 coeffs, 1 nn update, 2 dots, 3 gershgorin, 4 grid barrier (count, generation)
unsigned int *ctr(omm_handle *h, int i) { return h->counters + 64 * i; }
unsigned int *grid_bar(omm_handle *h) { return ctr(h, 4); }
double *scr(omm_handle *h, int i) {
    return h->scratch + (int64_t)i * omm::kRedBlocksMax * omm::kRedSlots;
}

// One CG step of the dense FP64 form (products, contractions, line search,
// update, energy + convergence, gradient, direction).
// Cholesky variant: the overlap of the reduced problem is I, so S D = D and
// S W = W are copies, not products.
bool s_identity(const omm_handle *h) { return h->opt.cholesky != 0 && !h->sparse; }

// electron pairs counted in the energy's 2 eta n_occ term: n, or fewer with the
// Kim functional's extra columns
int64_t n_occ(const omm_handle *h) { return h->opt.n_occupied > 0 ? h->opt.n_occupied : h->n; }

// CG dots, beta and direction of the dense FP64 form; with the kinetic-energy
// preconditioner the gradient is first multiplied by P (Eq. 6): Z = P G.
int dense_direction(omm_handle *h, int first) {
    const int64_t m = h->m, n = h->n, mn = m * n;
    cudaStream_t st = h->stream;
    const double *Zg = h->G;
    if (h->precon_on) {
        StageTimer t(h, OMM_STAGE_PRECON);
        omm::GemmBatch p{};
        p.A[0] = h->P; p.B[0] = h->G; p.C[0] = h->PG; p.Cin[0] = nullptr;
        TRY(omm::dgemm_batched(false, false, m, n, m, 1.0, p, 1, m, m, 0.0, m, m, h->dstate, st));
        Zg = h->PG;
    }
    StageTimer t(h, OMM_STAGE_DIRECTION);
    TRY(omm::launch_dots_beta(mn, h->G, Zg, h->Gp, h->WD + mn, scr(h, 2), ctr(h, 2), h->dstate, first, st));
    return omm::launch_direction(m, n, h->G, Zg, h->Gp, h->WD + mn, h->dstate, st);
}

int dense_iteration(omm_handle *h) {
    const int64_t m = h->m, n = h->n, mn = m * n;
    cudaStream_t st = h->stream;
    omm::DevState *s = h->dstate;
    omm::GemmBatch b{};
    // H'D and S D
    b.A[0] = h->HS;          b.B[0] = h->WD + mn; b.C[0] = h->HDSD;      b.Cin[0] = nullptr;
    b.A[1] = h->HS + m * m;  b.B[1] = h->WD + mn; b.C[1] = h->HDSD + mn; b.Cin[1] = nullptr;
    {
        StageTimer t(h, OMM_STAGE_PRODUCTS);
        TRY(omm::dgemm_batched(false, false, m, n, m, 1.0, b, s_identity(h) ? 1 : 2, m, m, 0.0, m, m, s, st));
        if (s_identity(h))
            OMM_CUDA_TRY(cudaMemcpyAsync(h->HDSD + mn, h->WD + mn, mn * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    // Z = [W D]^T [H'D SD]
    omm::GemmBatch z{};
    z.A[0] = h->WD; z.B[0] = h->HDSD; z.C[0] = h->Z;
    { StageTimer t(h, OMM_STAGE_CONTRACT); TRY(omm::dgemm_batched(true, false, 2 * n, 2 * n, m, 1.0, z, 1, m, m, 0.0, 2 * n, 2 * n, s, st)); }
    // quartic coefficients and its minimum
    { StageTimer t(h, OMM_STAGE_LINESEARCH);
      TRY(omm::launch_coeffs_linemin((int)n, h->h0s0, h->h0s0 + n, 2 * n, h->Z, 2 * n, scr(h, 0),
                                     ctr(h, 0), s, nullptr, st, true)); }
    // W += x D, H'W += x H'D, SW += x SD; then H_W, S_W update, energy, RelTol test
    { StageTimer t(h, OMM_STAGE_UPDATE);
      TRY(omm::launch_update(m, n, h->WD, h->WD + mn, h->SWHW + mn, h->HDSD, h->SWHW, h->HDSD + mn, s,
                             omm::DigitOut{nullptr, 0, 0}, omm::DigitOut{nullptr, 0, 0}, st));
      TRY(omm::launch_nn_update_energy((int)n, h->h0s0, h->h0s0 + n, 2 * n, h->Z, 2 * n, scr(h, 1),
                                       ctr(h, 1), s, 0, st)); }
    // G = 4 H'W - 2 [SW H'W][H_W ; S_W]
    omm::GemmBatch g{};
    g.A[0] = h->SWHW; g.B[0] = h->h0s0; g.Cin[0] = h->SWHW + mn; g.C[0] = h->G;
    { StageTimer t(h, OMM_STAGE_GRADIENT); TRY(omm::dgemm_batched(false, false, m, n, 2 * n, -2.0, g, 1, m, 2 * n, 4.0, m, m, s, st)); }
    return dense_direction(h, 0);
}

int dense_start(omm_handle *h) {
    const int64_t m = h->m, n = h->n, mn = m * n;
    cudaStream_t st = h->stream;
    omm::DevState *s = h->dstate;
    omm::GemmBatch b{};
    // SW = S W, H'W = H' W
    b.A[0] = h->HS;         b.B[0] = h->WD; b.C[0] = h->SWHW + mn;
    b.A[1] = h->HS + m * m; b.B[1] = h->WD; b.C[1] = h->SWHW;
    TRY(omm::dgemm_batched(false, false, m, n, m, 1.0, b, s_identity(h) ? 1 : 2, m, m, 0.0, m, m, s, st));
    if (s_identity(h))
        OMM_CUDA_TRY(cudaMemcpyAsync(h->SWHW, h->WD, mn * sizeof(double), cudaMemcpyDeviceToDevice, st));
    // H_W = W^T H'W, S_W = W^T S W
    omm::GemmBatch c{};
    c.A[0] = h->WD; c.B[0] = h->SWHW + mn; c.C[0] = h->h0s0;
    c.A[1] = h->WD; c.B[1] = h->SWHW;      c.C[1] = h->h0s0 + n;
    TRY(omm::dgemm_batched(true, false, n, n, m, 1.0, c, 2, m, m, 0.0, 2 * n, 2 * n, s, st));
    TRY(omm::launch_nn_update_energy((int)n, h->h0s0, h->h0s0 + n, 2 * n, h->Z, 2 * n, scr(h, 1),
                                     ctr(h, 1), s, 1, st));
    omm::GemmBatch g{};
    g.A[0] = h->SWHW; g.B[0] = h->h0s0; g.Cin[0] = h->SWHW + mn; g.C[0] = h->G;
    TRY(omm::dgemm_batched(false, false, m, n, 2 * n, -2.0, g, 1, m, 2 * n, 4.0, m, m, s, st));
    return dense_direction(h, 1);
}

// ---------------------------------------------------------------- mixed precision
constexpr int kDig = 3;
// K-block width of the split products.  With two digits a 64-wide K block
// (128-byte swizzle, two 96 KB stages) is read by the tensor cores without
// the shared-memory bank conflicts of the 64-byte swizzle; three digits keep
// 32-wide blocks (a 64-wide stage would leave room for only one).
int split_bk(int digits) { return digits == 2 ? 64 : 32; }
constexpr int kBN = 256;  // output tile width of the split products (UMMA N = 256)

// The 128-row-box map of a split product's B operand when the handle runs its
// split products on CTA pairs (omm_options.gemm_pair), else nullptr (one CTA per tile).
const CUtensorMap *pair_map(omm_handle *h, const CUtensorMap &half) {
    return h->opt.gemm_pair ? &half : nullptr;
}

omm::tc::TcArgs tc_args(omm_handle *h, int M, int N, int K) {
    omm::tc::TcArgs a{};
    omm::tc::pairs_for_digits(h->cur_dig, a);
    a.bk = h->mx.bk;
    a.M = M;
    a.N = N;
    a.K = K;
    a.alpha = 1.0;
    a.beta = 0.0;
    a.state = h->dstate;
    a.err = &h->dstate->wait_timeout;
    return a;
}

int mixed_alloc(omm_handle *h) {
    const int64_t m = h->m, n = h->n;
    MixedBufs &x = h->mx;
    x.ldm = (m + 7) / 8 * 8;
    x.bk = split_bk(h->opt.split_digits);
    const int kBK = x.bk;
    x.ld2n = (2 * n + 7) / 8 * 8;
    TRY(dalloc(&x.HSd, (size_t)(kDig * 2 * m * x.ldm)));
    TRY(dalloc(&x.WDd, (size_t)(kDig * 2 * n * x.ldm)));
    TRY(dalloc(&x.HDSDd, (size_t)(kDig * 2 * n * x.ldm)));
    TRY(dalloc(&x.SWHWd, (size_t)(kDig * m * x.ld2n)));
    TRY(dalloc(&x.HSWd, (size_t)(kDig * n * x.ld2n)));
    TRY(dalloc(&x.HDSD32, (size_t)(2 * m * n)));
    TRY(dalloc(&x.Z32, (size_t)(4 * n * n)));
    TRY(dalloc(&x.G32, (size_t)(m * n)));
    TRY(dalloc(&x.Gp32, (size_t)(m * n)));
    TRY(dalloc(&x.D32, (size_t)(m * n)));
    if (h->opt.dir_digits == 1) TRY(dalloc(&x.Df32, (size_t)(m * n)));
    TRY(omm::tc::make_digit_map(&x.mapHS_A, x.HSd, m, 2 * m, x.ldm, 2 * m * x.ldm, kDig, 128, kBK));
    TRY(omm::tc::make_digit_map(&x.mapWD_A, x.WDd, m, 2 * n, x.ldm, 2 * n * x.ldm, kDig, 128, kBK));
    TRY(omm::tc::make_digit_map(&x.mapWD_B, x.WDd, m, 2 * n, x.ldm, 2 * n * x.ldm, kDig, kBN, kBK));
    TRY(omm::tc::make_digit_map(&x.mapHDSD_B, x.HDSDd, m, 2 * n, x.ldm, 2 * n * x.ldm, kDig, kBN, kBK));
    TRY(omm::tc::make_digit_map(&x.mapSWHW_A, x.SWHWd, 2 * n, m, x.ld2n, m * x.ld2n, kDig, 128, kBK));
    TRY(omm::tc::make_digit_map(&x.mapHSW_B, x.HSWd, 2 * n, n, x.ld2n, n * x.ld2n, kDig, kBN, kBK));
    TRY(omm::tc::make_digit_map(&x.mapHDSD_H, x.HDSDd, m, 2 * n, x.ldm, 2 * n * x.ldm, kDig, 128, kBK));
    TRY(omm::tc::make_digit_map(&x.mapHSW_H, x.HSWd, 2 * n, n, x.ld2n, n * x.ld2n, kDig, 128, kBK));
    return OMM_OK;
}

int pack_W(omm_handle *h) {
    const MixedBufs &x = h->mx;
    return omm::tc::pack_cm(h->m, h->n, h->WD, h->m, x.WDd, x.ldm, 2 * h->n * x.ldm, kDig, h->dstate,
                            h->stream);
}
int pack_D(omm_handle *h) {
    const MixedBufs &x = h->mx;
    return omm::tc::pack_cm(h->m, h->n, h->WD + h->m * h->n, h->m, x.WDd + h->n * x.ldm, x.ldm,
                            2 * h->n * x.ldm, kDig, h->dstate, h->stream);
}
int pack_SWHW(omm_handle *h) {
    const MixedBufs &x = h->mx;
    return omm::tc::pack_t(h->m, 2 * h->n, h->SWHW, h->m, x.SWHWd, x.ld2n, h->m * x.ld2n, kDig, h->dstate,
                           h->stream);
}
int pack_HSW(omm_handle *h) {
    const MixedBufs &x = h->mx;
    return omm::tc::pack_cm(2 * h->n, h->n, h->h0s0, 2 * h->n, x.HSWd, x.ld2n, h->n * x.ld2n, kDig,
                            h->dstate, h->stream);
}

// Digit outputs fused into the elementwise kernels of the mixed form.
// digit outputs carry as many planes as the current phase's products read
omm::DigitOut dig_W(omm_handle *h) { return {h->mx.WDd, h->mx.ldm, 2 * h->n * h->mx.ldm, h->cur_dig}; }
omm::DigitOut dig_D(omm_handle *h) {
    return {h->mx.WDd + h->n * h->mx.ldm, h->mx.ldm, 2 * h->n * h->mx.ldm, h->cur_dig};
}
omm::DigitOut dig_SWHW(omm_handle *h) { return {h->mx.SWHWd, h->mx.ld2n, h->m * h->mx.ld2n, h->cur_dig}; }
omm::DigitOut dig_HSW(omm_handle *h) { return {h->mx.HSWd, h->mx.ld2n, h->n * h->mx.ld2n, h->cur_dig}; }
constexpr omm::DigitOut kNoDigits{nullptr, 0, 0};

// A split product of the mixed CG step: its arguments, operand maps and batch count.
struct SplitCall {
    omm::tc::TcArgs a;
    const CUtensorMap *mA = nullptr, *mB = nullptr, *mBh = nullptr;   // B with 256-row / 128-row boxes
    int nbatch = 1;
    // the B planes, for a map with another box (tile lists of narrow problems)
    const __nv_bfloat16 *b_base = nullptr;
    int64_t b_K = 0, b_rows = 0, b_ld = 0, b_plane = 0;
};

// [H'; S] times the digits of W (rows b_row0 = 0) or D (b_row0 = n) of WDd:
// FP64 results to C (H' part) and C + c_step (S part), digits to HDSDd.
SplitCall products_call(omm_handle *h, int b_row0, double *C, float *C32, int64_t c_step, int64_t dout_row0,
                        int64_t dout_step) {
    const int64_t m = h->m, n = h->n;
    MixedBufs &x = h->mx;
    SplitCall c;
    omm::tc::TcArgs &a = c.a;
    a = tc_args(h, (int)m, (int)n, (int)m);
    a.a_row0 = 0;
    a.a_row_step = (int)m;
    a.b_row0 = b_row0;
    a.b_row_step = 0;
    a.C = C;
    a.C32 = C32;
    a.ldc = m;
    a.c_step = c_step;
    a.Dout = x.HDSDd + dout_row0 * x.ldm;
    a.ldd = x.ldm;
    a.dplane = 2 * n * x.ldm;
    a.dout_step = dout_step * x.ldm;
    a.ndig = h->cur_dig;
    if (b_row0 == (int)n && h->opt.dir_digits == 1) {
        // one BF16 digit of D: the pairs (p, 1) of A's digits with it, smallest first
        omm::tc::pairs_one_b(h->cur_dig, a);
    }
    c.mA = &x.mapHS_A;
    c.mB = &x.mapWD_B;
    c.mBh = &x.mapWD_A;
    c.nbatch = s_identity(h) ? 1 : 2;
    c.b_base = x.WDd;
    c.b_K = m;
    c.b_rows = 2 * n;
    c.b_ld = x.ldm;
    c.b_plane = 2 * n * x.ldm;
    return c;
}

// Z = [W D]^T [H'D SD]
SplitCall contract_call(omm_handle *h) {
    const int64_t m = h->m, n = h->n;
    MixedBufs &x = h->mx;
    SplitCall c;
    c.a = tc_args(h, (int)(2 * n), (int)(2 * n), (int)m);
    if (h->opt.dir_digits == 1) c.a.a_split_row = (int)n;   // the rows of D^T carry one digit
    c.a.C32 = x.Z32;
    c.a.ldc = 2 * n;
    c.mA = &x.mapWD_A;
    c.mB = &x.mapHDSD_B;
    c.mBh = &x.mapHDSD_H;
    c.b_base = x.HDSDd;
    c.b_K = m;
    c.b_rows = 2 * n;
    c.b_ld = x.ldm;
    c.b_plane = 2 * n * x.ldm;
    return c;
}

// G = 4 H'W - 2 [SW H'W][H_W ; S_W]
SplitCall gradient_call(omm_handle *h) {
    const int64_t m = h->m, n = h->n;
    MixedBufs &x = h->mx;
    SplitCall c;
    c.a = tc_args(h, (int)m, (int)n, (int)(2 * n));
    c.a.alpha = -2.0;
    c.a.beta = 4.0;
    c.a.Cin = h->SWHW + m * n;
    c.a.ldcin = m;
    c.a.C32 = x.G32;
    c.a.ldc = m;
    c.mA = &x.mapSWHW_A;
    c.mB = &x.mapHSW_B;
    c.mBh = &x.mapHSW_H;
    c.b_base = x.HSWd;
    c.b_K = 2 * n;
    c.b_rows = n;
    c.b_ld = x.ld2n;
    c.b_plane = n * x.ld2n;
    return c;
}

// Tile-list form of one of the step's three split products (0 products, 1
// contraction, 2 gradient) for a persistent launch (omm_options.gemm_persistent):
// the arguments are fixed for the handle's life, so the list is built once.
int list_mode(omm_handle *h) { return h->opt.gemm_pair ? omm::tc::LIST_PAIR : omm::tc::LIST_SINGLE; }

int list_ctas(int mode, int64_t ntiles) {
    int64_t c = mode == omm::tc::LIST_PAIR ? 2 * ntiles : ntiles;
    if (c > 152) c = 152;
    return (int)c;
}

int tile_problem(const SplitCall &c, int mode, omm::tc::TileProblem &p) {
    memset(&p, 0, sizeof(p));
    p.mapA = *c.mA;
    p.a = c.a;
    omm::tc::list_prepare(p.a);
    p.bn = omm::tc::list_tile_width(c.a.N, mode);
    const int box = mode == omm::tc::LIST_PAIR ? p.bn / 2 : p.bn;
    if (box == 256 && mode != omm::tc::LIST_PAIR) {
        p.mapB = *c.mB;
    } else if (box == 128 && mode == omm::tc::LIST_PAIR) {
        p.mapB = *c.mBh;
    } else {
        TRY(omm::tc::make_digit_map(&p.mapB, c.b_base, c.b_K, c.b_rows, c.b_ld, c.b_plane, kDig, box, c.a.bk));
    }
    return OMM_OK;
}

int run_split(omm_handle *h, const SplitCall &c, int slot) {
    const bool list = slot >= 0 && h->opt.gemm_persistent && c.a.bk == 64 && c.a.nA + c.a.nB <= 4;
    if (!list) return omm::tc::gemm(*c.mA, *c.mB, c.a, c.nbatch, kBN, h->stream, pair_map(h, *c.mBh));
    HandleList &L = h->lists[slot];
    const int mode = list_mode(h);
    if (L.probs == nullptr) {
        omm::tc::TileProblem p;
        TRY(tile_problem(c, mode, p));
        std::vector<omm::tc::TileRef> tiles;
        omm::tc::list_tiles(0, p.a, c.nbatch, mode, p.bn, tiles);
        OMM_CUDA_TRY(cudaMalloc((void **)&L.probs, sizeof(p)));
        OMM_CUDA_TRY(cudaMalloc((void **)&L.tiles, tiles.size() * sizeof(omm::tc::TileRef)));
        OMM_CUDA_TRY(cudaMemcpy(L.probs, &p, sizeof(p), cudaMemcpyHostToDevice));
        OMM_CUDA_TRY(cudaMemcpy(L.tiles, tiles.data(), tiles.size() * sizeof(omm::tc::TileRef), cudaMemcpyHostToDevice));
        L.ntiles = (int)tiles.size();
    }
    return omm::tc::gemm_list(L.probs, L.tiles, L.ntiles, mode, list_ctas(mode, L.ntiles), c.a.nA, c.a.nB, h->stream);
}

int split_products(omm_handle *h, int b_row0, double *C, float *C32, int64_t c_step, int64_t dout_row0,
                   int64_t dout_step) {
    const int64_t m = h->m, n = h->n;
    MixedBufs &x = h->mx;
    const SplitCall c = products_call(h, b_row0, C, C32, c_step, dout_row0, dout_step);
    // the iteration's products (D, FP32 out) have fixed arguments: list slot 0
    TRY(run_split(h, c, (C32 != nullptr && b_row0 == (int)n) ? 0 : -1));
    if (!s_identity(h)) return OMM_OK;
    // z = 1 (S times the B rows) is the B rows themselves: their FP32/FP64 values and digits
    const int64_t mn = m * n;
    if (C32 != nullptr)   // iteration: S D = D
        OMM_CUDA_TRY(cudaMemcpyAsync(C32 + c_step, x.D32, mn * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    else                  // start: S W = W
        OMM_CUDA_TRY(cudaMemcpyAsync(C + c_step, h->WD + b_row0 * m, mn * sizeof(double), cudaMemcpyDeviceToDevice,
                                     h->stream));
    const size_t pitch = (size_t)(2 * n * x.ldm) * sizeof(__nv_bfloat16);
    OMM_CUDA_TRY(cudaMemcpy2DAsync(x.HDSDd + (dout_row0 + dout_step) * x.ldm, pitch, x.WDd + b_row0 * x.ldm, pitch,
                                   (size_t)(n * x.ldm) * sizeof(__nv_bfloat16), h->cur_dig, cudaMemcpyDeviceToDevice,
                                   h->stream));
    return OMM_OK;
}

int split_contract(omm_handle *h) { return run_split(h, contract_call(h), 1); }

int split_gradient(omm_handle *h) { return run_split(h, gradient_call(h), 2); }

// FP64 gradient (CUDA cores), rounded to the FP32 gradient of the mixed form
int fp64_gradient(omm_handle *h) {
    const int64_t m = h->m, n = h->n, mn = m * n;
    omm::GemmBatch g{};
    g.A[0] = h->SWHW; g.B[0] = h->h0s0; g.Cin[0] = h->SWHW + mn; g.C[0] = h->G;
    TRY(omm::dgemm_batched(false, false, m, n, 2 * n, -2.0, g, 1, m, 2 * n, 4.0, m, m, h->dstate, h->stream));
    return omm::mx_round(mn, h->G, h->mx.G32, h->dstate, h->stream);
}

int exact_alloc(omm_handle *h) {
    const int64_t m = h->m, n = h->n;
    const MixedBufs &x = h->mx;
    ExactBufs &e = h->ex;
    e.s = h->opt.exact_digits;
    const int s = e.s;
    TRY(dalloc(&e.HSx, (size_t)(s * 2 * m * x.ldm)));
    TRY(dalloc(&e.Wx, (size_t)(s * n * x.ldm)));
    TRY(dalloc(&e.HWSWx, (size_t)(s * 2 * n * x.ldm)));
    TRY(dalloc(&e.SWHWx, (size_t)(s * m * x.ld2n)));
    TRY(dalloc(&e.HSWx, (size_t)(s * n * x.ld2n)));
    TRY(dalloc(&e.e, (size_t)(2 * m + n + 2 * n + m + n)));
    e.eHS = e.e;
    e.eW = e.eHS + 2 * m;
    e.eHWSW = e.eW + n;
    e.eSWHW = e.eHWSW + 2 * n;
    e.eHSW = e.eSWHW + m;
    TRY(omm::tc::make_digit_map(&e.mapHS_A, e.HSx, m, 2 * m, x.ldm, 2 * m * x.ldm, s, 128));
    TRY(omm::tc::make_digit_map(&e.mapW, e.Wx, m, n, x.ldm, n * x.ldm, s, 128));
    TRY(omm::tc::make_digit_map(&e.mapHWSW_B, e.HWSWx, m, 2 * n, x.ldm, 2 * n * x.ldm, s, 128));
    TRY(omm::tc::make_digit_map(&e.mapSWHW_A, e.SWHWx, 2 * n, m, x.ld2n, m * x.ld2n, s, 128));
    TRY(omm::tc::make_digit_map(&e.mapHSW_B, e.HSWx, 2 * n, n, x.ld2n, n * x.ld2n, s, 128));
    return OMM_OK;
}

omm::tc::ExactArgs exact_args(omm_handle *h, int M, int N, int K) {
    omm::tc::ExactArgs a{};
    omm::tc::exact_pairs(h->ex.s, a);
    a.M = M;
    a.N = N;
    a.K = K;
    a.alpha = 1.0;
    a.beta = 0.0;
    a.state = h->dstate;
    a.err = &h->dstate->wait_timeout;
    return a;
}

// G = 4 H'W - 2 [SW H'W][H_W ; S_W] with exact-digit products
int exact_gradient(omm_handle *h) {
    const int64_t m = h->m, n = h->n;
    const MixedBufs &x = h->mx;
    ExactBufs &e = h->ex;
    cudaStream_t st = h->stream;
    // The gradient is consumed in FP32, but its digits must beat the
    // cancellation between 4 H'W and 2 [SW H_W + H'W S_W] near convergence.
    // Six digits (21 pair products instead of 28; error ~2^-41 of the terms)
    // keep the refinement's step count at m = 4096 and on the batched systems;
    // five digits (~2^-34) stalled it at m = 4096.
    const int sg = e.s < 6 ? e.s : 6;
    {
        StageTimer t(h, OMM_STAGE_PACK);
        TRY(omm::tc::exact_pack(false, m, 2 * n, h->SWHW, m, e.eSWHW, e.SWHWx, x.ld2n, m * x.ld2n, sg, h->dstate, st));
        TRY(omm::tc::exact_pack(true, 2 * n, n, h->h0s0, 2 * n, e.eHSW, e.HSWx, x.ld2n, n * x.ld2n, sg, h->dstate, st));
    }
    StageTimer t(h, OMM_STAGE_GRADIENT);
    omm::tc::ExactArgs a = exact_args(h, (int)m, (int)n, (int)(2 * n));
    omm::tc::exact_pairs(sg, a);
    a.alpha = -2.0;
    a.beta = 4.0;
    a.Cin = h->SWHW + m * n;
    a.ldcin = m;
    a.C32 = h->mx.G32;
    a.ldc = m;
    a.eA = e.eSWHW;
    a.eB = e.eHSW;
    return omm::tc::exact_gemm(e.mapSWHW_A, e.mapHSW_B, a, 1, st);
}

// Refinement start with exact-digit products: H'W, SW, H_W, S_W, energy, G, D.
// Six digits (21 pair products instead of 28; ~2^-41 of |A||B|) anchor the
// state far below what the refinement's RelTol and orthonormality bars can
// see; omm_set_HS packs six digits of H' and S for it.
int exact_anchor(omm_handle *h) {
    const int64_t m = h->m, n = h->n, mn = m * n;
    const MixedBufs &x = h->mx;
    ExactBufs &e = h->ex;
    cudaStream_t st = h->stream;
    omm::DevState *s = h->dstate;
    const int sa = e.s < 6 ? e.s : 6;
    {
        StageTimer t(h, OMM_STAGE_ANCHOR);
        TRY(omm::tc::exact_pack(true, m, n, h->WD, m, e.eW, e.Wx, x.ldm, n * x.ldm, sa, s, st));
        // z = 0: H'W -> SWHW + mn;  z = 1: SW -> SWHW
        omm::tc::ExactArgs a = exact_args(h, (int)m, (int)n, (int)m);
        omm::tc::exact_pairs(sa, a);
        a.a_row_step = (int)m;
        a.C = h->SWHW + mn;
        a.ldc = m;
        a.c_step = -mn;
        a.eA = e.eHS;
        a.eA_step = m;
        a.eB = e.eW;
        TRY(omm::tc::exact_gemm(e.mapHS_A, e.mapW, a, s_identity(h) ? 1 : 2, st));
        if (s_identity(h))
            OMM_CUDA_TRY(cudaMemcpyAsync(h->SWHW, h->WD, mn * sizeof(double), cudaMemcpyDeviceToDevice, st));
        TRY(omm::tc::exact_pack(true, m, n, h->SWHW + mn, m, e.eHWSW, e.HWSWx, x.ldm, 2 * n * x.ldm, sa, s, st));
        TRY(omm::tc::exact_pack(true, m, n, h->SWHW, m, e.eHWSW + n, e.HWSWx + n * x.ldm, x.ldm, 2 * n * x.ldm, sa,
                                s, st));
        // z = 0: H_W = W^T H'W -> rows [0, n) of h0s0;  z = 1: S_W -> rows [n, 2n)
        omm::tc::ExactArgs b = exact_args(h, (int)n, (int)n, (int)m);
        omm::tc::exact_pairs(sa, b);
        b.b_row_step = (int)n;
        b.C = h->h0s0;
        b.ldc = 2 * n;
        b.c_step = n;
        b.eA = e.eW;
        b.eB = e.eHWSW;
        b.eB_step = n;
        TRY(omm::tc::exact_gemm(e.mapW, e.mapHWSW_B, b, 2, st));
    }
    TRY(omm::launch_nn_update_energy((int)n, h->h0s0, h->h0s0 + n, 2 * n, h->Z, 2 * n, scr(h, 1),
                                     ctr(h, 1), s, 1, st));
    TRY(exact_gradient(h));
    return OMM_OK;
}

// CG dots + direction of the mixed form (FP32 G, Gp, D; digits of D).  With the
// kinetic-energy preconditioner: digits of G, then the split product
// Z = P G in FP32 (Eq. 6), which forms the direction and beta.
int mixed_direction(omm_handle *h, int first) {
    const int64_t m = h->m, n = h->n;
    MixedBufs &x = h->mx;
    const float *Zg = nullptr;
    if (h->precon_on) {
        // Z = P G only shapes the search direction (the line search is exact along
        // any direction, and beta and the restart test take the same Z), so it is
        // formed from the leading BF16 digit of P and of G: one pair product
        StageTimer t(h, OMM_STAGE_PRECON);
        TRY(omm::mx_digits(m, n, x.G32, h->dstate, omm::DigitOut{x.Gd, x.ldm, n * x.ldm, 1}, h->stream));
        omm::tc::TcArgs a = tc_args(h, (int)m, (int)n, (int)m);
        a.npairs = 1;
        a.pa[0] = 0;
        a.pb[0] = 0;
        a.nA = 1;
        a.nB = 1;
        a.C32 = x.PG32;
        a.ldc = m;
        TRY(omm::tc::gemm(x.mapP_A, x.mapG_B, a, 1, kBN, h->stream, pair_map(h, x.mapG_H)));
        Zg = x.PG32;
    }
    StageTimer t(h, OMM_STAGE_DIRECTION);
    // with one-digit directions the recurrence (beta, the restart test, the next
    // direction) runs on the unrounded Df32 and the line search along D32
    const bool round1 = h->opt.dir_digits == 1;
    float *Df = round1 ? x.Df32 : x.D32;
    // the slope parts go to reduction slot 3 (otherwise used by omm_set_HS only);
    // one cooperative launch where it applies, else the dots and direction kernels
    const int rc = omm::mx_dots_direction(m, n, x.G32, Zg, x.Gp32, Df, x.D32, h->dstate, dig_D(h), round1,
                                          scr(h, 3), &h->slope_blocks, scr(h, 2), grid_bar(h), first, h->stream);
    if (rc != OMM_ERR_UNSUPPORTED) return rc;
    TRY(omm::mx_dots_beta(m * n, x.G32, Zg, x.Gp32, Df, scr(h, 2), ctr(h, 2), h->dstate, first, h->stream));
    return omm::mx_direction(m, n, x.G32, Zg, x.Gp32, Df, x.D32, h->dstate, dig_D(h), round1, scr(h, 3),
                             &h->slope_blocks, h->stream);
}

// Start of the split-precision phase: H'W, SW, H_W, S_W, energy, G, D from W.
int mixed_start(omm_handle *h) {
    const int64_t m = h->m, n = h->n, mn = m * n;
    h->cur_dig = h->opt.split_digits;
    cudaStream_t st = h->stream;
    omm::DevState *s = h->dstate;
    { StageTimer t(h, OMM_STAGE_PACK); TRY(pack_W(h)); }
    // H'W -> SWHW + mn, SW -> SWHW (FP64 state); their digits to HDSDd rows [0, n) and [n, 2n)
    { StageTimer t(h, OMM_STAGE_PRODUCTS); TRY(split_products(h, 0, h->SWHW + mn, nullptr, -mn, 0, n)); }
    {
        StageTimer t(h, OMM_STAGE_CONTRACT);
        omm::tc::TcArgs a = tc_args(h, (int)n, (int)n, (int)m);
        a.b_row_step = (int)n;    // z = 0: H'W digits, z = 1: SW digits
        a.C = h->h0s0;
        a.ldc = 2 * n;
        a.c_step = n;             // H_W in rows [0, n), S_W in rows [n, 2n)
        TRY(omm::tc::gemm(h->mx.mapWD_A, h->mx.mapHDSD_B, a, 2, kBN, st, pair_map(h, h->mx.mapHDSD_H)));
    }
    TRY(omm::launch_nn_update_energy((int)n, h->h0s0, h->h0s0 + n, 2 * n, h->Z, 2 * n, scr(h, 1),
                                     ctr(h, 1), s, 1, st));
    { StageTimer t(h, OMM_STAGE_PACK); TRY(pack_SWHW(h)); TRY(pack_HSW(h)); }
    { StageTimer t(h, OMM_STAGE_GRADIENT); TRY(split_gradient(h)); }
    return mixed_direction(h, 1);
}

// Line minimum and state updates of a mixed step (after the contractions).
int mixed_glue1(omm_handle *h, bool accurate_gradient) {
    const int64_t m = h->m, n = h->n, mn = m * n;
    cudaStream_t st = h->stream;
    omm::DevState *s = h->dstate;
    MixedBufs &x = h->mx;
    { StageTimer t(h, OMM_STAGE_LINESEARCH);
      TRY(omm::mx_coeffs_linemin((int)n, h->h0s0, h->h0s0 + n, 2 * n, x.Z32, 2 * n, scr(h, 0), ctr(h, 0), s,
                                 scr(h, 3), h->slope_blocks, st)); }
    { StageTimer t(h, OMM_STAGE_UPDATE);
      // the n x n update (H_W, S_W, energy, stop test) reads and writes nothing the
      // m x n update touches: for large systems it runs beside it on the handle's
      // second stream (in a grouped batch, and for small systems, the extra fork
      // and join cost more than the overlap gains)
      const bool fork = !h->grouped && m * n >= ((int64_t)1 << 21) && st != cudaStreamLegacy &&
                        st != cudaStreamPerThread && st != nullptr;
      cudaStream_t sn = fork ? h->aux : st;
      if (fork) {
          OMM_CUDA_TRY(cudaEventRecord(h->ev_fork, st));
          OMM_CUDA_TRY(cudaStreamWaitEvent(sn, h->ev_fork, 0));
      }
      TRY(omm::mx_nn_update((int)n, h->h0s0, h->h0s0 + n, 2 * n, x.Z32, 2 * n, scr(h, 1), ctr(h, 1), s,
                            accurate_gradient ? kNoDigits : dig_HSW(h), sn));
      TRY(omm::mx_update(m, n, h->WD, x.D32, h->SWHW + mn, x.HDSD32, h->SWHW, x.HDSD32 + mn, s, dig_W(h),
                         accurate_gradient ? kNoDigits : dig_SWHW(h), st));
      if (fork) {
          OMM_CUDA_TRY(cudaEventRecord(h->ev_join, sn));
          OMM_CUDA_TRY(cudaStreamWaitEvent(st, h->ev_join, 0));
      } }
    return OMM_OK;
}

// One CG step of the mixed form: split-precision products with FP32 outputs,
// FP64 state updated from FP32 increments; accurate_gradient selects the
// accurate gradient of the refinement sweep (exact-digit or FP64 products).
int mixed_iteration(omm_handle *h, bool accurate_gradient) {
    const int64_t m = h->m, n = h->n, mn = m * n;
    // the increments keep the split digit count in both phases: in the
    // refinement they are small against the exactly re-anchored state and the
    // exact-digit gradient, so two digits cost no extra steps at C2
    h->cur_dig = h->opt.split_digits;
    MixedBufs &x = h->mx;
    { StageTimer t(h, OMM_STAGE_PRODUCTS); TRY(split_products(h, (int)n, nullptr, x.HDSD32, mn, 0, n)); }
    { StageTimer t(h, OMM_STAGE_CONTRACT); TRY(split_contract(h)); }
    TRY(mixed_glue1(h, accurate_gradient));
    if (accurate_gradient) {
        if (h->opt.refine == OMM_REFINE_EXACT) {
            TRY(exact_gradient(h));
        } else {
            StageTimer t(h, OMM_STAGE_GRADIENT);
            TRY(fp64_gradient(h));
        }
    } else {
        StageTimer t(h, OMM_STAGE_GRADIENT);
        TRY(split_gradient(h));
    }
    return mixed_direction(h, 0);
}

// ---------------------------------------------------------------- linear-scaling form
// With screening on (omm_options.screen_eps > 0) each product skips the block
// pairs whose norm product is below eps; the squared block norms of every
// operand are refreshed right after the operand is written (omm::sp::norms is a
// no-op otherwise, and the nullptr norm arguments select the plain kernels).
int sparse_start(omm_handle *h) {
    omm::sp::Dev &d = h->sd;
    cudaStream_t st = h->stream;
    omm::DevState *s = h->dstate;
    const bool sc = d.screening();
    { StageTimer t(h, OMM_STAGE_PRODUCTS);
      TRY(omm::sp::norms(d, omm::sp::NRM_W, s, st));
      TRY(omm::sp::products(d, d.W, d.HW, d.SW, sc ? d.nW : nullptr, s, st));
      TRY(omm::sp::norms(d, omm::sp::NRM_HWSW, s, st)); }
    // H_W = W^T H'W and S_W = W^T S W through the contraction kernel (D := W)
    { StageTimer t(h, OMM_STAGE_CONTRACT);
      TRY(omm::sp::contract(d, d.W, d.W, d.HW, d.SW, d.h0, d.s0, d.h2, d.s2, sc ? d.nW : nullptr, d.nW, d.nHW,
                            d.nSW, s, st)); }
    TRY(omm::sp::nn_update(d, h->n, 1, scr(h, 1), ctr(h, 1), s, st));
    { StageTimer t(h, OMM_STAGE_GRADIENT);
      TRY(omm::sp::norms(d, omm::sp::NRM_N, s, st));
      TRY(omm::sp::gradient(d, s, st)); }
    { StageTimer t(h, OMM_STAGE_DIRECTION);
      TRY(omm::sp::dots(d, 1, scr(h, 2), ctr(h, 2), s, st));
      TRY(omm::sp::direction(d, s, st));
      TRY(omm::sp::norms(d, omm::sp::NRM_D, s, st)); }
    return OMM_OK;
}

int sparse_iteration(omm_handle *h) {
    omm::sp::Dev &d = h->sd;
    cudaStream_t st = h->stream;
    omm::DevState *s = h->dstate;
    const bool sc = d.screening();
    { StageTimer t(h, OMM_STAGE_PRODUCTS);
      TRY(omm::sp::products(d, d.D, d.HD, d.SD, sc ? d.nD : nullptr, s, st));
      TRY(omm::sp::norms(d, omm::sp::NRM_HDSD, s, st)); }
    { StageTimer t(h, OMM_STAGE_CONTRACT);
      TRY(omm::sp::contract(d, d.W, d.D, d.HD, d.SD, d.X, d.Y, d.h2, d.s2, sc ? d.nW : nullptr, d.nD, d.nHD,
                            d.nSD, s, st)); }
    { StageTimer t(h, OMM_STAGE_LINESEARCH); TRY(omm::sp::coeffs(d, scr(h, 0), ctr(h, 0), s, st)); }
    { StageTimer t(h, OMM_STAGE_UPDATE);
      TRY(omm::sp::axpy(d, s, st));
      TRY(omm::sp::nn_update(d, h->n, 0, scr(h, 1), ctr(h, 1), s, st));
      TRY(omm::sp::norms(d, omm::sp::NRM_W | omm::sp::NRM_HWSW | omm::sp::NRM_N, s, st)); }
    { StageTimer t(h, OMM_STAGE_GRADIENT); TRY(omm::sp::gradient(d, s, st)); }
    { StageTimer t(h, OMM_STAGE_DIRECTION);
      TRY(omm::sp::dots(d, 0, scr(h, 2), ctr(h, 2), s, st));
      TRY(omm::sp::direction(d, s, st));
      TRY(omm::sp::norms(d, omm::sp::NRM_D, s, st)); }
    return OMM_OK;
}

// One first-phase step of the mixed sparse form (FP32 increments on FP64 state).
int sparse_mixed_iteration(omm_handle *h) {
    omm::sp::Dev &d = h->sd;
    cudaStream_t st = h->stream;
    omm::DevState *s = h->dstate;
    { StageTimer t(h, OMM_STAGE_PRODUCTS); TRY(omm::sp::mixed_products(d, s, st)); }
    { StageTimer t(h, OMM_STAGE_CONTRACT); TRY(omm::sp::mixed_contract(d, s, st)); }
    { StageTimer t(h, OMM_STAGE_LINESEARCH); TRY(omm::sp::mixed_coeffs(d, scr(h, 0), ctr(h, 0), s, st)); }
    { StageTimer t(h, OMM_STAGE_UPDATE); TRY(omm::sp::mixed_update(d, scr(h, 1), ctr(h, 1), s, st)); }
    { StageTimer t(h, OMM_STAGE_GRADIENT); TRY(omm::sp::mixed_gradient(d, s, st)); }
    { StageTimer t(h, OMM_STAGE_DIRECTION); TRY(omm::sp::mixed_direction(d, scr(h, 2), ctr(h, 2), s, st)); }
    return OMM_OK;
}

// Solve phases of the asynchronous driver (omm_solve_begin / _progress / _end)
enum { PH_IDLE = 0, PH_MIXED = 1, PH_REFINE = 2, PH_FP64 = 3, PH_SPARSE = 4, PH_FINISHED = 5, PH_SPARSE_MIXED = 6 };

double *w_dev(omm_handle *h) { return h->sparse ? h->sd.W : h->WD; }
int64_t w_len(omm_handle *h) { return h->sparse ? h->sd.nnzW * h->sd.bm * h->sd.bn : h->m * h->n; }

// Enqueue one chunk of CG steps of the current phase, then the state copy
// and the event the host polls.  Kernels of a finished solve return at once.
int chunk_body(omm_handle *h) {
    for (int c = 0; c < h->chunk; ++c) {
        switch (h->phase) {
            case PH_MIXED: TRY(mixed_iteration(h, false)); break;
            case PH_REFINE: TRY(mixed_iteration(h, true)); break;
            case PH_FP64: TRY(dense_iteration(h)); break;
            case PH_SPARSE: TRY(sparse_iteration(h)); break;
            case PH_SPARSE_MIXED: TRY(sparse_mixed_iteration(h)); break;
            default: return OMM_ERR_STATE;
        }
    }
    return OMM_OK;
}

// A chunk's launches are the same every time for a phase (every kernel reads
// its scalars from the device state), so after one eager chunk the sequence is
// captured into a graph and replayed: one launch from the host instead of
// ~100, which is what bounds small systems driven together.  Not on the
// legacy default stream (it cannot be captured) nor while profiling.
int run_chunk(omm_handle *h) {
    const int ph = h->phase;
    const bool capturable = h->opt.graphs != 0 && !h->profiling && h->stream != nullptr &&
                            h->stream != cudaStreamLegacy && h->stream != cudaStreamPerThread;
    if (!capturable) return chunk_body(h);
    if (h->graph[ph] == nullptr && h->graph_eager[ph] == 0) {
        ++h->graph_eager[ph];
        return chunk_body(h);
    }
    if (h->graph[ph] == nullptr) {
        const int64_t before = omm_kernel_launches();
        OMM_CUDA_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        const int rc = chunk_body(h);
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(h->stream, &g);
        if (rc != OMM_OK || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            omm::set_error("chunk capture failed: %s", cudaGetErrorString(ce));
            return rc != OMM_OK ? rc : OMM_ERR_CUDA;
        }
        const cudaError_t ie = cudaGraphInstantiate(&h->graph[ph], g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            h->graph[ph] = nullptr;
            omm::set_error("chunk graph instantiation failed: %s", cudaGetErrorString(ie));
            return OMM_ERR_CUDA;
        }
        // captured launches are counted each time the graph runs
        h->graph_kernels[ph] = omm_kernel_launches() - before;
        omm::count_launch(-h->graph_kernels[ph]);
    }
    OMM_CUDA_TRY(cudaGraphLaunch(h->graph[ph], h->stream));
    omm::count_launch(h->graph_kernels[ph]);
    return OMM_OK;
}

int enqueue_chunk(omm_handle *h) {
    TRY(run_chunk(h));
    OMM_CUDA_TRY(cudaMemcpyAsync(h->hstate, h->dstate, sizeof(omm::DevState), cudaMemcpyDeviceToHost, h->stream));
    OMM_CUDA_TRY(cudaEventRecord(h->ev_poll, h->stream));
    return OMM_OK;
}

// Buffers of the kinetic-energy preconditioner (T, P, P G; the exact-digit GEMM
// workspace and L^-1 of its Cholesky factor; the mixed form's digit planes).
int precon_alloc(omm_handle *h) {
    const int64_t m = h->m, n = h->n;
    h->cw.s = h->opt.exact_digits;
    h->cw.bytes = omm::chol::work_bytes(m, n, h->cw.s);
    TRY(dalloc(&h->Tk, (size_t)(m * m)));
    TRY(dalloc(&h->P, (size_t)(m * m)));
    TRY(dalloc(&h->PG, (size_t)(m * n)));
    TRY(dalloc(&h->cw.Linv, (size_t)omm::chol::linv_elems(m)));
    if (cudaMalloc(&h->cw.ws, (size_t)h->cw.bytes) != cudaSuccess) {
        h->cw.ws = nullptr;
        return OMM_ERR_NOMEM;
    }
    if (h->opt.precision == OMM_PREC_MIXED) {
        MixedBufs &x = h->mx;
        TRY(dalloc(&x.Pd, (size_t)(kDig * m * x.ldm)));
        TRY(dalloc(&x.Gd, (size_t)(kDig * n * x.ldm)));
        TRY(dalloc(&x.PG32, (size_t)(m * n)));
        TRY(omm::tc::make_digit_map(&x.mapP_A, x.Pd, m, m, x.ldm, m * x.ldm, kDig, 128, x.bk));
        TRY(omm::tc::make_digit_map(&x.mapG_B, x.Gd, m, n, x.ldm, n * x.ldm, kDig, kBN, x.bk));
        TRY(omm::tc::make_digit_map(&x.mapG_H, x.Gd, m, n, x.ldm, n * x.ldm, kDig, 128, x.bk));
    }
    return OMM_OK;
}

// P = (S + T / tau)^-1 for the current S and T (synchronous; OMM_ERR_NOT_SPD
// when S + T / tau is not positive definite), and its digits for the mixed form.
int precon_build(omm_handle *h) {
    const int64_t m = h->m;
    cudaStream_t st = h->stream;
    omm::DevState init{};
    *h->hstate = init;
    OMM_CUDA_TRY(cudaMemcpyAsync(h->dstate, h->hstate, sizeof(omm::DevState), cudaMemcpyHostToDevice, st));
    {
        StageTimer t(h, OMM_STAGE_SETUP);
        TRY(omm::chol::precon(h->HS + m * m, h->Tk, h->opt.tau_T, h->P, m, h->cw, h->dstate, st));
        if (h->opt.precision == OMM_PREC_MIXED)
            TRY(omm::tc::pack_cm(m, m, h->P, m, h->mx.Pd, h->mx.ldm, m * h->mx.ldm, kDig, nullptr, st));
    }
    OMM_CUDA_TRY(cudaMemcpyAsync(h->hstate, h->dstate, sizeof(omm::DevState), cudaMemcpyDeviceToHost, st));
    OMM_CUDA_TRY(cudaStreamSynchronize(st));
    if (h->hstate->status != OMM_OK) return h->hstate->status;
    h->p_ready = true;
    return OMM_OK;
}

// Captured chunk graphs hold the launches of one choice of preconditioning.
void drop_graphs(omm_handle *h) {
    for (int i = 0; i < omm_handle::kPhases; ++i) {
        if (h->graph[i]) cudaGraphExecDestroy(h->graph[i]);
        h->graph[i] = nullptr;
        h->graph_kernels[i] = 0;
        h->graph_eager[i] = 0;
    }
}

// Dense setup for omm_set_HS (S given) and omm_set_H (S == nullptr: the
// previous S, and with the Cholesky variant its factor, are kept).
int dense_set(omm_handle *h, const double *H, const double *S, bool on_device) {
    const int64_t m = h->m, mm = m * m;
    h->solved = false;
    cudaStream_t st = h->stream;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const bool chol = h->opt.cholesky != 0;
    // S goes to its slot (kept by omm_set_H; with the Cholesky variant restored
    // from its copy, since the slot then holds I); H is staged in the H' slot
    // and shifted in place
    if (S != nullptr) {
        h->have_S = false;
        h->p_ready = false;
        OMM_CUDA_TRY(cudaMemcpyAsync(h->HS + mm, S, mm * sizeof(double), kind, st));
        if (chol) OMM_CUDA_TRY(cudaMemcpyAsync(h->S0, h->HS + mm, mm * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else if (chol) {
        OMM_CUDA_TRY(cudaMemcpyAsync(h->HS + mm, h->S0, mm * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    OMM_CUDA_TRY(cudaMemcpyAsync(h->HS, H, mm * sizeof(double), kind, st));
    omm::DevState init{};
    init.eta = h->opt.eta;
    *h->hstate = init;
    OMM_CUDA_TRY(cudaMemcpyAsync(h->dstate, h->hstate, sizeof(omm::DevState), cudaMemcpyHostToDevice, st));
    {
        StageTimer t(h, OMM_STAGE_SETUP);
        if (h->opt.eta_auto)
            TRY(omm::launch_gershgorin(m, h->HS, h->HS + mm, scr(h, 3), ctr(h, 3), h->dstate, st));
        TRY(omm::launch_shift(mm, h->HS, h->HS + mm, h->HS, h->dstate, st));
        if (chol) {
            if (S != nullptr) TRY(omm::chol::factor(h->HS + mm, h->L, m, h->cw, h->dstate, st));
            TRY(omm::chol::transform(h->HS, h->HS + mm, m, h->cw, st));
        }
    }
    if (h->opt.precision == OMM_PREC_MIXED) {
        // columns of [H' | S] become the K-major rows of the A operand (symmetric);
        // omm_set_H and the Cholesky variant's S = I repack H' only
        StageTimer t(h, OMM_STAGE_PACK);
        const int64_t cols = (S == nullptr || s_identity(h)) ? m : 2 * m;
        // the split products of both phases read split_digits planes
        TRY(omm::tc::pack_cm(m, cols, h->HS, m, h->mx.HSd, h->mx.ldm, 2 * m * h->mx.ldm, h->opt.split_digits, nullptr,
                             st));
        // the re-anchor reads six digits of H' and S (see exact_anchor)
        if (h->opt.refine == OMM_REFINE_EXACT)
            TRY(omm::tc::exact_pack(true, m, cols, h->HS, m, h->ex.eHS, h->ex.HSx, h->mx.ldm, 2 * m * h->mx.ldm,
                                    h->ex.s < 6 ? h->ex.s : 6, nullptr, st));
    }
    OMM_CUDA_TRY(cudaMemcpyAsync(h->hstate, h->dstate, sizeof(omm::DevState), cudaMemcpyDeviceToHost, st));
    OMM_CUDA_TRY(cudaEventRecord(h->ev1, st));
    OMM_CUDA_TRY(cudaStreamSynchronize(st));
    harvest_stage_times(h);
    if (h->hstate->status != OMM_OK) return h->hstate->status;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    h->diag.t_setup_ms = ms;
    h->diag.eta = h->hstate->eta;
    h->have_HS = true;
    h->have_S = true;
    return OMM_OK;
}

// Position of every block of `to`'s W pattern in `from`'s W pattern (-1 where
// `from` has no such block): a merge of the sorted column lists of each row.
void w_block_map(const omm::sp::Host &to, const omm::sp::Host &from, std::vector<int64_t> &map) {
    const int64_t nbr = (int64_t)to.Wrp.size() - 1;
    map.assign((size_t)to.Wrp[nbr], -1);
    for (int64_t I = 0; I < nbr; ++I) {
        int64_t a = from.Wrp[I];
        const int64_t ae = from.Wrp[I + 1];
        for (int64_t b = to.Wrp[I]; b < to.Wrp[I + 1]; ++b) {
            while (a < ae && from.Wcol[a] < to.Wcol[b]) ++a;
            if (a < ae && from.Wcol[a] == to.Wcol[b]) map[b] = a;
        }
    }
}

// Resident W in the original basis (the Cholesky variant keeps it in Wsave)
double *w_orig(omm_handle *h) {
    if (h->sparse) return h->sd.W;
    return h->opt.cholesky ? h->Wsave : h->WD;
}

bool idle(const omm_handle *h) { return h->phase == PH_IDLE || h->phase == PH_FINISHED; }

}  // namespace

namespace {
int begin_setup(omm_handle *h, const double *W0, int32_t W0_on_device, double tol);
int drive_batch(omm_handle **handles, int32_t count, double *E_out, int32_t *iters_out, int32_t *status_out);
}

extern "C" {

void omm_default_options(omm_options *opt) {
    if (opt == nullptr) return;
    memset(opt, 0, sizeof(*opt));
    opt->eta = 0.0;
    opt->eta_auto = 1;
    opt->precision = OMM_PREC_FP64;
    opt->cholesky = 0;
    opt->max_iter = 10000;
    opt->orth_tol = 0.0;
    opt->filter_eps = 1e-8;
    opt->stream = nullptr;
    opt->refine = OMM_REFINE_EXACT;
    opt->exact_digits = 7;
    opt->split_digits = 2;
    opt->graphs = 1;
    opt->n_occupied = 0;
    opt->precon = 0;
    opt->tau_T = 136.05693122994;   // 10 Ry in eV
    opt->screen_eps = 0.0;
    opt->gemm_pair = 1;
    opt->gemm_persistent = 0;
    opt->dir_digits = 1;
}

const char *omm_status_str(int status) {
    switch (status) {
        case OMM_OK: return "ok";
        case OMM_ERR_ARG: return "invalid argument";
        case OMM_ERR_NOMEM: return "out of memory";
        case OMM_ERR_CUDA: return "CUDA error";
        case OMM_ERR_NOT_SPD: return "overlap matrix not positive definite";
        case OMM_ERR_LINESEARCH: return "line-search quartic has no minimum";
        case OMM_ERR_MAXITER: return "maximum number of CG iterations reached";
        case OMM_ERR_PATTERN: return "invalid or inconsistent sparsity pattern";
        case OMM_ERR_NONFINITE: return "non-finite energy or line-search data";
        case OMM_ERR_TIMEOUT: return "bounded device wait timed out";
        case OMM_ERR_STATE: return "call out of order";
        case OMM_ERR_UNSUPPORTED: return "unsupported option combination";
        default: return "unknown status";
    }
}

int omm_create(int64_t m, int64_t n, int32_t block_size, const omm_pattern *pattern,
               const omm_options *opt, omm_handle **out) {
    if (out == nullptr) return OMM_ERR_ARG;
    *out = nullptr;
    if (m <= 0 || n <= 0 || n > m) return OMM_ERR_ARG;
    if (n > 2147483647 / 2 || m > ((int64_t)1 << 31)) return OMM_ERR_ARG;
    if (block_size < 0) return OMM_ERR_ARG;
    if (pattern != nullptr) {
        if (pattern->bm <= 0 || pattern->bn <= 0 || pattern->bm != block_size || pattern->nbr * pattern->bm != m ||
            pattern->nbc * pattern->bn != n || pattern->H_rowptr == nullptr || pattern->H_col == nullptr ||
            pattern->W_rowptr == nullptr || pattern->W_col == nullptr)
            return OMM_ERR_PATTERN;
        if (pattern->bm != 8 || pattern->bn != 2) return OMM_ERR_UNSUPPORTED;
        if (opt != nullptr && (opt->cholesky != 0 || opt->precon != 0 ||
                               (opt->precision == OMM_PREC_MIXED && opt->screen_eps > 0.0)))
            return OMM_ERR_UNSUPPORTED;
    }
    omm_handle *h = new (std::nothrow) omm_handle();
    if (h == nullptr) return OMM_ERR_NOMEM;
    h->m = m;
    h->n = n;
    h->bm = block_size;
    if (opt) h->opt = *opt; else omm_default_options(&h->opt);
    if (h->opt.max_iter < 0 || (h->opt.refine != OMM_REFINE_EXACT && h->opt.refine != OMM_REFINE_FP64) ||
        h->opt.exact_digits < 1 || h->opt.exact_digits > omm::tc::kExactMaxDigits || h->opt.split_digits < 2 ||
        h->opt.split_digits > 3 || h->opt.n_occupied < 0 || h->opt.n_occupied > n ||
        (h->opt.n_occupied > 0 && h->opt.n_occupied < n && h->opt.eta_auto) ||
        (h->opt.precon != 0 && !(h->opt.tau_T > 0.0 && isfinite(h->opt.tau_T))) ||
        !(h->opt.screen_eps >= 0.0 && isfinite(h->opt.screen_eps)) || h->opt.dir_digits < 0 ||
        h->opt.dir_digits > 1) {
        delete h;
        return OMM_ERR_ARG;
    }
    if (h->opt.precon != 0 && h->opt.cholesky != 0) {   // two answers to the same ill-conditioning
        delete h;
        return OMM_ERR_UNSUPPORTED;
    }
    if (h->opt.precision != OMM_PREC_FP64 && h->opt.precision != OMM_PREC_MIXED) {
        delete h;
        return OMM_ERR_UNSUPPORTED;
    }
    int rc = OMM_OK;
    if (h->opt.stream) {
        h->stream = (cudaStream_t)h->opt.stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete h;
            return OMM_ERR_CUDA;
        }
        h->own_stream = true;
    }
    const int64_t mn = m * n;
    if (pattern != nullptr) {
        h->sparse = true;
        omm::sp::Pattern P;
        P.bm = pattern->bm;
        P.bn = pattern->bn;
        P.nbr = pattern->nbr;
        P.nbc = pattern->nbc;
        P.Hrp = pattern->H_rowptr;
        P.Hcol = pattern->H_col;
        P.Wrp = pattern->W_rowptr;
        P.Wcol = pattern->W_col;
        if ((rc = omm::sp::build(P, h->sh)) || (rc = omm::sp::upload(h->sh, h->sd)) ||
            (rc = omm::sp::screen_alloc(h->sd, h->opt.screen_eps)) ||
            (rc = dalloc(&h->scratch, (size_t)(4 * omm::kRedBlocksMax * omm::kRedSlots))) ||
            (rc = dalloc(&h->counters, (size_t)(64 * 8))) || (rc = dalloc(&h->dstate, 1))) {
            free_handle(h);
            return rc;
        }
        h->diag.nnzb_H = h->sd.nnzH;
        h->diag.nnzb_W = h->sd.nnzW;
        h->diag.nnzb_HW = h->sd.nnzHW;
        h->diag.nnzb_N = h->sd.nnzN;
    } else if ((rc = dalloc(&h->HS, (size_t)(2 * m * m))) ||
        (rc = dalloc(&h->WD, (size_t)(2 * mn))) || (rc = dalloc(&h->HDSD, (size_t)(2 * mn))) ||
        (rc = dalloc(&h->SWHW, (size_t)(2 * mn))) || (rc = dalloc(&h->h0s0, (size_t)(2 * n * n))) ||
        (rc = dalloc(&h->Z, (size_t)(4 * n * n))) || (rc = dalloc(&h->G, (size_t)mn)) ||
        (rc = dalloc(&h->Gp, (size_t)mn)) ||
        (rc = dalloc(&h->scratch, (size_t)(4 * omm::kRedBlocksMax * omm::kRedSlots))) ||
        (rc = dalloc(&h->counters, (size_t)(64 * 8))) || (rc = dalloc(&h->dstate, 1))) {
        free_handle(h);
        return rc;
    }
    if (h->opt.precision == OMM_PREC_MIXED && (rc = h->sparse ? omm::sp::mixed_alloc(h->sh, h->sd) : mixed_alloc(h))) {
        free_handle(h);
        return rc;
    }
    if (!h->sparse && h->opt.cholesky) {
        h->cw.s = h->opt.exact_digits;
        h->cw.bytes = omm::chol::work_bytes(m, n, h->cw.s);
        if ((rc = dalloc(&h->L, (size_t)(m * m))) || (rc = dalloc(&h->Wsave, (size_t)mn)) ||
            (rc = dalloc(&h->S0, (size_t)(m * m))) ||
            (rc = dalloc(&h->cw.Linv, (size_t)omm::chol::linv_elems(m))) ||
            (cudaMalloc(&h->cw.ws, (size_t)h->cw.bytes) != cudaSuccess ? (rc = OMM_ERR_NOMEM) : 0)) {
            free_handle(h);
            return rc;
        }
    }
    if (!h->sparse && h->opt.precision == OMM_PREC_MIXED && h->opt.refine == OMM_REFINE_EXACT &&
        (rc = exact_alloc(h))) {
        free_handle(h);
        return rc;
    }
    if (!h->sparse && h->opt.precon != 0 && (rc = precon_alloc(h))) {
        free_handle(h);
        return rc;
    }
    if (cudaMallocHost((void **)&h->hstate, sizeof(omm::DevState)) != cudaSuccess) {
        h->hstate = nullptr;
        free_handle(h);
        return OMM_ERR_NOMEM;
    }
    if (cudaMemsetAsync(h->counters, 0, 64 * 8 * sizeof(unsigned int), h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->dstate, 0, sizeof(omm::DevState), h->stream) != cudaSuccess ||
        cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_poll, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        free_handle(h);
        return OMM_ERR_CUDA;
    }
    *out = h;
    return OMM_OK;
}

int omm_set_HS(omm_handle *h, const double *H, const double *S, int32_t on_device) {
    if (h == nullptr || H == nullptr || S == nullptr) return OMM_ERR_ARG;
    if (h->phase != PH_IDLE && h->phase != PH_FINISHED) return OMM_ERR_STATE;
    cudaStream_t st = h->stream;
    h->have_HS = false;   // set again only when this setup succeeds
    h->solved = false;
    OMM_CUDA_TRY(cudaEventRecord(h->ev0, st));
    if (h->sparse) {
        omm::DevState init{};
        init.eta = h->opt.eta;
        *h->hstate = init;
        OMM_CUDA_TRY(cudaMemcpyAsync(h->dstate, h->hstate, sizeof(omm::DevState), cudaMemcpyHostToDevice, st));
        {
            StageTimer t(h, OMM_STAGE_SETUP);
            TRY(omm::sp::set_HS(h->sd, H, S, on_device != 0, h->opt.filter_eps, h->opt.eta_auto != 0, scr(h, 3),
                                ctr(h, 3), h->dstate, st));
            if (h->sd.mixed) TRY(omm::sp::mixed_shadow_HS(h->sd, st));
        }
        OMM_CUDA_TRY(cudaMemcpyAsync(h->hstate, h->dstate, sizeof(omm::DevState), cudaMemcpyDeviceToHost, st));
        OMM_CUDA_TRY(cudaEventRecord(h->ev1, st));
        OMM_CUDA_TRY(cudaStreamSynchronize(st));
        harvest_stage_times(h);
        if (h->hstate->status != OMM_OK) return h->hstate->status;
        // stored H/S pattern after filtering
        std::vector<unsigned char> keep((size_t)h->sd.nnzH);
        OMM_CUDA_TRY(cudaMemcpy(keep.data(), h->sd.keep, keep.size(), cudaMemcpyDeviceToHost));
        int64_t kept = 0;
        for (unsigned char k : keep) kept += k != 0;
        h->diag.nnzb_H = kept;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, h->ev0, h->ev1);
        h->diag.t_setup_ms = ms;
        h->diag.eta = h->hstate->eta;
        h->have_HS = true;
        return OMM_OK;
    }
    return dense_set(h, H, S, on_device != 0);
}

int omm_set_H(omm_handle *h, const double *H, int32_t on_device) {
    if (h == nullptr || H == nullptr) return OMM_ERR_ARG;
    if (h->sparse) return OMM_ERR_UNSUPPORTED;
    if (h->phase != PH_IDLE && h->phase != PH_FINISHED) return OMM_ERR_STATE;
    if (!h->have_S) return OMM_ERR_STATE;
    h->have_HS = false;
    OMM_CUDA_TRY(cudaEventRecord(h->ev0, h->stream));
    return dense_set(h, H, nullptr, on_device != 0);
}

int omm_set_T(omm_handle *h, const double *T, int32_t on_device) {
    if (h == nullptr || T == nullptr) return OMM_ERR_ARG;
    if (h->sparse || h->opt.precon == 0) return OMM_ERR_UNSUPPORTED;
    if (h->phase != PH_IDLE && h->phase != PH_FINISHED) return OMM_ERR_STATE;
    h->have_T = false;
    h->p_ready = false;
    OMM_CUDA_TRY(cudaMemcpyAsync(h->Tk, T, (size_t)(h->m * h->m) * sizeof(double),
                                 on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    OMM_CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->have_T = true;
    h->precon_left = h->opt.precon > 0 ? h->opt.precon : 0;
    return OMM_OK;
}

int omm_md_guess(omm_handle *dst, omm_handle *prev, omm_handle *prev2) {
    if (dst == nullptr || prev == nullptr) return OMM_ERR_ARG;
    for (omm_handle *x : {prev, prev2}) {
        if (x == nullptr) continue;
        if (x->sparse != dst->sparse || x->m != dst->m || x->n != dst->n) return OMM_ERR_ARG;
        if (x->sparse && (x->sd.bm != dst->sd.bm || x->sd.bn != dst->sd.bn || x->sd.nbr != dst->sd.nbr ||
                          x->sd.nbc != dst->sd.nbc))
            return OMM_ERR_ARG;
        if (!x->have_W || !idle(x)) return OMM_ERR_STATE;
    }
    if (!idle(dst)) return OMM_ERR_STATE;
    // the sources' W are complete: their last writes were on their own streams
    OMM_CUDA_TRY(cudaStreamSynchronize(prev->stream));
    if (prev2 != nullptr) OMM_CUDA_TRY(cudaStreamSynchronize(prev2->stream));
    cudaStream_t st = dst->stream;
    const double *W1 = w_orig(prev), *W2 = prev2 != nullptr ? w_orig(prev2) : nullptr;
    int rc = OMM_OK;
    if (!dst->sparse) {
        rc = omm::launch_md_guess(dst->m * dst->n, 1, w_orig(dst), W1, nullptr, W2, nullptr, st);
        if (rc == OMM_OK) OMM_CUDA_TRY(cudaStreamSynchronize(st));
    } else {
        // index maps of dst's W blocks in the sources' patterns, uploaded for the gather
        std::vector<int64_t> map1, map2;
        w_block_map(dst->sh, prev->sh, map1);
        if (prev2 != nullptr) w_block_map(dst->sh, prev2->sh, map2);
        const int64_t nnz = dst->sd.nnzW, blk = (int64_t)dst->sd.bm * dst->sd.bn;
        int64_t *dmap = nullptr;
        TRY(dalloc(&dmap, (size_t)(2 * nnz)));
        if (cudaMemcpyAsync(dmap, map1.data(), nnz * sizeof(int64_t), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            (prev2 != nullptr && cudaMemcpyAsync(dmap + nnz, map2.data(), nnz * sizeof(int64_t),
                                                 cudaMemcpyHostToDevice, st) != cudaSuccess))
            rc = OMM_ERR_CUDA;
        if (rc == OMM_OK)
            rc = omm::launch_md_guess(nnz, (int)blk, dst->sd.W, W1, dmap, W2, prev2 != nullptr ? dmap + nnz : nullptr,
                                      st);
        if (cudaStreamSynchronize(st) != cudaSuccess && rc == OMM_OK) rc = OMM_ERR_CUDA;
        cudaFree(dmap);
    }
    if (rc != OMM_OK) return rc;
    dst->have_W = true;
    dst->solved = false;
    return OMM_OK;
}

int omm_solve_begin(omm_handle *h, const double *W0, int32_t W0_on_device, double tol) {
    TRY(begin_setup(h, W0, W0_on_device, tol));
    return enqueue_chunk(h);
}

}  // extern "C"

namespace {
// Everything of omm_solve_begin but the first chunk: W0 in place, the phase's
// device state, and the phase's start (H'W, SW, H_W, S_W, energy, G, D).
int begin_setup(omm_handle *h, const double *W0, int32_t W0_on_device, double tol) {
    if (h == nullptr || !(tol >= 0.0)) return OMM_ERR_ARG;
    h->solved = false;
    if (!h->have_HS) return OMM_ERR_STATE;
    if (W0 == nullptr && !h->have_W) return OMM_ERR_STATE;
    if (h->phase != PH_IDLE && h->phase != PH_FINISHED) return OMM_ERR_STATE;
    if (h->opt.precon != 0 && !h->have_T) return OMM_ERR_STATE;
    const int64_t n = h->n;
    cudaStream_t st = h->stream;
    OMM_CUDA_TRY(cudaEventRecord(h->ev0, st));
    h->precon_on = h->opt.precon < 0 || (h->opt.precon > 0 && h->precon_left > 0);
    if (h->precon_on) {
        if (!h->p_ready) TRY(precon_build(h));
        if (h->opt.precon > 0) --h->precon_left;
    }
    if (h->precon_on != h->graph_precon) {
        drop_graphs(h);
        h->graph_precon = h->precon_on;
    }
    if (h->opt.cholesky && !h->sparse) {
        // W~ = L^T W: W0, or the previous solution kept in the original basis
        if (W0 != nullptr)
            OMM_CUDA_TRY(cudaMemcpyAsync(h->Wsave, W0, w_len(h) * sizeof(double),
                                         W0_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        StageTimer t(h, OMM_STAGE_SETUP);
        TRY(omm::chol::lt_times(h->L, h->m, h->Wsave, h->WD, h->n, h->cw, st));
    } else if (W0 != nullptr) {
        OMM_CUDA_TRY(cudaMemcpyAsync(w_dev(h), W0, w_len(h) * sizeof(double),
                                     W0_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    }
    omm::DevState init{};
    init.eta = h->diag.eta;
    init.e_shift = 2.0 * h->diag.eta * (double)n_occ(h);
    init.tol = tol;
    init.orth_tol = h->opt.orth_tol;
    init.max_iter = h->opt.max_iter;
    init.n = (int)n;
    h->tol_target = tol;
    h->k_mixed = 0;
    h->status = OMM_OK;
    if (h->sparse && h->sd.mixed) {
        // first phase with FP32 increments: from the FP64 start, to RelTol
        // max(0.1 tol, 1e-12) or until the FP32 increments' noise makes the energy
        // rise; an FP64 refinement, re-anchored from W, takes it to tol
        h->phase = PH_SPARSE_MIXED;
        omm::DevState ph = init;
        ph.tol = fmax(0.1 * tol, 1e-12);
        ph.orth_tol = 0.0;
        *h->hstate = ph;
        OMM_CUDA_TRY(cudaMemcpyAsync(h->dstate, h->hstate, sizeof(omm::DevState), cudaMemcpyHostToDevice, st));
        { StageTimer t(h, OMM_STAGE_START);
          TRY(sparse_start(h));
          TRY(omm::sp::mixed_begin(h->sd, h->dstate, st)); }
    } else if (h->sparse) {
        h->phase = PH_SPARSE;
        *h->hstate = init;
        OMM_CUDA_TRY(cudaMemcpyAsync(h->dstate, h->hstate, sizeof(omm::DevState), cudaMemcpyHostToDevice, st));
        { StageTimer t(h, OMM_STAGE_START); TRY(sparse_start(h)); }
    } else if (h->opt.precision == OMM_PREC_MIXED) {
        // phase 1: split-precision CG.  With three digits it runs to a
        // tolerance a decade below the target.  With two, the increments carry
        // ~1e-5 relative error and the phase-1 state drifts at that level, so
        // its energy changes cannot fall far below it: phase 1 stops at 1e-7
        // and the refinement, re-anchored exactly, takes the solve the rest of
        // the way (at m = 4096 a tighter first phase only adds iterations; a
        // looser one adds refinement steps, which cost twice as much).
        h->phase = PH_MIXED;
        omm::DevState ph = init;
        ph.tol = h->opt.split_digits == 2 ? fmax(0.1 * tol, 1e-7) : fmax(0.1 * tol, 1e-12);
        ph.orth_tol = 0.0;
        *h->hstate = ph;
        OMM_CUDA_TRY(cudaMemcpyAsync(h->dstate, h->hstate, sizeof(omm::DevState), cudaMemcpyHostToDevice, st));
        { StageTimer t(h, OMM_STAGE_START); TRY(mixed_start(h)); }
    } else {
        h->phase = PH_FP64;
        *h->hstate = init;
        OMM_CUDA_TRY(cudaMemcpyAsync(h->dstate, h->hstate, sizeof(omm::DevState), cudaMemcpyHostToDevice, st));
        { StageTimer t(h, OMM_STAGE_START); TRY(dense_start(h)); }
    }
    h->have_W = true;
    return OMM_OK;
}
}  // namespace

extern "C" {

int omm_solve_progress(omm_handle *h, int32_t blocking, int32_t *done) {
    if (h == nullptr || done == nullptr) return OMM_ERR_ARG;
    *done = 0;
    if (h->phase == PH_IDLE) return OMM_ERR_STATE;
    if (h->phase == PH_FINISHED) {
        *done = 1;
        return OMM_OK;
    }
    if (blocking) {
        OMM_CUDA_TRY(cudaEventSynchronize(h->ev_poll));
    } else {
        const cudaError_t q = cudaEventQuery(h->ev_poll);
        if (q == cudaErrorNotReady) return OMM_OK;
        OMM_CUDA_TRY(q);
    }
    harvest_stage_times(h);
    if (h->hstate->wait_timeout) {
        omm::set_error("a bounded mbarrier wait in the tensor-core GEMM timed out");
        h->status = OMM_ERR_TIMEOUT;
        h->phase = PH_FINISHED;
        *done = 1;
        return OMM_OK;
    }
    if (!h->hstate->done) return enqueue_chunk(h);
    if (h->phase == PH_SPARSE_MIXED && h->hstate->status == OMM_OK) {
        // refinement of the sparse form: FP64 steps, re-anchored from W
        h->k_mixed = h->hstate->k;
        omm::DevState rf{};
        rf.eta = h->diag.eta;
        rf.e_shift = 2.0 * h->diag.eta * (double)n_occ(h);
        rf.tol = h->tol_target;
        rf.orth_tol = h->opt.orth_tol;
        rf.max_iter = h->opt.max_iter;
        rf.n = (int)h->n;
        rf.k = h->k_mixed;
        *h->hstate = rf;
        OMM_CUDA_TRY(cudaMemcpyAsync(h->dstate, h->hstate, sizeof(omm::DevState), cudaMemcpyHostToDevice, h->stream));
        { StageTimer t(h, OMM_STAGE_ANCHOR); TRY(sparse_start(h)); }
        h->phase = PH_SPARSE;
        return enqueue_chunk(h);
    }
    if (h->phase == PH_MIXED && h->hstate->status == OMM_OK) {
        // phase 2: refinement sweep -- accurate re-anchoring of H'W, SW, H_W,
        // S_W and G, then CG steps with an accurate gradient
        const int64_t mn = h->m * h->n;
        cudaStream_t st = h->stream;
        h->k_mixed = h->hstate->k;
        omm::DevState rf{};
        rf.eta = h->diag.eta;
        rf.e_shift = 2.0 * h->diag.eta * (double)n_occ(h);
        rf.tol = h->tol_target;
        rf.orth_tol = h->opt.orth_tol;
        rf.max_iter = h->opt.max_iter;
        rf.n = (int)h->n;
        rf.k = h->k_mixed;
        *h->hstate = rf;
        OMM_CUDA_TRY(cudaMemcpyAsync(h->dstate, h->hstate, sizeof(omm::DevState), cudaMemcpyHostToDevice, st));
        if (h->opt.refine == OMM_REFINE_EXACT) {
            TRY(exact_anchor(h));
        } else {
            StageTimer t(h, OMM_STAGE_ANCHOR);
            TRY(dense_start(h));
            TRY(omm::mx_round(mn, h->G, h->mx.G32, h->dstate, st));
        }
        h->cur_dig = h->opt.split_digits;
        TRY(mixed_direction(h, 1));
        { StageTimer t(h, OMM_STAGE_PACK); TRY(pack_W(h)); }
        h->phase = PH_REFINE;
        return enqueue_chunk(h);
    }
    // a first phase that ended without reaching its tolerance (step limit, line
    // search, non-finite data) ends the solve: its steps are first-phase steps
    if (h->phase == PH_MIXED || h->phase == PH_SPARSE_MIXED) h->k_mixed = h->hstate->k;
    h->status = h->hstate->status;
    h->phase = PH_FINISHED;
    OMM_CUDA_TRY(cudaEventRecord(h->ev1, h->stream));
    *done = 1;
    return OMM_OK;
}

int omm_solve_end(omm_handle *h, double *W_out, int32_t W_out_on_device, double *E_out, int32_t *iters_out) {
    if (h == nullptr) return OMM_ERR_ARG;
    if (h->phase != PH_FINISHED) return OMM_ERR_STATE;
    cudaStream_t st = h->stream;
    const double *Wres = w_dev(h);
    if (h->opt.cholesky && !h->sparse) {
        // W = L^-T W~, kept for warm starts in the original basis
        TRY(omm::chol::lt_times(h->cw.Linv, h->m, h->WD, h->Wsave, h->n, h->cw, st));
        Wres = h->Wsave;
    }
    if (W_out != nullptr)
        OMM_CUDA_TRY(cudaMemcpyAsync(W_out, Wres, w_len(h) * sizeof(double),
                                     W_out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    OMM_CUDA_TRY(cudaStreamSynchronize(st));
    const omm::DevState &s = *h->hstate;
    const int64_t n = h->n;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    h->diag.t_solve_ms = ms;
    h->diag.E = s.E;
    h->diag.E_rel_change = s.rel;
    h->diag.orth = sqrt(s.orth2 > 0.0 ? s.orth2 : 0.0);
    // n_e = 2 Tr[(2I - S_W) S_W] = 2 (2 tr S_W - ||S_W||^2); from ||S_W - I||^2 =
    // ||S_W||^2 - 2 tr S_W + n:  n_e = 2 (n - ||S_W - I||^2)
    h->diag.charge = 2.0 * ((double)n - s.orth2);
    h->diag.iters = s.k;
    h->diag.status = h->status;
    h->diag.iters_mixed = h->k_mixed;
    h->diag.iters_refine = s.k - h->k_mixed;
    if (E_out) *E_out = s.E;
    if (iters_out) *iters_out = s.k;
    h->phase = PH_IDLE;
    h->solved = true;
    return h->status;
}

int omm_solve(omm_handle *h, const double *W0, int32_t W0_on_device, double tol, double *W_out,
              int32_t W_out_on_device, double *E_out, int32_t *iters_out) {
    TRY(omm_solve_begin(h, W0, W0_on_device, tol));
    for (int32_t done = 0; !done;) TRY(omm_solve_progress(h, 1, &done));
    return omm_solve_end(h, W_out, W_out_on_device, E_out, iters_out);
}

int omm_batch_solve(omm_handle **handles, int32_t count, const double *const *W0, int32_t W0_on_device, double tol,
                    double *E_out, int32_t *iters_out, int32_t *status_out) {
    if (handles == nullptr || count < 0) return OMM_ERR_ARG;
    for (int32_t i = 0; i < count; ++i) {
        if (handles[i] == nullptr) return OMM_ERR_ARG;
        for (int32_t j = 0; j < i; ++j)
            if (handles[j] == handles[i]) return OMM_ERR_ARG;
    }
    for (int32_t i = 0; i < count; ++i) {
        const int rc = omm_solve_begin(handles[i], W0 ? W0[i] : nullptr, W0_on_device, tol);
        if (rc != OMM_OK) return rc;
    }
    return drive_batch(handles, count, E_out, iters_out, status_out);
}

}  // extern "C"

namespace {
// Poll every handle of a batch whose solves are under way, enqueue each one's
// next chunk as its previous one completes, and collect the results.
int drive_batch(omm_handle **handles, int32_t count, double *E_out, int32_t *iters_out, int32_t *status_out) {
    std::vector<int32_t> done(count, 0);
    int32_t remaining = count;
    while (remaining > 0) {
        int ready = 0, first_open = -1;
        for (int32_t i = 0; i < count; ++i) {
            if (done[i]) continue;
            if (first_open < 0) first_open = i;
            if (cudaEventQuery(handles[i]->ev_poll) == cudaErrorNotReady) continue;
            ++ready;
            const int rc = omm_solve_progress(handles[i], 0, &done[i]);   // enqueues the next chunk
            if (rc != OMM_OK) return rc;
            if (done[i]) --remaining;
        }
        if (remaining > 0 && ready == 0) {
            // nothing ready: wait for the oldest open chunk instead of spinning
            const int rc = omm_solve_progress(handles[first_open], 1, &done[first_open]);
            if (rc != OMM_OK) return rc;
            if (done[first_open]) --remaining;
        }
    }
    int worst = OMM_OK;
    for (int32_t i = 0; i < count; ++i) {
        double E = 0.0;
        int32_t it = 0;
        const int st = omm_solve_end(handles[i], nullptr, 0, &E, &it);
        if (E_out) E_out[i] = E;
        if (iters_out) iters_out[i] = it;
        if (status_out) status_out[i] = st;
        if (st != OMM_OK && worst == OMM_OK) worst = st;
    }
    return worst;
}
}  // namespace

extern "C" {

}  // extern "C"

// ---------------------------------------------------------------- grouped batch
namespace {

// One stage's tile list over every system of a group (device copy).
struct GroupList {
    omm::tc::TileProblem *probs = nullptr;
    omm::tc::TileRef *tiles = nullptr;
    int ntiles = 0;
    int nA = 0, nB = 0;   // digit planes of every problem's operands
    void release() {
        cudaFree(probs);
        cudaFree(tiles);
        probs = nullptr;
        tiles = nullptr;
        ntiles = 0;
    }
};

SplitCall stage_call(omm_handle *h, int stage) {
    const int64_t m = h->m, n = h->n;
    if (stage == 0) return products_call(h, (int)n, nullptr, h->mx.HDSD32, m * n, 0, n);
    return stage == 1 ? contract_call(h) : gradient_call(h);
}

// Tiles of every system's split product of one stage, the systems with the longest
// K loop first (a longest-first list over the persistent CTAs).
int build_group_list(omm_handle **hs, int count, int stage, int mode, GroupList &L) {
    std::vector<omm::tc::TileProblem> probs((size_t)count);
    std::vector<int> order((size_t)count);
    std::vector<int> nb((size_t)count);
    for (int i = 0; i < count; ++i) {
        const SplitCall c = stage_call(hs[i], stage);
        TRY(tile_problem(c, mode, probs[i]));
        nb[i] = c.nbatch;
        order[i] = i;
        if (i > 0 && (c.a.nA != probs[0].a.nA || c.a.nB != probs[0].a.nB)) return OMM_ERR_UNSUPPORTED;
    }
    L.nA = probs[0].a.nA;
    L.nB = probs[0].a.nB;
    // longest tiles first: K loop times tile width
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (int64_t)probs[a].a.K * probs[a].bn > (int64_t)probs[b].a.K * probs[b].bn;
    });
    std::vector<omm::tc::TileRef> tiles;
    for (int i : order) omm::tc::list_tiles(i, probs[i].a, nb[i], mode, probs[i].bn, tiles);
    OMM_CUDA_TRY(cudaMalloc((void **)&L.probs, probs.size() * sizeof(omm::tc::TileProblem)));
    OMM_CUDA_TRY(cudaMalloc((void **)&L.tiles, tiles.size() * sizeof(omm::tc::TileRef)));
    OMM_CUDA_TRY(cudaMemcpy(L.probs, probs.data(), probs.size() * sizeof(omm::tc::TileProblem), cudaMemcpyHostToDevice));
    OMM_CUDA_TRY(cudaMemcpy(L.tiles, tiles.data(), tiles.size() * sizeof(omm::tc::TileRef), cudaMemcpyHostToDevice));
    L.ntiles = (int)tiles.size();
    return OMM_OK;
}

int run_group_list(const GroupList &L, int mode, omm_handle *h0, cudaStream_t st) {
    (void)h0;
    return omm::tc::gemm_list(L.probs, L.tiles, L.ntiles, mode, list_ctas(mode, L.ntiles), L.nA, L.nB, st);
}

// Tile modes chosen by the autotuner per group signature (the systems' (m, n) in
// order): timed once, then reused, so a group always runs the same schedule.  Both
// modes give the same bits, so the choice never changes a result.
struct TuneEntry {
    std::vector<int64_t> sig;
    int mode[3];
    float ms[3][2];
};
std::mutex g_tune_mu;
std::vector<TuneEntry> g_tune;
TuneEntry g_last_tune;

// Fork every system's stream off the group stream, run fn(h) on each, join back.
template <class F>
int fork_join(omm_handle **hs, int count, cudaStream_t gs, cudaEvent_t ev_fork, cudaEvent_t *ev_join, F fn) {
    OMM_CUDA_TRY(cudaEventRecord(ev_fork, gs));
    for (int i = 0; i < count; ++i) {
        OMM_CUDA_TRY(cudaStreamWaitEvent(hs[i]->stream, ev_fork, 0));
        TRY(fn(hs[i]));
        OMM_CUDA_TRY(cudaEventRecord(ev_join[i], hs[i]->stream));
        OMM_CUDA_TRY(cudaStreamWaitEvent(gs, ev_join[i], 0));
    }
    return OMM_OK;
}

// One first-phase CG step of every system: the three split products as grouped
// persistent launches on the group stream, the per-system line minimum, updates
// and direction on the systems' own streams in between.
int group_iteration(omm_handle **hs, int count, const GroupList *L, const int *mode, cudaStream_t gs,
                    cudaEvent_t ev_fork, cudaEvent_t *ev_join) {
    TRY(run_group_list(L[0], mode[0], hs[0], gs));
    TRY(run_group_list(L[1], mode[1], hs[0], gs));
    TRY(fork_join(hs, count, gs, ev_fork, ev_join, [](omm_handle *h) { return mixed_glue1(h, false); }));
    TRY(run_group_list(L[2], mode[2], hs[0], gs));
    return fork_join(hs, count, gs, ev_fork, ev_join, [](omm_handle *h) { return mixed_direction(h, 0); });
}

}  // namespace

extern "C" {

int omm_batch_solve_grouped(omm_handle **handles, int32_t count, const double *const *W0, int32_t W0_on_device,
                            double tol, int32_t tile_mode, double *E_out, int32_t *iters_out, int32_t *status_out) {
    using omm::tc::LIST_PAIR;
    using omm::tc::LIST_SINGLE;
    if (handles == nullptr || count < 1 || tile_mode < -1 || tile_mode > 1) return OMM_ERR_ARG;
    for (int32_t i = 0; i < count; ++i) {
        omm_handle *h = handles[i];
        if (h == nullptr) return OMM_ERR_ARG;
        for (int32_t j = 0; j < i; ++j)
            if (handles[j] == h) return OMM_ERR_ARG;
        if (h->sparse || h->opt.precision != OMM_PREC_MIXED || h->opt.split_digits != 2 || h->opt.cholesky ||
            h->opt.precon != 0 || h->profiling || h->stream == nullptr || h->stream == cudaStreamLegacy ||
            h->stream == cudaStreamPerThread || h->opt.dir_digits != handles[0]->opt.dir_digits) {
            omm::set_error("omm_batch_solve_grouped: handle %d is not a dense mixed-precision handle with two "
                           "split digits, no Cholesky or preconditioning, profiling off, its own stream and "
                           "the first handle's dir_digits", i);
            return OMM_ERR_UNSUPPORTED;
        }
        for (int32_t j = 0; j < i; ++j)
            if (handles[j]->stream == h->stream) {
                omm::set_error("omm_batch_solve_grouped: handles %d and %d share a stream", j, i);
                return OMM_ERR_UNSUPPORTED;
            }
    }
    // ---- phase 1 of every system in lock step
    for (int32_t i = 0; i < count; ++i) TRY(begin_setup(handles[i], W0 ? W0[i] : nullptr, W0_on_device, tol));
    struct Ungroup {
        omm_handle **hs;
        int32_t count;
        ~Ungroup() {
            for (int32_t i = 0; i < count; ++i) hs[i]->grouped = false;
        }
    } ungroup{handles, count};
    for (int32_t i = 0; i < count; ++i) handles[i]->grouped = true;
    cudaStream_t gs = nullptr;
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_join((size_t)count, nullptr);
    GroupList lists[2][3];
    cudaGraphExec_t gexec = nullptr;
    int rc = OMM_OK;
    auto cleanup = [&]() {
        if (gs) cudaStreamSynchronize(gs);
        if (gexec) cudaGraphExecDestroy(gexec);
        for (auto &row : lists)
            for (auto &L : row) L.release();
        for (auto e : ev_join)
            if (e) cudaEventDestroy(e);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (gs) cudaStreamDestroy(gs);
    };
#define GTRY(x)                  \
    do {                         \
        rc = (x);                \
        if (rc != OMM_OK) {      \
            cleanup();           \
            return rc;           \
        }                        \
    } while (0)
#define GCUDA(x) GTRY((x) == cudaSuccess ? OMM_OK : (omm::set_error("%s failed", #x), OMM_ERR_CUDA))
    GCUDA(cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking));
    GCUDA(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
    for (auto &e : ev_join) GCUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    for (int32_t i = 0; i < count; ++i) {
        GCUDA(cudaEventRecord(ev_join[i], handles[i]->stream));
        GCUDA(cudaStreamWaitEvent(gs, ev_join[i], 0));
    }
    // ---- tile modes: given, stored for this group, or timed now (each stage's product
    // is a function of operands the start has already written, so timing both modes
    // once and then running the step changes nothing)
    int mode[3] = {tile_mode, tile_mode, tile_mode};
    TuneEntry te;
    for (int k = 0; k < 3; ++k) {
        te.mode[k] = tile_mode;
        te.ms[k][0] = te.ms[k][1] = 0.f;
    }
    for (int32_t i = 0; i < count; ++i) {
        te.sig.push_back(handles[i]->m);
        te.sig.push_back(handles[i]->n);
    }
    bool tuned = tile_mode >= 0;
    if (!tuned) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        for (const auto &e : g_tune)
            if (e.sig == te.sig) {
                for (int k = 0; k < 3; ++k) mode[k] = e.mode[k];
                te = e;
                tuned = true;
            }
    }
    for (int k = 0; k < 3; ++k)
        for (int md : {LIST_SINGLE, LIST_PAIR})
            if (!tuned || mode[k] == md) GTRY(build_group_list(handles, count, k, md, lists[md][k]));
    if (!tuned) {
        cudaEvent_t t0, t1;
        GCUDA(cudaEventCreate(&t0));
        GCUDA(cudaEventCreate(&t1));
        for (int k = 0; k < 3; ++k) {
            for (int md : {LIST_SINGLE, LIST_PAIR}) {
                float best = 1e30f;
                for (int rep = 0; rep < 3; ++rep) {
                    GCUDA(cudaEventRecord(t0, gs));
                    GTRY(run_group_list(lists[md][k], md, handles[0], gs));
                    GCUDA(cudaEventRecord(t1, gs));
                    GCUDA(cudaEventSynchronize(t1));
                    float ms = 0.f;
                    GCUDA(cudaEventElapsedTime(&ms, t0, t1));
                    if (rep > 0 && ms < best) best = ms;
                }
                te.ms[k][md] = best;
            }
            mode[k] = te.ms[k][LIST_PAIR] <= te.ms[k][LIST_SINGLE] ? LIST_PAIR : LIST_SINGLE;
            te.mode[k] = mode[k];
        }
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune.push_back(te);
    }
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_last_tune = te;
        for (int k = 0; k < 3; ++k) g_last_tune.mode[k] = mode[k];
    }
    GroupList use[3] = {lists[mode[0]][0], lists[mode[1]][1], lists[mode[2]][2]};
    // ---- a chunk of first-phase steps, captured once, replayed until every system is done
    const int chunk = 8;
    const int64_t before = omm_kernel_launches();
    GCUDA(cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal));
    int crc = OMM_OK;
    for (int c = 0; c < chunk && crc == OMM_OK; ++c)
        crc = group_iteration(handles, count, use, mode, gs, ev_fork, ev_join.data());
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(gs, &graph);
    if (crc != OMM_OK || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        omm::set_error("grouped chunk capture failed: %s", cudaGetErrorString(ce));
        cleanup();
        return crc != OMM_OK ? crc : OMM_ERR_CUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
        gexec = nullptr;
        omm::set_error("grouped chunk graph instantiation failed: %s", cudaGetErrorString(ie));
        cleanup();
        return OMM_ERR_CUDA;
    }
    const int64_t per_chunk = omm_kernel_launches() - before;
    omm::count_launch(-per_chunk);
    for (;;) {
        GCUDA(cudaGraphLaunch(gexec, gs));
        omm::count_launch(per_chunk);
        for (int32_t i = 0; i < count; ++i)
            GCUDA(cudaMemcpyAsync(handles[i]->hstate, handles[i]->dstate, sizeof(omm::DevState),
                                  cudaMemcpyDeviceToHost, gs));
        GCUDA(cudaStreamSynchronize(gs));
        bool all = true;
        for (int32_t i = 0; i < count; ++i)
            if (!handles[i]->hstate->done && !handles[i]->hstate->wait_timeout) all = false;
        if (all) break;
    }
    // ---- phase 2 (refinement) per system on its own stream, as omm_batch_solve
    for (int32_t i = 0; i < count; ++i) handles[i]->grouped = false;
    GCUDA(cudaEventRecord(ev_fork, gs));
    for (int32_t i = 0; i < count; ++i) {
        GCUDA(cudaStreamWaitEvent(handles[i]->stream, ev_fork, 0));
        GCUDA(cudaEventRecord(handles[i]->ev_poll, handles[i]->stream));
    }
    cleanup();
#undef GTRY
#undef GCUDA
    return drive_batch(handles, count, E_out, iters_out, status_out);
}

int omm_batch_last_tuning(int32_t *modes, float *ms) {
    if (modes == nullptr) return OMM_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (int k = 0; k < 3; ++k) {
        modes[k] = g_last_tune.mode[k];
        if (ms) {
            ms[2 * k] = g_last_tune.ms[k][0];
            ms[2 * k + 1] = g_last_tune.ms[k][1];
        }
    }
    return OMM_OK;
}

int omm_get_diag(omm_handle *h, omm_diag *d) {
    if (h == nullptr || d == nullptr) return OMM_ERR_ARG;
    *d = h->diag;
    return OMM_OK;
}

int omm_get_density(omm_handle *h, int32_t which, double *dst, int32_t on_device) {
    if (h == nullptr || dst == nullptr || (which != OMM_DENSITY_RHO && which != OMM_DENSITY_RHO_E))
        return OMM_ERR_ARG;
    if (!h->solved || h->phase != PH_IDLE) return OMM_ERR_STATE;
    if (h->sparse) {
        // rho / rho_E on the pattern of S (section "Solver library"): P_H's blocks
        omm::sp::Dev &d = h->sd;
        if (d.Trp == nullptr) {
            omm::sp::DensHost dh;
            TRY(omm::sp::build_density(h->sh, dh));
            TRY(omm::sp::upload_density(dh, d));
        }
        const int64_t len = d.nnzH * d.bm * d.bm;
        double *out = dst;
        if (!on_device) {
            if (h->dOut == nullptr) TRY(dalloc(&h->dOut, (size_t)len));
            out = h->dOut;
        }
        TRY(omm::sp::density(d, which == OMM_DENSITY_RHO_E ? 1 : 0, h->diag.eta, out, h->stream));
        if (!on_device)
            OMM_CUDA_TRY(cudaMemcpyAsync(dst, out, (size_t)len * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        OMM_CUDA_TRY(cudaStreamSynchronize(h->stream));
        return OMM_OK;
    }
    const int64_t m = h->m, n = h->n, mm = m * m;
    cudaStream_t st = h->stream;
    const int s = h->opt.exact_digits;
    if (h->dK == nullptr) {
        const int64_t b1 = omm_op_exact_gemm_workspace_bytes(m, n, m, s);   // [H'|S] W
        const int64_t b2 = omm_op_exact_gemm_workspace_bytes(m, m, n, s);   // 2 T W^T
        h->dWs_bytes = b1 > b2 ? b1 : b2;
        TRY(dalloc(&h->dK, (size_t)(3 * n * n)));   // K, then [H'_W ; S_W] (2n x n)
        TRY(dalloc(&h->dT, (size_t)(m * n)));
        if (cudaMalloc(&h->dWs, (size_t)h->dWs_bytes) != cudaSuccess) return OMM_ERR_NOMEM;
    }
    double *out = dst;
    if (!on_device) {
        if (h->dOut == nullptr) TRY(dalloc(&h->dOut, (size_t)mm));
        out = h->dOut;
    }
    // H'_W and S_W afresh from the returned W (Eq. 5 defines rho from W; the
    // solve's running copies carry its increments' rounding), in the basis the
    // CG ran in: W~ with H~ and S = I for the Cholesky variant (W~^T W~ = W^T S W)
    const double *Wr = h->WD;
    const double *Wout = h->opt.cholesky ? h->Wsave : h->WD;   // the solution in the original basis
    double *K = h->dK, *HSW = h->dK + n * n;                    // HSW: [H'_W ; S_W], ld 2n
    const int need_h = which == OMM_DENSITY_RHO_E;
    for (int part = need_h ? 0 : 1; part < 2; ++part) {
        const double *A = h->HS + part * mm;                    // part 0: H', part 1: S
        TRY(omm_op_exact_gemm(0, 0, m, n, m, s, 1.0, A, m, Wr, m, 0.0, nullptr, m, h->dT, m, h->dWs, h->dWs_bytes,
                              st));
        TRY(omm_op_exact_gemm(1, 0, n, n, m, s, 1.0, Wr, m, h->dT, m, 0.0, nullptr, n, HSW + part * n, 2 * n,
                              h->dWs, h->dWs_bytes, st));
    }
    TRY(omm::launch_density_K(n, HSW, h->diag.eta, need_h, K, st));
    // T = W K, then 2 T W^T, both with exact-digit tensor-core products
    TRY(omm_op_exact_gemm(0, 0, m, n, n, s, 1.0, Wout, m, K, n, 0.0, nullptr, m, h->dT, m, h->dWs, h->dWs_bytes,
                          st));
    TRY(omm_op_exact_gemm(0, 1, m, m, n, s, 2.0, h->dT, m, Wout, m, 0.0, nullptr, m, out, m, h->dWs, h->dWs_bytes,
                          st));
    if (!on_device) OMM_CUDA_TRY(cudaMemcpyAsync(dst, out, (size_t)mm * sizeof(double), cudaMemcpyDeviceToHost, st));
    OMM_CUDA_TRY(cudaStreamSynchronize(st));
    return OMM_OK;
}

int omm_get_array(omm_handle *h, int32_t which, double *dst, int32_t on_device) {
    if (h == nullptr || dst == nullptr) return OMM_ERR_ARG;
    if (h->sparse) {
        const omm::sp::Dev &d = h->sd;
        const int64_t bw = (int64_t)d.bm * d.bn, bq = (int64_t)d.bn * d.bn;
        const double *src = nullptr;
        int64_t len = 0;
        switch (which) {
            case 0: src = d.W; len = d.nnzW * bw; break;
            case 1: src = d.HW; len = d.nnzHW * bw; break;
            case 2: src = d.SW; len = d.nnzHW * bw; break;
            case 3: src = d.G; len = d.nnzW * bw; break;
            case 4: src = d.D; len = d.nnzW * bw; break;
            case 5: src = d.h0; len = d.nnzN * bq; break;
            case 6: src = d.s0; len = d.nnzN * bq; break;
            default: return OMM_ERR_ARG;
        }
        OMM_CUDA_TRY(cudaMemcpyAsync(dst, src, len * sizeof(double),
                                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
        OMM_CUDA_TRY(cudaStreamSynchronize(h->stream));
        return OMM_OK;
    }
    const int64_t m = h->m, n = h->n, mn = m * n;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaStream_t st = h->stream;
    switch (which) {
        case 0: OMM_CUDA_TRY(cudaMemcpyAsync(dst, h->opt.cholesky ? h->Wsave : h->WD, mn * 8, kind, st)); break;
        case 1: OMM_CUDA_TRY(cudaMemcpyAsync(dst, h->SWHW + mn, mn * 8, kind, st)); break;
        case 2: OMM_CUDA_TRY(cudaMemcpyAsync(dst, h->SWHW, mn * 8, kind, st)); break;
        case 3: OMM_CUDA_TRY(cudaMemcpyAsync(dst, h->G, mn * 8, kind, st)); break;
        case 4: OMM_CUDA_TRY(cudaMemcpyAsync(dst, h->WD + mn, mn * 8, kind, st)); break;
        case 5:
        case 6: {
            const double *src = h->h0s0 + (which == 6 ? n : 0);
            OMM_CUDA_TRY(cudaMemcpy2DAsync(dst, n * 8, src, 2 * n * 8, n * 8, n, kind, st));
            break;
        }
        default: return OMM_ERR_ARG;
    }
    OMM_CUDA_TRY(cudaStreamSynchronize(st));
    return OMM_OK;
}

void omm_destroy(omm_handle *h) { free_handle(h); }

int omm_get_pattern(omm_handle *h, int32_t which, int64_t *rowptr, int32_t *col) {
    if (h == nullptr || !h->sparse || rowptr == nullptr || col == nullptr) return OMM_ERR_ARG;
    const omm::sp::Host &hs = h->sh;
    const int64_t nbr = hs.P.nbr;
    switch (which) {
        case OMM_PATTERN_H: {
            if (!h->have_HS) return OMM_ERR_STATE;
            std::vector<unsigned char> keep((size_t)h->sd.nnzH);
            OMM_CUDA_TRY(cudaMemcpy(keep.data(), h->sd.keep, keep.size(), cudaMemcpyDeviceToHost));
            int64_t k = 0;
            rowptr[0] = 0;
            for (int64_t I = 0; I < nbr; ++I) {
                for (int64_t b = hs.Hrp[I]; b < hs.Hrp[I + 1]; ++b)
                    if (keep[b]) col[k++] = hs.Hcol[b];
                rowptr[I + 1] = k;
            }
            return OMM_OK;
        }
        case OMM_PATTERN_W:
            std::copy(hs.Wrp.begin(), hs.Wrp.end(), rowptr);
            std::copy(hs.Wcol.begin(), hs.Wcol.end(), col);
            return OMM_OK;
        case OMM_PATTERN_HW:
            std::copy(hs.HWrp.begin(), hs.HWrp.end(), rowptr);
            std::copy(hs.HWcol.begin(), hs.HWcol.end(), col);
            return OMM_OK;
        case OMM_PATTERN_N:
            std::copy(hs.Nrp.begin(), hs.Nrp.end(), rowptr);
            std::copy(hs.Ncol.begin(), hs.Ncol.end(), col);
            return OMM_OK;
        default:
            return OMM_ERR_ARG;
    }
}

int omm_set_profiling(omm_handle *h, int32_t on) {
    if (h == nullptr) return OMM_ERR_ARG;
    h->profiling = on != 0;
    return OMM_OK;
}

int omm_get_stage_times(omm_handle *h, double *ms, int64_t *launches, int32_t nstages, int32_t reset) {
    if (h == nullptr || nstages < 0) return OMM_ERR_ARG;
    for (int i = 0; i < nstages && i < OMM_NSTAGES; ++i) {
        if (ms) ms[i] = h->stage_ms[i];
        if (launches) launches[i] = h->stage_launches[i];
    }
    if (reset) {
        for (int i = 0; i < OMM_NSTAGES; ++i) {
            h->stage_ms[i] = 0.0;
            h->stage_launches[i] = 0;
        }
    }
    return OMM_OK;
}

int64_t omm_kernel_launches(void) { return omm::launch_count(); }

}  // extern "C"
