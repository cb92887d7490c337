// Linear-scaling form: host pattern structures and device pieces (sparse.cu).
#pragma once

#include <stdint.h>

#include <vector>

#include "omm_internal.cuh"

namespace omm {
namespace sp {

// Block patterns as given by the caller (block CSR over basis-atom rows).
struct Pattern {
    int32_t bm = 0, bn = 0;
    int64_t nbr = 0, nbc = 0;
    const int64_t *Hrp = nullptr;
    const int32_t *Hcol = nullptr;
    const int64_t *Wrp = nullptr;
    const int32_t *Wcol = nullptr;
};

// Host copy of the patterns, the structural product patterns and the gather lists.
struct Host {
    Pattern P;
    std::vector<int64_t> Hrp, Wrp, HWrp, Nrp;
    std::vector<int32_t> Hcol, Wcol, HWcol, Ncol;
    std::vector<int32_t> Ntr;               // transpose index within P_N
    std::vector<unsigned char> Ndiag;       // block on the diagonal of P_N
    std::vector<int32_t> WtoHW;             // position of each W block inside P_HW
    std::vector<int64_t> Prp;               // products: per P_HW block
    std::vector<int32_t> Ph, Pw;
    std::vector<int64_t> Crp;               // contractions: per P_N block
    std::vector<int32_t> Ca, Cb;
    std::vector<int64_t> Grp;               // gradient: per P_W block
    std::vector<int32_t> Gb, Gq;
    std::vector<int64_t> WcolRp, WcolIdx;   // W blocks by column
};

// Gather lists of the density matrices (built at their first request):
//   T = W (2I - S_W) on P_HW: block (I, b) <- W block (I, a) x N block (a, b);
//   rho on P_H:              block (I, J) <- T block (I, b) x W block (J, b)^T.
struct DensHost {
    std::vector<int64_t> Trp, Rrp;
    std::vector<int32_t> Tw, Tq, Rt, Rw;
};

// Device arrays of one sparse handle.
struct Dev {
    int32_t bm = 0, bn = 0;
    int64_t nbr = 0, nbc = 0, nnzH = 0, nnzW = 0, nnzHW = 0, nnzN = 0;
    int64_t *Hrp = nullptr, *Prp = nullptr, *Crp = nullptr, *Grp = nullptr;
    int32_t *Hcol = nullptr, *Ph = nullptr, *Pw = nullptr, *Ca = nullptr, *Cb = nullptr, *Gb = nullptr,
            *Gq = nullptr, *WtoHW = nullptr, *Ntr = nullptr;
    unsigned char *Ndiag = nullptr, *keep = nullptr;
    double *HS = nullptr, *Hin = nullptr;
    double *W = nullptr, *D = nullptr, *G = nullptr, *Gp = nullptr;
    double *HW = nullptr, *SW = nullptr, *HD = nullptr, *SD = nullptr;
    double *h0 = nullptr, *s0 = nullptr, *X = nullptr, *Y = nullptr, *h2 = nullptr, *s2 = nullptr;
    // density matrices (allocated with their lists)
    int64_t *Trp = nullptr, *Rrp = nullptr;
    int32_t *Tw = nullptr, *Tq = nullptr, *Rt = nullptr, *Rw = nullptr;
    double *K = nullptr, *T = nullptr;
    // norm-based screening of the block products (allocated when eps > 0): squared
    // Frobenius norms of H' and S ([nnzH][2]), W, D, H'W, SW, H'D, SD, H_W, S_W blocks
    double screen_eps2 = 0.0;
    double *nrm = nullptr;
    double *nHS = nullptr, *nW = nullptr, *nD = nullptr, *nHW = nullptr, *nSW = nullptr, *nHD = nullptr,
           *nSD = nullptr, *nh0 = nullptr, *ns0 = nullptr;
    bool screening() const { return screen_eps2 > 0.0; }
    // mixed form (allocated by mixed_alloc): FP32 shadows of H' and S ([nnzH][2]), W,
    // H'W, SW, H_W, S_W, and the FP32 increments D, G, Gp, H'D, SD, X, Y, h2, s2
    bool mixed = false;
    float *fbuf = nullptr;
    float *HS32 = nullptr, *W32 = nullptr, *D32 = nullptr, *G32 = nullptr, *Gp32 = nullptr, *HW32 = nullptr,
          *SW32 = nullptr, *HD32 = nullptr, *SD32 = nullptr, *h032 = nullptr, *s032 = nullptr, *X32 = nullptr,
          *Y32 = nullptr, *h232 = nullptr, *s232 = nullptr;
    // the FP32 contraction by P_N rows (mixed form): row J's W and D blocks (W's
    // column J, WcolRp / WcolIdx) staged in shared memory, each triple's W block
    // named by its slot in that column (CaSlot); maxcol = 0: not built (a column
    // longer than the staging allows), the per-block kernel runs instead
    int64_t *Nrp = nullptr, *WcolRp = nullptr;
    int32_t *WcolIdx = nullptr;
    uint16_t *CaSlot = nullptr;
    int maxcol = 0;
};

// which block norms to refresh (norms())
enum { NRM_HS = 1, NRM_W = 2, NRM_D = 4, NRM_HWSW = 8, NRM_HDSD = 16, NRM_N = 32 };

// Validate the caller's patterns and build everything host-side (OMM_ERR_PATTERN on malformed input).
int build(const Pattern &P, Host &out);
int upload(const Host &hs, Dev &d);
void release(Dev &d);

// Per-(H,S) setup: copy, block filtering, Gershgorin eta (optional), shift and pack.
int set_HS(Dev &d, const double *H, const double *S, bool on_device, double eps, bool eta_auto, double *scratch,
           unsigned int *counter, DevState *state, cudaStream_t st);

int build_density(const Host &hs, DensHost &out);
int upload_density(const DensHost &dh, Dev &d);
// rho (mode 0) or rho_E (mode 1) on P_H into out (nnzH blocks of bm x bm, row-major,
// P_H's CSR order), from W with S_W and H'_W formed afresh
int density(Dev &d, int mode, double eta, double *out, cudaStream_t st);

// Norm-based screening of the CG's block products: a block product A_ik B_kj is
// skipped when ||A_ik||_F ||B_kj||_F < eps (squared norms compared with eps^2).
// eps <= 0 leaves screening off and allocates nothing.
int screen_alloc(Dev &d, double eps);
// refresh the squared norms named by `which` (NRM_* flags); no-op when screening is off
int norms(Dev &d, int which, const DevState *state, cudaStream_t st);

// One step's pieces.  The n* arguments are the squared norms of the right-hand
// operand blocks (products: of Din; contract: of W-side, D-side, H'D-side and
// SD-side operands); nullptr, or screening off, multiplies every block pair.
int products(Dev &d, const double *Din, double *HDo, double *SDo, const double *nDin, const DevState *state,
             cudaStream_t st);
int contract(Dev &d, const double *Wl, const double *Dl, const double *HDr, const double *SDr, double *Xo,
             double *Yo, double *h2o, double *s2o, const double *nWl, const double *nDl, const double *nHDr,
             const double *nSDr, const DevState *state, cudaStream_t st);
int gradient(Dev &d, const DevState *state, cudaStream_t st);

// Mixed form.  mixed_alloc: the FP32 arrays (about 60% of the FP64 ones).
// mixed_shadow_HS: FP32 copies of H' and S (after set_HS).  mixed_begin: FP32
// shadows and increments from the FP64 start (W, H'W, SW, H_W, S_W, G, Gp, D).
// One first-phase CG step, in order: mixed_products (H'D, SD), mixed_contract
// (X, Y, h2, s2), mixed_coeffs (quartic and line minimum), mixed_update (FP64
// W, H'W, SW, H_W, S_W from FP32 increments, shadows, energy and stop test),
// mixed_gradient, mixed_direction.
int mixed_alloc(const Host &hs, Dev &d);
int mixed_shadow_HS(Dev &d, cudaStream_t st);
int mixed_begin(Dev &d, const DevState *state, cudaStream_t st);
int mixed_products(Dev &d, const DevState *state, cudaStream_t st);
int mixed_contract(Dev &d, const DevState *state, cudaStream_t st);
int mixed_coeffs(Dev &d, double *scratch, unsigned int *counter, DevState *state, cudaStream_t st);
int mixed_update(Dev &d, double *scratch, unsigned int *counter, DevState *state, cudaStream_t st);
int mixed_gradient(Dev &d, const DevState *state, cudaStream_t st);
int mixed_direction(Dev &d, double *scratch, unsigned int *counter, DevState *state, cudaStream_t st);
int coeffs(Dev &d, double *scratch, unsigned int *counter, DevState *state, cudaStream_t st);
int nn_update(Dev &d, int64_t n, int mode, double *scratch, unsigned int *counter, DevState *state, cudaStream_t st);
int axpy(Dev &d, const DevState *state, cudaStream_t st);
int dots(Dev &d, int first, double *scratch, unsigned int *counter, DevState *state, cudaStream_t st);
int direction(Dev &d, const DevState *state, cudaStream_t st);

}  // namespace sp
}  // namespace omm
