// Linear-scaling (block-sparse) form of the OMM CG step.
//
// H and S share one block pattern P_H of bm x bm blocks; W (and D, G) live on
// the localisation pattern P_W of bm x bn blocks, fixed for the whole
// minimisation, and the gradient is kept on it (section "Solver library").
// The products live on structural patterns built once on the host:
//   P_HW = P_H . P_W            (H'W, SW, H'D, SD; contains P_W)
//   P_N  = P_W^T . P_HW         (H_W, S_W, X, Y, h2, s2; symmetric)
// Every output block is a gather over a precomputed list of operand-block
// pairs, summed in list order: no atomics, bitwise repeatable results.
//
// Device storage (FP64, blocks row-major, in pattern order):
//   HS   [nnzH][2][bm*bm]   H' and S block k side by side
//   W, D, G, Gp  [nnzW][bm*bn]
//   HW, SW, HD, SD [nnzHW][bm*bn]
//   h0, s0, X, Y, h2, s2  [nnzN][bn*bn]
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "fp_convert.cuh"
#include "linemin.cuh"
#include "omm_internal.cuh"
#include "sparse.cuh"

namespace omm {
namespace sp {

// ======================================================================== host: patterns
namespace {

// union of the W rows K over K in P_H(I, :): row I of P_HW
void build_hw(const Pattern &P, std::vector<int64_t> &rp, std::vector<int32_t> &col) {
    const int64_t nbr = P.nbr;
    rp.assign(nbr + 1, 0);
    col.clear();
    std::vector<int32_t> mark(P.nbc, -1);
    std::vector<int32_t> row;
    for (int64_t I = 0; I < nbr; ++I) {
        row.clear();
        for (int64_t h = P.Hrp[I]; h < P.Hrp[I + 1]; ++h) {
            const int32_t K = P.Hcol[h];
            for (int64_t w = P.Wrp[K]; w < P.Wrp[K + 1]; ++w) {
                const int32_t J = P.Wcol[w];
                if (mark[J] != (int32_t)I) {
                    mark[J] = (int32_t)I;
                    row.push_back(J);
                }
            }
        }
        std::sort(row.begin(), row.end());
        col.insert(col.end(), row.begin(), row.end());
        rp[I + 1] = (int64_t)col.size();
    }
}

// P_N = P_W^T P_HW via one bitset row per W block column
void build_n(const Pattern &P, const std::vector<int64_t> &hwrp, const std::vector<int32_t> &hwcol,
             std::vector<int64_t> &rp, std::vector<int32_t> &col) {
    const int64_t nbc = P.nbc, words = (nbc + 63) / 64;
    std::vector<uint64_t> bits((size_t)(nbc * words), 0ull);
    std::vector<uint64_t> rowbits((size_t)words);
    for (int64_t I = 0; I < P.nbr; ++I) {
        std::fill(rowbits.begin(), rowbits.end(), 0ull);
        for (int64_t b = hwrp[I]; b < hwrp[I + 1]; ++b) rowbits[hwcol[b] >> 6] |= 1ull << (hwcol[b] & 63);
        for (int64_t a = P.Wrp[I]; a < P.Wrp[I + 1]; ++a) {
            uint64_t *dst = &bits[(size_t)P.Wcol[a] * words];
            for (int64_t q = 0; q < words; ++q) dst[q] |= rowbits[q];
        }
    }
    rp.assign(nbc + 1, 0);
    col.clear();
    for (int64_t J = 0; J < nbc; ++J) {
        const uint64_t *src = &bits[(size_t)J * words];
        for (int64_t q = 0; q < words; ++q) {
            uint64_t v = src[q];
            while (v) {
                const int t = __builtin_ctzll(v);
                col.push_back((int32_t)(q * 64 + t));
                v &= v - 1;
            }
        }
        rp[J + 1] = (int64_t)col.size();
    }
}

}  // namespace

int build(const Pattern &P, Host &out) {
    // ---- validate
    if (P.nbr <= 0 || P.nbc <= 0 || P.bm <= 0 || P.bn <= 0) return OMM_ERR_PATTERN;
    for (int which = 0; which < 2; ++which) {
        const int64_t *rp = which ? P.Wrp : P.Hrp;
        const int32_t *c = which ? P.Wcol : P.Hcol;
        const int64_t ncol = which ? P.nbc : P.nbr;
        if (rp[0] != 0) return OMM_ERR_PATTERN;
        for (int64_t I = 0; I < P.nbr; ++I) {
            if (rp[I + 1] < rp[I]) return OMM_ERR_PATTERN;
            for (int64_t k = rp[I]; k < rp[I + 1]; ++k) {
                if (c[k] < 0 || c[k] >= ncol) return OMM_ERR_PATTERN;
                if (k > rp[I] && c[k] <= c[k - 1]) return OMM_ERR_PATTERN;   // sorted, unique
            }
        }
    }
    // H must hold its diagonal blocks and be structurally symmetric
    for (int64_t I = 0; I < P.nbr; ++I) {
        const int32_t *b = P.Hcol + P.Hrp[I], *e = P.Hcol + P.Hrp[I + 1];
        if (!std::binary_search(b, e, (int32_t)I)) return OMM_ERR_PATTERN;
        for (const int32_t *k = b; k < e; ++k) {
            const int32_t *b2 = P.Hcol + P.Hrp[*k], *e2 = P.Hcol + P.Hrp[*k + 1];
            if (!std::binary_search(b2, e2, (int32_t)I)) return OMM_ERR_PATTERN;
        }
    }
    out.P = P;
    out.Hrp.assign(P.Hrp, P.Hrp + P.nbr + 1);
    out.Hcol.assign(P.Hcol, P.Hcol + P.Hrp[P.nbr]);
    out.Wrp.assign(P.Wrp, P.Wrp + P.nbr + 1);
    out.Wcol.assign(P.Wcol, P.Wcol + P.Wrp[P.nbr]);
    out.P.Hrp = out.Hrp.data();
    out.P.Hcol = out.Hcol.data();
    out.P.Wrp = out.Wrp.data();
    out.P.Wcol = out.Wcol.data();
    const Pattern &Q = out.P;
    build_hw(Q, out.HWrp, out.HWcol);
    build_n(Q, out.HWrp, out.HWcol, out.Nrp, out.Ncol);
    const int64_t nnzH = Q.Hrp[Q.nbr], nnzW = Q.Wrp[Q.nbr];
    const int64_t nnzHW = out.HWrp[Q.nbr], nnzN = out.Nrp[Q.nbc];

    // ---- transpose of P_N (symmetric pattern): index of (J2, J1) for each (J1, J2)
    out.Ntr.assign(nnzN, -1);
    out.Ndiag.assign(nnzN, 0);
    for (int64_t J = 0; J < Q.nbc; ++J)
        for (int64_t q = out.Nrp[J]; q < out.Nrp[J + 1]; ++q) {
            const int32_t J2 = out.Ncol[q];
            const int32_t *b = out.Ncol.data() + out.Nrp[J2], *e = out.Ncol.data() + out.Nrp[J2 + 1];
            const int32_t *f = std::lower_bound(b, e, (int32_t)J);
            if (f == e || *f != (int32_t)J) return OMM_ERR_PATTERN;
            out.Ntr[q] = (int32_t)(f - out.Ncol.data());
            out.Ndiag[q] = (J2 == J) ? 1 : 0;
        }
    // ---- W block -> its position inside P_HW
    out.WtoHW.assign(nnzW, -1);
    for (int64_t I = 0; I < Q.nbr; ++I)
        for (int64_t a = Q.Wrp[I]; a < Q.Wrp[I + 1]; ++a) {
            const int32_t *b = out.HWcol.data() + out.HWrp[I], *e = out.HWcol.data() + out.HWrp[I + 1];
            const int32_t *f = std::lower_bound(b, e, Q.Wcol[a]);
            out.WtoHW[a] = (int32_t)(f - out.HWcol.data());
        }
    // ---- product lists: HW block o = (I, J) <- (H block (I, K), W block (K, J)), K ascending
    {
        std::vector<int32_t> pos(Q.nbc, -1);
        out.Prp.assign(nnzHW + 1, 0);
        for (int pass = 0; pass < 2; ++pass) {
            std::vector<int64_t> fill;
            if (pass == 1) {
                for (int64_t o = 0; o < nnzHW; ++o) out.Prp[o + 1] += out.Prp[o];
                out.Ph.resize(out.Prp[nnzHW]);
                out.Pw.resize(out.Prp[nnzHW]);
                fill.assign(out.Prp.begin(), out.Prp.end() - 1);
            }
            for (int64_t I = 0; I < Q.nbr; ++I) {
                for (int64_t o = out.HWrp[I]; o < out.HWrp[I + 1]; ++o) pos[out.HWcol[o]] = (int32_t)o;
                for (int64_t h = Q.Hrp[I]; h < Q.Hrp[I + 1]; ++h) {
                    const int32_t K = Q.Hcol[h];
                    for (int64_t w = Q.Wrp[K]; w < Q.Wrp[K + 1]; ++w) {
                        const int32_t o = pos[Q.Wcol[w]];
                        if (pass == 0) {
                            out.Prp[o + 1] += 1;
                        } else {
                            out.Ph[fill[o]] = (int32_t)h;
                            out.Pw[fill[o]] = (int32_t)w;
                            ++fill[o];
                        }
                    }
                }
            }
        }
    }
    // ---- contraction lists: N block q = (J1, J2) <- (W block (I, J1), HW block (I, J2)), I ascending
    {
        // W blocks by column: (I, a) pairs with Wcol[a] = J, I ascending
        std::vector<int64_t> crp(Q.nbc + 1, 0);
        for (int64_t a = 0; a < nnzW; ++a) crp[Q.Wcol[a] + 1] += 1;
        for (int64_t J = 0; J < Q.nbc; ++J) crp[J + 1] += crp[J];
        std::vector<int64_t> cidx(nnzW), cfill(crp.begin(), crp.end() - 1);
        std::vector<int32_t> crow(nnzW);
        for (int64_t I = 0; I < Q.nbr; ++I)
            for (int64_t a = Q.Wrp[I]; a < Q.Wrp[I + 1]; ++a) {
                cidx[cfill[Q.Wcol[a]]] = a;
                crow[cfill[Q.Wcol[a]]++] = (int32_t)I;
            }
        out.WcolRp = crp;
        out.WcolIdx = cidx;
        std::vector<int32_t> pos(Q.nbc, -1);
        out.Crp.assign(nnzN + 1, 0);
        for (int pass = 0; pass < 2; ++pass) {
            std::vector<int64_t> fill;
            if (pass == 1) {
                for (int64_t q = 0; q < nnzN; ++q) out.Crp[q + 1] += out.Crp[q];
                out.Ca.resize(out.Crp[nnzN]);
                out.Cb.resize(out.Crp[nnzN]);
                fill.assign(out.Crp.begin(), out.Crp.end() - 1);
            }
            for (int64_t J1 = 0; J1 < Q.nbc; ++J1) {
                for (int64_t q = out.Nrp[J1]; q < out.Nrp[J1 + 1]; ++q) pos[out.Ncol[q]] = (int32_t)q;
                for (int64_t c = crp[J1]; c < crp[J1 + 1]; ++c) {
                    const int64_t a = cidx[c];
                    const int32_t I = crow[c];
                    for (int64_t b = out.HWrp[I]; b < out.HWrp[I + 1]; ++b) {
                        const int32_t q = pos[out.HWcol[b]];
                        if (pass == 0) {
                            out.Crp[q + 1] += 1;
                        } else {
                            out.Ca[fill[q]] = (int32_t)a;
                            out.Cb[fill[q]] = (int32_t)b;
                            ++fill[q];
                        }
                    }
                }
                for (int64_t q = out.Nrp[J1]; q < out.Nrp[J1 + 1]; ++q) pos[out.Ncol[q]] = -1;
            }
        }
    }
    // ---- gradient lists: W block o = (I, J) <- (HW block (I, K), N block (K, J)), K ascending
    {
        std::vector<int32_t> posJ(Q.nbc, -1);
        out.Grp.assign(nnzW + 1, 0);
        for (int pass = 0; pass < 2; ++pass) {
            std::vector<int64_t> fill;
            if (pass == 1) {
                for (int64_t o = 0; o < nnzW; ++o) out.Grp[o + 1] += out.Grp[o];
                out.Gb.resize(out.Grp[nnzW]);
                out.Gq.resize(out.Grp[nnzW]);
                fill.assign(out.Grp.begin(), out.Grp.end() - 1);
            }
            for (int64_t J = 0; J < Q.nbc; ++J) {
                // row J of P_N: posJ[K] = index of (J, K); (K, J) is its transpose
                for (int64_t q = out.Nrp[J]; q < out.Nrp[J + 1]; ++q) posJ[out.Ncol[q]] = (int32_t)q;
                for (int64_t c = out.WcolRp[J]; c < out.WcolRp[J + 1]; ++c) {
                    const int64_t o = out.WcolIdx[c];
                    int64_t I = 0;
                    {   // row of W block o
                        const int64_t *f = std::upper_bound(out.Wrp.data(), out.Wrp.data() + Q.nbr + 1, o);
                        I = (f - out.Wrp.data()) - 1;
                    }
                    for (int64_t b = out.HWrp[I]; b < out.HWrp[I + 1]; ++b) {
                        const int32_t qJK = posJ[out.HWcol[b]];
                        if (qJK < 0) continue;
                        if (pass == 0) {
                            out.Grp[o + 1] += 1;
                        } else {
                            out.Gb[fill[o]] = (int32_t)b;
                            out.Gq[fill[o]] = out.Ntr[qJK];
                            ++fill[o];
                        }
                    }
                }
                for (int64_t q = out.Nrp[J]; q < out.Nrp[J + 1]; ++q) posJ[out.Ncol[q]] = -1;
            }
        }
    }
    (void)nnzH;
    return OMM_OK;
}

int build_density(const Host &hs, DensHost &out) {
    const Pattern &Q = hs.P;
    const int64_t nnzH = Q.Hrp[Q.nbr], nnzHW = hs.HWrp[Q.nbr];
    // T lists: (I, b) in P_HW <- W (I, a), N (a, b)
    {
        std::vector<int32_t> pos(Q.nbc, -1);
        out.Trp.assign(nnzHW + 1, 0);
        for (int pass = 0; pass < 2; ++pass) {
            std::vector<int64_t> fill;
            if (pass == 1) {
                for (int64_t o = 0; o < nnzHW; ++o) out.Trp[o + 1] += out.Trp[o];
                out.Tw.resize(out.Trp[nnzHW]);
                out.Tq.resize(out.Trp[nnzHW]);
                fill.assign(out.Trp.begin(), out.Trp.end() - 1);
            }
            for (int64_t I = 0; I < Q.nbr; ++I) {
                for (int64_t o = hs.HWrp[I]; o < hs.HWrp[I + 1]; ++o) pos[hs.HWcol[o]] = (int32_t)o;
                for (int64_t w = Q.Wrp[I]; w < Q.Wrp[I + 1]; ++w) {
                    const int32_t a = Q.Wcol[w];
                    for (int64_t q = hs.Nrp[a]; q < hs.Nrp[a + 1]; ++q) {
                        const int32_t o = pos[hs.Ncol[q]];
                        if (o < 0) continue;
                        if (pass == 0) {
                            out.Trp[o + 1] += 1;
                        } else {
                            out.Tw[fill[o]] = (int32_t)w;
                            out.Tq[fill[o]] = (int32_t)q;
                            ++fill[o];
                        }
                    }
                }
                for (int64_t o = hs.HWrp[I]; o < hs.HWrp[I + 1]; ++o) pos[hs.HWcol[o]] = -1;
            }
        }
    }
    // rho lists: (I, J) in P_H <- T (I, b), W (J, b) for b in row J of P_W
    // ((I, b) is in P_HW since J is in row I of P_H)
    {
        std::vector<int32_t> pos(Q.nbc, -1);
        out.Rrp.assign(nnzH + 1, 0);
        for (int64_t I = 0; I < Q.nbr; ++I)
            for (int64_t h = Q.Hrp[I]; h < Q.Hrp[I + 1]; ++h) {
                const int32_t J = Q.Hcol[h];
                out.Rrp[h + 1] = out.Rrp[h] + (Q.Wrp[J + 1] - Q.Wrp[J]);
            }
        out.Rt.resize(out.Rrp[nnzH]);
        out.Rw.resize(out.Rrp[nnzH]);
        for (int64_t I = 0; I < Q.nbr; ++I) {
            for (int64_t o = hs.HWrp[I]; o < hs.HWrp[I + 1]; ++o) pos[hs.HWcol[o]] = (int32_t)o;
            for (int64_t h = Q.Hrp[I]; h < Q.Hrp[I + 1]; ++h) {
                const int32_t J = Q.Hcol[h];
                int64_t f = out.Rrp[h];
                for (int64_t w = Q.Wrp[J]; w < Q.Wrp[J + 1]; ++w, ++f) {
                    const int32_t o = pos[Q.Wcol[w]];
                    if (o < 0) return OMM_ERR_PATTERN;   // cannot happen for P_HW = P_H P_W
                    out.Rt[f] = o;
                    out.Rw[f] = (int32_t)w;
                }
            }
            for (int64_t o = hs.HWrp[I]; o < hs.HWrp[I + 1]; ++o) pos[hs.HWcol[o]] = -1;
        }
    }
    return OMM_OK;
}

// ======================================================================== device kernels
namespace {

constexpr int NT = 256;

// Block sum / last-block combination (fixed order; same scheme as the dense kernels)
template <int NV>
__device__ void block_sum(double (&v)[NV], double *red) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double s = v[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        v[q] = s;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) red[warp * NV + q] = v[q];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double s = 0.0;
            for (int w = 0; w < NT / 32; ++w) s += red[w * NV + q];
            v[q] = s;
        }
    }
    __syncthreads();
}

template <int NV>
__device__ bool publish_and_collect(const double (&v)[NV], double *partials, unsigned int *counter,
                                    double (&tot)[NV], double *red) {
    __shared__ bool is_last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) partials[blockIdx.x * NV + q] = v[q];
        __threadfence();
        is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    // warp w sums values w, w + NT/32, ...: its lanes take blocks lane, lane + 32,
    // ... in order, then a fixed shuffle tree (one dependent chain per value on
    // the long-latency FP64 unit, instead of a block-wide tree per value)
    for (int q = threadIdx.x >> 5; q < NV; q += NT / 32) {
        double s = 0.0;
        // the lane's blocks in order, eight loads in flight at a time
        unsigned b = threadIdx.x & 31;
        for (; b + 224 < gridDim.x; b += 256) {
            double p[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) p[k] = __ldcg(&partials[(b + 32 * k) * NV + q]);
#pragma unroll
            for (int k = 0; k < 8; ++k) s += p[k];
        }
        for (; b < gridDim.x; b += 32) s += __ldcg(&partials[b * NV + q]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if ((threadIdx.x & 31) == 0) red[q] = s;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) tot[q] = red[q];
    if (threadIdx.x == 0) *counter = 0u;
    __syncthreads();   // red is free again for the caller
    return true;
}

__device__ __forceinline__ bool done(const DevState *s) { return s != nullptr && *((volatile const int *)&s->done); }

// ---- block filtering: keep[b] = ||H_b||^2 >= eps^2 or ||S_b||^2 >= eps^2, squares
// summed in row-major element order with one rounded product and add each.
__global__ void filter_kernel(int64_t nnzH, int bb, const double *H, const double *S, double eps2,
                              unsigned char *keep) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nnzH; b += (int64_t)gridDim.x * blockDim.x) {
        double sh = 0.0, ss = 0.0;
        for (int t = 0; t < bb; ++t) {
            sh = __dadd_rn(sh, __dmul_rn(H[b * bb + t], H[b * bb + t]));
            ss = __dadd_rn(ss, __dmul_rn(S[b * bb + t], S[b * bb + t]));
        }
        keep[b] = !(sh < eps2) || !(ss < eps2);
    }
}

// HS[b] = (keep ? H_b - eta S_b : 0, keep ? S_b : 0)
__global__ void shift_pack_kernel(int64_t nnzH, int bb, const double *H, const double *S,
                                  const unsigned char *keep, const DevState *state, double *HS) {
    const double eta = state->eta;
    const int64_t total = nnzH * bb;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = t / bb;
        const int e = (int)(t - b * bb);
        const bool k = keep[b] != 0;
        const double s = k ? S[t] : 0.0;
        HS[(b * 2) * bb + e] = k ? H[t] - eta * s : 0.0;
        HS[(b * 2 + 1) * bb + e] = s;
    }
}

// Gershgorin bound over the block rows: thread per matrix row
__global__ void __launch_bounds__(NT) gershgorin_kernel(int64_t nbr, int bm, const int64_t *Hrp, const int32_t *Hcol,
                                                         const double *H, const double *S, double *partials,
                                                         unsigned int *counter, DevState *state) {
    __shared__ double red[(NT / 32) * 3];
    double gmax = -INFINITY, lomin = INFINITY, himax = -INFINITY;
    const int64_t nrows = nbr * bm;
    for (int64_t row = (int64_t)blockIdx.x * NT + threadIdx.x; row < nrows; row += (int64_t)gridDim.x * NT) {
        const int64_t I = row / bm;
        const int r = (int)(row - I * bm);
        double sh = 0.0, ss = 0.0, dh = 0.0, ds = 0.0;
        for (int64_t b = Hrp[I]; b < Hrp[I + 1]; ++b) {
            const bool diag = Hcol[b] == (int32_t)I;
            for (int c = 0; c < bm; ++c) {
                const double vh = H[(b * bm + r) * bm + c], vs = S[(b * bm + r) * bm + c];
                if (diag && c == r) { dh = vh; ds = vs; }
                else { sh += fabs(vh); ss += fabs(vs); }
            }
        }
        gmax = fmax(gmax, dh + sh);
        lomin = fmin(lomin, ds - ss);
        himax = fmax(himax, ds + ss);
    }
    // block max/min then last-block combination (order-independent)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        gmax = fmax(gmax, __shfl_down_sync(0xffffffffu, gmax, off));
        lomin = fmin(lomin, __shfl_down_sync(0xffffffffu, lomin, off));
        himax = fmax(himax, __shfl_down_sync(0xffffffffu, himax, off));
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { red[w * 3] = gmax; red[w * 3 + 1] = lomin; red[w * 3 + 2] = himax; }
    __syncthreads();
    __shared__ bool is_last;
    if (threadIdx.x == 0) {
        double v0 = -INFINITY, v1 = INFINITY, v2 = -INFINITY;
        for (int q = 0; q < NT / 32; ++q) {
            v0 = fmax(v0, red[q * 3]);
            v1 = fmin(v1, red[q * 3 + 1]);
            v2 = fmax(v2, red[q * 3 + 2]);
        }
        partials[blockIdx.x * 3] = v0;
        partials[blockIdx.x * 3 + 1] = v1;
        partials[blockIdx.x * 3 + 2] = v2;
        __threadfence();
        is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last || threadIdx.x != 0) return;
    __threadfence();
    double g = -INFINITY, lo = INFINITY, hi = -INFINITY;
    for (unsigned b = 0; b < gridDim.x; ++b) {
        g = fmax(g, __ldcg(&partials[b * 3]));
        lo = fmin(lo, __ldcg(&partials[b * 3 + 1]));
        hi = fmax(hi, __ldcg(&partials[b * 3 + 2]));
    }
    *counter = 0u;
    if (!(lo > 0.0)) {
        state->status = OMM_ERR_NOT_SPD;
        state->eta = NAN;
        return;
    }
    state->eta = (g >= 0.0) ? g / lo : g / hi;
}

// FP32 gathers of the mixed form (8x2 blocks, no screening) in the products and
// gradient kernels load whole block rows and blocks as 8- and 16-byte vectors
// (every FP32 block array is 16-byte aligned: its blocks hold 64, 16 or 4 floats)
// instead of one scalar per element; the FMAs run in the scalar paths' order, so
// the results are the same bits.
template <typename T, int BM, int BN, bool SCREEN>
struct VecGather {
    static constexpr bool on = std::is_same<T, float>::value && BM == 8 && BN == 2 && !SCREEN;
};
__device__ __forceinline__ float4 ld4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }

// ---- products: HD_o = sum H'_(I,K) D_(K,J), SD_o likewise; warp per P_HW block,
// lanes 0..15 -> H'D element (r, c), lanes 16..31 -> SD element.
// Screening (SCREEN): the block product H'_(I,K) D_(K,J) (or S_(I,K) D_(K,J)) is
// skipped when ||H'_(I,K)||^2 ||D_(K,J)||^2 < eps^2, from the squared block norms
// nHS ([nnzH][2]: H', S) and nB (one per D block).
template <int BM, int BN, bool SCREEN, typename T = double>
__global__ void __launch_bounds__(NT) products_kernel(int64_t nnzHW, const int64_t *__restrict__ Prp,
                                                       const int32_t *__restrict__ Ph, const int32_t *__restrict__ Pw,
                                                       const T *__restrict__ HS, const T *__restrict__ D,
                                                       T *HD, T *SD, const double *__restrict__ nHS,
                                                       const double *__restrict__ nB, double eps2,
                                                       const DevState *state) {
    if (done(state)) return;
    if constexpr (VecGather<T, BM, BN, SCREEN>::on) {
        // FP32 (8x2 blocks): lane (which, r) computes both columns of row r from
        // its A row (two 16-byte loads) and the whole D block (four): two P_HW
        // blocks per warp, half the L1 bytes of a lane per output element; the
        // FMAs of each output run in k order, as in the scalar form
        const int lane = threadIdx.x & 31;
        const int r = lane & 7, which = (lane >> 3) & 1;
        const int64_t ngroups = ((int64_t)gridDim.x * NT) >> 4;
        for (int64_t o = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 4; o < nnzHW; o += ngroups) {
            float acc0 = 0.f, acc1 = 0.f;
#pragma unroll 2
            for (int64_t t = Prp[o]; t < Prp[o + 1]; ++t) {
                const float *A = HS + ((int64_t)Ph[t] * 2 + which) * 64 + r * 8;
                const float *B = D + (int64_t)Pw[t] * 16;
                const float4 a0 = ld4(A), a1 = ld4(A + 4);
                const float4 b0 = ld4(B), b1 = ld4(B + 4), b2 = ld4(B + 8), b3 = ld4(B + 12);
                acc0 = fmaf(a0.x, b0.x, acc0);
                acc1 = fmaf(a0.x, b0.y, acc1);
                acc0 = fmaf(a0.y, b0.z, acc0);
                acc1 = fmaf(a0.y, b0.w, acc1);
                acc0 = fmaf(a0.z, b1.x, acc0);
                acc1 = fmaf(a0.z, b1.y, acc1);
                acc0 = fmaf(a0.w, b1.z, acc0);
                acc1 = fmaf(a0.w, b1.w, acc1);
                acc0 = fmaf(a1.x, b2.x, acc0);
                acc1 = fmaf(a1.x, b2.y, acc1);
                acc0 = fmaf(a1.y, b2.z, acc0);
                acc1 = fmaf(a1.y, b2.w, acc1);
                acc0 = fmaf(a1.z, b3.x, acc0);
                acc1 = fmaf(a1.z, b3.y, acc1);
                acc0 = fmaf(a1.w, b3.z, acc0);
                acc1 = fmaf(a1.w, b3.w, acc1);
            }
            *reinterpret_cast<float2 *>((which ? SD : HD) + o * 16 + r * 2) = make_float2(acc0, acc1);
        }
    } else {
        const int lane = threadIdx.x & 31;
        constexpr int NE = BM * BN;          // outputs per block
        const int which = lane / 16, e = lane % 16;   // which: 0 = H', 1 = S
        const bool active = e < NE;
        const int r = e / BN, c = e % BN;
        const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
        for (int64_t o = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5; o < nnzHW; o += nwarps) {
            T acc = T(0);
#pragma unroll 4
            for (int64_t t = Prp[o]; t < Prp[o + 1]; ++t) {
                if (SCREEN && nHS[(int64_t)Ph[t] * 2 + which] * nB[Pw[t]] < eps2) continue;
                const T *A = HS + ((int64_t)Ph[t] * 2 + which) * BM * BM + r * BM;
                const T *B = D + (int64_t)Pw[t] * BM * BN + c;
                if (active) {
#pragma unroll
                    for (int k = 0; k < BM; ++k) acc = fma(A[k], B[k * BN], acc);
                }
            }
            if (active) (which ? SD : HD)[o * NE + e] = acc;
        }
    }
}

// ---- contractions on P_N: warp per N block q; 16 outputs (X, Y, h2, s2 of 2x2)
// with two lanes each splitting the basis index k.
// Screening: the pair (L block a, R block b) is skipped when ||L_a||^2 ||R_b||^2 < eps^2,
// with L = W or D and R = H'D or SD as the output matrix takes them.
template <int BM, int BN, bool SCREEN, typename T = double>
__global__ void __launch_bounds__(NT) contract_kernel(int64_t nnzN, const int64_t *__restrict__ Crp,
                                                       const int32_t *__restrict__ Ca, const int32_t *__restrict__ Cb,
                                                       const T *__restrict__ W, const T *__restrict__ D,
                                                       const T *__restrict__ HD, const T *__restrict__ SD,
                                                       T *X, T *Y, T *h2, T *s2,
                                                       const double *__restrict__ nW, const double *__restrict__ nD,
                                                       const double *__restrict__ nHD, const double *__restrict__ nSD,
                                                       double eps2, const int32_t *__restrict__ Ntr,
                                                       const DevState *state) {
    if (done(state)) return;
    const int lane = threadIdx.x & 31;
    static_assert(BN == 2, "contraction lanes assume 2 orbitals per W block");
    const int v = lane >> 1, half = lane & 1;
    const int mat = v >> 2, a = (v >> 1) & 1, b = v & 1;   // mat: 0 X, 1 Y, 2 h2, 3 s2
    const T *L = (mat < 2) ? W : D;
    const T *R = (mat == 0 || mat == 2) ? HD : SD;
    T *out = mat == 0 ? X : mat == 1 ? Y : mat == 2 ? h2 : s2;
    const double *nL = SCREEN ? ((mat < 2) ? nW : nD) : nullptr;
    const double *nR = SCREEN ? ((mat == 0 || mat == 2) ? nHD : nSD) : nullptr;
    // lower-triangle blocks with `Ntr` given: D^T H'D and D^T S D are symmetric, so
    // only X and Y are formed there (their transposes' blocks give h2, s2), each
    // output by four lanes splitting the basis index k
    const int v4 = lane >> 2, quarter = lane & 3;
    const int mat4 = v4 >> 2, a4 = (v4 >> 1) & 1, b4 = v4 & 1;   // mat4: 0 X, 1 Y
    const T *R4 = mat4 == 0 ? HD : SD;
    T *out4 = mat4 == 0 ? X : Y;
    const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
    if constexpr (VecGather<T, BM, BN, SCREEN>::on) {
        // FP32 (8x2 blocks): each eight-lane group of a warp takes one P_N block,
        // lane k of the group basis row k: per block triple it loads row k of the
        // W, D, H'D and SD blocks once (the L1's return bandwidth bounds these
        // gathers: 256 bytes per triple, each byte fetched once) and updates all
        // sixteen outputs (2x2 each of X, Y, h2, s2; X and Y only on the lower-
        // triangle blocks), which the group then sums over k.
        const int k = lane & 7, grp = lane >> 3;
        // warp-uniform loop: the four groups of a warp take blocks qb .. qb + 3, and
        // every lane runs the sums (a group past the end accumulates nothing)
        for (int64_t qb = (((int64_t)blockIdx.x * NT + threadIdx.x) >> 5) * 4; qb < nnzN; qb += nwarps * 4) {
            const int64_t q = qb + grp;
            const bool valid = q < nnzN;
            const bool lower = valid && Ntr != nullptr && Ntr[q] < q;
            float acc[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[i] = 0.f;
            const int64_t t1 = valid ? Crp[q + 1] : 0;
#pragma unroll 2
            for (int64_t t = valid ? Crp[q] : 0; t < t1; ++t) {
                const int64_t ia = (int64_t)Ca[t] * 16 + 2 * k, ib = (int64_t)Cb[t] * 16 + 2 * k;
                const float2 w = __ldg(reinterpret_cast<const float2 *>(W + ia));
                const float2 hd = __ldg(reinterpret_cast<const float2 *>(HD + ib));
                const float2 sd = __ldg(reinterpret_cast<const float2 *>(SD + ib));
                acc[0] = fmaf(w.x, hd.x, acc[0]);
                acc[1] = fmaf(w.x, hd.y, acc[1]);
                acc[2] = fmaf(w.y, hd.x, acc[2]);
                acc[3] = fmaf(w.y, hd.y, acc[3]);
                acc[4] = fmaf(w.x, sd.x, acc[4]);
                acc[5] = fmaf(w.x, sd.y, acc[5]);
                acc[6] = fmaf(w.y, sd.x, acc[6]);
                acc[7] = fmaf(w.y, sd.y, acc[7]);
                if (!lower) {
                    const float2 dd = __ldg(reinterpret_cast<const float2 *>(D + ia));
                    acc[8] = fmaf(dd.x, hd.x, acc[8]);
                    acc[9] = fmaf(dd.x, hd.y, acc[9]);
                    acc[10] = fmaf(dd.y, hd.x, acc[10]);
                    acc[11] = fmaf(dd.y, hd.y, acc[11]);
                    acc[12] = fmaf(dd.x, sd.x, acc[12]);
                    acc[13] = fmaf(dd.x, sd.y, acc[13]);
                    acc[14] = fmaf(dd.y, sd.x, acc[14]);
                    acc[15] = fmaf(dd.y, sd.y, acc[15]);
                }
            }
            // sums over the group's eight lanes (xor 1, 2, 4 stay inside the group)
#pragma unroll
            for (int off = 1; off < 8; off <<= 1)
#pragma unroll
                for (int i = 0; i < 16; ++i) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], off);
            // lanes 0..3 of the group store X, Y, h2, s2 (X and Y on lower blocks)
            if (valid && k < (lower ? 2 : 4)) {
                float *o = k == 0 ? X : k == 1 ? Y : k == 2 ? h2 : s2;
                const float4 v = k == 0   ? make_float4(acc[0], acc[1], acc[2], acc[3])
                                 : k == 1 ? make_float4(acc[4], acc[5], acc[6], acc[7])
                                 : k == 2 ? make_float4(acc[8], acc[9], acc[10], acc[11])
                                          : make_float4(acc[12], acc[13], acc[14], acc[15]);
                *reinterpret_cast<float4 *>(o + q * 4) = v;
            }
        }
    } else {
    for (int64_t q = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5; q < nnzN; q += nwarps) {
        if (!SCREEN && Ntr != nullptr && Ntr[q] < q) {
            T acc = T(0);
#pragma unroll 4
            for (int64_t t = Crp[q]; t < Crp[q + 1]; ++t) {
                const T *l = W + (int64_t)Ca[t] * BM * BN + a4;
                const T *rr = R4 + (int64_t)Cb[t] * BM * BN + b4;
#pragma unroll
                for (int kk = 0; kk < BM / 4; ++kk) {
                    const int k = quarter * (BM / 4) + kk;
                    acc = fma(l[k * BN], rr[k * BN], acc);
                }
            }
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            if (quarter == 0) out4[q * 4 + a4 * 2 + b4] = acc;
            continue;
        }
        // (16-byte vector loads measured slower here than these scalar ones: each
        // lane needs every other element of its block rows)
        T acc = T(0);
#pragma unroll 4
        for (int64_t t = Crp[q]; t < Crp[q + 1]; ++t) {
            if (SCREEN && nL[Ca[t]] * nR[Cb[t]] < eps2) continue;
            const T *l = L + (int64_t)Ca[t] * BM * BN + a;
            const T *rr = R + (int64_t)Cb[t] * BM * BN + b;
#pragma unroll
            for (int kk = 0; kk < BM / 2; ++kk) {
                const int k = half * (BM / 2) + kk;
                acc = fma(l[k * BN], rr[k * BN], acc);
            }
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        if (half == 0) out[q * 4 + a * 2 + b] = acc;
    }
    }
}

// The FP32 contraction by P_N rows: a CTA takes row J (outputs (J, J2)); the
// W and D blocks of W's column J (every triple of the row draws its left block
// from them) are staged in shared memory once, so per triple only the H'D and
// SD rows come from the L1 and L2; CaSlot names the left block's slot in the
// column.  Lanes as in contract_kernel's FP32 form: an eight-lane group per
// output block, lane k holding all sixteen outputs for basis row k.
__global__ void __launch_bounds__(NT) contract_rows_kernel(int64_t nbc, const int64_t *__restrict__ Nrp,
                                                            const int64_t *__restrict__ WcolRp,
                                                            const int32_t *__restrict__ WcolIdx,
                                                            const int64_t *__restrict__ Crp,
                                                            const uint16_t *__restrict__ CaSlot,
                                                            const int32_t *__restrict__ Cb, const float *__restrict__ W,
                                                            const float *__restrict__ D, const float *__restrict__ HD,
                                                            const float *__restrict__ SD, float *X, float *Y, float *h2,
                                                            float *s2, const int32_t *__restrict__ Ntr,
                                                            const DevState *state) {
    if (done(state)) return;
    extern __shared__ float4 stage4[];   // W rows of the column, then D rows (nc x 16 floats each)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, k = lane & 7, grp = lane >> 3;
    for (int64_t J = blockIdx.x; J < nbc; J += gridDim.x) {
        const int64_t c0 = WcolRp[J];
        const int nc = (int)(WcolRp[J + 1] - c0);
        float *sW = reinterpret_cast<float *>(stage4), *sD = sW + (int64_t)nc * 16;
        __syncthreads();   // the previous row's readers are done with the stage
        for (int e = threadIdx.x; e < nc * 4; e += NT) {   // one float4 per thread and step
            const int64_t a = WcolIdx[c0 + (e >> 2)];
            reinterpret_cast<float4 *>(sW)[e] = __ldg(reinterpret_cast<const float4 *>(W + a * 16) + (e & 3));
            reinterpret_cast<float4 *>(sD)[e] = __ldg(reinterpret_cast<const float4 *>(D + a * 16) + (e & 3));
        }
        __syncthreads();
        const int64_t q1 = Nrp[J + 1];
        // warp-uniform loop: the four groups of a warp take blocks qb .. qb + 3
        for (int64_t qb = Nrp[J] + 4 * warp; qb < q1; qb += 4 * (NT / 32)) {
            const int64_t q = qb + grp;
            const bool valid = q < q1;
            const bool lower = valid && Ntr[q] < q;
            float acc[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[i] = 0.f;
            const int64_t t1 = valid ? Crp[q + 1] : 0;
#pragma unroll 2
            for (int64_t t = valid ? Crp[q] : 0; t < t1; ++t) {
                const int ia = (int)CaSlot[t] * 16 + 2 * k;
                const int64_t ib = (int64_t)Cb[t] * 16 + 2 * k;
                const float2 w = *reinterpret_cast<const float2 *>(sW + ia);
                const float2 hd = __ldg(reinterpret_cast<const float2 *>(HD + ib));
                const float2 sd = __ldg(reinterpret_cast<const float2 *>(SD + ib));
                acc[0] = fmaf(w.x, hd.x, acc[0]);
                acc[1] = fmaf(w.x, hd.y, acc[1]);
                acc[2] = fmaf(w.y, hd.x, acc[2]);
                acc[3] = fmaf(w.y, hd.y, acc[3]);
                acc[4] = fmaf(w.x, sd.x, acc[4]);
                acc[5] = fmaf(w.x, sd.y, acc[5]);
                acc[6] = fmaf(w.y, sd.x, acc[6]);
                acc[7] = fmaf(w.y, sd.y, acc[7]);
                if (!lower) {
                    const float2 dd = *reinterpret_cast<const float2 *>(sD + ia);
                    acc[8] = fmaf(dd.x, hd.x, acc[8]);
                    acc[9] = fmaf(dd.x, hd.y, acc[9]);
                    acc[10] = fmaf(dd.y, hd.x, acc[10]);
                    acc[11] = fmaf(dd.y, hd.y, acc[11]);
                    acc[12] = fmaf(dd.x, sd.x, acc[12]);
                    acc[13] = fmaf(dd.x, sd.y, acc[13]);
                    acc[14] = fmaf(dd.y, sd.x, acc[14]);
                    acc[15] = fmaf(dd.y, sd.y, acc[15]);
                }
            }
#pragma unroll
            for (int off = 1; off < 8; off <<= 1)
#pragma unroll
                for (int i = 0; i < 16; ++i) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], off);
            if (valid && k < (lower ? 2 : 4)) {
                float *o = k == 0 ? X : k == 1 ? Y : k == 2 ? h2 : s2;
                const float4 v = k == 0   ? make_float4(acc[0], acc[1], acc[2], acc[3])
                                 : k == 1 ? make_float4(acc[4], acc[5], acc[6], acc[7])
                                 : k == 2 ? make_float4(acc[8], acc[9], acc[10], acc[11])
                                          : make_float4(acc[12], acc[13], acc[14], acc[15]);
                *reinterpret_cast<float4 *>(o + q * 4) = v;
            }
        }
    }
}

// h2, s2 on the lower-triangle blocks of P_N from their transposes' blocks
template <typename T>
__global__ void mirror_kernel(int64_t nnzN, const int32_t *__restrict__ Ntr, T *h2, T *s2, const DevState *state) {
    if (done(state)) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnzN * 4;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = i >> 2;
        const int64_t tq = Ntr[q];
        if (tq >= q) continue;
        const int e = (int)(i & 3), a = e >> 1, b = e & 1;
        h2[i] = h2[tq * 4 + b * 2 + a];
        s2[i] = s2[tq * 4 + b * 2 + a];
    }
}

// ---- gradient on P_W: G_o = 2 (2 H'W_o - sum (SW_(I,K) h0_(K,J) + H'W_(I,K) s0_(K,J)))
// half-warp per W block, one lane per element (r, c).
// Screening: SW_(I,K) h0_(K,J) and H'W_(I,K) s0_(K,J) are skipped separately when
// the product of their squared block norms is below eps^2.
template <int BM, int BN, bool SCREEN, typename T = double>
__global__ void __launch_bounds__(NT) gradient_kernel(int64_t nnzW, const int64_t *__restrict__ Grp,
                                                       const int32_t *__restrict__ Gb, const int32_t *__restrict__ Gq,
                                                       const int32_t *__restrict__ WtoHW, const T *__restrict__ HW,
                                                       const T *__restrict__ SW, const T *__restrict__ h0,
                                                       const T *__restrict__ s0, T *G,
                                                       const double *__restrict__ nHW, const double *__restrict__ nSW,
                                                       const double *__restrict__ nh0, const double *__restrict__ ns0,
                                                       double eps2, const DevState *state) {
    if (done(state)) return;
    if constexpr (VecGather<T, BM, BN, SCREEN>::on) {
        // FP32 (8x2 blocks): lane per block row r computing both columns from one
        // row of the SW and H'W blocks and the whole 2x2 h0, s0 blocks (half the
        // L1 bytes of a lane per output element), four W blocks per warp; the
        // FMAs of each output run in the same order as the scalar form's
        const int r = threadIdx.x & 7;
        const int64_t ngroups = ((int64_t)gridDim.x * NT) >> 3;
        for (int64_t o = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 3; o < nnzW; o += ngroups) {
            float acc0 = 0.f, acc1 = 0.f;
#pragma unroll 2
            for (int64_t t = Grp[o]; t < Grp[o + 1]; ++t) {
                const int64_t gb = (int64_t)Gb[t] * 16 + r * 2, gq = (int64_t)Gq[t] * 4;
                const float2 sw = __ldg(reinterpret_cast<const float2 *>(SW + gb));
                const float2 hw = __ldg(reinterpret_cast<const float2 *>(HW + gb));
                const float4 hq = ld4(h0 + gq), sq = ld4(s0 + gq);
                acc0 = fmaf(sw.x, hq.x, acc0);
                acc0 = fmaf(hw.x, sq.x, acc0);
                acc0 = fmaf(sw.y, hq.z, acc0);
                acc0 = fmaf(hw.y, sq.z, acc0);
                acc1 = fmaf(sw.x, hq.y, acc1);
                acc1 = fmaf(hw.x, sq.y, acc1);
                acc1 = fmaf(sw.y, hq.w, acc1);
                acc1 = fmaf(hw.y, sq.w, acc1);
            }
            const float2 hwo = *reinterpret_cast<const float2 *>(HW + (int64_t)WtoHW[o] * 16 + r * 2);
            *reinterpret_cast<float2 *>(G + o * 16 + r * 2) =
                make_float2(2.0f * (2.0f * hwo.x - acc0), 2.0f * (2.0f * hwo.y - acc1));
        }
    } else {
        const int e = threadIdx.x & 15;
        if (e >= BM * BN) return;
        const int r = e / BN, c = e % BN;
        const int64_t ngroups = ((int64_t)gridDim.x * NT) >> 4;
        for (int64_t o = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 4; o < nnzW; o += ngroups) {
            T acc = T(0);
#pragma unroll 4
            for (int64_t t = Grp[o]; t < Grp[o + 1]; ++t) {
                const T *sw = SW + (int64_t)Gb[t] * BM * BN + r * BN;
                const T *hw = HW + (int64_t)Gb[t] * BM * BN + r * BN;
                const T *hq = h0 + (int64_t)Gq[t] * BN * BN + c;
                const T *sq = s0 + (int64_t)Gq[t] * BN * BN + c;
                if constexpr (SCREEN) {
                    const bool use_s = !(nSW[Gb[t]] * nh0[Gq[t]] < eps2),
                               use_h = !(nHW[Gb[t]] * ns0[Gq[t]] < eps2);
#pragma unroll
                    for (int k = 0; k < BN; ++k) {
                        if (use_s) acc = fma(sw[k], hq[k * BN], acc);
                        if (use_h) acc = fma(hw[k], sq[k * BN], acc);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < BN; ++k) {
                        acc = fma(sw[k], hq[k * BN], acc);
                        acc = fma(hw[k], sq[k * BN], acc);
                    }
                }
            }
            G[o * BM * BN + e] = T(2) * (T(2) * HW[(int64_t)WtoHW[o] * BM * BN + e] - acc);
        }
    }
}

// ---- quartic coefficients and line minimum on P_N (2x2 blocks)
constexpr int NC = 13;

__global__ void __launch_bounds__(NT) coeffs_kernel(int64_t nnzN, const int32_t *__restrict__ Ntr,
                                                     const unsigned char *__restrict__ Ndiag,
                                                     const double *__restrict__ h0, const double *__restrict__ s0,
                                                     const double *__restrict__ X, const double *__restrict__ Y,
                                                     const double *__restrict__ h2, const double *__restrict__ s2,
                                                     double *partials, unsigned int *counter, DevState *state) {
    if (done(state)) return;
    __shared__ double red[(NT / 32) * NC];
    double v[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) v[q] = 0.0;
    const int64_t total = nnzN * 4;
    for (int64_t t = (int64_t)blockIdx.x * NT + threadIdx.x; t < total; t += (int64_t)gridDim.x * NT) {
        const int64_t q = t >> 2;
        const int e = (int)(t & 3), a = e >> 1, b = e & 1;
        const int64_t tt = (int64_t)Ntr[q] * 4 + b * 2 + a;   // transposed element
        const double vh0 = h0[t], vs0 = s0[t], vx = X[t], vy = Y[t], vh2 = h2[t], vs2 = s2[t];
        if (Ndiag[q] && a == b) { v[0] += vh0; v[2] += vx; v[5] += vh2; }
        v[1] = fma(vs0, vh0, v[1]);
        v[3] = fma(vs0, vx, v[3]);
        v[4] = fma(vy, vh0, v[4]);
        v[6] = fma(vs0, vh2, v[6]);
        v[7] = fma(vy, vx, v[7]);
        v[8] = fma(vy, X[tt], v[8]);
        v[9] = fma(vs2, vh0, v[9]);
        v[10] = fma(vy, vh2, v[10]);
        v[11] = fma(vs2, vx, v[11]);
        v[12] = fma(vs2, vh2, v[12]);
    }
    block_sum<NC>(v, red);
    double tot[NC] = {};
    if (!publish_and_collect<NC>(v, partials, counter, tot, red)) return;
    if (threadIdx.x >= 32) return;   // warp 0: the line minimum
#pragma unroll
    for (int q = 0; q < NC; ++q) tot[q] = __shfl_sync(0xffffffffu, tot[q], 0);
    double c[5];
    c[0] = 2.0 * (2.0 * tot[0] - tot[1]);
    c[1] = 2.0 * (4.0 * tot[2] - 2.0 * tot[3] - 2.0 * tot[4]);
    c[2] = 2.0 * (2.0 * tot[5] - tot[6] - 2.0 * (tot[7] + tot[8]) - tot[9]);
    c[3] = 2.0 * (-2.0 * tot[10] - 2.0 * tot[11]);
    c[4] = -2.0 * tot[12];
    double x = 0.0;
    const int st = lm::quartic_min_warp(c, &x);
    if (threadIdx.x != 0) return;
    for (int q = 0; q < 5; ++q) state->c[q] = c[q];
    state->x = x;
    if (st != OMM_OK) {
        state->status = st;
        state->done = 1;
    }
}

// ---- h0, s0 update on P_N + energy/orthonormality + RelTol test (mode 0), or
// energy only (mode 1, start)
constexpr int NE3 = 3;
__global__ void __launch_bounds__(NT) nn_update_kernel(int64_t nnzN, const int32_t *__restrict__ Ntr,
                                                        const unsigned char *__restrict__ Ndiag, double *h0, double *s0,
                                                        const double *__restrict__ X, const double *__restrict__ Y,
                                                        const double *__restrict__ h2, const double *__restrict__ s2,
                                                        int64_t n, double *partials, unsigned int *counter,
                                                        DevState *state, int mode) {
    if (done(state)) return;
    __shared__ double red[(NT / 32) * NE3];
    const double x = state->x;
    double v[NE3] = {0.0, 0.0, 0.0};
    const int64_t total = nnzN * 4;
    for (int64_t t = (int64_t)blockIdx.x * NT + threadIdx.x; t < total; t += (int64_t)gridDim.x * NT) {
        const int64_t q = t >> 2;
        const int e = (int)(t & 3), a = e >> 1, b = e & 1;
        const int64_t tt = (int64_t)Ntr[q] * 4 + b * 2 + a;
        double vh = h0[t], vs = s0[t];
        if (mode == 0) {
            vh = vh + x * ((X[t] + X[tt]) + x * (0.5 * (h2[t] + h2[tt])));
            vs = vs + x * ((Y[t] + Y[tt]) + x * (0.5 * (s2[t] + s2[tt])));
            h0[t] = vh;
            s0[t] = vs;
        }
        const bool dg = Ndiag[q] && a == b;
        if (dg) v[0] += vh;
        v[1] = fma(vs, vh, v[1]);
        const double ee = vs - (dg ? 1.0 : 0.0);
        v[2] = fma(ee, ee, v[2]);
    }
    block_sum<NE3>(v, red);
    double tot[NE3];
    if (!publish_and_collect<NE3>(v, partials, counter, tot, red)) return;
    if (threadIdx.x != 0) return;
    const double E = 2.0 * (2.0 * tot[0] - tot[1]) + state->e_shift;
    state->orth2 = tot[2];
    if (!isfinite(E)) {
        state->status = OMM_ERR_NONFINITE;
        state->done = 1;
        state->E = E;
        return;
    }
    if (mode == 1) {
        state->E = E;
        state->E_prev = E;
        state->rel = 0.0;
        if (state->max_iter <= 0) {
            state->status = OMM_ERR_MAXITER;
            state->done = 1;
        }
        return;
    }
    const double Ep = state->E;
    const double rel = fabs(2.0 * (E - Ep) / (E + Ep));
    state->E_prev = Ep;
    state->E = E;
    state->rel = rel;
    state->k += 1;
    const bool orth_ok = !(state->orth_tol > 0.0) || sqrt(tot[2]) < state->orth_tol;
    if (rel < state->tol && orth_ok) {
        state->status = OMM_OK;
        state->done = 1;
    } else if (state->k >= state->max_iter) {
        state->status = OMM_ERR_MAXITER;
        state->done = 1;
    }
}

// ---- W += x D on P_W; H'W += x H'D, SW += x SD on P_HW
__global__ void axpy_kernel(int64_t nW, double *W, const double *__restrict__ D, int64_t nHW, double *HW,
                            const double *__restrict__ HD, double *SW, const double *__restrict__ SD,
                            const DevState *state) {
    if (done(state)) return;
    const double x = state->x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nHW; i += (int64_t)gridDim.x * blockDim.x) {
        HW[i] = fma(x, HD[i], HW[i]);
        SW[i] = fma(x, SD[i], SW[i]);
        if (i < nW) W[i] = fma(x, D[i], W[i]);
    }
}

constexpr int ND = 3;
template <typename T>
__global__ void __launch_bounds__(NT) dots_kernel(int64_t len, const T *__restrict__ G,
                                                   const T *__restrict__ Gp, const T *__restrict__ D,
                                                   double *partials, unsigned int *counter, DevState *state, int first) {
    if (done(state)) return;
    __shared__ double red[(NT / 32) * ND];
    double v[ND] = {0.0, 0.0, 0.0};
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < len; i += (int64_t)gridDim.x * NT) {
        const double g = G[i];
        v[0] = fma(g, g, v[0]);
        if (!first) {
            v[1] = fma(g, Gp[i], v[1]);
            v[2] = fma(g, D[i], v[2]);
        }
    }
    block_sum<ND>(v, red);
    double tot[ND];
    if (!publish_and_collect<ND>(v, partials, counter, tot, red)) return;
    if (threadIdx.x != 0) return;
    const double gg = tot[0];
    double beta = 0.0;
    int restart = 1;
    if (!first) {
        const double gpgp = state->gg_prev;
        beta = (gpgp > 0.0) ? fmax(0.0, (gg - tot[1]) / gpgp) : 0.0;
        restart = (-gg + beta * tot[2] >= 0.0) ? 1 : 0;
        if (restart) beta = 0.0;
    }
    if (!isfinite(gg) || !isfinite(beta)) {
        state->status = OMM_ERR_NONFINITE;
        state->done = 1;
        return;
    }
    state->gg = gg;
    state->gg_prev = gg;
    state->beta = beta;
    state->restart = restart;
}

template <typename T>
__global__ void direction_kernel(int64_t len, const T *__restrict__ G, T *Gp, T *D, const DevState *state) {
    if (done(state)) return;
    const T beta = (T)state->beta;
    const bool restart = state->restart != 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        const T g = G[i];
        D[i] = restart ? -g : fma(beta, D[i], -g);
        Gp[i] = g;
    }
}

// ======================================================================== mixed form
// FP32 increments on FP64 state: the first phase of a mixed-precision sparse solve
// forms H'D, SD, the contractions and the gradient in FP32 (the GB300 FP32 pipe is
// ~60x the FP64 one) from FP32 copies ("shadows") of H', S, W, H'W, SW, H_W, S_W,
// and adds each FP32 increment to the FP64 state; energies and the stop test stay
// FP64.  A refinement in FP64, re-anchored from W, finishes the solve.
struct ConvJob {
    const double *src;
    float *dst;
    int64_t n;
};
struct ConvJobs {
    ConvJob j[8];
    int n;
};

__global__ void shadow_kernel(ConvJobs jobs, const DevState *state) {
    if (done(state)) return;
    for (int q = 0; q < jobs.n; ++q) {
        const ConvJob J = jobs.j[q];
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < J.n; i += (int64_t)gridDim.x * blockDim.x)
            J.dst[i] = sw_d2f(J.src[i]);
    }
}

// quartic coefficients from FP32 shadows and increments, FP32 per-thread sums
// combined in FP64; c0 is the FP64 energy of the current state
__global__ void __launch_bounds__(NT) mx_coeffs_kernel(int64_t nnzN, const int32_t *__restrict__ Ntr,
                                                        const unsigned char *__restrict__ Ndiag,
                                                        const float *__restrict__ h0, const float *__restrict__ s0,
                                                        const float *__restrict__ X, const float *__restrict__ Y,
                                                        const float *__restrict__ h2, const float *__restrict__ s2,
                                                        double *partials, unsigned int *counter, DevState *state) {
    if (done(state)) return;
    __shared__ double red[(NT / 32) * NC];
    float f[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) f[q] = 0.f;
    const int64_t total = nnzN * 4;
    for (int64_t t = (int64_t)blockIdx.x * NT + threadIdx.x; t < total; t += (int64_t)gridDim.x * NT) {
        const int64_t q = t >> 2;
        const int e = (int)(t & 3), a = e >> 1, b = e & 1;
        const int64_t tt = (int64_t)Ntr[q] * 4 + b * 2 + a;
        const float vh0 = h0[t], vs0 = s0[t], vx = X[t], vy = Y[t], vh2 = h2[t], vs2 = s2[t], vxt = X[tt];
        if (Ndiag[q] && a == b) { f[0] += vh0; f[2] += vx; f[5] += vh2; }
        f[1] = fmaf(vs0, vh0, f[1]);
        f[3] = fmaf(vs0, vx, f[3]);
        f[4] = fmaf(vy, vh0, f[4]);
        f[6] = fmaf(vs0, vh2, f[6]);
        f[7] = fmaf(vy, vx, f[7]);
        f[8] = fmaf(vy, vxt, f[8]);
        f[9] = fmaf(vs2, vh0, f[9]);
        f[10] = fmaf(vy, vh2, f[10]);
        f[11] = fmaf(vs2, vx, f[11]);
        f[12] = fmaf(vs2, vh2, f[12]);
    }
    double v[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) v[q] = sw_f2d(f[q]);
    block_sum<NC>(v, red);
    double tot[NC] = {};
    if (!publish_and_collect<NC>(v, partials, counter, tot, red)) return;
    if (threadIdx.x >= 32) return;
#pragma unroll
    for (int q = 0; q < NC; ++q) tot[q] = __shfl_sync(0xffffffffu, tot[q], 0);
    double c[5];
    c[0] = state->E - state->e_shift;
    c[1] = 2.0 * (4.0 * tot[2] - 2.0 * tot[3] - 2.0 * tot[4]);
    c[2] = 2.0 * (2.0 * tot[5] - tot[6] - 2.0 * (tot[7] + tot[8]) - tot[9]);
    c[3] = 2.0 * (-2.0 * tot[10] - 2.0 * tot[11]);
    c[4] = -2.0 * tot[12];
    double x = 0.0;
    const int st = lm::quartic_min_warp(c, &x);
    if (threadIdx.x != 0) return;
    for (int q = 0; q < 5; ++q) state->c[q] = c[q];
    state->x = x;
    state->x_f = (float)x;
    if (st != OMM_OK) {
        state->status = st;
        state->done = 1;
    }
}

// W += x D, H'W += x H'D, SW += x SD (FP64 state, FP32 increments) and their shadows
__global__ void mx_axpy_kernel(int64_t nW, double *W, const float *__restrict__ D, float *Ws, int64_t nHW, double *HW,
                               const float *__restrict__ HD, float *HWs, double *SW, const float *__restrict__ SD,
                               float *SWs, const DevState *state) {
    if (done(state)) return;
    const double x = state->x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nHW; i += (int64_t)gridDim.x * blockDim.x) {
        const double hw = fma(x, sw_f2d(HD[i]), HW[i]);
        const double sw = fma(x, sw_f2d(SD[i]), SW[i]);
        HW[i] = hw;
        SW[i] = sw;
        HWs[i] = sw_d2f(hw);
        SWs[i] = sw_d2f(sw);
        if (i < nW) {
            const double w = fma(x, sw_f2d(D[i]), W[i]);
            W[i] = w;
            Ws[i] = sw_d2f(w);
        }
    }
}

// h0, s0 += x (X + X^T) + x^2 sym(h2 / s2) in FP64 from FP32 increments, their shadows,
// energy, ||S_W - I||, and the first phase's stop: RelTol, or an energy that rose
// (the FP32 increments' noise floor), or max_iter
__global__ void __launch_bounds__(NT) mx_nn_update_kernel(int64_t nnzN, const int32_t *__restrict__ Ntr,
                                                           const unsigned char *__restrict__ Ndiag, double *h0,
                                                           double *s0, const float *__restrict__ X,
                                                           const float *__restrict__ Y, const float *__restrict__ h2,
                                                           const float *__restrict__ s2, float *h0s, float *s0s,
                                                           double *partials, unsigned int *counter, DevState *state) {
    if (done(state)) return;
    __shared__ double red[(NT / 32) * NE3];
    const double x = state->x;
    double v[NE3] = {0.0, 0.0, 0.0};
    const int64_t total = nnzN * 4;
    for (int64_t t = (int64_t)blockIdx.x * NT + threadIdx.x; t < total; t += (int64_t)gridDim.x * NT) {
        const int64_t q = t >> 2;
        const int e = (int)(t & 3), a = e >> 1, b = e & 1;
        const int64_t tt = (int64_t)Ntr[q] * 4 + b * 2 + a;
        const float fx = (float)x;
        const float dh = fx * fmaf(fx, 0.5f * (h2[t] + h2[tt]), X[t] + X[tt]);
        const float ds = fx * fmaf(fx, 0.5f * (s2[t] + s2[tt]), Y[t] + Y[tt]);
        const double vh = h0[t] + sw_f2d(dh), vs = s0[t] + sw_f2d(ds);
        h0[t] = vh;
        s0[t] = vs;
        h0s[t] = sw_d2f(vh);
        s0s[t] = sw_d2f(vs);
        const bool dg = Ndiag[q] && a == b;
        if (dg) v[0] += vh;
        v[1] = fma(vs, vh, v[1]);
        const double ee = vs - (dg ? 1.0 : 0.0);
        v[2] = fma(ee, ee, v[2]);
    }
    block_sum<NE3>(v, red);
    double tot[NE3];
    if (!publish_and_collect<NE3>(v, partials, counter, tot, red)) return;
    if (threadIdx.x != 0) return;
    const double E = 2.0 * (2.0 * tot[0] - tot[1]) + state->e_shift;
    state->orth2 = tot[2];
    if (!isfinite(E)) {
        state->status = OMM_ERR_NONFINITE;
        state->done = 1;
        state->E = E;
        return;
    }
    const double Ep = state->E;
    const double rel = fabs(2.0 * (E - Ep) / (E + Ep));
    state->E_prev = Ep;
    state->E = E;
    state->rel = rel;
    state->k += 1;
    if (rel < state->tol || E > Ep) {
        state->status = OMM_OK;
        state->done = 1;
    } else if (state->k >= state->max_iter) {
        state->status = OMM_ERR_MAXITER;
        state->done = 1;
    }
}

// ---- density matrices
// K = 2I - S_W (mode 0) or H'_W + eta (2I - S_W) (mode 1) on P_N (bn x bn blocks)
__global__ void density_K_kernel(int64_t nnzN, int bn, const unsigned char *__restrict__ Ndiag,
                                 const double *__restrict__ HW_N, const double *__restrict__ SW_N, int mode,
                                 double eta, double *K) {
    const int64_t bb = (int64_t)bn * bn;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnzN * bb;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = i / bb;
        const int e = (int)(i % bb);
        const double t = ((Ndiag[q] && e / bn == e % bn) ? 2.0 : 0.0) - SW_N[i];
        K[i] = mode == 0 ? t : fma(eta, t, HW_N[i]);
    }
}

// T_(I,b) = sum W_(I,a) K_(a,b): half-warp per P_HW block, one lane per element
template <int BM, int BN>
__global__ void __launch_bounds__(NT) density_T_kernel(int64_t nnzHW, const int64_t *__restrict__ Trp,
                                                        const int32_t *__restrict__ Tw, const int32_t *__restrict__ Tq,
                                                        const double *__restrict__ W, const double *__restrict__ K,
                                                        double *T) {
    const int e = threadIdx.x & 15;
    if (e >= BM * BN) return;
    const int r = e / BN, c = e % BN;
    const int64_t ngroups = ((int64_t)gridDim.x * NT) >> 4;
    for (int64_t o = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 4; o < nnzHW; o += ngroups) {
        double acc = 0.0;
        for (int64_t t = Trp[o]; t < Trp[o + 1]; ++t) {
            const double *w = W + (int64_t)Tw[t] * BM * BN + r * BN;
            const double *k = K + (int64_t)Tq[t] * BN * BN + c;
#pragma unroll
            for (int j = 0; j < BN; ++j) acc = fma(w[j], k[j * BN], acc);
        }
        T[o * BM * BN + e] = acc;
    }
}

// rho_(I,J) = 2 sum T_(I,b) W_(J,b)^T: two warps' worth of lanes per P_H block
// (BM*BM = 64 outputs), each lane two outputs
template <int BM, int BN>
__global__ void __launch_bounds__(NT) density_rho_kernel(int64_t nnzH, const int64_t *__restrict__ Rrp,
                                                          const int32_t *__restrict__ Rt,
                                                          const int32_t *__restrict__ Rw,
                                                          const double *__restrict__ T,
                                                          const double *__restrict__ W, double *rho) {
    const int lane = threadIdx.x & 31;
    constexpr int NE = BM * BM;
    const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
    for (int64_t h = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5; h < nnzH; h += nwarps) {
        for (int e = lane; e < NE; e += 32) {
            const int r = e / BM, c = e % BM;
            double acc = 0.0;
            for (int64_t t = Rrp[h]; t < Rrp[h + 1]; ++t) {
                const double *tt = T + (int64_t)Rt[t] * BM * BN + r * BN;
                const double *ww = W + (int64_t)Rw[t] * BM * BN + c * BN;
#pragma unroll
                for (int j = 0; j < BN; ++j) acc = fma(tt[j], ww[j], acc);
            }
            rho[h * NE + e] = 2.0 * acc;
        }
    }
}

// ---- squared Frobenius norms of blocks, for screening: one thread per block,
// up to four arrays per launch
struct NormJob {
    const double *vals;
    double *out;
    int64_t nblocks;
    int bs;                 // values per block
};
struct NormJobs {
    NormJob j[4];
    int n;
};

__global__ void norms_kernel(NormJobs jobs, const DevState *state) {
    if (done(state)) return;
    for (int q = 0; q < jobs.n; ++q) {
        const NormJob J = jobs.j[q];
        for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < J.nblocks;
             b += (int64_t)gridDim.x * blockDim.x) {
            const double *v = J.vals + b * J.bs;
            double s = 0.0;
            for (int t = 0; t < J.bs; ++t) s = fma(v[t], v[t], s);
            J.out[b] = s;
        }
    }
}

int blocks_for(int64_t work, int per) {
    int64_t nb = ceil_div(work, per);
    if (nb > 152 * 16) nb = 152 * 16;
    return (int)(nb < 1 ? 1 : nb);
}
int red_blocks(int64_t work) {
    int64_t nb = ceil_div(work, (int64_t)NT * 4);
    if (nb > kRedBlocksMax) nb = kRedBlocksMax;
    return (int)(nb < 1 ? 1 : nb);
}

#define LAUNCHED()                             \
    do {                                       \
        count_launch();                        \
        OMM_CUDA_TRY(cudaGetLastError());      \
    } while (0)

}  // namespace

// ======================================================================== device side: handle pieces
int upload(const Host &hs, Dev &d) {
    auto up = [](auto **dst, const auto &src) -> int {
        using T = typename std::remove_reference<decltype(src[0])>::type;
        const size_t n = src.size() ? src.size() : 1;
        if (cudaMalloc((void **)dst, n * sizeof(T)) != cudaSuccess) return OMM_ERR_NOMEM;
        if (!src.empty() && cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
            return OMM_ERR_CUDA;
        return OMM_OK;
    };
    const Pattern &P = hs.P;
    d.bm = P.bm;
    d.bn = P.bn;
    d.nbr = P.nbr;
    d.nbc = P.nbc;
    d.nnzH = P.Hrp[P.nbr];
    d.nnzW = P.Wrp[P.nbr];
    d.nnzHW = hs.HWrp[P.nbr];
    d.nnzN = hs.Nrp[P.nbc];
    int rc;
    if ((rc = up(&d.Hrp, hs.Hrp)) || (rc = up(&d.Hcol, hs.Hcol)) || (rc = up(&d.Prp, hs.Prp)) ||
        (rc = up(&d.Ph, hs.Ph)) || (rc = up(&d.Pw, hs.Pw)) || (rc = up(&d.Crp, hs.Crp)) || (rc = up(&d.Ca, hs.Ca)) ||
        (rc = up(&d.Cb, hs.Cb)) || (rc = up(&d.Grp, hs.Grp)) || (rc = up(&d.Gb, hs.Gb)) || (rc = up(&d.Gq, hs.Gq)) ||
        (rc = up(&d.WtoHW, hs.WtoHW)) || (rc = up(&d.Ntr, hs.Ntr)) || (rc = up(&d.Ndiag, hs.Ndiag)))
        return rc;
    const int64_t bb = (int64_t)P.bm * P.bm, bw = (int64_t)P.bm * P.bn, bq = (int64_t)P.bn * P.bn;
    auto al = [](double **p, int64_t n) -> int {
        return cudaMalloc((void **)p, (size_t)(n > 0 ? n : 1) * sizeof(double)) == cudaSuccess ? OMM_OK : OMM_ERR_NOMEM;
    };
    if ((rc = al(&d.HS, 2 * d.nnzH * bb)) || (rc = al(&d.Hin, 2 * d.nnzH * bb)) || (rc = al(&d.W, d.nnzW * bw)) ||
        (rc = al(&d.D, d.nnzW * bw)) || (rc = al(&d.G, d.nnzW * bw)) || (rc = al(&d.Gp, d.nnzW * bw)) ||
        (rc = al(&d.HW, d.nnzHW * bw)) || (rc = al(&d.SW, d.nnzHW * bw)) || (rc = al(&d.HD, d.nnzHW * bw)) ||
        (rc = al(&d.SD, d.nnzHW * bw)) || (rc = al(&d.h0, d.nnzN * bq)) || (rc = al(&d.s0, d.nnzN * bq)) ||
        (rc = al(&d.X, d.nnzN * bq)) || (rc = al(&d.Y, d.nnzN * bq)) || (rc = al(&d.h2, d.nnzN * bq)) ||
        (rc = al(&d.s2, d.nnzN * bq)))
        return rc;
    if (cudaMalloc((void **)&d.keep, (size_t)(d.nnzH > 0 ? d.nnzH : 1)) != cudaSuccess) return OMM_ERR_NOMEM;
    return OMM_OK;
}

void release(Dev &d) {
    void *ptrs[] = {d.Trp, d.Rrp, d.Tw, d.Tq, d.Rt, d.Rw, d.K, d.T,
                    d.Hrp, d.Hcol, d.Prp, d.Ph, d.Pw, d.Crp, d.Ca, d.Cb, d.Grp, d.Gb, d.Gq, d.WtoHW, d.Ntr,
                    d.Ndiag, d.HS, d.Hin, d.W, d.D, d.G, d.Gp, d.HW, d.SW, d.HD, d.SD, d.h0, d.s0, d.X,
                    d.Y, d.h2, d.s2, d.keep, d.nrm, d.fbuf, d.Nrp, d.WcolRp, d.WcolIdx, d.CaSlot};
    for (void *p : ptrs) cudaFree(p);
    d = Dev{};
}

int set_HS(Dev &d, const double *H, const double *S, bool on_device, double eps, bool eta_auto, double *scratch,
           unsigned int *counter, DevState *state, cudaStream_t st) {
    const int64_t bb = (int64_t)d.bm * d.bm;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    double *Hc = d.Hin, *Sc = d.Hin + d.nnzH * bb;
    OMM_CUDA_TRY(cudaMemcpyAsync(Hc, H, d.nnzH * bb * sizeof(double), kind, st));
    OMM_CUDA_TRY(cudaMemcpyAsync(Sc, S, d.nnzH * bb * sizeof(double), kind, st));
    filter_kernel<<<blocks_for(d.nnzH, 256), 256, 0, st>>>(d.nnzH, (int)bb, Hc, Sc, eps * eps, d.keep);
    LAUNCHED();
    if (eta_auto) {
        gershgorin_kernel<<<red_blocks(d.nbr * d.bm), NT, 0, st>>>(d.nbr, d.bm, d.Hrp, d.Hcol, Hc, Sc, scratch,
                                                                    counter, state);
        LAUNCHED();
    }
    shift_pack_kernel<<<blocks_for(d.nnzH * bb, 256), 256, 0, st>>>(d.nnzH, (int)bb, Hc, Sc, d.keep, state, d.HS);
    LAUNCHED();
    return norms(d, NRM_HS, nullptr, st);
}

#define DISPATCH_BLOCKS(BMv, BNv, CALL)                              \
    do {                                                             \
        if ((BMv) == 8 && (BNv) == 2) { constexpr int BM = 8, BN = 2; CALL; } \
        else return OMM_ERR_UNSUPPORTED;                             \
    } while (0)

int screen_alloc(Dev &d, double eps) {
    if (!(eps > 0.0)) return OMM_OK;
    const int64_t total = 2 * d.nnzH + 2 * d.nnzW + 4 * d.nnzHW + 2 * d.nnzN;
    if (cudaMalloc((void **)&d.nrm, (size_t)(total > 0 ? total : 1) * sizeof(double)) != cudaSuccess)
        return OMM_ERR_NOMEM;
    d.screen_eps2 = eps * eps;
    d.nHS = d.nrm;
    d.nW = d.nHS + 2 * d.nnzH;
    d.nD = d.nW + d.nnzW;
    d.nHW = d.nD + d.nnzW;
    d.nSW = d.nHW + d.nnzHW;
    d.nHD = d.nSW + d.nnzHW;
    d.nSD = d.nHD + d.nnzHW;
    d.nh0 = d.nSD + d.nnzHW;
    d.ns0 = d.nh0 + d.nnzN;
    return OMM_OK;
}

int norms(Dev &d, int which, const DevState *state, cudaStream_t st) {
    if (!d.screening()) return OMM_OK;
    const int bb = d.bm * d.bm, bw = d.bm * d.bn, bq = d.bn * d.bn;
    NormJobs jobs{};
    auto add = [&](const double *v, double *o, int64_t nb, int bs) { jobs.j[jobs.n++] = NormJob{v, o, nb, bs}; };
    auto flush = [&]() -> int {
        if (jobs.n == 0) return OMM_OK;
        int64_t most = 0;
        for (int q = 0; q < jobs.n; ++q) most = std::max(most, jobs.j[q].nblocks);
        norms_kernel<<<blocks_for(most, 256), 256, 0, st>>>(jobs, state);
        LAUNCHED();
        jobs.n = 0;
        return OMM_OK;
    };
    int rc;
    if (which & NRM_HS) add(d.HS, d.nHS, 2 * d.nnzH, bb);
    if (which & NRM_W) add(d.W, d.nW, d.nnzW, bw);
    if (which & NRM_D) add(d.D, d.nD, d.nnzW, bw);
    if ((rc = flush())) return rc;
    if (which & NRM_HWSW) { add(d.HW, d.nHW, d.nnzHW, bw); add(d.SW, d.nSW, d.nnzHW, bw); }
    if (which & NRM_HDSD) { add(d.HD, d.nHD, d.nnzHW, bw); add(d.SD, d.nSD, d.nnzHW, bw); }
    if ((rc = flush())) return rc;
    if (which & NRM_N) { add(d.h0, d.nh0, d.nnzN, bq); add(d.s0, d.ns0, d.nnzN, bq); }
    return flush();
}

int products(Dev &d, const double *Din, double *HDo, double *SDo, const double *nDin, const DevState *state,
             cudaStream_t st) {
    if (nDin != nullptr && d.screening()) {
        DISPATCH_BLOCKS(d.bm, d.bn, (products_kernel<BM, BN, true><<<blocks_for(d.nnzHW * 32, NT), NT, 0, st>>>(
                                         d.nnzHW, d.Prp, d.Ph, d.Pw, d.HS, Din, HDo, SDo, d.nHS, nDin,
                                         d.screen_eps2, state)));
    } else {
        DISPATCH_BLOCKS(d.bm, d.bn, (products_kernel<BM, BN, false><<<blocks_for(d.nnzHW * 32, NT), NT, 0, st>>>(
                                         d.nnzHW, d.Prp, d.Ph, d.Pw, d.HS, Din, HDo, SDo, nullptr, nullptr, 0.0,
                                         state)));
    }
    LAUNCHED();
    return OMM_OK;
}

int contract(Dev &d, const double *Wl, const double *Dl, const double *HDr, const double *SDr, double *Xo,
             double *Yo, double *h2o, double *s2o, const double *nWl, const double *nDl, const double *nHDr,
             const double *nSDr, const DevState *state, cudaStream_t st) {
    if (nWl != nullptr && d.screening()) {
        DISPATCH_BLOCKS(d.bm, d.bn, (contract_kernel<BM, BN, true><<<blocks_for(d.nnzN * 32, NT), NT, 0, st>>>(
                                         d.nnzN, d.Crp, d.Ca, d.Cb, Wl, Dl, HDr, SDr, Xo, Yo, h2o, s2o, nWl, nDl,
                                         nHDr, nSDr, d.screen_eps2, nullptr, state)));
        LAUNCHED();
        return OMM_OK;
    }
    // without screening D^T H'D and D^T S D are formed on the upper triangle of P_N
    // and mirrored to the lower one (H' and S are symmetric); with D = W (the start,
    // the density matrices) every block of every output is formed
    const bool sym = Dl != Wl;
    DISPATCH_BLOCKS(d.bm, d.bn, (contract_kernel<BM, BN, false><<<blocks_for(d.nnzN * 32, NT), NT, 0, st>>>(
                                     d.nnzN, d.Crp, d.Ca, d.Cb, Wl, Dl, HDr, SDr, Xo, Yo, h2o, s2o, nullptr,
                                     nullptr, nullptr, nullptr, 0.0, sym ? d.Ntr : nullptr, state)));
    LAUNCHED();
    if (sym) {
        mirror_kernel<double><<<blocks_for(d.nnzN * 4, 256), 256, 0, st>>>(d.nnzN, d.Ntr, h2o, s2o, state);
        LAUNCHED();
    }
    return OMM_OK;
}

int upload_density(const DensHost &dh, Dev &d) {
    auto up64 = [](int64_t **dst, const std::vector<int64_t> &v) -> int {
        if (cudaMalloc(dst, std::max<size_t>(1, v.size()) * sizeof(int64_t)) != cudaSuccess) return OMM_ERR_NOMEM;
        return cudaMemcpy(*dst, v.data(), v.size() * sizeof(int64_t), cudaMemcpyHostToDevice) == cudaSuccess
                   ? OMM_OK : OMM_ERR_CUDA;
    };
    auto up32 = [](int32_t **dst, const std::vector<int32_t> &v) -> int {
        if (cudaMalloc(dst, std::max<size_t>(1, v.size()) * sizeof(int32_t)) != cudaSuccess) return OMM_ERR_NOMEM;
        return cudaMemcpy(*dst, v.data(), v.size() * sizeof(int32_t), cudaMemcpyHostToDevice) == cudaSuccess
                   ? OMM_OK : OMM_ERR_CUDA;
    };
    int rc;
    if ((rc = up64(&d.Trp, dh.Trp)) || (rc = up32(&d.Tw, dh.Tw)) || (rc = up32(&d.Tq, dh.Tq)) ||
        (rc = up64(&d.Rrp, dh.Rrp)) || (rc = up32(&d.Rt, dh.Rt)) || (rc = up32(&d.Rw, dh.Rw)))
        return rc;
    if (cudaMalloc(&d.K, (size_t)(d.nnzN * d.bn * d.bn) * sizeof(double)) != cudaSuccess) return OMM_ERR_NOMEM;
    if (cudaMalloc(&d.T, (size_t)(d.nnzHW * d.bm * d.bn) * sizeof(double)) != cudaSuccess) return OMM_ERR_NOMEM;
    return OMM_OK;
}

int density(Dev &d, int mode, double eta, double *out, cudaStream_t st) {
    // H'W, SW on P_HW and H'_W = W^T H'W, S_W = W^T SW on P_N, afresh from W
    int rc;
    if ((rc = products(d, d.W, d.HD, d.SD, nullptr, nullptr, st))) return rc;
    if ((rc = contract(d, d.W, d.W, d.HD, d.SD, d.X, d.Y, d.h2, d.s2, nullptr, nullptr, nullptr, nullptr, nullptr,
                       st)))
        return rc;
    const int64_t bb = (int64_t)d.bn * d.bn;
    density_K_kernel<<<blocks_for(d.nnzN * bb, 256), 256, 0, st>>>(d.nnzN, d.bn, d.Ndiag, d.X, d.Y, mode, eta, d.K);
    LAUNCHED();
    DISPATCH_BLOCKS(d.bm, d.bn, (density_T_kernel<BM, BN><<<blocks_for(d.nnzHW * 16, NT), NT, 0, st>>>(
                                     d.nnzHW, d.Trp, d.Tw, d.Tq, d.W, d.K, d.T)));
    LAUNCHED();
    DISPATCH_BLOCKS(d.bm, d.bn, (density_rho_kernel<BM, BN><<<blocks_for(d.nnzH * 32, NT), NT, 0, st>>>(
                                     d.nnzH, d.Rrp, d.Rt, d.Rw, d.T, d.W, out)));
    LAUNCHED();
    return OMM_OK;
}

int gradient(Dev &d, const DevState *state, cudaStream_t st) {
    if (d.screening()) {
        DISPATCH_BLOCKS(d.bm, d.bn, (gradient_kernel<BM, BN, true><<<blocks_for(d.nnzW * 16, NT), NT, 0, st>>>(
                                         d.nnzW, d.Grp, d.Gb, d.Gq, d.WtoHW, d.HW, d.SW, d.h0, d.s0, d.G, d.nHW,
                                         d.nSW, d.nh0, d.ns0, d.screen_eps2, state)));
    } else {
        DISPATCH_BLOCKS(d.bm, d.bn, (gradient_kernel<BM, BN, false><<<blocks_for(d.nnzW * 16, NT), NT, 0, st>>>(
                                         d.nnzW, d.Grp, d.Gb, d.Gq, d.WtoHW, d.HW, d.SW, d.h0, d.s0, d.G, nullptr,
                                         nullptr, nullptr, nullptr, 0.0, state)));
    }
    LAUNCHED();
    return OMM_OK;
}

namespace {
// Shared-memory budget of the row-staged contraction: W and D rows of one
// column of W (16 floats each per block)
constexpr int kRowStageMaxCol = 256;   // 32 KB
}

int mixed_alloc(const Host &hs, Dev &d) {
    // row-staged FP32 contraction: slot of every W block in its column, per triple
    {
        const int64_t nbc = hs.P.nbc, nnzW = (int64_t)hs.WcolIdx.size();
        int64_t maxcol = 0;
        for (int64_t J = 0; J < nbc; ++J) maxcol = std::max(maxcol, hs.WcolRp[J + 1] - hs.WcolRp[J]);
        if (maxcol > 0 && maxcol <= kRowStageMaxCol) {
            std::vector<uint16_t> wslot(nnzW);
            std::vector<int32_t> widx(nnzW);
            for (int64_t J = 0; J < nbc; ++J)
                for (int64_t c = hs.WcolRp[J]; c < hs.WcolRp[J + 1]; ++c) {
                    wslot[hs.WcolIdx[c]] = (uint16_t)(c - hs.WcolRp[J]);
                    widx[c] = (int32_t)hs.WcolIdx[c];
                }
            std::vector<uint16_t> slot(hs.Ca.size());
            for (size_t t = 0; t < hs.Ca.size(); ++t) slot[t] = wslot[hs.Ca[t]];
            auto up = [](auto **dst, const auto &v) -> int {
                const size_t bytes = (v.empty() ? 1 : v.size()) * sizeof(v[0]);
                if (cudaMalloc((void **)dst, bytes) != cudaSuccess) return OMM_ERR_NOMEM;
                if (!v.empty() && cudaMemcpy(*dst, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice) != cudaSuccess)
                    return OMM_ERR_CUDA;
                return OMM_OK;
            };
            int rc;
            if ((rc = up(&d.Nrp, hs.Nrp)) || (rc = up(&d.WcolRp, hs.WcolRp)) || (rc = up(&d.WcolIdx, widx)) ||
                (rc = up(&d.CaSlot, slot)))
                return rc;
            d.maxcol = (int)maxcol;
        }
    }
    const int64_t bb = (int64_t)d.bm * d.bm, bw = (int64_t)d.bm * d.bn, bq = (int64_t)d.bn * d.bn;
    const int64_t nHS = 2 * d.nnzH * bb, nW = d.nnzW * bw, nHW = d.nnzHW * bw, nN = d.nnzN * bq;
    const int64_t total = nHS + 4 * nW + 4 * nHW + 6 * nN;
    if (cudaMalloc((void **)&d.fbuf, (size_t)(total > 0 ? total : 1) * sizeof(float)) != cudaSuccess)
        return OMM_ERR_NOMEM;
    float *p = d.fbuf;
    auto take = [&](float **dst, int64_t n) { *dst = p; p += n; };
    take(&d.HS32, nHS);
    take(&d.W32, nW);
    take(&d.D32, nW);
    take(&d.G32, nW);
    take(&d.Gp32, nW);
    take(&d.HW32, nHW);
    take(&d.SW32, nHW);
    take(&d.HD32, nHW);
    take(&d.SD32, nHW);
    take(&d.h032, nN);
    take(&d.s032, nN);
    take(&d.X32, nN);
    take(&d.Y32, nN);
    take(&d.h232, nN);
    take(&d.s232, nN);
    d.mixed = true;
    return OMM_OK;
}

namespace {
int convert(ConvJobs &jobs, const DevState *state, cudaStream_t st) {
    if (jobs.n == 0) return OMM_OK;
    int64_t most = 0;
    for (int q = 0; q < jobs.n; ++q) most = std::max(most, jobs.j[q].n);
    shadow_kernel<<<blocks_for(most, 256), 256, 0, st>>>(jobs, state);
    LAUNCHED();
    jobs.n = 0;
    return OMM_OK;
}
}  // namespace

int mixed_shadow_HS(Dev &d, cudaStream_t st) {
    ConvJobs jobs{};
    jobs.j[jobs.n++] = ConvJob{d.HS, d.HS32, 2 * d.nnzH * d.bm * d.bm};
    return convert(jobs, nullptr, st);
}

int mixed_begin(Dev &d, const DevState *state, cudaStream_t st) {
    const int64_t bw = (int64_t)d.bm * d.bn, bq = (int64_t)d.bn * d.bn;
    ConvJobs jobs{};
    jobs.j[jobs.n++] = ConvJob{d.W, d.W32, d.nnzW * bw};
    jobs.j[jobs.n++] = ConvJob{d.D, d.D32, d.nnzW * bw};
    jobs.j[jobs.n++] = ConvJob{d.G, d.G32, d.nnzW * bw};
    jobs.j[jobs.n++] = ConvJob{d.Gp, d.Gp32, d.nnzW * bw};
    jobs.j[jobs.n++] = ConvJob{d.HW, d.HW32, d.nnzHW * bw};
    jobs.j[jobs.n++] = ConvJob{d.SW, d.SW32, d.nnzHW * bw};
    jobs.j[jobs.n++] = ConvJob{d.h0, d.h032, d.nnzN * bq};
    jobs.j[jobs.n++] = ConvJob{d.s0, d.s032, d.nnzN * bq};
    return convert(jobs, state, st);
}

int mixed_products(Dev &d, const DevState *state, cudaStream_t st) {
    DISPATCH_BLOCKS(d.bm, d.bn, (products_kernel<BM, BN, false, float><<<blocks_for(d.nnzHW * 16, NT), NT, 0, st>>>(
                                     d.nnzHW, d.Prp, d.Ph, d.Pw, d.HS32, d.D32, d.HD32, d.SD32, nullptr, nullptr, 0.0,
                                     state)));
    LAUNCHED();
    return OMM_OK;
}

int mixed_contract(Dev &d, const DevState *state, cudaStream_t st) {
    if (d.maxcol > 0 && d.bm == 8 && d.bn == 2) {
        const size_t smem = (size_t)d.maxcol * 16 * 2 * sizeof(float);
        const int64_t nb = d.nbc < 152 * 8 ? d.nbc : 152 * 8;
        contract_rows_kernel<<<(unsigned)(nb < 1 ? 1 : nb), NT, smem, st>>>(
            d.nbc, d.Nrp, d.WcolRp, d.WcolIdx, d.Crp, d.CaSlot, d.Cb, d.W32, d.D32, d.HD32, d.SD32, d.X32, d.Y32,
            d.h232, d.s232, d.Ntr, state);
        LAUNCHED();
    } else {
        DISPATCH_BLOCKS(d.bm, d.bn, (contract_kernel<BM, BN, false, float><<<blocks_for(d.nnzN * 8, NT), NT, 0, st>>>(
                                         d.nnzN, d.Crp, d.Ca, d.Cb, d.W32, d.D32, d.HD32, d.SD32, d.X32, d.Y32,
                                         d.h232, d.s232, nullptr, nullptr, nullptr, nullptr, 0.0, d.Ntr, state)));
        LAUNCHED();
    }
    mirror_kernel<float><<<blocks_for(d.nnzN * 4, 256), 256, 0, st>>>(d.nnzN, d.Ntr, d.h232, d.s232, state);
    LAUNCHED();
    return OMM_OK;
}

int mixed_coeffs(Dev &d, double *scratch, unsigned int *counter, DevState *state, cudaStream_t st) {
    mx_coeffs_kernel<<<red_blocks(d.nnzN * 4), NT, 0, st>>>(d.nnzN, d.Ntr, d.Ndiag, d.h032, d.s032, d.X32, d.Y32,
                                                              d.h232, d.s232, scratch, counter, state);
    LAUNCHED();
    return OMM_OK;
}

int mixed_update(Dev &d, double *scratch, unsigned int *counter, DevState *state, cudaStream_t st) {
    const int64_t bw = (int64_t)d.bm * d.bn;
    mx_axpy_kernel<<<blocks_for(d.nnzHW * bw, 256 * 4), 256, 0, st>>>(d.nnzW * bw, d.W, d.D32, d.W32, d.nnzHW * bw,
                                                                         d.HW, d.HD32, d.HW32, d.SW, d.SD32, d.SW32,
                                                                         state);
    LAUNCHED();
    mx_nn_update_kernel<<<red_blocks(d.nnzN * 4), NT, 0, st>>>(d.nnzN, d.Ntr, d.Ndiag, d.h0, d.s0, d.X32, d.Y32,
                                                                 d.h232, d.s232, d.h032, d.s032, scratch, counter,
                                                                 state);
    LAUNCHED();
    return OMM_OK;
}

int mixed_gradient(Dev &d, const DevState *state, cudaStream_t st) {
    DISPATCH_BLOCKS(d.bm, d.bn, (gradient_kernel<BM, BN, false, float><<<blocks_for(d.nnzW * 8, NT), NT, 0, st>>>(
                                     d.nnzW, d.Grp, d.Gb, d.Gq, d.WtoHW, d.HW32, d.SW32, d.h032, d.s032, d.G32,
                                     nullptr, nullptr, nullptr, nullptr, 0.0, state)));
    LAUNCHED();
    return OMM_OK;
}

int mixed_direction(Dev &d, double *scratch, unsigned int *counter, DevState *state, cudaStream_t st) {
    const int64_t len = d.nnzW * d.bm * d.bn;
    dots_kernel<float><<<red_blocks(len), NT, 0, st>>>(len, d.G32, d.Gp32, d.D32, scratch, counter, state, 0);
    LAUNCHED();
    direction_kernel<float><<<blocks_for(len, 256 * 4), 256, 0, st>>>(len, d.G32, d.Gp32, d.D32, state);
    LAUNCHED();
    return OMM_OK;
}

int coeffs(Dev &d, double *scratch, unsigned int *counter, DevState *state, cudaStream_t st) {
    coeffs_kernel<<<red_blocks(d.nnzN * 4), NT, 0, st>>>(d.nnzN, d.Ntr, d.Ndiag, d.h0, d.s0, d.X, d.Y, d.h2,
                                                           d.s2, scratch, counter, state);
    LAUNCHED();
    return OMM_OK;
}

int nn_update(Dev &d, int64_t n, int mode, double *scratch, unsigned int *counter, DevState *state, cudaStream_t st) {
    nn_update_kernel<<<red_blocks(d.nnzN * 4), NT, 0, st>>>(d.nnzN, d.Ntr, d.Ndiag, d.h0, d.s0, d.X, d.Y, d.h2,
                                                              d.s2, n, scratch, counter, state, mode);
    LAUNCHED();
    return OMM_OK;
}

int axpy(Dev &d, const DevState *state, cudaStream_t st) {
    const int64_t bw = (int64_t)d.bm * d.bn;
    axpy_kernel<<<blocks_for(d.nnzHW * bw, 256 * 4), 256, 0, st>>>(d.nnzW * bw, d.W, d.D, d.nnzHW * bw, d.HW, d.HD,
                                                                      d.SW, d.SD, state);
    LAUNCHED();
    return OMM_OK;
}

int dots(Dev &d, int first, double *scratch, unsigned int *counter, DevState *state, cudaStream_t st) {
    const int64_t len = d.nnzW * d.bm * d.bn;
    dots_kernel<double><<<red_blocks(len), NT, 0, st>>>(len, d.G, d.Gp, d.D, scratch, counter, state, first);
    LAUNCHED();
    return OMM_OK;
}

int direction(Dev &d, const DevState *state, cudaStream_t st) {
    const int64_t len = d.nnzW * d.bm * d.bn;
    direction_kernel<double><<<blocks_for(len, 256 * 4), 256, 0, st>>>(len, d.G, d.Gp, d.D, state);
    LAUNCHED();
    return OMM_OK;
}

}  // namespace sp
}  // namespace omm
