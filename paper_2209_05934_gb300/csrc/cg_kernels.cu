// Reductions, line search and CG updates of the OMM step (FP64 state).
//
// Every reduction uses a fixed number of blocks for a given size, a fixed
// per-thread traversal, warp-shuffle trees and a "last block" that sums the
// per-block partials in block order, so equal inputs give bitwise equal
// results (needed for the batched and serving forms, whose results must not
// depend on what else runs).
#include <cuda_bf16.h>
#include <math.h>

#include <mutex>

#include "linemin.cuh"
#include "omm_internal.cuh"

namespace omm {
namespace {

constexpr int NT = 256;
constexpr int TILE = 32;

template <int NV>
__device__ void block_sum(double (&v)[NV], double *red /* smem NV*8 */) {
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

// Publish this block's NV partials; returns true in the last block to finish,
// whose threads then all hold the totals in `tot`.  The last block sums the
// partials in a fixed order (warp per value, lane-strided blocks, shuffle tree),
// so the result does not depend on which block finished last.
template <int NV>
__device__ bool publish_and_collect(const double (&v)[NV], double *partials, unsigned int *counter,
                                    double (&tot)[NV], double *red) {
    __shared__ bool is_last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) partials[blockIdx.x * NV + q] = v[q];
        __threadfence();
        const unsigned prev = atomicAdd(counter, 1u);
        is_last = (prev == gridDim.x - 1);
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

__device__ inline bool finite(double x) { return isfinite(x); }

// Three BF16 digits d1 = bf16(v), d2 = bf16(v - d1), d3 = bf16(v - d1 - d2),
// written to the planes of a DigitOut at element offset o.
__device__ __forceinline__ void put3(const DigitOut &d, int64_t o, double v) {
    const __nv_bfloat16 d1 = __double2bfloat16(v);
    const double r1 = v - (double)__bfloat162float(d1);
    const __nv_bfloat16 d2 = __double2bfloat16(r1);
    const __nv_bfloat16 d3 = __double2bfloat16(r1 - (double)__bfloat162float(d2));
    __nv_bfloat16 *p = (__nv_bfloat16 *)d.ptr;
    p[o] = d1;
    p[d.plane + o] = d2;
    if (d.nd > 2) p[2 * d.plane + o] = d3;
}

// ---------------------------------------------------------------- coefficients
// partial sums: 0 tr h0, 1 <s0,h0>, 2 tr X, 3 <s0,X>, 4 <Y,h0>, 5 tr h2, 6 <s0,h2>,
// 7 <Y,X>, 8 <Y,X^T>, 9 <s2,h0>, 10 <Y,h2>, 11 <s2,X>, 12 <s2,h2>
constexpr int NC = 13;

__global__ void __launch_bounds__(NT) coeffs_kernel(int n, const double *__restrict__ h0,
                                                     const double *__restrict__ s0, int64_t ldh,
                                                     const double *__restrict__ X,
                                                     const double *__restrict__ Y,
                                                     const double *__restrict__ h2,
                                                     const double *__restrict__ s2, int64_t ldz,
                                                     double *partials, unsigned int *counter,
                                                     DevState *state, double *coeffs_out,
                                                     int do_linemin) {
    if (state != nullptr && *((volatile int *)&state->done)) return;
    __shared__ double Xt[TILE][TILE + 1];
    __shared__ double red[(NT / 32) * NC];
    const int lx = threadIdx.x % TILE, ly = threadIdx.x / TILE;
    const int T = (n + TILE - 1) / TILE;
    const int64_t ntiles = (int64_t)T * T;
    double v[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) v[q] = 0.0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int ti = (int)(t % T), tj = (int)(t / T);
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int a = ly + 8 * r;
            const int64_t gi = (int64_t)tj * TILE + lx, gj = (int64_t)ti * TILE + a;
            Xt[a][lx] = (gi < n && gj < n) ? X[gi + gj * ldz] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int64_t i = (int64_t)ti * TILE + lx, j = (int64_t)tj * TILE + ly + 8 * r;
            if (i >= n || j >= n) continue;
            const double vh0 = h0[i + j * ldh], vs0 = s0[i + j * ldh];
            const double vx = X[i + j * ldz], vy = Y[i + j * ldz];
            const double vh2 = h2[i + j * ldz], vs2 = s2[i + j * ldz];
            const double vxt = Xt[lx][ly + 8 * r];
            if (i == j) { v[0] += vh0; v[2] += vx; v[5] += vh2; }
            v[1] = fma(vs0, vh0, v[1]);
            v[3] = fma(vs0, vx, v[3]);
            v[4] = fma(vy, vh0, v[4]);
            v[6] = fma(vs0, vh2, v[6]);
            v[7] = fma(vy, vx, v[7]);
            v[8] = fma(vy, vxt, v[8]);
            v[9] = fma(vs2, vh0, v[9]);
            v[10] = fma(vy, vh2, v[10]);
            v[11] = fma(vs2, vx, v[11]);
            v[12] = fma(vs2, vh2, v[12]);
        }
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
    int st = OMM_OK;
    if (state != nullptr && do_linemin) st = lm::quartic_min_warp(c, &x);
    if (threadIdx.x != 0) return;
    if (coeffs_out != nullptr)
        for (int q = 0; q < 5; ++q) coeffs_out[q] = c[q];
    if (state != nullptr) {
        for (int q = 0; q < 5; ++q) state->c[q] = c[q];
        if (do_linemin) {
            state->x = x;
            if (st != OMM_OK) {
                state->status = st;
                state->done = 1;
            }
        }
    }
}

// ---------------------------------------------------------------- n x n update + energy
// partials: 0 tr h0, 1 <s0,h0>, 2 ||s0 - I||^2
constexpr int NE = 3;

__global__ void __launch_bounds__(NT) nn_update_kernel(int n, double *h0, double *s0, int64_t ldh,
                                                        const double *__restrict__ X,
                                                        const double *__restrict__ Y,
                                                        const double *__restrict__ h2,
                                                        const double *__restrict__ s2,
                                                        int64_t ldz, double *partials,
                                                        unsigned int *counter, DevState *state,
                                                        int mode, DigitOut hsw) {
    if (*((volatile int *)&state->done)) return;
    __shared__ double Tt[4][TILE][TILE + 1];
    __shared__ double red[(NT / 32) * NE];
    const int lx = threadIdx.x % TILE, ly = threadIdx.x / TILE;
    const int T = (n + TILE - 1) / TILE;
    const int64_t ntiles = (int64_t)T * T;
    const double x = state->x;
    double v[NE] = {0.0, 0.0, 0.0};
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int ti = (int)(t % T), tj = (int)(t / T);
        if (mode == 0) {
            __syncthreads();
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int a = ly + 8 * r;
                const int64_t gi = (int64_t)tj * TILE + lx, gj = (int64_t)ti * TILE + a;
                const bool in = gi < n && gj < n;
                Tt[0][a][lx] = in ? X[gi + gj * ldz] : 0.0;
                Tt[1][a][lx] = in ? Y[gi + gj * ldz] : 0.0;
                Tt[2][a][lx] = in ? h2[gi + gj * ldz] : 0.0;
                Tt[3][a][lx] = in ? s2[gi + gj * ldz] : 0.0;
            }
            __syncthreads();
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int64_t i = (int64_t)ti * TILE + lx, j = (int64_t)tj * TILE + ly + 8 * r;
            if (i >= n || j >= n) continue;
            double vh = h0[i + j * ldh], vs = s0[i + j * ldh];
            if (mode == 0) {
                const int b = ly + 8 * r;
                const double xs = X[i + j * ldz] + Tt[0][lx][b];
                const double ys = Y[i + j * ldz] + Tt[1][lx][b];
                const double h2s = 0.5 * (h2[i + j * ldz] + Tt[2][lx][b]);
                const double s2s = 0.5 * (s2[i + j * ldz] + Tt[3][lx][b]);
                vh = vh + x * (xs + x * h2s);
                vs = vs + x * (ys + x * s2s);
                h0[i + j * ldh] = vh;
                s0[i + j * ldh] = vs;
            }
            if (hsw.ptr != nullptr) {   // column j of [H_W ; S_W] is digit row j, K index i and n + i
                put3(hsw, j * hsw.ld + i, vh);
                put3(hsw, j * hsw.ld + n + i, vs);
            }
            if (i == j) v[0] += vh;
            v[1] = fma(vs, vh, v[1]);
            const double e = vs - (i == j ? 1.0 : 0.0);
            v[2] = fma(e, e, v[2]);
        }
    }
    block_sum<NE>(v, red);
    double tot[NE];
    if (!publish_and_collect<NE>(v, partials, counter, tot, red)) return;
    if (threadIdx.x != 0) return;
    const double E = 2.0 * (2.0 * tot[0] - tot[1]) + state->e_shift;
    state->trh0 = tot[0];
    state->sh = tot[1];
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

// ---------------------------------------------------------------- m x n kernels
// W += x D, H'W += x H'D, SW += x SD over 32 x 32 tiles of the m x n arrays
// (column-major, ld = m); optionally writes the digits of the new W (column
// j = digit row j) and of the rows of [SW | H'W] (digit row i, K index j and
// n + j) through a shared-memory transpose.
__global__ void __launch_bounds__(NT) update_kernel(int m, int n, double *W, const double *__restrict__ D,
                                                     double *HW, const double *__restrict__ HD, double *SW,
                                                     const double *__restrict__ SD, const DevState *state,
                                                     DigitOut wd, DigitOut swhw) {
    if (*((volatile const int *)&state->done)) return;
    __shared__ double tH[TILE][TILE + 1];
    __shared__ double tS[TILE][TILE + 1];
    const double x = state->x;
    const int lx = threadIdx.x % TILE, ly = threadIdx.x / TILE;
    const int Tm = (m + TILE - 1) / TILE, Tn = (n + TILE - 1) / TILE;
    for (int t = blockIdx.x; t < Tm * Tn; t += gridDim.x) {
        const int ti = t % Tm, tj = t / Tm;
        const int i = ti * TILE + lx;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int jl = ly + 8 * r, j = tj * TILE + jl;
            if (i < m && j < n) {
                const int64_t o = (int64_t)j * m + i;
                const double w = fma(x, D[o], W[o]);
                const double hw = fma(x, HD[o], HW[o]);
                const double sw = fma(x, SD[o], SW[o]);
                W[o] = w;
                HW[o] = hw;
                SW[o] = sw;
                if (wd.ptr != nullptr) put3(wd, (int64_t)j * wd.ld + i, w);
                tH[jl][lx] = hw;
                tS[jl][lx] = sw;
            }
        }
        if (swhw.ptr != nullptr) {
            __syncthreads();
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int il = ly + 8 * r, ii = ti * TILE + il, jj = tj * TILE + lx;
                if (ii < m && jj < n) {
                    put3(swhw, (int64_t)ii * swhw.ld + jj, tS[lx][il]);
                    put3(swhw, (int64_t)ii * swhw.ld + n + jj, tH[lx][il]);
                }
            }
            __syncthreads();
        }
    }
}

// <Z,G>, <Z,Gp>, <G,D> with Z = P G the preconditioned gradient (Z = G without
// preconditioning: then <G,G>, <G,Gp>, <G,D>)
constexpr int ND = 3;

__global__ void __launch_bounds__(NT) dots_kernel(int64_t mn, const double *__restrict__ G,
                                                   const double *__restrict__ Zg,
                                                   const double *__restrict__ Gp,
                                                   const double *__restrict__ D, double *partials,
                                                   unsigned int *counter, DevState *state,
                                                   int first) {
    if (*((volatile int *)&state->done)) return;
    __shared__ double red[(NT / 32) * ND];
    double v[ND] = {0.0, 0.0, 0.0};
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < mn; i += (int64_t)gridDim.x * NT) {
        const double g = G[i], z = Zg[i];
        v[0] = fma(z, g, v[0]);
        if (!first) {
            v[1] = fma(z, Gp[i], v[1]);
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
        // <G, -Z + beta D> >= 0 means no descent: restart with -Z
        restart = (-gg + beta * tot[2] >= 0.0) ? 1 : 0;
        if (restart) beta = 0.0;
    }
    if (!isfinite(gg) || !isfinite(beta)) {
        state->status = OMM_ERR_NONFINITE;
        state->done = 1;
        return;
    }
    state->gg = gg;
    state->ggp = tot[1];
    state->gd = tot[2];
    state->gg_prev = gg;
    state->beta = beta;
    state->restart = restart;
}

// D = -Z + beta D (D = -Z on a restart); Gp <- G
__global__ void direction_kernel(int m, int n, const double *__restrict__ G, const double *__restrict__ Zg,
                                 double *Gp, double *D, const DevState *state, DigitOut dd) {
    if (*((volatile const int *)&state->done)) return;
    const double beta = state->beta;
    const bool restart = state->restart != 0;
    for (int j = blockIdx.y; j < n; j += gridDim.y)
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
            const int64_t o = (int64_t)j * m + i;
            const double g = G[o], z = Zg[o];
            const double d = restart ? -z : fma(beta, D[o], -z);
            D[o] = d;
            Gp[o] = g;
            if (dd.ptr != nullptr) put3(dd, (int64_t)j * dd.ld + i, d);
        }
}

// one element per thread-iteration; every element reads only its own source
// elements, so Wd may alias W1 or W2 when the maps are the identity
__global__ void md_guess_kernel(int64_t nblk, int blk, double *Wd, const double *W1, const int64_t *i1,
                                const double *W2, const int64_t *i2) {
    const int64_t total = nblk * blk;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = e / blk, k = e - b * blk;
        const int64_t a1 = i1 != nullptr ? i1[b] : b;
        double v = 0.0;
        if (a1 >= 0) {
            const double w1 = W1[a1 * blk + k];
            if (W2 == nullptr) {
                v = w1;
            } else {
                const int64_t a2 = i2 != nullptr ? i2[b] : b;
                v = fma(2.0, w1, a2 >= 0 ? -W2[a2 * blk + k] : 0.0);   // 2 w1 exact: one rounding
            }
        }
        Wd[e] = v;
    }
}

__global__ void shift_kernel(int64_t mm, const double *H, const double *__restrict__ S, double *Hs,
                             const DevState *state) {
    const double eta = state->eta;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < mm;
         i += (int64_t)gridDim.x * blockDim.x)
        Hs[i] = H[i] - eta * S[i];
}

// per column j (= row j, symmetric): g = H_jj + sum_{i!=j} |H_ij|,
// lo = S_jj - sum_{i!=j} |S_ij|, hi = S_jj + sum_{i!=j} |S_ij|; then max/min.
__global__ void __launch_bounds__(NT) gershgorin_kernel(int64_t m, const double *__restrict__ H,
                                                         const double *__restrict__ S,
                                                         double *partials, unsigned int *counter,
                                                         DevState *state) {
    __shared__ double red[(NT / 32) * 3];
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
    double gmax = -INFINITY, lomin = INFINITY, himax = -INFINITY;
    for (int64_t j = warp; j < m; j += nwarps) {
        double sh = 0.0, ss = 0.0;
        for (int64_t i = lane; i < m; i += 32) {
            if (i == j) continue;
            sh += fabs(H[i + j * m]);
            ss += fabs(S[i + j * m]);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            sh += __shfl_down_sync(0xffffffffu, sh, off);
            ss += __shfl_down_sync(0xffffffffu, ss, off);
        }
        if (lane == 0) {
            gmax = fmax(gmax, H[j + j * m] + sh);
            lomin = fmin(lomin, S[j + j * m] - ss);
            himax = fmax(himax, S[j + j * m] + ss);
        }
    }
    // max/min reduction across the block (order-independent)
    const int w = threadIdx.x >> 5;
    if (lane == 0) { red[w * 3] = gmax; red[w * 3 + 1] = lomin; red[w * 3 + 2] = himax; }
    __syncthreads();
    double v[3];
    if (threadIdx.x == 0) {
        v[0] = -INFINITY; v[1] = INFINITY; v[2] = -INFINITY;
        for (int q = 0; q < NT / 32; ++q) {
            v[0] = fmax(v[0], red[q * 3]);
            v[1] = fmin(v[1], red[q * 3 + 1]);
            v[2] = fmax(v[2], red[q * 3 + 2]);
        }
    }
    __shared__ bool is_last;
    if (threadIdx.x == 0) {
        for (int q = 0; q < 3; ++q) partials[blockIdx.x * 3 + q] = v[q];
        __threadfence();
        is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last || threadIdx.x != 0) return;
    __threadfence();
    volatile const double *p = partials;
    double g = -INFINITY, lo = INFINITY, hi = -INFINITY;
    for (unsigned b = 0; b < gridDim.x; ++b) {
        g = fmax(g, p[b * 3]);
        lo = fmin(lo, p[b * 3 + 1]);
        hi = fmax(hi, p[b * 3 + 2]);
    }
    *counter = 0u;
    if (!(lo > 0.0)) {
        state->status = OMM_ERR_NOT_SPD;
        state->eta = NAN;
        return;
    }
    state->eta = (g >= 0.0) ? g / lo : g / hi;
}

int red_blocks_for_tiles(int n) {
    const int64_t T = ceil_div(n, TILE);
    int64_t nb = T * T;
    if (nb > kRedBlocksMax) nb = kRedBlocksMax;
    if (nb < 1) nb = 1;
    return (int)nb;
}

int red_blocks_for_len(int64_t len) {
    int64_t nb = ceil_div(len, (int64_t)NT * 8);
    if (nb > kRedBlocksMax) nb = kRedBlocksMax;
    if (nb < 1) nb = 1;
    return (int)nb;
}

int ew_blocks(int64_t len) {
    int64_t nb = ceil_div(len, (int64_t)NT * 4);
    if (nb > 152 * 8) nb = 152 * 8;
    if (nb < 1) nb = 1;
    return (int)nb;
}

}  // namespace

int64_t red_scratch_bytes() { return (int64_t)kRedBlocksMax * kRedSlots * sizeof(double); }

int launch_coeffs_linemin(int n, const double *h0, const double *s0, int64_t ldh, const double *Z,
                          int64_t ldz, double *scratch, unsigned int *counter, DevState *state,
                          double *coeffs_out, cudaStream_t st, bool do_linemin) {
    const double *X = Z;
    const double *Y = Z + (int64_t)n * ldz;
    const double *h2 = Z + n;
    const double *s2 = Z + n + (int64_t)n * ldz;
    coeffs_kernel<<<red_blocks_for_tiles(n), NT, 0, st>>>(n, h0, s0, ldh, X, Y, h2, s2, ldz, scratch,
                                                          counter, state, coeffs_out, do_linemin ? 1 : 0);
    omm::count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

int launch_update(int64_t m, int64_t n, double *W, const double *D, double *HW, const double *HD, double *SW,
                  const double *SD, const DevState *state, DigitOut wd, DigitOut swhw, cudaStream_t st) {
    int64_t nb = ceil_div(m, TILE) * ceil_div(n, TILE);
    if (nb > 152 * 8) nb = 152 * 8;
    update_kernel<<<(unsigned)nb, NT, 0, st>>>((int)m, (int)n, W, D, HW, HD, SW, SD, state, wd, swhw);
    omm::count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

int launch_nn_update_energy(int n, double *h0, double *s0, int64_t ldh, const double *Z,
                            int64_t ldz, double *scratch, unsigned int *counter, DevState *state,
                            int mode, cudaStream_t st, DigitOut hsw) {
    const double *X = Z;
    const double *Y = Z + (int64_t)n * ldz;
    const double *h2 = Z + n;
    const double *s2 = Z + n + (int64_t)n * ldz;
    nn_update_kernel<<<red_blocks_for_tiles(n), NT, 0, st>>>(n, h0, s0, ldh, X, Y, h2, s2, ldz,
                                                             scratch, counter, state, mode, hsw);
    omm::count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

int launch_dots_beta(int64_t mn, const double *G, const double *Zg, const double *Gp, const double *D,
                     double *scratch, unsigned int *counter, DevState *state, int first,
                     cudaStream_t st) {
    dots_kernel<<<red_blocks_for_len(mn), NT, 0, st>>>(mn, G, Zg, Gp, D, scratch, counter, state, first);
    omm::count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

int launch_direction(int64_t m, int64_t n, const double *G, const double *Zg, double *Gp, double *D,
                     const DevState *state, cudaStream_t st, DigitOut dd) {
    dim3 grid((unsigned)ceil_div(m, NT), (unsigned)(n < 1024 ? n : 1024));
    direction_kernel<<<grid, NT, 0, st>>>((int)m, (int)n, G, Zg, Gp, D, state, dd);
    omm::count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

int launch_md_guess(int64_t nblk, int blk, double *Wd, const double *W1, const int64_t *i1, const double *W2,
                    const int64_t *i2, cudaStream_t st) {
    int64_t nb = ceil_div(nblk * blk, (int64_t)NT);
    if (nb > 152 * 8) nb = 152 * 8;
    md_guess_kernel<<<(unsigned)(nb < 1 ? 1 : nb), NT, 0, st>>>(nblk, blk, Wd, W1, i1, W2, i2);
    omm::count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

int launch_shift(int64_t mm, const double *H, const double *S, double *Hs, const DevState *state,
                 cudaStream_t st) {
    shift_kernel<<<ew_blocks(mm), NT, 0, st>>>(mm, H, S, Hs, state);
    omm::count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

namespace {
// K = 2I - S_W (mode 0) or H'_W + eta (2I - S_W) (mode 1), n x n column-major,
// from [H'_W ; S_W] (2n x n, ld 2n)
__global__ void density_K_kernel(int64_t n, const double *__restrict__ h0s0, double eta, int mode, double *K) {
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n * n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx % n, j = idx / n;
        const double t = (i == j ? 2.0 : 0.0) - h0s0[(n + i) + j * 2 * n];
        K[i + j * n] = mode == 0 ? t : fma(eta, t, h0s0[i + j * 2 * n]);
    }
}
}  // namespace

int launch_density_K(int64_t n, const double *h0s0, double eta, int mode, double *K, cudaStream_t st) {
    int64_t nb = ceil_div(n * n, 256);
    if (nb > 152 * 8) nb = 152 * 8;
    density_K_kernel<<<(unsigned)(nb < 1 ? 1 : nb), 256, 0, st>>>(n, h0s0, eta, mode, K);
    count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

int launch_gershgorin(int64_t m, const double *H, const double *S, double *scratch,
                      unsigned int *counter, DevState *state, cudaStream_t st) {
    int64_t nb = ceil_div(m, NT / 32);
    if (nb > kRedBlocksMax) nb = kRedBlocksMax;
    gershgorin_kernel<<<(unsigned)nb, NT, 0, st>>>(m, H, S, scratch, counter, state);
    omm::count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

// ---------------------------------------------------------------- op-level entries
namespace {
// one warp
__global__ void line_min_kernel(const double *c, double *x_out, int32_t *status_out) {
    double cc[5];
    for (int q = 0; q < 5; ++q) cc[q] = c[q];
    double x = 0.0;
    const int st = lm::quartic_min_warp(cc, &x);
    if (threadIdx.x != 0) return;
    *x_out = x;
    *status_out = st;
}
}  // namespace

}  // namespace omm

extern "C" int64_t omm_op_quartic_coeffs_scratch_bytes(int64_t n) {
    (void)n;
    // per-block partials (<= kRedBlocksMax blocks x 13 doubles) + the counter
    return (int64_t)omm::kRedBlocksMax * 13 * (int64_t)sizeof(double) + 256;
}

extern "C" int omm_op_quartic_coeffs(int64_t n, const double *h0, const double *s0, int64_t ld_h,
                                     const double *X, const double *Y, const double *h2,
                                     const double *s2, int64_t ld_z, double *coeffs, void *scratch,
                                     int64_t scratch_bytes, void *stream) {
    if (n < 0 || n > 2147483647) return OMM_ERR_ARG;
    if (coeffs == nullptr || scratch == nullptr) return OMM_ERR_ARG;
    if (scratch_bytes < omm_op_quartic_coeffs_scratch_bytes(n)) return OMM_ERR_ARG;
    if (((uintptr_t)scratch) & 15u) return OMM_ERR_ARG;
    if (n > 0 && (h0 == nullptr || s0 == nullptr || X == nullptr || Y == nullptr || h2 == nullptr ||
                  s2 == nullptr || ld_h < n || ld_z < n))
        return OMM_ERR_ARG;
    double *partials = (double *)scratch;
    unsigned int *counter =
        (unsigned int *)((char *)scratch + (int64_t)omm::kRedBlocksMax * 13 * sizeof(double));
    cudaStream_t st = (cudaStream_t)stream;
    omm::coeffs_kernel<<<omm::red_blocks_for_tiles((int)n), omm::NT, 0, st>>>(
        (int)n, h0, s0, ld_h, X, Y, h2, s2, ld_z, partials, counter, nullptr, coeffs, 0);
    omm::count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

extern "C" int omm_op_line_min(const double *coeffs, double *x_out, int32_t *status_out,
                               void *stream) {
    if (coeffs == nullptr || x_out == nullptr || status_out == nullptr) return OMM_ERR_ARG;
    omm::line_min_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(coeffs, x_out, status_out);
    omm::count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

// ---------------------------------------------------------------- allocation-free variant
// Some callers cannot allocate device memory at the point where they need the
// line-search coefficients: code running under a memory budget that forbids
// cudaMalloc on the hot path, or a caller that only owns the six input arrays
// and the 5-double output.  For them the reduction's scratch (per-block
// partial sums and the completion counter) lives in this file-scope array,
// which every GPU that loads the library holds until the process exits.
namespace {
constexpr int64_t kCoeffPartialsBytes = (int64_t)omm::kRedBlocksMax * 13 * (int64_t)sizeof(double);
constexpr int64_t kCoeffStaticBytes = kCoeffPartialsBytes + 256;   // + the counter, own 256-byte slot
static __device__ __align__(256) unsigned char g_coeff_scratch[kCoeffStaticBytes];

// red_blocks_for_tiles never launches more than kRedBlocksMax blocks, so every
// n in [0, 2^31 - 1] fits the array.
static_assert(kCoeffPartialsBytes >= (int64_t)omm::kRedBlocksMax * 13 * (int64_t)sizeof(double),
              "one partial-sum slot per block of the largest launch");

constexpr int kMaxDevices = 64;
std::mutex g_coeff_mu;
void *g_coeff_ptr[kMaxDevices] = {};   // device address of g_coeff_scratch last seen, per device

// With the device current: look up the array's device address (its host-side
// name is only a stand-in).  The lookup runs on every call, so a module loaded
// again after a device reset is found at its new address; the counter is zeroed
// (synchronously, before any kernel may use it) the first time an address is seen.
int coeff_scratch_for_current_device(void **out) {
    int dev = -1;
    OMM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        omm::set_error("omm_op_quartic_coeffs_static: device ordinal %d outside 0..%d", dev, kMaxDevices - 1);
        return OMM_ERR_ARG;
    }
    void *p = nullptr;
    OMM_CUDA_TRY(cudaGetSymbolAddress(&p, g_coeff_scratch));
    std::lock_guard<std::mutex> lock(g_coeff_mu);
    if (g_coeff_ptr[dev] != p) {
        OMM_CUDA_TRY(cudaMemset((char *)p + kCoeffPartialsBytes, 0, 256));
        OMM_CUDA_TRY(cudaDeviceSynchronize());
        g_coeff_ptr[dev] = p;
    }
    *out = p;
    return OMM_OK;
}
}  // namespace

extern "C" int64_t omm_op_quartic_coeffs_static_max_bytes(void) { return kCoeffStaticBytes; }

extern "C" int omm_op_quartic_coeffs_static(int64_t n, const double *h0, const double *s0, int64_t ld_h,
                                            const double *X, const double *Y, const double *h2,
                                            const double *s2, int64_t ld_z, double *coeffs, void *stream) {
    if (n < 0 || n > 2147483647) {
        omm::set_error("omm_op_quartic_coeffs_static: n = %lld outside 0..2147483647", (long long)n);
        return OMM_ERR_ARG;
    }
    const int64_t blocks = omm::red_blocks_for_tiles((int)n);   // at most kRedBlocksMax
    if (coeffs == nullptr) {
        omm::set_error("omm_op_quartic_coeffs_static: coeffs is NULL");
        return OMM_ERR_ARG;
    }
    if (n > 0 && (h0 == nullptr || s0 == nullptr || X == nullptr || Y == nullptr || h2 == nullptr ||
                  s2 == nullptr)) {
        omm::set_error("omm_op_quartic_coeffs_static: an input array is NULL with n = %lld", (long long)n);
        return OMM_ERR_ARG;
    }
    if (n > 0 && (ld_h < n || ld_z < n)) {
        omm::set_error("omm_op_quartic_coeffs_static: ld_h = %lld, ld_z = %lld below n = %lld", (long long)ld_h,
                       (long long)ld_z, (long long)n);
        return OMM_ERR_ARG;
    }
    void *scratch = nullptr;
    const int rc = coeff_scratch_for_current_device(&scratch);
    if (rc != OMM_OK) return rc;
    double *partials = (double *)scratch;
    unsigned int *counter = (unsigned int *)((char *)scratch + kCoeffPartialsBytes);
    cudaStream_t st = (cudaStream_t)stream;
    omm::coeffs_kernel<<<(unsigned)blocks, omm::NT, 0, st>>>((int)n, h0, s0, ld_h, X, Y, h2, s2, ld_z,
                                                             partials, counter, nullptr, coeffs, 0);
    omm::count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}
