// FP32 "glue" kernels of the mixed-precision CG step.
//
// GB300 runs FP64 (and conversions from FP64) on a small unit: about two FP64
// operations per clock per SM against thousands of tensor-core flops.  So the
// mixed form keeps FP64 only for the state that must stay accurate -- W, H'W,
// SW, H_W, S_W -- and carries every increment in FP32: the products H'D, SD
// and the contractions X, Y, h2, s2 come out of the split tensor-core GEMMs as
// FP32, the gradient and search direction are FP32, and each state update is
// one FP32 increment added in FP64.  The increments are only as accurate as
// the 24-bit split products that feed them, so nothing is lost by rounding
// them to FP32.  Reductions multiply and accumulate in FP32 per thread and
// combine per-block partials in FP64 in a fixed order (bitwise repeatable).
//
// Two quantities avoid cancellation by construction:
//   c1 = 2 <G, D>   the slope of the line, taken from the CG dot products
//                   (it equals 2 [4 tr X - 2 <S_W, X> - 2 <Y, H_W>] exactly);
//   E_{k+1} = c0 + c1 x + c2 x^2 + c3 x^3 + c4 x^4  at the line minimum x,
//                   the quartic being exact along the line.
#include <cuda_bf16.h>
#include <math.h>

#include "fp_convert.cuh"
#include "linemin.cuh"
#include "omm_internal.cuh"

namespace omm {
namespace {

constexpr int NT = 256;
constexpr int TILE = 32;

// Three BF16 digits of an FP32 value (exact: 3 x 8 significant bits)
__device__ __forceinline__ void put3f(const DigitOut &d, int64_t o, float v) {
    const __nv_bfloat16 d1 = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(d1);
    const __nv_bfloat16 d2 = __float2bfloat16_rn(r1);
    const __nv_bfloat16 d3 = __float2bfloat16_rn(r1 - __bfloat162float(d2));
    __nv_bfloat16 *p = (__nv_bfloat16 *)d.ptr;
    p[o] = d1;
    if (d.nd > 1) p[d.plane + o] = d2;
    if (d.nd > 2) p[2 * d.plane + o] = d3;
}

// Digits of four consecutive FP32 values (8-byte aligned offset o): same
// rounding as put3f, two values per conversion, one 8-byte store per plane.
__device__ __forceinline__ void put3f4(const DigitOut &d, int64_t o, float4 v) {
    const __nv_bfloat162 a1 = __floats2bfloat162_rn(v.x, v.y), b1 = __floats2bfloat162_rn(v.z, v.w);
    const float2 fa1 = __bfloat1622float2(a1), fb1 = __bfloat1622float2(b1);
    const float r0 = v.x - fa1.x, r1 = v.y - fa1.y, r2 = v.z - fb1.x, r3 = v.w - fb1.y;
    const __nv_bfloat162 a2 = __floats2bfloat162_rn(r0, r1), b2 = __floats2bfloat162_rn(r2, r3);
    const float2 fa2 = __bfloat1622float2(a2), fb2 = __bfloat1622float2(b2);
    const __nv_bfloat162 a3 = __floats2bfloat162_rn(r0 - fa2.x, r1 - fa2.y);
    const __nv_bfloat162 b3 = __floats2bfloat162_rn(r2 - fb2.x, r3 - fb2.y);
    __nv_bfloat16 *p = (__nv_bfloat16 *)d.ptr;
    auto pack = [](__nv_bfloat162 lo, __nv_bfloat162 hi) {
        uint2 u;
        u.x = *reinterpret_cast<const uint32_t *>(&lo);
        u.y = *reinterpret_cast<const uint32_t *>(&hi);
        return u;
    };
    *reinterpret_cast<uint2 *>(p + o) = pack(a1, b1);
    if (d.nd > 1) *reinterpret_cast<uint2 *>(p + d.plane + o) = pack(a2, b2);
    if (d.nd > 2) *reinterpret_cast<uint2 *>(p + 2 * d.plane + o) = pack(a3, b3);
}

// Digits of two consecutive FP32 values (4-byte aligned offset o), as put3f.
__device__ __forceinline__ void put3f2(const DigitOut &d, int64_t o, float v0, float v1) {
    const __nv_bfloat162 a1 = __floats2bfloat162_rn(v0, v1);
    const float2 f1 = __bfloat1622float2(a1);
    const float r0 = v0 - f1.x, r1 = v1 - f1.y;
    const __nv_bfloat162 a2 = __floats2bfloat162_rn(r0, r1);
    const float2 f2 = __bfloat1622float2(a2);
    const __nv_bfloat162 a3 = __floats2bfloat162_rn(r0 - f2.x, r1 - f2.y);
    __nv_bfloat16 *p = (__nv_bfloat16 *)d.ptr;
    *reinterpret_cast<__nv_bfloat162 *>(p + o) = a1;
    if (d.nd > 1) *reinterpret_cast<__nv_bfloat162 *>(p + d.plane + o) = a2;
    if (d.nd > 2) *reinterpret_cast<__nv_bfloat162 *>(p + 2 * d.plane + o) = a3;
}

// FP32 per-thread partials: summed across the warp in FP32 (their inputs are
// FP32 products, so this adds error of the same order), then converted to
// FP64 on the integer pipe; block_sum then adds the warps' values in FP64.
template <int NV>
__device__ __forceinline__ void to_f64(const float (&f)[NV], double (&v)[NV]) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        float t = f[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
        v[q] = (threadIdx.x & 31) == 0 ? sw_f2d(t) : 0.0;
    }
}

template <int NV>
__device__ void block_sum(double (&v)[NV], double *red, bool lane0_only = false) {
    if (!lane0_only) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double s = v[q];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
            v[q] = s;
        }
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

// ---------------------------------------------------------------- coefficients
// partials: 0 tr h2, 1 <s0,h2>, 2 <Y,X>, 3 <Y,X^T>, 4 <s2,h0>, 5 <Y,h2>, 6 <s2,X>, 7 <s2,h2>
constexpr int NC = 8;

__global__ void __launch_bounds__(NT) mx_coeffs_kernel(int n, const double *__restrict__ h0,
                                                        const double *__restrict__ s0, int64_t ldh,
                                                        const float *__restrict__ Z, int64_t ldz,
                                                        double *partials, unsigned int *counter,
                                                        DevState *state, const double *__restrict__ slope,
                                                        int nslope) {
    if (*((volatile int *)&state->done)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) state->done_upd = 1;
        return;
    }
    __shared__ float Xt[TILE][TILE + 1];
    __shared__ double red[(NT / 32) * NC];
    const float *X = Z, *Y = Z + (int64_t)n * ldz, *h2 = Z + n, *s2 = Z + n + (int64_t)n * ldz;
    const int lx = threadIdx.x % TILE, ly = threadIdx.x / TILE;
    const int T = (n + TILE - 1) / TILE;
    float f[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) f[q] = 0.f;
    for (int t = blockIdx.x; t < T * T; t += gridDim.x) {
        const int ti = t % T, tj = t / T;
        // every load of the tile is issued before any is used (zero outside the
        // matrix instead of a branch), so a thread has ~30 loads in flight
        float xt[4], vx[4], vy[4], vh2[4], vs2[4];
        double dh0[4], ds0[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int a = ly + 8 * r, gi = tj * TILE + lx, gj = ti * TILE + a;
            xt[r] = (gi < n && gj < n) ? X[gi + (int64_t)gj * ldz] : 0.f;
            const int i = ti * TILE + lx, j = tj * TILE + a;
            const bool in = i < n && j < n;
            const int64_t oz = i + (int64_t)j * ldz, oh = i + (int64_t)j * ldh;
            vx[r] = in ? X[oz] : 0.f;
            vy[r] = in ? Y[oz] : 0.f;
            vh2[r] = in ? h2[oz] : 0.f;
            vs2[r] = in ? s2[oz] : 0.f;
            dh0[r] = in ? h0[oh] : 0.0;
            ds0[r] = in ? s0[oh] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 4; ++r) Xt[ly + 8 * r][lx] = xt[r];
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = ti * TILE + lx, j = tj * TILE + ly + 8 * r;
            const float vh0 = sw_d2f(dh0[r]), vs0 = sw_d2f(ds0[r]), vxt = Xt[lx][ly + 8 * r];
            if (i == j && i < n) f[0] += vh2[r];
            f[1] = fmaf(vs0, vh2[r], f[1]);
            f[2] = fmaf(vy[r], vx[r], f[2]);
            f[3] = fmaf(vy[r], vxt, f[3]);
            f[4] = fmaf(vs2[r], vh0, f[4]);
            f[5] = fmaf(vy[r], vh2[r], f[5]);
            f[6] = fmaf(vs2[r], vx[r], f[6]);
            f[7] = fmaf(vs2[r], vh2[r], f[7]);
        }
    }
    double v[NC];
    to_f64<NC>(f, v);
    block_sum<NC>(v, red, true);
    double tot[NC] = {};
    if (!publish_and_collect<NC>(v, partials, counter, tot, red)) return;
    // the slope <G, D>: the direction kernel's per-block parts (one-digit
    // directions), else the dots kernel's value
    double gd[1] = {0.0};
    if (nslope > 0) {
        for (int b = threadIdx.x; b < nslope; b += NT) gd[0] += __ldcg(&slope[b]);
        block_sum<1>(gd, red);
    }
    if (threadIdx.x >= 32) return;   // warp 0: the line minimum
#pragma unroll
    for (int q = 0; q < NC; ++q) tot[q] = __shfl_sync(0xffffffffu, tot[q], 0);
    const double gD = nslope > 0 ? __shfl_sync(0xffffffffu, gd[0], 0) : state->gD;
    double c[5];
    c[0] = state->E - state->e_shift;   // the shifted functional at x = 0
    c[1] = 2.0 * gD;
    c[2] = 2.0 * (2.0 * tot[0] - tot[1] - 2.0 * (tot[2] + tot[3]) - tot[4]);
    c[3] = 2.0 * (-2.0 * tot[5] - 2.0 * tot[6]);
    c[4] = -2.0 * tot[7];
    double x = 0.0;
    const int st = lm::quartic_min_warp(c, &x);
    if (threadIdx.x != 0) return;
    state->gD = gD;
    for (int q = 0; q < 5; ++q) state->c[q] = c[q];
    state->x = x;
    state->x_f = (float)x;
    state->E_next = lm::quartic_val(c, x) + state->e_shift;
    if (st != OMM_OK) {
        state->status = st;
        state->done = 1;
    }
    state->done_upd = st != OMM_OK ? 1 : 0;
}

// ---------------------------------------------------------------- H_W, S_W update
// h0 += x (X + X^T) + x^2 sym(h2), s0 likewise (FP32 increments, FP64 sums);
// ||s0 - I||_F^2 for the orthonormality test; digits of [H_W ; S_W] columns.
__global__ void __launch_bounds__(NT, 4) mx_nn_update_kernel(int n, double *h0, double *s0, int64_t ldh,
                                                           const float *__restrict__ Z, int64_t ldz,
                                                           double *partials, unsigned int *counter,
                                                           DevState *state, DigitOut hsw) {
    if (*((volatile int *)&state->done)) return;
    __shared__ float Tt[4][TILE][TILE + 1];
    __shared__ double red[(NT / 32)];
    const float *X = Z, *Y = Z + (int64_t)n * ldz, *h2 = Z + n, *s2 = Z + n + (int64_t)n * ldz;
    const int lx = threadIdx.x % TILE, ly = threadIdx.x / TILE;
    const int T = (n + TILE - 1) / TILE;
    const float x = state->x_f;
    float orth = 0.f;
    for (int t = blockIdx.x; t < T * T; t += gridDim.x) {
        const int ti = t % T, tj = t / T;
        // all loads of the tile first (zero outside the matrix), then the transposes
        // through shared memory, then the updates
        float tx[4][4], vz[4][4];
        double dh0[4], ds0[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int a = ly + 8 * r, gi = tj * TILE + lx, gj = ti * TILE + a;
            const bool tin = gi < n && gj < n;
            const int64_t to = gi + (int64_t)gj * ldz;
            tx[0][r] = tin ? X[to] : 0.f;
            tx[1][r] = tin ? Y[to] : 0.f;
            tx[2][r] = tin ? h2[to] : 0.f;
            tx[3][r] = tin ? s2[to] : 0.f;
            const int i = ti * TILE + lx, j = tj * TILE + a;
            const bool in = i < n && j < n;
            const int64_t oz = i + (int64_t)j * ldz, oh = i + (int64_t)j * ldh;
            vz[0][r] = in ? X[oz] : 0.f;
            vz[1][r] = in ? Y[oz] : 0.f;
            vz[2][r] = in ? h2[oz] : 0.f;
            vz[3][r] = in ? s2[oz] : 0.f;
            dh0[r] = in ? h0[oh] : 0.0;
            ds0[r] = in ? s0[oh] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) Tt[q][ly + 8 * r][lx] = tx[q][r];
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = ti * TILE + lx, j = tj * TILE + ly + 8 * r, b = ly + 8 * r;
            if (i >= n || j >= n) continue;
            const int64_t oh = i + (int64_t)j * ldh;
            const float xs = vz[0][r] + Tt[0][lx][b], ys = vz[1][r] + Tt[1][lx][b];
            const float h2s = 0.5f * (vz[2][r] + Tt[2][lx][b]), s2s = 0.5f * (vz[3][r] + Tt[3][lx][b]);
            const double vh = dh0[r] + sw_f2d(x * fmaf(x, h2s, xs));
            const double vs = ds0[r] + sw_f2d(x * fmaf(x, s2s, ys));
            h0[oh] = vh;
            s0[oh] = vs;
            const float fvs = sw_d2f(vs);
            const float e = (i == j) ? sw_d2f(vs - 1.0) : fvs;
            orth = fmaf(e, e, orth);
            if (hsw.ptr != nullptr) {
                put3f(hsw, (int64_t)j * hsw.ld + i, sw_d2f(vh));
                put3f(hsw, (int64_t)j * hsw.ld + n + i, fvs);
            }
        }
    }
    const float fo[1] = {orth};
    double v[1];
    to_f64<1>(fo, v);
    block_sum<1>(v, red, true);
    double tot[1];
    if (!publish_and_collect<1>(v, partials, counter, tot, red)) return;
    if (threadIdx.x != 0) return;
    const double E = state->E_next;
    state->orth2 = tot[0];
    if (!isfinite(E)) {
        state->status = OMM_ERR_NONFINITE;
        state->done = 1;
        return;
    }
    const double Ep = state->E;
    const double rel = fabs(2.0 * (E - Ep) / (E + Ep));
    state->E_prev = Ep;
    state->E = E;
    state->rel = rel;
    state->k += 1;
    const bool orth_ok = !(state->orth_tol > 0.0) || sqrt(tot[0]) < state->orth_tol;
    if (rel < state->tol && orth_ok) {
        state->status = OMM_OK;
        state->done = 1;
    } else if (state->k >= state->max_iter) {
        state->status = OMM_ERR_MAXITER;
        state->done = 1;
    }
}

// ---------------------------------------------------------------- W, H'W, SW update
__global__ void __launch_bounds__(NT) mx_update_kernel(int m, int n, double *W, const float *__restrict__ D,
                                                        double *HW, const float *__restrict__ HD, double *SW,
                                                        const float *__restrict__ SD, const DevState *state,
                                                        DigitOut wd, DigitOut swhw) {
    if (*((volatile const int *)&state->done_upd)) return;
    __shared__ float tH[TILE][TILE + 1];
    __shared__ float tS[TILE][TILE + 1];
    const float x = state->x_f;
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
                const double w = W[o] + sw_f2d(x * D[o]);
                const double hw = HW[o] + sw_f2d(x * HD[o]);
                const double sw = SW[o] + sw_f2d(x * SD[o]);
                W[o] = w;
                HW[o] = hw;
                SW[o] = sw;
                if (wd.ptr != nullptr) put3f(wd, (int64_t)j * wd.ld + i, sw_d2f(w));
                tH[jl][lx] = sw_d2f(hw);
                tS[jl][lx] = sw_d2f(sw);
            }
        }
        if (swhw.ptr != nullptr) {
            __syncthreads();
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int il = ly + 8 * r, ii = ti * TILE + il, jj = tj * TILE + lx;
                if (ii < m && jj < n) {
                    put3f(swhw, (int64_t)ii * swhw.ld + jj, tS[lx][il]);
                    put3f(swhw, (int64_t)ii * swhw.ld + n + jj, tH[lx][il]);
                }
            }
            __syncthreads();
        }
    }
}

// Two consecutive rows per thread on 64 x 32 tiles (m even, 16-byte aligned
// FP64 arrays): double2 / float2 accesses, paired digit conversions.
constexpr int TI2 = 64;
__global__ void __launch_bounds__(NT) mx_update2_kernel(int m, int n, double2 *W, const float2 *__restrict__ D,
                                                         double2 *HW, const float2 *__restrict__ HD, double2 *SW,
                                                         const float2 *__restrict__ SD, const DevState *state,
                                                         DigitOut wd, DigitOut swhw) {
    if (*((volatile const int *)&state->done_upd)) return;
    __shared__ float tH[TILE][TI2 + 1];
    __shared__ float tS[TILE][TI2 + 1];
    const float x = state->x_f;
    const int lx = threadIdx.x % 32, ly = threadIdx.x / 32;
    const int Tm = (m + TI2 - 1) / TI2, Tn = (n + TILE - 1) / TILE;
    for (int t = blockIdx.x; t < Tm * Tn; t += gridDim.x) {
        const int ti = t % Tm, tj = t / Tm;
        const int i = ti * TI2 + 2 * lx;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int jl = ly + 8 * r, j = tj * TILE + jl;
            if (i < m && j < n) {
                const int64_t o2 = ((int64_t)j * m + i) >> 1;
                const float2 d = D[o2], hd = HD[o2], sd = SD[o2];
                double2 w = W[o2], hw = HW[o2], sw = SW[o2];
                w.x += sw_f2d(x * d.x);
                w.y += sw_f2d(x * d.y);
                hw.x += sw_f2d(x * hd.x);
                hw.y += sw_f2d(x * hd.y);
                sw.x += sw_f2d(x * sd.x);
                sw.y += sw_f2d(x * sd.y);
                W[o2] = w;
                HW[o2] = hw;
                SW[o2] = sw;
                if (wd.ptr != nullptr) put3f2(wd, (int64_t)j * wd.ld + i, sw_d2f(w.x), sw_d2f(w.y));
                tH[jl][2 * lx] = sw_d2f(hw.x);
                tH[jl][2 * lx + 1] = sw_d2f(hw.y);
                tS[jl][2 * lx] = sw_d2f(sw.x);
                tS[jl][2 * lx + 1] = sw_d2f(sw.y);
            }
        }
        if (swhw.ptr != nullptr) {
            __syncthreads();
#pragma unroll
            for (int r = 0; r < TI2 / 8; ++r) {
                const int il = ly + 8 * r, ii = ti * TI2 + il, jj = tj * TILE + lx;
                if (ii < m && jj < n) {
                    put3f(swhw, (int64_t)ii * swhw.ld + jj, tS[lx][il]);
                    put3f(swhw, (int64_t)ii * swhw.ld + n + jj, tH[lx][il]);
                }
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------- CG dots and direction
// <Z,G>, <Z,Gp>, <G,D> with Z = P G (PRE) or Z = G
constexpr int ND = 3;

template <bool PRE>
__global__ void __launch_bounds__(NT) mx_dots_kernel(int64_t mn, const float *__restrict__ G,
                                                      const float *__restrict__ Zg, const float *__restrict__ Gp,
                                                      const float *__restrict__ D, double *partials,
                                                      unsigned int *counter, DevState *state, int first) {
    if (*((volatile int *)&state->done)) return;
    __shared__ double red[(NT / 32) * ND];
    float f[ND] = {0.f, 0.f, 0.f};
    const int64_t n4 = mn / 4, stride = (int64_t)gridDim.x * NT;
    const float4 *G4 = reinterpret_cast<const float4 *>(G), *Gp4 = reinterpret_cast<const float4 *>(Gp),
                 *D4 = reinterpret_cast<const float4 *>(D), *Z4 = reinterpret_cast<const float4 *>(Zg);
#pragma unroll 4
    for (int64_t k = (int64_t)blockIdx.x * NT + threadIdx.x; k < n4; k += stride) {
        const float4 g = G4[k];
        const float4 z = PRE ? Z4[k] : g;
        f[0] = fmaf(z.x, g.x, fmaf(z.y, g.y, fmaf(z.z, g.z, fmaf(z.w, g.w, f[0]))));
        if (!first) {
            const float4 p = Gp4[k], d = D4[k];
            f[1] = fmaf(z.x, p.x, fmaf(z.y, p.y, fmaf(z.z, p.z, fmaf(z.w, p.w, f[1]))));
            f[2] = fmaf(g.x, d.x, fmaf(g.y, d.y, fmaf(g.z, d.z, fmaf(g.w, d.w, f[2]))));
        }
    }
    for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * NT + threadIdx.x; i < mn; i += stride) {   // tail
        const float g = G[i], z = PRE ? Zg[i] : g;
        f[0] = fmaf(z, g, f[0]);
        if (!first) {
            f[1] = fmaf(z, Gp[i], f[1]);
            f[2] = fmaf(g, D[i], f[2]);
        }
    }
    double v[ND];
    to_f64<ND>(f, v);
    block_sum<ND>(v, red, true);
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
    state->ggp = tot[1];
    state->gd = tot[2];
    state->gg_prev = gg;
    state->beta = beta;
    state->beta_f = (float)beta;
    state->restart = restart;
    state->gD = restart ? -gg : -gg + beta * tot[2];   // <G, D_new>
}

// Df = -Z + beta Df (Df = -Z on a restart), Z = P G (Zg) or G; Gp <- G.  Df is
// the direction of the CG recurrence.  ROUND1: the line search runs along D, Df
// rounded to one BF16 digit (its digit planes past the first are zero), while
// the recurrence keeps Df unrounded; each block leaves its part of the slope
// <G, D> of the rounded direction in slope[blockIdx.x], which the coefficients
// kernel sums (c1 / 2 of the quartic; no serial tail here).  Without ROUND1, D
// and Df are the same array.
template <bool ROUND1>
__device__ __forceinline__ void direction_slope(float gd, double *slope) {
    if (!ROUND1) return;
    __shared__ double red[NT / 32];
    const float f[1] = {gd};
    double v[1];
    to_f64<1>(f, v);
    block_sum<1>(v, red, true);
    if (threadIdx.x == 0) slope[blockIdx.x] = v[0];
}

template <bool ROUND1>
__global__ void __launch_bounds__(NT) mx_direction_kernel(int m, int64_t mn, const float *__restrict__ G,
                                                           const float *__restrict__ Zg, float *Gp, float *Df,
                                                           float *D, DevState *state, DigitOut dd, double *slope) {
    if (*((volatile const int *)&state->done)) return;
    const float beta = state->beta_f;
    const bool restart = state->restart != 0;
    float gd = 0.f;
    for (int64_t o = (int64_t)blockIdx.x * NT + threadIdx.x; o < mn; o += (int64_t)gridDim.x * NT) {
        const float g = G[o], z = Zg != nullptr ? Zg[o] : g;
        const float d = restart ? -z : fmaf(beta, Df[o], -z);
        Df[o] = d;
        Gp[o] = g;
        const int64_t j = o / m, i = o - j * m;
        if (ROUND1) {
            const __nv_bfloat16 b = __float2bfloat16_rn(d);
            const float r = __bfloat162float(b);
            gd = fmaf(g, r, gd);
            D[o] = r;
            if (dd.ptr != nullptr) {
                __nv_bfloat16 *p = (__nv_bfloat16 *)dd.ptr;
                const int64_t q = j * dd.ld + i;
                p[q] = b;
                for (int t = 1; t < dd.nd; ++t) p[t * dd.plane + q] = __float2bfloat16_rn(0.f);
            }
        } else if (dd.ptr != nullptr) {
            put3f(dd, j * dd.ld + i, d);
        }
    }
    direction_slope<ROUND1>(gd, slope);
}

// four consecutive rows of one column per thread (m % 4 == 0, 16-byte aligned arrays)
template <bool PRE, bool ROUND1>
__global__ void __launch_bounds__(NT) mx_direction4_kernel(int m, int64_t mn, const float4 *__restrict__ G,
                                                            const float4 *__restrict__ Zg, float4 *Gp, float4 *Df,
                                                            float4 *D, DevState *state, DigitOut dd,
                                                            double *slope) {
    if (*((volatile const int *)&state->done)) return;
    const float beta = state->beta_f;
    const bool restart = state->restart != 0;
    const int64_t n4 = mn / 4;
    float gd = 0.f;
    for (int64_t k = (int64_t)blockIdx.x * NT + threadIdx.x; k < n4; k += (int64_t)gridDim.x * NT) {
        const float4 g = G[k];
        const float4 z = PRE ? Zg[k] : g;
        float4 d = Df[k];
        if (restart) {
            d = make_float4(-z.x, -z.y, -z.z, -z.w);
        } else {
            d.x = fmaf(beta, d.x, -z.x);
            d.y = fmaf(beta, d.y, -z.y);
            d.z = fmaf(beta, d.z, -z.z);
            d.w = fmaf(beta, d.w, -z.w);
        }
        Df[k] = d;
        Gp[k] = g;
        const int64_t o = 4 * k, j = o / m, i = o - j * m;
        if (ROUND1) {
            const __nv_bfloat162 b01 = __floats2bfloat162_rn(d.x, d.y), b23 = __floats2bfloat162_rn(d.z, d.w);
            const float2 f01 = __bfloat1622float2(b01), f23 = __bfloat1622float2(b23);
            const float4 r = make_float4(f01.x, f01.y, f23.x, f23.y);
            gd = fmaf(g.x, r.x, fmaf(g.y, r.y, fmaf(g.z, r.z, fmaf(g.w, r.w, gd))));
            D[k] = r;
            if (dd.ptr != nullptr) {
                __nv_bfloat16 *p = (__nv_bfloat16 *)dd.ptr;
                uint2 u;
                u.x = *reinterpret_cast<const uint32_t *>(&b01);
                u.y = *reinterpret_cast<const uint32_t *>(&b23);
                *reinterpret_cast<uint2 *>(p + j * dd.ld + i) = u;
                for (int t = 1; t < dd.nd; ++t)
                    *reinterpret_cast<uint2 *>(p + t * dd.plane + j * dd.ld + i) = make_uint2(0u, 0u);
            }
        } else if (dd.ptr != nullptr) {
            put3f4(dd, j * dd.ld + i, d);
        }
    }
    direction_slope<ROUND1>(gd, slope);
}

// Grid-wide barrier of a cooperative launch (every block of the grid is
// resident), on two words kept for the handle: bar[0] counts the blocks that
// have arrived, bar[1] is the generation.  Each block reads the generation,
// then arrives; the last to arrive resets the count and advances the
// generation, which releases the others.  Nothing depends on the grid size of
// earlier launches.  The wait is bounded: past ~1 s (far beyond any skew
// between resident blocks) it records the error and the block goes on.
__device__ __forceinline__ void grid_barrier(unsigned int *bar, int *err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int gen;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(gen) : "l"(bar + 1) : "memory");
        __threadfence();
        const unsigned int arrived = atomicAdd(bar, 1u) + 1u;
        if (arrived == gridDim.x) {
            bar[0] = 0u;
            __threadfence();
            asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(bar + 1), "r"(gen + 1u) : "memory");
        } else {
            uint64_t t0;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
            for (uint32_t i = 0;; ++i) {
                unsigned int g;
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(bar + 1) : "memory");
                if (g != gen) break;
                if ((i & 255u) == 255u) {
                    uint64_t t;
                    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
                    if (t - t0 > 1000000000ull) {
                        atomicExch(err, 1);
                        break;
                    }
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// The CG dots and the direction in one cooperative launch (m % 4 == 0, 16-byte
// aligned arrays): each block sums its part of <Z,G>, <Z,Gp>, <G,Df> exactly as
// mx_dots_kernel does, the grid meets at a barrier, every block then forms the
// three totals from the per-block parts in the same fixed order (so every block
// holds the same beta and restart flag; block 0 writes them to the state), and
// the grid runs the direction pass of mx_direction4_kernel.  This replaces a
// second launch and the last block's serial pass of the dots kernel; G, Gp and
// Df are read twice, the second time mostly from L2.
template <bool PRE, bool ROUND1>
__global__ void __launch_bounds__(NT, 4) mx_dots_direction4_kernel(int m, int64_t mn, const float4 *__restrict__ G,
                                                                 const float4 *__restrict__ Zg, float4 *Gp,
                                                                 float4 *Df, float4 *D, DevState *state, DigitOut dd,
                                                                 double *slope, double *partials,
                                                                 unsigned int *bar, int first) {
    if (*((volatile const int *)&state->done)) return;
    __shared__ double red[(NT / 32) * ND];
    __shared__ float s_beta;
    __shared__ int s_restart, s_bad;
    // read before the barrier: block 0 overwrites it after
    const double gpgp = state->gg_prev;
    const int64_t n4 = mn / 4, stride = (int64_t)gridDim.x * NT;
    {
        float f[ND] = {0.f, 0.f, 0.f};
#pragma unroll 4
        for (int64_t k = (int64_t)blockIdx.x * NT + threadIdx.x; k < n4; k += stride) {
            const float4 g = G[k];
            const float4 z = PRE ? Zg[k] : g;
            f[0] = fmaf(z.x, g.x, fmaf(z.y, g.y, fmaf(z.z, g.z, fmaf(z.w, g.w, f[0]))));
            if (!first) {
                const float4 p = Gp[k], d = Df[k];
                f[1] = fmaf(z.x, p.x, fmaf(z.y, p.y, fmaf(z.z, p.z, fmaf(z.w, p.w, f[1]))));
                f[2] = fmaf(g.x, d.x, fmaf(g.y, d.y, fmaf(g.z, d.z, fmaf(g.w, d.w, f[2]))));
            }
        }
        double v[ND];
        to_f64<ND>(f, v);
        block_sum<ND>(v, red, true);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int q = 0; q < ND; ++q) partials[blockIdx.x * ND + q] = v[q];
        }
    }
    grid_barrier(bar, &state->wait_timeout);
    // the totals, warp q for value q, lanes over the blocks in order (as the
    // last block of a reduction kernel sums them)
    if ((threadIdx.x >> 5) < ND) {
        const int q = threadIdx.x >> 5;
        double s = 0.0;
        unsigned b = threadIdx.x & 31;
        for (; b + 224 < gridDim.x; b += 256) {
            double p[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) p[k] = __ldcg(&partials[(b + 32 * k) * ND + q]);
#pragma unroll
            for (int k = 0; k < 8; ++k) s += p[k];
        }
        for (; b < gridDim.x; b += 32) s += __ldcg(&partials[b * ND + q]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if ((threadIdx.x & 31) == 0) red[q] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double gg = red[0], ggp = red[1], gdot = red[2];
        double beta = 0.0;
        int restart = 1;
        if (!first) {
            beta = (gpgp > 0.0) ? fmax(0.0, (gg - ggp) / gpgp) : 0.0;
            restart = (-gg + beta * gdot >= 0.0) ? 1 : 0;
            if (restart) beta = 0.0;
        }
        const bool bad = !isfinite(gg) || !isfinite(beta);
        s_beta = (float)beta;
        s_restart = restart;
        s_bad = bad ? 1 : 0;
        if (blockIdx.x == 0) {
            if (bad) {
                state->status = OMM_ERR_NONFINITE;
                state->done = 1;
            } else {
                state->gg = gg;
                state->ggp = ggp;
                state->gd = gdot;
                state->gg_prev = gg;
                state->beta = beta;
                state->beta_f = (float)beta;
                state->restart = restart;
                state->gD = restart ? -gg : -gg + beta * gdot;   // <G, D_new>
            }
        }
    }
    __syncthreads();
    if (s_bad) return;
    // the direction pass (mx_direction4_kernel)
    const float beta = s_beta;
    const bool restart = s_restart != 0;
    float gd = 0.f;
    for (int64_t k = (int64_t)blockIdx.x * NT + threadIdx.x; k < n4; k += stride) {
        const float4 g = G[k];
        const float4 z = PRE ? Zg[k] : g;
        float4 d = Df[k];
        if (restart) {
            d = make_float4(-z.x, -z.y, -z.z, -z.w);
        } else {
            d.x = fmaf(beta, d.x, -z.x);
            d.y = fmaf(beta, d.y, -z.y);
            d.z = fmaf(beta, d.z, -z.z);
            d.w = fmaf(beta, d.w, -z.w);
        }
        Df[k] = d;
        Gp[k] = g;
        const int64_t o = 4 * k, j = o / m, i = o - j * m;
        if (ROUND1) {
            const __nv_bfloat162 b01 = __floats2bfloat162_rn(d.x, d.y), b23 = __floats2bfloat162_rn(d.z, d.w);
            const float2 f01 = __bfloat1622float2(b01), f23 = __bfloat1622float2(b23);
            const float4 r = make_float4(f01.x, f01.y, f23.x, f23.y);
            gd = fmaf(g.x, r.x, fmaf(g.y, r.y, fmaf(g.z, r.z, fmaf(g.w, r.w, gd))));
            D[k] = r;
            if (dd.ptr != nullptr) {
                __nv_bfloat16 *p = (__nv_bfloat16 *)dd.ptr;
                uint2 u;
                u.x = *reinterpret_cast<const uint32_t *>(&b01);
                u.y = *reinterpret_cast<const uint32_t *>(&b23);
                *reinterpret_cast<uint2 *>(p + j * dd.ld + i) = u;
                for (int t = 1; t < dd.nd; ++t)
                    *reinterpret_cast<uint2 *>(p + t * dd.plane + j * dd.ld + i) = make_uint2(0u, 0u);
            }
        } else if (dd.ptr != nullptr) {
            put3f4(dd, j * dd.ld + i, d);
        }
    }
    direction_slope<ROUND1>(gd, slope);
}

// Digits of four consecutive rows of one column per thread (m % 4 == 0)
__global__ void __launch_bounds__(NT) mx_digits4_kernel(int m, int64_t mn, const float4 *__restrict__ A,
                                                         const DevState *state, DigitOut dd) {
    if (*((volatile const int *)&state->done)) return;
    for (int64_t k = (int64_t)blockIdx.x * NT + threadIdx.x; k < mn / 4; k += (int64_t)gridDim.x * NT) {
        const int64_t o = 4 * k, j = o / m, i = o - j * m;
        put3f4(dd, j * dd.ld + i, A[k]);
    }
}

__global__ void mx_digits_kernel(int m, int n, const float *__restrict__ A, const DevState *state, DigitOut dd) {
    if (*((volatile const int *)&state->done)) return;
    for (int j = blockIdx.y; j < n; j += gridDim.y)
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
            put3f(dd, (int64_t)j * dd.ld + i, A[(int64_t)j * m + i]);
}

__global__ void mx_round_kernel(int64_t count, const double *__restrict__ src, float *dst, const DevState *state) {
    if (state != nullptr && *((volatile const int *)&state->done)) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = sw_d2f(src[i]);
}

int tiles_blocks(int64_t a, int64_t b) {
    int64_t nb = ceil_div(a, TILE) * ceil_div(b, TILE);
    if (nb > kRedBlocksMax) nb = kRedBlocksMax;
    return (int)(nb < 1 ? 1 : nb);
}

}  // namespace

int mx_coeffs_linemin(int n, const double *h0, const double *s0, int64_t ldh, const float *Z, int64_t ldz,
                      double *scratch, unsigned int *counter, DevState *state, const double *slope, int nslope,
                      cudaStream_t st) {
    if (nslope < 0 || nslope > kRedBlocksMax || (nslope > 0 && slope == nullptr)) return OMM_ERR_ARG;
    mx_coeffs_kernel<<<tiles_blocks(n, n), NT, 0, st>>>(n, h0, s0, ldh, Z, ldz, scratch, counter, state, slope,
                                                        nslope);
    count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

int mx_update(int64_t m, int64_t n, double *W, const float *D, double *HW, const float *HD, double *SW,
              const float *SD, const DevState *state, DigitOut wd, DigitOut swhw, cudaStream_t st) {
    const bool aligned = ((((uintptr_t)W) | ((uintptr_t)HW) | ((uintptr_t)SW)) & 15u) == 0 &&
                         ((((uintptr_t)D) | ((uintptr_t)HD) | ((uintptr_t)SD)) & 7u) == 0 &&
                         (wd.ptr == nullptr || ((((uintptr_t)wd.ptr) & 3u) == 0 && wd.ld % 2 == 0 && wd.plane % 2 == 0));
    if (m % 2 == 0 && aligned) {
        int64_t nb = ceil_div(m, TI2) * ceil_div(n, TILE);
        if (nb > 152 * 8) nb = 152 * 8;
        mx_update2_kernel<<<(unsigned)nb, NT, 0, st>>>(
            (int)m, (int)n, reinterpret_cast<double2 *>(W), reinterpret_cast<const float2 *>(D),
            reinterpret_cast<double2 *>(HW), reinterpret_cast<const float2 *>(HD), reinterpret_cast<double2 *>(SW),
            reinterpret_cast<const float2 *>(SD), state, wd, swhw);
        count_launch();
        OMM_CUDA_TRY(cudaGetLastError());
        return OMM_OK;
    }
    int64_t nb = ceil_div(m, TILE) * ceil_div(n, TILE);
    if (nb > 152 * 8) nb = 152 * 8;
    mx_update_kernel<<<(unsigned)nb, NT, 0, st>>>((int)m, (int)n, W, D, HW, HD, SW, SD, state, wd, swhw);
    count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

int mx_nn_update(int n, double *h0, double *s0, int64_t ldh, const float *Z, int64_t ldz, double *scratch,
                 unsigned int *counter, DevState *state, DigitOut hsw, cudaStream_t st) {
    mx_nn_update_kernel<<<tiles_blocks(n, n), NT, 0, st>>>(n, h0, s0, ldh, Z, ldz, scratch, counter, state, hsw);
    count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

int mx_dots_beta(int64_t mn, const float *G, const float *Zg, const float *Gp, const float *D, double *scratch,
                 unsigned int *counter, DevState *state, int first, cudaStream_t st) {
    if (((((uintptr_t)G) | ((uintptr_t)Gp) | ((uintptr_t)D) | ((uintptr_t)Zg)) & 15u) != 0) return OMM_ERR_ARG;
    // up to kRedBlocksMax blocks (the partial-sum slots): enough warps per SM to
    // keep the three streams' loads in flight
    int64_t nb = ceil_div(mn, (int64_t)NT * 8);
    if (nb > kRedBlocksMax) nb = kRedBlocksMax;
    const unsigned grid = (unsigned)(nb < 1 ? 1 : nb);
    if (Zg != nullptr)
        mx_dots_kernel<true><<<grid, NT, 0, st>>>(mn, G, Zg, Gp, D, scratch, counter, state, first);
    else
        mx_dots_kernel<false><<<grid, NT, 0, st>>>(mn, G, G, Gp, D, scratch, counter, state, first);
    count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

int mx_direction(int64_t m, int64_t n, const float *G, const float *Zg, float *Gp, float *Df, float *D,
                 DevState *state, DigitOut dd, bool round1, double *slope, int *slope_blocks, cudaStream_t st) {
    if (round1 && (slope == nullptr || D == nullptr || D == Df)) return OMM_ERR_ARG;
    if (!round1) D = Df;
    const int64_t mn = m * n;
    const bool aligned =
        ((((uintptr_t)G) | ((uintptr_t)Gp) | ((uintptr_t)Df) | ((uintptr_t)D) | ((uintptr_t)Zg)) & 15u) == 0 &&
        (dd.ptr == nullptr || ((((uintptr_t)dd.ptr) & 7u) == 0 && dd.ld % 4 == 0 && dd.plane % 4 == 0));
    // the rounding form leaves one slope partial per block: at most kRedBlocksMax
    const int64_t cap = round1 ? kRedBlocksMax : 152 * 8;
    const bool vec = m % 4 == 0 && aligned;
    int64_t nb = vec ? ceil_div(mn / 4, (int64_t)NT * 4) : ceil_div(mn, (int64_t)NT * 4);
    if (nb > cap) nb = cap;
    const unsigned grid = (unsigned)(nb < 1 ? 1 : nb);
    if (slope_blocks != nullptr) *slope_blocks = round1 ? (int)grid : 0;
    if (vec) {
        const float4 *G4 = reinterpret_cast<const float4 *>(G);
        const float4 *Z4 = Zg != nullptr ? reinterpret_cast<const float4 *>(Zg) : G4;
        float4 *Gp4 = reinterpret_cast<float4 *>(Gp), *Df4 = reinterpret_cast<float4 *>(Df),
               *D4 = reinterpret_cast<float4 *>(D);
        auto kern = Zg != nullptr ? (round1 ? mx_direction4_kernel<true, true> : mx_direction4_kernel<true, false>)
                                  : (round1 ? mx_direction4_kernel<false, true> : mx_direction4_kernel<false, false>);
        kern<<<grid, NT, 0, st>>>((int)m, mn, G4, Z4, Gp4, Df4, D4, state, dd, slope);
        count_launch();
        OMM_CUDA_TRY(cudaGetLastError());
        return OMM_OK;
    }
    if (round1)
        mx_direction_kernel<true><<<grid, NT, 0, st>>>((int)m, mn, G, Zg, Gp, Df, D, state, dd, slope);
    else
        mx_direction_kernel<false><<<grid, NT, 0, st>>>((int)m, mn, G, Zg, Gp, Df, D, state, dd, slope);
    count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

int mx_dots_direction(int64_t m, int64_t n, const float *G, const float *Zg, float *Gp, float *Df, float *D,
                      DevState *state, DigitOut dd, bool round1, double *slope, int *slope_blocks, double *scratch,
                      unsigned int *bar, int first, cudaStream_t st) {
    if (round1 && (slope == nullptr || D == nullptr || D == Df)) return OMM_ERR_ARG;
    if (!round1) D = Df;
    const int64_t mn = m * n;
    const bool aligned =
        ((((uintptr_t)G) | ((uintptr_t)Gp) | ((uintptr_t)Df) | ((uintptr_t)D) | ((uintptr_t)Zg)) & 15u) == 0 &&
        (dd.ptr == nullptr || ((((uintptr_t)dd.ptr) & 7u) == 0 && dd.ld % 4 == 0 && dd.plane % 4 == 0));
    if (m % 4 != 0 || !aligned || bar == nullptr || (((uintptr_t)bar) & 7u) != 0) return OMM_ERR_UNSUPPORTED;
    const int variant = (Zg != nullptr ? 2 : 0) + (round1 ? 1 : 0);
    auto kern = Zg != nullptr
                    ? (round1 ? mx_dots_direction4_kernel<true, true> : mx_dots_direction4_kernel<true, false>)
                    : (round1 ? mx_dots_direction4_kernel<false, true> : mx_dots_direction4_kernel<false, false>);
    // every block must be resident at once: the grid is capped by the occupancy
    static int coop = -1, sms = 0;
    if (coop < 0) {
        int dev = 0, c = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&c, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return OMM_ERR_CUDA;
        coop = c;
    }
    if (!coop) return OMM_ERR_UNSUPPORTED;
    static int occupancy[4] = {0, 0, 0, 0};
    if (occupancy[variant] == 0) OMM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occupancy[variant], kern, NT, 0));
    const int per_sm = occupancy[variant];
    int64_t nb = ceil_div(mn, (int64_t)NT * 8);
    if (nb > kRedBlocksMax) nb = kRedBlocksMax;
    if (nb > (int64_t)per_sm * sms) nb = (int64_t)per_sm * sms;
    if (nb < 1) return OMM_ERR_UNSUPPORTED;
    if (slope_blocks != nullptr) *slope_blocks = round1 ? (int)nb : 0;
    const float4 *G4 = reinterpret_cast<const float4 *>(G);
    const float4 *Z4 = Zg != nullptr ? reinterpret_cast<const float4 *>(Zg) : G4;
    float4 *Gp4 = reinterpret_cast<float4 *>(Gp), *Df4 = reinterpret_cast<float4 *>(Df),
           *D4 = reinterpret_cast<float4 *>(D);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nb, 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    OMM_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, (int)m, mn, G4, Z4, Gp4, Df4, D4, state, dd, slope, scratch, bar,
                                    first));
    count_launch();
    return OMM_OK;
}

int mx_digits(int64_t m, int64_t n, const float *A, const DevState *state, DigitOut dd, cudaStream_t st) {
    const bool aligned = (((uintptr_t)A) & 15u) == 0 && (((uintptr_t)dd.ptr) & 7u) == 0 && dd.ld % 4 == 0 &&
                         dd.plane % 4 == 0;
    if (m % 4 == 0 && aligned) {
        int64_t nb = ceil_div(m * n / 4, (int64_t)NT * 4);
        if (nb > 152 * 8) nb = 152 * 8;
        mx_digits4_kernel<<<(unsigned)(nb < 1 ? 1 : nb), NT, 0, st>>>((int)m, m * n,
                                                                       reinterpret_cast<const float4 *>(A), state, dd);
    } else {
        dim3 grid((unsigned)ceil_div(m, NT), (unsigned)(n < 1024 ? n : 1024));
        mx_digits_kernel<<<grid, NT, 0, st>>>((int)m, (int)n, A, state, dd);
    }
    count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

int mx_round(int64_t count, const double *src, float *dst, const DevState *state, cudaStream_t st) {
    int64_t nb = ceil_div(count, 256 * 4);
    if (nb > 152 * 8) nb = 152 * 8;
    mx_round_kernel<<<(unsigned)(nb < 1 ? 1 : nb), 256, 0, st>>>(count, src, dst, state);
    count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

}  // namespace omm
