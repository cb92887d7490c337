// Exact-digit BF16 tensor-core GEMM: near-FP64 products on tcgen05 (sm_103a).
//
// Error-free splitting in the manner of Ozaki, Ogita, Oishi & Rump (2012),
// applied to BF16 tensor cores as in Mukunoki et al. (2020): every K-major
// row r of an operand is scaled by 2^-e_r so its entries lie in (-1, 1), then
// cut into s fixed-point digits: the integer F = round(a 2^(6 + 7(s-1))) is
// written in balanced base 128, so a = sum_t d_t 2^-(7t-1) + O(2^-(7s)) with
// each |d_t| <= 64 (exact in BF16).
// A product of two digits is at most 2^12 in magnitude, so a sum of up to
// 4096 of them is an integer below 2^24: the tensor cores accumulate every
// digit pair (t, u) over a K chunk of <= 4096 exactly in FP32.  Pairs with
// t + u <= s + 1 are kept; pairs of one level L = t + u share the weight
// 2^-(7L-2).
//
// One CTA computes a 128 x 128 tile.  Warp 0 streams (A_t, B_u) digit tiles of
// each pair through a 6-stage TMA ring; warp 1 accumulates each (pair, chunk)
// unit in one of two tensor-memory buffers; warps 2..5 read a finished unit,
// convert its exact integers to int32 and add them to the level's integer
// sum (registers), and at the end of each level fold that sum into an FP64
// running sum kept in tensor memory.  The final epilogue scales by
// 2^(e_i + f_j) and writes C = alpha * A B + beta * Cin in FP64.
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>

#include "fp_convert.cuh"
#include "omm_internal.cuh"
#include "tc_exact.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace omm {
namespace tc {
namespace {

using namespace ptx;

constexpr int XBN = 128;
constexpr int XSTAGES = 6;
constexpr int XTILE_B_BYTES = XBN * BK * 2;
constexpr int XSTAGE_BYTES = TILE_A_BYTES + XTILE_B_BYTES;
constexpr int kChunkMax = 4096;     // 4096 * 64 * 64 = 2^24: exact FP32 integer sums
constexpr int kRunCol = 2 * XBN;    // tensor-memory column of the FP64 running sum

__global__ void __launch_bounds__(192, 1)
    tc_exact_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                    const ExactArgs args) {
    if (args.state != nullptr && *((volatile const int *)&args.state->done)) return;
    const int z = blockIdx.z;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[XSTAGES];
    __shared__ __align__(8) uint64_t empty_bar[XSTAGES];
    __shared__ __align__(8) uint64_t tfull_bar[2];
    __shared__ __align__(8) uint64_t tempty_bar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const uint64_t deadline = globaltimer_ns() + kWaitNs;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM;     // N tiles vary fastest: CTAs in flight share A tiles in L2
    const int n0 = blockIdx.x * XBN;
    const int nkb_total = (args.K + BK - 1) / BK;
    const int kb_per_chunk = kChunkMax / BK;
    const int nchunks = (nkb_total + kb_per_chunk - 1) / kb_per_chunk;
    const int nunits = args.npairs * nchunks;

    if (threadIdx.x == 0) {
        for (int s = 0; s < XSTAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull_bar[b], 1);
            mbar_init(&tempty_bar[b], 128);
        }
        abort_flag = 0;
        mbar_fence_init();
    }
    if (warp == 1) tmem_alloc(&tmem_base, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer: every unit's k-blocks, in unit order
        const int a_row = args.a_row0 + z * args.a_row_step + m0;
        const int b_row = args.b_row0 + z * args.b_row_step + n0;
        int it = 0;
        for (int u = 0; u < nunits && !abort_flag; ++u) {
            const int p = u / nchunks, c = u % nchunks;
            const int kb0 = c * kb_per_chunk;
            const int kb1 = min(nkb_total, kb0 + kb_per_chunk);
            for (int kb = kb0; kb < kb1; ++kb, ++it) {
                const int s = it % XSTAGES;
                const uint32_t ph = (uint32_t)((it / XSTAGES) & 1);
                if (!mbar_wait(&empty_bar[s], ph ^ 1u, deadline, &abort_flag, args.err)) break;
                mbar_arrive_expect_tx(&full_bar[s], (uint32_t)XSTAGE_BYTES);
                uint8_t *st = smem + s * XSTAGE_BYTES;
                tma_load_3d(st, &mapA, kb * BK, a_row, args.pa[p], &full_bar[s]);
                tma_load_3d(st + TILE_A_BYTES, &mapB, kb * BK, b_row, args.pb[p], &full_bar[s]);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer: unit u accumulates into buffer u & 1
        constexpr uint32_t idesc = idesc_bf16(BM, XBN);
        int it = 0;
        for (int u = 0; u < nunits; ++u) {
            const int c = u % nchunks;
            const int b = u & 1;
            if (!mbar_wait(&tempty_bar[b], (uint32_t)(((u >> 1) & 1) ^ 1), deadline, &abort_flag, args.err)) break;
            tc_fence_after();
            const uint32_t tacc = tmem + (uint32_t)(b * XBN);
            const int kb0 = c * kb_per_chunk;
            const int kb1 = min(nkb_total, kb0 + kb_per_chunk);
            bool ok = true;
            for (int kb = kb0; kb < kb1; ++kb, ++it) {
                const int s = it % XSTAGES;
                const uint32_t ph = (uint32_t)((it / XSTAGES) & 1);
                if (!mbar_wait(&full_bar[s], ph, deadline, &abort_flag, args.err)) { ok = false; break; }
                tc_fence_after();
                const uint32_t st = smem_u32(smem + s * XSTAGE_BYTES);
                const uint64_t da = sdesc_sw128(st), db = sdesc_sw128(st + TILE_A_BYTES);
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)
                    umma_bf16(tacc, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc,
                              (kb != kb0 || kk != 0) ? 1u : 0u);
                umma_commit(&empty_bar[s]);
            }
            umma_commit(&tfull_bar[b]);
            if (!ok) break;
        }
    } else if (warp >= 2) {
        // ---------------- epilogue
        const int q = warp & 3;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
        const int row = m0 + 32 * q + lane;
        int32_t acc[XBN];
#pragma unroll
        for (int j = 0; j < XBN; ++j) acc[j] = 0;
        // Running sum in tensor memory (two words per value): the integer
        // R = sum_L acc_L 2^(7 (Lr - L)) over the levels folded so far, counted
        // in units of level Lr, updated with integer instructions only:
        // R <- 128 R + acc_L (Lr <- L) while a bound on |R|, the same in every
        // thread, stays below 2^62; past that, Lr stays and a later level adds
        // acc_L 2^-7(L - Lr) rounded to an integer.  With 7 digits and K up to
        // 32768 every level is exact; otherwise the rounding is below 2^-47 of
        // the scaled operands' unit, far inside an FP64 GEMM's error bound.
        // The code stays compact on purpose: an unrolled per-element body
        // with heavy conversions overflows the instruction cache.
        int mode = 0;           // 0 empty, 1 growing, 2 fixed units
        int lvl_r = 0;          // level whose units R counts in
        double bound = 0.0;     // bound on |R|
        bool alive = true;
        for (int u = 0; u < nunits; ++u) {
            const int p = u / nchunks, c = u % nchunks;
            const int b = u & 1;
            bool got = alive && mbar_wait(&tfull_bar[b], (uint32_t)((u >> 1) & 1), deadline, &abort_flag, args.err);
            got = __all_sync(0xffffffffu, got);
            alive = got;
            tc_fence_after();
            if (got) {
                // four 16-column loads in flight per wait
#pragma unroll
                for (int c0 = 0; c0 < XBN; c0 += 64) {
                    uint32_t r0[16], r1[16], r2[16], r3[16];
                    const uint32_t t = lane_base + (uint32_t)(b * XBN + c0);
                    tmem_ld16_async(t, r0);
                    tmem_ld16_async(t + 16, r1);
                    tmem_ld16_async(t + 32, r2);
                    tmem_ld16_async(t + 48, r3);
                    tmem_wait_ld(r0);
                    tmem_pin16(r1);
                    tmem_pin16(r2);
                    tmem_pin16(r3);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        acc[c0 + j] += __float2int_rn(__uint_as_float(r0[j]));
                        acc[c0 + 16 + j] += __float2int_rn(__uint_as_float(r1[j]));
                        acc[c0 + 32 + j] += __float2int_rn(__uint_as_float(r2[j]));
                        acc[c0 + 48 + j] += __float2int_rn(__uint_as_float(r3[j]));
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&tempty_bar[b]);
            const int level = args.pa[p] + args.pb[p] + 2;
            const bool last_of_level =
                c == nchunks - 1 && (p == args.npairs - 1 || args.pa[p + 1] + args.pb[p + 1] + 2 != level);
            if (last_of_level && got) {
                int np = 0;   // pairs on this level
                for (int p2 = 0; p2 < args.npairs; ++p2) np += (args.pa[p2] + args.pb[p2] + 2 == level);
                const double add = (double)np * (double)nchunks * 16777216.0;   // |acc| < np nchunks 2^24
                int next = mode;
                if (mode == 0) next = 1;
                else if (mode == 1 && !(bound * 128.0 + add < 4.6e18)) next = 2;
                const int sh = next == 2 ? 7 * (level - lvl_r) : 0;            // fixed units: right shift
                const int64_t half = sh > 0 ? ((int64_t)1 << (sh - 1)) : 0;
#pragma unroll
                for (int c0 = 0; c0 < XBN; c0 += 32) {
                    uint32_t r[4][16];
                    const uint32_t t = lane_base + (uint32_t)(kRunCol + 2 * c0);
                    if (mode != 0) {
                        tmem_ld16_async(t, r[0]);
                        tmem_ld16_async(t + 16, r[1]);
                        tmem_ld16_async(t + 32, r[2]);
                        tmem_ld16_async(t + 48, r[3]);
                        tmem_wait_ld(r[0]);
                        tmem_pin16(r[1]);
                        tmem_pin16(r[2]);
                        tmem_pin16(r[3]);
                    }
#pragma unroll
                    for (int g = 0; g < 4; ++g)
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int64_t a = (int64_t)acc[c0 + 8 * g + j];
                            const int64_t old = mode == 0 ? 0 : (int64_t)(((uint64_t)r[g][2 * j + 1] << 32) | r[g][2 * j]);
                            const int64_t nv = next == 1 ? old * 128 + a : old + ((a + half) >> sh);
                            r[g][2 * j] = (uint32_t)(uint64_t)nv;
                            r[g][2 * j + 1] = (uint32_t)((uint64_t)nv >> 32);
                        }
                    tmem_st16_async(t, r[0]);
                    tmem_st16_async(t + 16, r[1]);
                    tmem_st16_async(t + 32, r[2]);
                    tmem_st16_async(t + 48, r[3]);
                }
                tmem_wait_st();
#pragma unroll
                for (int j = 0; j < XBN; ++j) acc[j] = 0;
                if (next == 1) {
                    bound = mode == 0 ? add : bound * 128.0 + add;
                    lvl_r = level;
                } else {
                    bound += add / ldexp(1.0, sh) + 1.0;
                }
                mode = next;
            }
        }
        // final: C = alpha 2^(eA + eB) R 2^-(7 Lr - 2) + beta Cin, one integer-op
        // conversion per value (rolled loop: compact code)
        const bool ok = __all_sync(0xffffffffu, alive && mode != 0);
        double *C = args.C != nullptr ? args.C + (int64_t)z * args.c_step : nullptr;
        float *C32 = args.C32 != nullptr ? args.C32 + (int64_t)z * args.c_step : nullptr;
        const double *Cin = args.Cin ? args.Cin + (int64_t)z * args.cin_step : nullptr;
        const int *eA = args.eA + (int64_t)z * args.eA_step;
        const int *eB = args.eB + (int64_t)z * args.eB_step;
        const int e_row = (row < args.M ? eA[row] : 0) - (7 * lvl_r - 2);
#pragma unroll 1
        for (int c0 = 0; c0 < XBN; c0 += 8) {
            uint32_t r[16];
            if (ok) {
                tmem_ld16_async(lane_base + (uint32_t)(kRunCol + 2 * c0), r);
                tmem_wait_ld(r);
            }
            if (row < args.M) {
                // Cin first: C may alias it as far as the compiler knows, so a load
                // after a store would wait for that store
                double cin[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int col = n0 + c0 + j;
                    cin[j] = (Cin != nullptr && col < args.N) ? __ldg(&Cin[row + (int64_t)col * args.ldcin]) : 0.0;
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int col = n0 + c0 + j;
                    if (col >= args.N) break;
                    double out = 0.0;
                    if (ok) {
                        const int64_t R = (int64_t)(((uint64_t)r[2 * j + 1] << 32) | r[2 * j]);
                        const int e = e_row + eB[col];
                        // normal-range results by integer ops; anything else (never for
                        // operands within 2^+-900) through ldexp
                        out = (e > -960 && e < 900) ? sw_i64_scaled(R, e) : ldexp((double)R, e);
                    }
                    if (args.alpha != 1.0) out *= args.alpha;
                    if (Cin != nullptr) out = fma(args.beta, cin[j], out);
                    if (C32 != nullptr) C32[row + (int64_t)col * args.ldc] = sw_d2f(out);
                    else C[row + (int64_t)col * args.ldc] = out;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// ------------------------------------------------------------------ digit packing
// All integer arithmetic: the FP64 unit of GB300 is far too narrow for
// per-element digit splitting.
//
// A row's exponent e makes the scaled row lie in (-1, 1): 2^e > max |a|.
// Magnitudes of non-negative doubles order like their bit patterns, so the
// row maximum is an integer max over the bits with the sign cleared.
__device__ __forceinline__ int exponent_from_maxbits(uint64_t mb) {
    const int be = (int)(mb >> 52);                 // biased exponent of max |a|
    if (be == 0) return 0;                           // zero (or subnormal) row
    int e = be - 1023 + 1;                           // 2^e > max |a| >= 2^(e-1)
    return e < -1000 ? -1000 : (e > 1000 ? 1000 : e);
}

// Digits of a = v 2^-e: F = round(v 2^(B-e)) with B = 6 + 7(s-1), then balanced
// base-128 digits from the bottom: F = sum_t d_t 128^(s-t), d_t in [-64, 64].
// d_t then carries the weight 2^-(7t-1) of the fixed-point splitting.
__device__ __forceinline__ void put_digits(double v, int e, int s, __nv_bfloat16 *dst, int64_t o, int64_t plane) {
    const uint64_t b = (uint64_t)__double_as_longlong(v);
    const int be = (int)((b >> 52) & 0x7FF);
    int64_t F = 0;
    if (be != 0) {
        const uint64_t mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);   // v = mant 2^(be - 1075)
        const int shift = be - 1075 + (6 + 7 * (s - 1)) - e;
        if (shift >= 0) {
            F = (int64_t)(mant << shift);             // |F| < 2^(6 + 7(s-1)) <= 2^55
        } else if (shift > -64) {
            F = (int64_t)((mant + (1ull << (-shift - 1))) >> (-shift));
        }
        if (b >> 63) F = -F;
    }
    for (int t = s - 1; t >= 1; --t) {
        const int64_t r = ((F + 64) & 127) - 64;      // in [-64, 63]
        dst[t * plane + o] = __float2bfloat16_rn((float)(int)r);   // small integers: exact, 32-bit convert
        F = (F - r) >> 7;
    }
    dst[o] = __float2bfloat16_rn((float)(int)F);      // |F| <= 64
}

// K along the source's rows: operand row r is source column r (warp per column).
__global__ void exp_cm_kernel(int64_t K, int64_t R, const double *__restrict__ X, int64_t ld, int *e,
                              const DevState *state) {
    if (state != nullptr && *((volatile const int *)&state->done)) return;
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t *Xb = (const uint64_t *)X;
    for (int64_t r = w; r < R; r += nw) {
        // four independent maxima: four loads of each lane in flight (with one warp
        // per column the grid holds few warps, so each must keep several loads going)
        unsigned long long m4[4] = {0, 0, 0, 0};
        int64_t k = lane;
        for (; k + 96 < K; k += 128)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const unsigned long long a = Xb[k + 32 * u + r * ld] & 0x7FFFFFFFFFFFFFFFull;
                m4[u] = a > m4[u] ? a : m4[u];
            }
        for (; k < K; k += 32) {
            const unsigned long long a = Xb[k + r * ld] & 0x7FFFFFFFFFFFFFFFull;
            m4[0] = a > m4[0] ? a : m4[0];
        }
        unsigned long long mx = m4[0] > m4[1] ? m4[0] : m4[1];
        const unsigned long long m23 = m4[2] > m4[3] ? m4[2] : m4[3];
        mx = m23 > mx ? m23 : mx;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, mx, off);
            mx = o > mx ? o : mx;
        }
        if (lane == 0) e[r] = exponent_from_maxbits(mx);
    }
}

// Row exponents when K runs along the source's columns, split over K: each warp
// takes 32 rows (one per lane, coalesced) and a slice of the columns, and folds
// the biased exponent of its largest magnitude into be[r] with an integer
// atomic max (be zeroed first); exp_finish_kernel turns be into exponents.
__global__ void exp_t_split_kernel(int64_t R, int64_t K, const double *__restrict__ X, int64_t ld, int *be,
                                   int64_t kslice, const DevState *state) {
    if (state != nullptr && *((volatile const int *)&state->done)) return;
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
    const int64_t r = (int64_t)blockIdx.x * 32 + lx;
    const int64_t k0 = (int64_t)blockIdx.y * kslice, k1 = k0 + kslice < K ? k0 + kslice : K;
    const uint64_t *Xb = (const uint64_t *)X;
    unsigned long long mx = 0;
    if (r < R)
        for (int64_t k = k0 + ly; k < k1; k += 8) {
            const unsigned long long a = Xb[r + k * ld] & 0x7FFFFFFFFFFFFFFFull;
            mx = a > mx ? a : mx;
        }
    if (r < R && mx != 0) atomicMax(&be[r], (int)(mx >> 52));
}

__global__ void exp_finish_kernel(int64_t R, int *e, const DevState *state) {
    if (state != nullptr && *((volatile const int *)&state->done)) return;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x)
        e[r] = exponent_from_maxbits((uint64_t)e[r] << 52);
}

__global__ void digits_cm_kernel(int64_t K, int64_t R, const double *__restrict__ X, int64_t ld,
                                 const int *__restrict__ e, __nv_bfloat16 *dst, int64_t ldk, int64_t plane,
                                 int s, const DevState *state) {
    if (state != nullptr && *((volatile const int *)&state->done)) return;
    for (int64_t r = blockIdx.y; r < R; r += gridDim.y) {
        const int er = e[r];
        for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < K; k += (int64_t)gridDim.x * blockDim.x)
            put_digits(X[k + r * ld], er, s, dst, r * ldk + k, plane);
    }
}

__global__ void digits_t_kernel(int64_t R, int64_t K, const double *__restrict__ X, int64_t ld,
                                const int *__restrict__ e, __nv_bfloat16 *dst, int64_t ldk, int64_t plane, int s,
                                const DevState *state) {
    if (state != nullptr && *((volatile const int *)&state->done)) return;
    __shared__ double tile[32][33];
    const int64_t tr = (int64_t)blockIdx.x * 32, tk = (int64_t)blockIdx.y * 32;
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
    for (int i = ly; i < 32; i += 8) {
        const int64_t r = tr + lx, k = tk + i;
        tile[i][lx] = (r < R && k < K) ? X[r + k * ld] : 0.0;
    }
    __syncthreads();
    for (int i = ly; i < 32; i += 8) {
        const int64_t r = tr + i, k = tk + lx;
        if (r < R && k < K) put_digits(tile[lx][i], e[r], s, dst, r * ldk + k, plane);
    }
}

int grid_for(int64_t work, int per_block) {
    int64_t nb = ceil_div(work, per_block);
    if (nb > 152 * 16) nb = 152 * 16;
    return (int)(nb < 1 ? 1 : nb);
}

}  // namespace

void exact_pairs(int s, ExactArgs &a) {
    int k = 0;
    for (int lvl = 2; lvl <= s + 1; ++lvl)
        for (int t = 1; t <= s; ++t) {
            const int u = lvl - t;
            if (u < 1 || u > s) continue;
            a.pa[k] = (uint8_t)(t - 1);
            a.pb[k] = (uint8_t)(u - 1);
            ++k;
        }
    a.npairs = k;
}

int exact_pack(bool k_along_rows, int64_t rows, int64_t cols, const double *X, int64_t ld, int *e,
               __nv_bfloat16 *dst, int64_t ldk, int64_t plane, int s, const DevState *state, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return OMM_OK;
    if (s < 1 || s > kExactMaxDigits) return OMM_ERR_ARG;
    if (k_along_rows) {   // K = rows, operand rows = cols
        exp_cm_kernel<<<grid_for(cols * 32, 256), 256, 0, st>>>(rows, cols, X, ld, e, state);
        count_launch();
        OMM_CUDA_TRY(cudaGetLastError());
        dim3 grid((unsigned)ceil_div(rows, 256 * 2), (unsigned)(cols < 8192 ? cols : 8192));
        digits_cm_kernel<<<grid, 256, 0, st>>>(rows, cols, X, ld, e, dst, ldk, plane, s, state);
        count_launch();
        OMM_CUDA_TRY(cudaGetLastError());
    } else {              // K = cols, operand rows = rows
        // biased exponents by an atomic max over K slices of 256 columns, then exponents
        OMM_CUDA_TRY(cudaMemsetAsync(e, 0, (size_t)rows * sizeof(int), st));
        const int64_t kslice = 256;
        dim3 eg((unsigned)ceil_div(rows, 32), (unsigned)ceil_div(cols, kslice));
        exp_t_split_kernel<<<eg, 256, 0, st>>>(rows, cols, X, ld, e, kslice, state);
        count_launch();
        OMM_CUDA_TRY(cudaGetLastError());
        exp_finish_kernel<<<grid_for(rows, 256), 256, 0, st>>>(rows, e, state);
        count_launch();
        OMM_CUDA_TRY(cudaGetLastError());
        dim3 grid((unsigned)ceil_div(rows, 32), (unsigned)ceil_div(cols, 32));
        digits_t_kernel<<<grid, 256, 0, st>>>(rows, cols, X, ld, e, dst, ldk, plane, s, state);
        count_launch();
        OMM_CUDA_TRY(cudaGetLastError());
    }
    return OMM_OK;
}

int exact_gemm(const CUtensorMap &mapA, const CUtensorMap &mapB, const ExactArgs &a, int nbatch, cudaStream_t st) {
    if (a.M <= 0 || a.N <= 0 || a.K <= 0 || a.npairs < 1 || a.npairs > kExactMaxPairs || nbatch < 1)
        return OMM_ERR_ARG;
    const int smem = XSTAGES * XSTAGE_BYTES + 1024;
    static int attr_bytes = 0;
    if (smem > attr_bytes) {
        OMM_CUDA_TRY(cudaFuncSetAttribute(tc_exact_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr_bytes = smem;
    }
    dim3 grid((unsigned)ceil_div(a.N, XBN), (unsigned)ceil_div(a.M, BM), (unsigned)nbatch);
    tc_exact_kernel<<<grid, 192, smem, st>>>(mapA, mapB, a);
    count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

}  // namespace tc
}  // namespace omm

// ---------------------------------------------------------------- op-level entry
extern "C" int64_t omm_op_exact_gemm_workspace_bytes(int64_t M, int64_t N, int64_t K, int32_t ndigits) {
    if (M < 0 || N < 0 || K < 0 || ndigits < 1 || ndigits > omm::tc::kExactMaxDigits) return -1;
    const int64_t ldk = (K + 7) / 8 * 8;
    return (int64_t)ndigits * (M + N) * ldk * 2 + (M + N) * 4 + 2048;
}

extern "C" int omm_op_exact_gemm(int32_t transA, int32_t transB, int64_t M, int64_t N, int64_t K,
                                 int32_t ndigits, double alpha, const double *A, int64_t lda,
                                 const double *B, int64_t ldb, double beta, const double *Cin,
                                 int64_t ldcin, double *C, int64_t ldc, void *workspace,
                                 int64_t workspace_bytes, void *stream) {
    using namespace omm;
    if (M <= 0 || N <= 0 || K <= 0 || ndigits < 1 || ndigits > tc::kExactMaxDigits) return OMM_ERR_ARG;
    if (M > (1 << 30) || N > (1 << 30) || K > (1 << 30)) return OMM_ERR_ARG;
    if (A == nullptr || B == nullptr || C == nullptr || workspace == nullptr) return OMM_ERR_ARG;
    if (lda < (transA ? K : M) || ldb < (transB ? N : K) || ldc < M) return OMM_ERR_ARG;
    if (beta != 0.0 && (Cin == nullptr || ldcin < M)) return OMM_ERR_ARG;
    if (workspace_bytes < omm_op_exact_gemm_workspace_bytes(M, N, K, ndigits)) return OMM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t ldk = (K + 7) / 8 * 8;
    uintptr_t base = ((uintptr_t)workspace + 255) & ~(uintptr_t)255;
    __nv_bfloat16 *Ad = (__nv_bfloat16 *)base;
    __nv_bfloat16 *Bd = Ad + (int64_t)ndigits * M * ldk;
    int *eA = (int *)(Bd + (int64_t)ndigits * N * ldk);
    int *eB = eA + M;
    int rc;
    // op(A) M x K: rows of op(A) are K-major operand rows
    if ((rc = tc::exact_pack(transA != 0, transA ? K : M, transA ? M : K, A, lda, eA, Ad, ldk, M * ldk, ndigits,
                             nullptr, st)))
        return rc;
    // op(B) K x N: columns of op(B) are K-major operand rows
    if ((rc = tc::exact_pack(transB == 0, transB ? N : K, transB ? K : N, B, ldb, eB, Bd, ldk, N * ldk, ndigits,
                             nullptr, st)))
        return rc;
    CUtensorMap ma, mb;
    if ((rc = tc::make_digit_map(&ma, Ad, K, M, ldk, M * ldk, ndigits, 128))) return rc;
    if ((rc = tc::make_digit_map(&mb, Bd, K, N, ldk, N * ldk, ndigits, 128))) return rc;
    tc::ExactArgs a{};
    tc::exact_pairs(ndigits, a);
    a.M = (int)M;
    a.N = (int)N;
    a.K = (int)K;
    a.alpha = alpha;
    a.beta = beta;
    a.Cin = beta != 0.0 ? Cin : nullptr;
    a.ldcin = ldcin;
    a.C = C;
    a.ldc = ldc;
    a.eA = eA;
    a.eB = eB;
    return tc::exact_gemm(ma, mb, a, 1, st);
}
