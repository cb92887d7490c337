// Split-BF16 tensor-core GEMM on tcgen05 (sm_103a), with FP64 epilogues.
//
// An FP64 operand x is carried as up to three BF16 "digits"
//     d1 = bf16(x),  d2 = bf16(x - d1),  d3 = bf16(x - d1 - d2),
// (24 significant bits in all; Markidis et al. 2018, Ootomo & Yokota 2022
// split a wide operand into narrow tensor-core operands the same way).
// Each BF16 x BF16 product is exact in the FP32 accumulator, so
//     C ~= sum over chosen digit pairs (p, q) of A_p B_q
// with FP32 accumulation in tensor memory.  The pairs with p + q <= 4
// ((1,1),(1,2),(2,1),(1,3),(2,2),(3,1)) keep FP32-level operands.  The tensor
// cores' FP32 accumulation loses accuracy with the number of accumulation
// steps, so the K range is cut into up to 512/BN contiguous pieces, each
// accumulated in its own tensor-memory columns, and the epilogue adds the
// pieces in FP64.
//
// Operands are K-major BF16 digit planes: A as [plane][M rows][lda], B as
// [plane][N rows][ldb], K contiguous (ld a multiple of 8 elements).  One CTA
// computes a 128 x BN tile: warp 0 issues TMA loads of every needed digit
// tile of a 64-wide K block into one pipeline stage (128-byte swizzle), warp 1
// issues tcgen05.mma for every digit pair on that stage, and warps 2..5 read
// the FP32 accumulator from tensor memory and write C = alpha acc + beta Cin
// in FP64 (column-major), optionally with the BF16 digits of C as well.
// Every mbarrier wait is bounded; on timeout the kernel records an error and
// unwinds (tensor memory is always released).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <string.h>

#include "fp_convert.cuh"
#include "omm_internal.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace omm {
namespace tc {
namespace {

using namespace ptx;

__device__ __forceinline__ void split3(double v, __nv_bfloat16 &d1, __nv_bfloat16 &d2, __nv_bfloat16 &d3) {
    d1 = __double2bfloat16(v);
    const double r1 = v - (double)__bfloat162float(d1);
    d2 = __double2bfloat16(r1);
    const double r2 = r1 - (double)__bfloat162float(d2);
    d3 = __double2bfloat16(r2);
}

// The same three digits taken from the double's float rounding: the FP64 -> FP32
// step on the integer pipe (sw_d2f), the splits in FP32.  They keep the same
// ~24 significant bits (d1 + d2 + d3 = RN24(v) up to the last bit of d3)
// without FP64 arithmetic or conversions, which are slow on this part; used by
// the packing kernels, which touch every element of H' and S.
__device__ __forceinline__ void split3_i(double v, __nv_bfloat16 &d1, __nv_bfloat16 &d2, __nv_bfloat16 &d3) {
    const float f = sw_d2f(v);
    d1 = __float2bfloat16_rn(f);
    const float r1 = f - __bfloat162float(d1);
    d2 = __float2bfloat16_rn(r1);
    d3 = __float2bfloat16_rn(r1 - __bfloat162float(d2));
}

// ------------------------------------------------------------------ epilogue
// One epilogue warp: TMEM lanes 32q..32q+31 (rows `row` = m0 + 32q + lane of the
// tile) x the tile columns [c_lo, c_hi) from n0 -> C = alpha acc + beta Cin (FP32
// or FP64, column-major), optionally with the result's BF16 digits.  nacc
// accumulators (K ranges x pair classes) are summed; have_acc false writes beta
// Cin only.  This is the general form; tc_epilogue_part takes the specialised one
// below where it applies.
template <int BN>
__device__ __forceinline__ void tc_epilogue(const TcArgs &args, uint32_t tmem, int q, int row, int n0, int z,
                                            int nacc, bool have_acc, int c_lo, int c_hi) {
    double *C = args.C != nullptr ? args.C + (int64_t)z * args.c_step : nullptr;
    const double *Cin = args.Cin ? args.Cin + (int64_t)z * args.cin_step : nullptr;
    __nv_bfloat16 *Dd = args.Dout ? args.Dout + (int64_t)z * args.dout_step : nullptr;
    if (args.C32 != nullptr) {
        // FP32 epilogue: no FP64 arithmetic except reading an FP64 Cin
        float *C32 = args.C32 + (int64_t)z * args.c_step;
        const float alpha = (float)args.alpha, beta = (float)args.beta;
        // Cin is fetched one 16-column chunk ahead as raw FP64 and converted
        // only when used: the compiler cannot rule out that C32 aliases Cin,
        // so a load placed after a store, or tied to a branchy conversion,
        // would wait out one DRAM round trip per output
        const bool rd = Cin != nullptr && row < args.M;
        auto load_cin = [&](int c0, double (&dst)[16]) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int col = n0 + c0 + i;
                dst[i] = (rd && col < args.N) ? __ldg(&Cin[row + (int64_t)col * args.ldcin]) : 0.0;
            }
        };
        double cin[16], cin_next[16];
        load_cin(c_lo, cin);
        for (int c0 = c_lo; c0 < c_hi; c0 += 16) {
            if (c0 + 16 < c_hi) load_cin(c0 + 16, cin_next);
            float v[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = 0.f;
            if (have_acc) {
                for (int ac = 0; ac < nacc; ++ac) {
                    float f[16];
                    tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(ac * BN + c0), f);
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] += f[i];
                }
            }
            if (row < args.M) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int col = n0 + c0 + i;
                    if (col >= args.N) break;
                    float out = alpha * v[i];
                    if (Cin != nullptr) out = fmaf(beta, sw_d2f(cin[i]), out);
                    C32[row + (int64_t)col * args.ldc] = out;
                    if (Dd != nullptr) {
                        const int64_t o = row + (int64_t)col * args.ldd;
                        const __nv_bfloat16 d1 = __float2bfloat16_rn(out);
                        const float r1 = out - __bfloat162float(d1);
                        const __nv_bfloat16 d2 = __float2bfloat16_rn(r1);
                        Dd[o] = d1;
                        if (args.ndig > 1) Dd[args.dplane + o] = d2;
                        if (args.ndig > 2) Dd[2 * args.dplane + o] = __float2bfloat16_rn(r1 - __bfloat162float(d2));
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) cin[i] = cin_next[i];
        }
    } else {
        // Cin one chunk ahead of the stores, as in the FP32 epilogue
        const bool rd = Cin != nullptr && row < args.M;
        auto load_cin = [&](int c0, double (&dst)[16]) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int col = n0 + c0 + i;
                dst[i] = (rd && col < args.N) ? __ldg(&Cin[row + (int64_t)col * args.ldcin]) : 0.0;
            }
        };
        double cin[16], cin_next[16];
        load_cin(c_lo, cin);
        for (int c0 = c_lo; c0 < c_hi; c0 += 16) {
            if (c0 + 16 < c_hi) load_cin(c0 + 16, cin_next);
            double v[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = 0.0;
            if (have_acc) {
                for (int ac = 0; ac < nacc; ++ac) {
                    float f[16];
                    tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(ac * BN + c0), f);
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] += (double)f[i];
                }
            }
            if (row < args.M) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int col = n0 + c0 + i;
                    if (col >= args.N) break;
                    double out = args.alpha * v[i];
                    if (Cin != nullptr) out = fma(args.beta, cin[i], out);
                    C[row + (int64_t)col * args.ldc] = out;
                    if (Dd != nullptr) {
                        __nv_bfloat16 d1, d2, d3;
                        split3(out, d1, d2, d3);
                        const int64_t o = row + (int64_t)col * args.ldd;
                        Dd[o] = d1;
                        if (args.ndig > 1) Dd[args.dplane + o] = d2;
                        if (args.ndig > 2) Dd[2 * args.dplane + o] = d3;
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) cin[i] = cin_next[i];
        }
    }
}

// The FP32 epilogue specialised at compile time on the launch's options: CIN (an
// FP64 Cin is read) and NDIG (BF16 digit planes written).  Same arithmetic and
// rounding as the FP32 branch of tc_epilogue, element for element (the sum of
// the accumulators starts from +0 there too), but every option test and every
// 64-bit index product leaves the per-element loop: the outputs advance by
// pointer steps, and only a chunk that crosses column N tests its columns.  The
// general form spent about 60 instructions per element on one warp per
// scheduler, which made the epilogue of a 128 x 256 tile longer than half of
// its MMAs.  Up to two accumulators (nacc <= 2).
template <int BN, bool CIN, int NDIG>
__device__ __forceinline__ void tc_epilogue_fast(const TcArgs &args, uint32_t lane_base, int row, int n0, int z,
                                                 int nacc, bool have_acc, int c_lo, int c_hi) {
    const bool row_ok = row < args.M;
    const int nlim = args.N - n0;   // tile columns inside N
    const float alpha = (float)args.alpha, beta = (float)args.beta;
    const int64_t ldc = args.ldc, ldd = NDIG > 0 ? args.ldd : 0, ldi = CIN ? args.ldcin : 0;
    const int64_t dpl = NDIG > 1 ? args.dplane : 0;
    float *pc = args.C32 + (int64_t)z * args.c_step + row + (int64_t)(n0 + c_lo) * ldc;
    __nv_bfloat16 *pd =
        NDIG > 0 ? args.Dout + (int64_t)z * args.dout_step + row + (int64_t)(n0 + c_lo) * ldd : nullptr;
    const double *pi = CIN ? args.Cin + (int64_t)z * args.cin_step + row + (int64_t)(n0 + c_lo) * ldi : nullptr;
    double cin[16], cin_next[16];
    // Cin of the 16 columns from tile column c0 (p points at column c0), zero past N
    auto load_cin = [&](const double *p, int c0, double (&dst)[16]) {
        if (c0 + 16 <= nlim) {
#pragma unroll
            for (int i = 0; i < 16; ++i) dst[i] = __ldg(p + i * ldi);
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) dst[i] = c0 + i < nlim ? __ldg(p + i * ldi) : 0.0;
        }
    };
    // one output element: column i of the chunk at pc / pd
    auto put = [&](int i, float acc, double cin_i) {
        float out = alpha * acc;
        if (CIN) out = fmaf(beta, sw_d2f(cin_i), out);
        pc[i * ldc] = out;
        if (NDIG > 0) {
            const __nv_bfloat16 d1 = __float2bfloat16_rn(out);
            pd[i * ldd] = d1;
            if (NDIG > 1) {
                const float r1 = out - __bfloat162float(d1);
                const __nv_bfloat16 d2 = __float2bfloat16_rn(r1);
                pd[dpl + i * ldd] = d2;
                if (NDIG > 2) pd[2 * dpl + i * ldd] = __float2bfloat16_rn(r1 - __bfloat162float(d2));
            }
        }
    };
    if (CIN && row_ok && c_lo < nlim) load_cin(pi, c_lo, cin);
    for (int c0 = c_lo; c0 < c_hi; c0 += 16) {
        if (c0 >= nlim) break;   // the rest of the tile lies past N (uniform over the warp)
        if (CIN && row_ok && c0 + 16 < c_hi && c0 + 16 < nlim) load_cin(pi + 16 * ldi, c0 + 16, cin_next);
        uint32_t r0[16], r1[16];
        if (have_acc) {
            tmem_ld16_async(lane_base + (uint32_t)c0, r0);
            if (nacc > 1) tmem_ld16_async(lane_base + (uint32_t)(BN + c0), r1);
            tmem_wait_ld(r0);
            tmem_pin16(r1);
        }
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            v[i] = 0.f;
            if (have_acc) {
                v[i] += __uint_as_float(r0[i]);
                if (nacc > 1) v[i] += __uint_as_float(r1[i]);
            }
        }
        if (row_ok) {
            if (c0 + 16 <= nlim) {
#pragma unroll
                for (int i = 0; i < 16; ++i) put(i, v[i], CIN ? cin[i] : 0.0);
            } else {
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (c0 + i < nlim) put(i, v[i], CIN ? cin[i] : 0.0);
            }
        }
        pc += 16 * ldc;
        if (NDIG > 0) pd += 16 * ldd;
        if (CIN) {
            pi += 16 * ldi;
#pragma unroll
            for (int i = 0; i < 16; ++i) cin[i] = cin_next[i];
        }
    }
}

// The epilogue of columns [c_lo, c_hi) of a tile: the specialised FP32 form for
// FP32 outputs from at most two accumulators, the general form otherwise.
template <int BN>
__device__ __forceinline__ void tc_epilogue_part(const TcArgs &args, uint32_t tmem, int q, int row, int n0, int z,
                                                 int nacc, bool have_acc, int c_lo, int c_hi) {
    if (args.C32 != nullptr && nacc <= 2) {
        const uint32_t lb = tmem + ((uint32_t)(32 * q) << 16);
        const int ndig = args.Dout != nullptr ? args.ndig : 0;
        if (args.Cin != nullptr) {
            switch (ndig) {
            case 0: tc_epilogue_fast<BN, true, 0>(args, lb, row, n0, z, nacc, have_acc, c_lo, c_hi); return;
            case 1: tc_epilogue_fast<BN, true, 1>(args, lb, row, n0, z, nacc, have_acc, c_lo, c_hi); return;
            case 2: tc_epilogue_fast<BN, true, 2>(args, lb, row, n0, z, nacc, have_acc, c_lo, c_hi); return;
            case 3: tc_epilogue_fast<BN, true, 3>(args, lb, row, n0, z, nacc, have_acc, c_lo, c_hi); return;
            default: break;
            }
        } else {
            switch (ndig) {
            case 0: tc_epilogue_fast<BN, false, 0>(args, lb, row, n0, z, nacc, have_acc, c_lo, c_hi); return;
            case 1: tc_epilogue_fast<BN, false, 1>(args, lb, row, n0, z, nacc, have_acc, c_lo, c_hi); return;
            case 2: tc_epilogue_fast<BN, false, 2>(args, lb, row, n0, z, nacc, have_acc, c_lo, c_hi); return;
            case 3: tc_epilogue_fast<BN, false, 3>(args, lb, row, n0, z, nacc, have_acc, c_lo, c_hi); return;
            default: break;
            }
        }
    }
    tc_epilogue<BN>(args, tmem, q, row, n0, z, nacc, have_acc, c_lo, c_hi);
}

// The same with only the three forms the solver's split products take (digits of
// the products with two planes, the contraction without, the gradient with Cin),
// for the tile-list kernel, whose roles leave less room for inlined code.
template <int BN>
__device__ __forceinline__ void tc_epilogue_part3(const TcArgs &args, uint32_t tmem, int q, int row, int n0, int z,
                                                  int nacc, bool have_acc, int c_lo, int c_hi) {
    if (args.C32 != nullptr && nacc <= 2) {
        const uint32_t lb = tmem + ((uint32_t)(32 * q) << 16);
        const int ndig = args.Dout != nullptr ? args.ndig : 0;
        if (args.Cin != nullptr && ndig == 0) {
            tc_epilogue_fast<BN, true, 0>(args, lb, row, n0, z, nacc, have_acc, c_lo, c_hi);
            return;
        }
        if (args.Cin == nullptr && ndig == 0) {
            tc_epilogue_fast<BN, false, 0>(args, lb, row, n0, z, nacc, have_acc, c_lo, c_hi);
            return;
        }
        if (args.Cin == nullptr && ndig == 2) {
            tc_epilogue_fast<BN, false, 2>(args, lb, row, n0, z, nacc, have_acc, c_lo, c_hi);
            return;
        }
    }
    tc_epilogue<BN>(args, tmem, q, row, n0, z, nacc, have_acc, c_lo, c_hi);
}

// Epilogue warps per tensor-memory lane quarter in the CTA-pair kernel: two, each
// taking half of the tile's columns, so that every scheduler runs two epilogue
// warps and hides the latency of the other's chain (10 warps: at most 168
// registers a thread).
constexpr int kEpiWarpsPerQuarter = 2;
constexpr int kPairThreads = 64 + 128 * kEpiWarpsPerQuarter;

// ------------------------------------------------------------------ the GEMM kernel
template <int BN, int STAGES, int BKT>
__global__ void __launch_bounds__(192, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   const TcArgs args) {
    if (args.state != nullptr && *((volatile const int *)&args.state->done)) return;
    const int z = blockIdx.z;
    const int nA = args.nA, nB = args.nB;
    constexpr int TILE_A = BM * BKT * 2;
    const int tileB = BN * BKT * 2;
    const int stage_bytes = nA * TILE_A + nB * tileB;

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[STAGES];
    __shared__ __align__(8) uint64_t empty_bar[STAGES];
    __shared__ __align__(8) uint64_t acc_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const uint64_t deadline = globaltimer_ns() + kWaitNs;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM;     // N tiles vary fastest: CTAs in flight share A tiles in L2
    const int n0 = blockIdx.x * BN;
    const int nkb = (args.K + BKT - 1) / BKT;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&acc_bar, 1);
        abort_flag = 0;
        mbar_fence_init();
    }
    // Accumulators in tensor memory: kacc contiguous K ranges x ncls pair classes
    // (class 0: the leading digit pair (1,1); class 1: every smaller pair).
    const int kacc = args.kacc, ncls = args.ncls;
    const uint32_t tmem_cols = (uint32_t)(BN * kacc * ncls);
    if (warp == 1) tmem_alloc(&tmem_base, tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer
        const int a_row = args.a_row0 + z * args.a_row_step + m0;
        const int b_row = args.b_row0 + z * args.b_row_step + n0;
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % STAGES;
            const uint32_t ph = (uint32_t)((kb / STAGES) & 1);
            if (!mbar_wait(&empty_bar[s], ph ^ 1u, deadline, &abort_flag, args.err)) break;
            mbar_arrive_expect_tx(&full_bar[s], (uint32_t)stage_bytes);
            uint8_t *st = smem + s * stage_bytes;
            for (int p = 0; p < nA; ++p)
                tma_load_3d(st + p * TILE_A, &mapA, kb * BKT, a_row, p, &full_bar[s]);
            for (int q = 0; q < nB; ++q)
                tma_load_3d(st + nA * TILE_A + q * tileB, &mapB, kb * BKT, b_row, q, &full_bar[s]);
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        constexpr uint32_t idesc = idesc_bf16(BM, BN);
        bool ok = true;
        uint32_t written = 0;   // accumulators already holding a partial sum
        for (int kb = 0; kb < nkb && ok; ++kb) {
            const int s = kb % STAGES;
            const uint32_t ph = (uint32_t)((kb / STAGES) & 1);
            if (!mbar_wait(&full_bar[s], ph, deadline, &abort_flag, args.err)) { ok = false; break; }
            tc_fence_after();
            const uint32_t st = smem_u32(smem + s * stage_bytes);
            // k-block kb feeds K slot (kb * kacc) / nkb; the first MMA into an accumulator overwrites it
            const int slot = (kb * kacc) / nkb;
            for (int pr = 0; pr < args.npairs; ++pr) {
                const int cls = (ncls == 2 && (args.pa[pr] != 0 || args.pb[pr] != 0)) ? 1 : 0;
                const int acc = slot * ncls + cls;
                const uint32_t tacc = tmem + (uint32_t)(acc * BN);
                const uint32_t sa = st + args.pa[pr] * TILE_A;
                const uint32_t sb = st + nA * TILE_A + args.pb[pr] * tileB;
                const uint64_t da = BKT == 64 ? sdesc_sw128(sa) : sdesc_sw64(sa);
                const uint64_t db = BKT == 64 ? sdesc_sw128(sb) : sdesc_sw64(sb);
#pragma unroll
                for (int kk = 0; kk < BKT / 16; ++kk) {
                    // advance 16 elements (32 bytes) along K inside the swizzle row
                    umma_bf16(tacc, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc,
                              ((written >> acc) & 1u) ? 1u : 0u);
                    written |= 1u << acc;
                }
            }
            umma_commit(&empty_bar[s]);
        }
        umma_commit(&acc_bar);
    } else if (warp >= 2) {
        // ---------------- epilogue: TMEM -> registers -> FP64 global
        const int q = warp & 3;              // TMEM lane quarter this warp may access
        const int row = m0 + 32 * q + lane;
        bool got = nkb > 0 && mbar_wait(&acc_bar, 0, deadline, &abort_flag, args.err);
        const bool have_acc = __all_sync(0xffffffffu, got);   // tcgen05.ld is warp-collective
        tc_fence_after();
        const int nacc = (nkb < kacc ? nkb : kacc) * ncls;   // accumulators that were written
        tc_epilogue_part<BN>(args, tmem, q, row, n0, z, nacc, have_acc, 0, BN);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, tmem_cols);
    }
}

// ------------------------------------------------------------------ the GEMM on CTA pairs
// A cluster of two CTAs computes a 256 x 256 tile with the pair MMA
// (tcgen05.mma.cta_group::2, M = 256): CTA r holds A rows 128r..128r+127 and
// B rows (output columns) 128r..128r+127 of the tile in its shared memory, and
// its tensor memory receives output rows 128r..128r+127 for all 256 columns.
// Each SM thus pulls half of the B tile through its shared memory per MMA
// instead of all of it.  Roles:
//   warp 0 (both CTAs): TMA of the CTA's own A and B digit tiles; every copy
//     completes on CTA 0's full barrier of the stage, which CTA 0's producer
//     arms with the bytes of both CTAs;
//   warp 1, CTA 0: waits for the stage, issues the pair MMAs and commits to
//     the empty barriers of both CTAs (multicast), finally to both
//     accumulator barriers;
//   warps 2..9 (both CTAs): the epilogue of the CTA's 128 rows, two warps per
//     tensor-memory lane quarter, each writing half of the tile's columns.
// All waits are bounded; the pair meets at cluster barriers only after every
// role's loop has ended, and tensor memory is released by both CTAs together.
template <int STAGES, int BKT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kPairThreads, 1)
    tc_gemm_pair_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                        const TcArgs args) {
    // state->done only changes between launches, so both CTAs of a pair return here together
    if (args.state != nullptr && *((volatile const int *)&args.state->done)) return;
    constexpr int BN = 256, BNH = 128;
    const uint32_t rank = cluster_ctarank();
    const int z = blockIdx.z;
    const int nA = args.nA, nB = args.nB;
    constexpr int TILE_A = BM * BKT * 2;
    constexpr int TILE_B = BNH * BKT * 2;
    const int stage_bytes = nA * TILE_A + nB * TILE_B;
    // A planes this pair tile reads: one where the whole tile lies in A's one-digit rows
    const int nA_t = (args.a_split_row > 0 && (int)blockIdx.y * (2 * BM) >= args.a_split_row) ? 1 : nA;

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[STAGES];    // (CTA 0) both CTAs' copies of a stage landed
    __shared__ __align__(8) uint64_t empty_bar[STAGES];   // the pair's MMAs of a stage completed
    __shared__ __align__(8) uint64_t acc_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const uint64_t deadline = globaltimer_ns() + kWaitNs;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * (2 * BM) + BM * (int)rank;   // this CTA's output rows
    const int n0 = (blockIdx.x >> 1) * BN;                   // the pair's output columns
    const int nb0 = n0 + BNH * (int)rank;                    // this CTA's B rows
    const int nkb = (args.K + BKT - 1) / BKT;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&acc_bar, 1);
        abort_flag = 0;
        mbar_fence_init();
    }
    const int kacc = args.kacc, ncls = args.ncls;
    const uint32_t tmem_cols = (uint32_t)(BN * kacc * ncls);
    if (warp == 1) tmem_alloc_pair(&tmem_base, tmem_cols);
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();   // barriers of both CTAs initialised before any copy signals them
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    int issued = 0;       // producer: k-blocks whose copies were issued

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer (both CTAs)
        const int a_row = args.a_row0 + z * args.a_row_step + m0;
        const int b_row = args.b_row0 + z * args.b_row_step + nb0;
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % STAGES;
            const uint32_t ph = (uint32_t)((kb / STAGES) & 1);
            if (!mbar_wait(&empty_bar[s], ph ^ 1u, deadline, &abort_flag, args.err)) break;
            uint8_t *st = smem + s * stage_bytes;
            if (rank == 0) {
                mbar_arrive_expect_tx(&full_bar[s], (uint32_t)(2 * (nA_t * TILE_A + nB * TILE_B)));
                for (int p = 0; p < nA_t; ++p)
                    tma_load_3d(st + p * TILE_A, &mapA, kb * BKT, a_row, p, &full_bar[s]);
                for (int q = 0; q < nB; ++q)
                    tma_load_3d(st + nA * TILE_A + q * TILE_B, &mapB, kb * BKT, b_row, q, &full_bar[s]);
            } else {
                const uint32_t fb = mapa_shared(smem_u32(&full_bar[s]), 0u);
                for (int p = 0; p < nA_t; ++p)
                    tma_load_3d_pair(st + p * TILE_A, &mapA, kb * BKT, a_row, p, fb);
                for (int q = 0; q < nB; ++q)
                    tma_load_3d_pair(st + nA * TILE_A + q * TILE_B, &mapB, kb * BKT, b_row, q, fb);
            }
            issued = kb + 1;
        }
    } else if (warp == 1 && lane == 0 && rank == 0) {
        // ---------------- pair MMA issuer (CTA 0)
        constexpr uint32_t idesc = idesc_bf16(2 * BM, BN);
        uint32_t written = 0;
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % STAGES;
            const uint32_t ph = (uint32_t)((kb / STAGES) & 1);
            if (!mbar_wait_cluster(&full_bar[s], ph, deadline, &abort_flag, args.err)) break;
            tc_fence_after();
            const uint32_t st = smem_u32(smem + s * stage_bytes);
            const int slot = (kb * kacc) / nkb;
            for (int pr = 0; pr < args.npairs; ++pr) {
                if (args.pa[pr] >= nA_t) continue;   // a zero plane of A: the pair adds nothing
                const int cls = (ncls == 2 && (args.pa[pr] != 0 || args.pb[pr] != 0)) ? 1 : 0;
                const int acc = slot * ncls + cls;
                const uint32_t tacc = tmem + (uint32_t)(acc * BN);
                const uint32_t sa = st + args.pa[pr] * TILE_A, sb = st + nA * TILE_A + args.pb[pr] * TILE_B;
                const uint64_t da = BKT == 64 ? sdesc_sw128(sa) : sdesc_sw64(sa);
                const uint64_t db = BKT == 64 ? sdesc_sw128(sb) : sdesc_sw64(sb);
#pragma unroll
                for (int kk = 0; kk < BKT / 16; ++kk) {
                    umma_bf16_pair(tacc, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc,
                                   ((written >> acc) & 1u) ? 1u : 0u);
                    written |= 1u << acc;
                }
            }
            umma_commit_pair_mc(&empty_bar[s], (uint16_t)0x3);
        }
        umma_commit_pair_mc(&acc_bar, (uint16_t)0x3);
    } else if (warp >= 2) {
        // ---------------- epilogue (both CTAs): this CTA's 128 rows
        const int q = warp & 3;
        const int row = m0 + 32 * q + lane;
        bool got = nkb > 0 && mbar_wait(&acc_bar, 0, deadline, &abort_flag, args.err);
        const bool have_acc = __all_sync(0xffffffffu, got);
        tc_fence_after();
        const int nacc = (nkb < kacc ? nkb : kacc) * ncls;
        const int c_lo = (warp - 2) < 4 ? 0 : BN / 2;   // two warps per lane quarter, half the columns each
        tc_epilogue_part<BN>(args, tmem, q, row, n0, z, nacc, have_acc, c_lo, c_lo + BN / 2);
    }
    if (warp == 0 && lane == 0 && abort_flag) {
        // an aborted pipeline: let the issued copies land before the CTA can exit.  CTA 0
        // watches its full barriers (they count both CTAs' copies); CTA 1 cannot see
        // its copies complete and waits out a fixed 1 ms, far beyond a copy's latency.
        const uint64_t now = globaltimer_ns();
        if (rank == 0) {
            const uint64_t until = now + 200000000ull;
            for (int kb = issued - STAGES < 0 ? 0 : issued - STAGES; kb < issued; ++kb) {
                const uint32_t addr = smem_u32(&full_bar[kb % STAGES]);
                const uint32_t ph = (uint32_t)((kb / STAGES) & 1);
                while (!mbar_try_wait_cluster(addr, ph) && globaltimer_ns() < until) {
                }
            }
        } else {
            while (globaltimer_ns() < now + 1000000ull) {
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();   // neither CTA leaves while the pair's MMAs or copies may touch it
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc_pair(tmem, tmem_cols);
    }
}

// ------------------------------------------------------------------ persistent tile-list GEMM
// One launch over a list of 256-column output tiles drawn from many problems
// (the grouped products of many systems, or one system's tiles in a persistent
// schedule).  CTA c (pair c with PAIR) takes tiles c, c + G, c + 2G, ... of the
// list; a tile whose problem's solve has finished (state->done, fixed during
// the launch) is skipped by every role alike.  The shared-memory ring and its
// barrier phases run on across tiles, so the producer fills the next tile's
// first stages while the epilogue drains the last one.  The accumulator
// occupies all 512 tensor-memory columns (two pair classes of 256), so the MMA
// of a tile waits for the epilogue warps of the previous tile (tmem_empty,
// arrived by the four epilogue warps of each CTA).
template <bool PAIR, int STAGES, int BKT>
__global__ void __launch_bounds__(192, 1)
    tc_gemm_list_kernel(const TileProblem *__restrict__ probs, const TileRef *__restrict__ tiles, int ntiles) {
    constexpr int BN = 256;                        // accumulator columns per pair class
    constexpr int BNC = PAIR ? 128 : 256;          // most B rows per CTA (a problem's tiles may be narrower)
    constexpr int TILE_A = BM * BKT * 2;
    constexpr int TILE_B = BNC * BKT * 2;
    const uint32_t rank = PAIR ? cluster_ctarank() : 0u;
    const int group = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
    const int ngroups = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;
    const int nA = probs[0].a.nA, nB = probs[0].a.nB;
    const int stage_bytes = nA * TILE_A + nB * TILE_B;

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[STAGES];
    __shared__ __align__(8) uint64_t empty_bar[STAGES];
    __shared__ __align__(8) uint64_t acc_bar;
    __shared__ __align__(8) uint64_t tmem_empty_bar;   // (CTA 0) epilogues drained the accumulator
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const uint64_t deadline = globaltimer_ns() + kWaitNs;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    int *err = probs[0].a.err;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&acc_bar, 1);
        mbar_init(&tmem_empty_bar, PAIR ? 8 : 4);
        abort_flag = 0;
        mbar_fence_init();
    }
    constexpr uint32_t tmem_cols = 512;
    if (warp == 1) {
        if (PAIR) tmem_alloc_pair(&tmem_base, tmem_cols);
        else tmem_alloc(&tmem_base, tmem_cols);
    }
    tc_fence_before();
    __syncthreads();
    if (PAIR) cluster_sync_all();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    auto live = [&](const TcArgs &a) {
        return a.state == nullptr || !*((volatile const int *)&a.state->done);
    };
    int issued = 0;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer: the ring runs on across tiles
        uint32_t g = 0;   // k-blocks issued so far
        bool ok = true;
        for (int t = group; t < ntiles && ok; t += ngroups) {
            const TileRef tr = tiles[t];
            const TileProblem *P = probs + tr.p;
            const TcArgs a = P->a;   // a register copy: the stores of other roles cannot alias it
            if (!live(a)) continue;
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&P->mapA)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&P->mapB)) : "memory");
            const int bn = P->bn, bnc = PAIR ? bn / 2 : bn;   // this problem's tile width, B rows per CTA
            const uint32_t tile_bytes = (uint32_t)(nA * TILE_A + nB * bnc * BKT * 2);
            const int m0 = tr.mi * (PAIR ? 2 * BM : BM) + BM * (int)rank;
            const int a_row = a.a_row0 + tr.z * a.a_row_step + m0;
            const int b_row = a.b_row0 + tr.z * a.b_row_step + tr.ni * bn + bnc * (int)rank;
            const int nkb = (a.K + BKT - 1) / BKT;
            for (int kb = 0; kb < nkb; ++kb, ++g) {
                const int s = (int)(g % STAGES);
                const uint32_t ph = (g / STAGES) & 1u;
                if (!mbar_wait(&empty_bar[s], ph ^ 1u, deadline, &abort_flag, err)) { ok = false; break; }
                uint8_t *st = smem + s * stage_bytes;
                if (rank == 0) {
                    mbar_arrive_expect_tx(&full_bar[s], (PAIR ? 2u : 1u) * tile_bytes);
                    for (int p = 0; p < nA; ++p)
                        tma_load_3d(st + p * TILE_A, &P->mapA, kb * BKT, a_row, p, &full_bar[s]);
                    for (int q = 0; q < nB; ++q)
                        tma_load_3d(st + nA * TILE_A + q * TILE_B, &P->mapB, kb * BKT, b_row, q, &full_bar[s]);
                } else {
                    const uint32_t fb = mapa_shared(smem_u32(&full_bar[s]), 0u);
                    for (int p = 0; p < nA; ++p)
                        tma_load_3d_pair(st + p * TILE_A, &P->mapA, kb * BKT, a_row, p, fb);
                    for (int q = 0; q < nB; ++q)
                        tma_load_3d_pair(st + nA * TILE_A + q * TILE_B, &P->mapB, kb * BKT, b_row, q, fb);
                }
                issued = (int)g + 1;
            }
        }
    } else if (warp == 1 && lane == 0 && rank == 0) {
        // ---------------- MMA issuer (the single CTA, or CTA 0 of the pair)
        uint32_t g = 0, tile_it = 0;
        bool ok = true;
        for (int t = group; t < ntiles && ok; t += ngroups) {
            const TcArgs a = probs[tiles[t].p].a;
            if (!live(a)) continue;
            const uint32_t idesc = idesc_bf16(PAIR ? 2 * BM : BM, probs[tiles[t].p].bn);
            // the previous tile's epilogues must have read the accumulator out
            if (!mbar_wait_cluster(&tmem_empty_bar, (tile_it & 1u) ^ 1u, deadline, &abort_flag, err)) break;
            tc_fence_after();
            const int nkb = (a.K + BKT - 1) / BKT;
            const int ncls = a.ncls, npairs = a.npairs;
            uint32_t written = 0;
            for (int kb = 0; kb < nkb; ++kb, ++g) {
                const int s = (int)(g % STAGES);
                const uint32_t ph = (g / STAGES) & 1u;
                if (!mbar_wait_cluster(&full_bar[s], ph, deadline, &abort_flag, err)) { ok = false; break; }
                tc_fence_after();
                const uint32_t st = smem_u32(smem + s * stage_bytes);
#pragma unroll
                for (int pr = 0; pr < 9; ++pr) {   // unrolled: the pair table stays in registers
                    if (pr >= npairs) break;
                    const int cls = (ncls == 2 && (a.pa[pr] != 0 || a.pb[pr] != 0)) ? 1 : 0;
                    const uint32_t tacc = tmem + (uint32_t)(cls * BN);
                    const uint64_t da = sdesc_sw128(st + a.pa[pr] * TILE_A);
                    const uint64_t db = sdesc_sw128(st + nA * TILE_A + a.pb[pr] * TILE_B);
#pragma unroll
                    for (int kk = 0; kk < BKT / 16; ++kk) {
                        const uint32_t accum = ((written >> cls) & 1u) ? 1u : 0u;
                        if (PAIR) umma_bf16_pair(tacc, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc, accum);
                        else umma_bf16(tacc, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc, accum);
                        written |= 1u << cls;
                    }
                }
                if (PAIR) umma_commit_pair_mc(&empty_bar[s], (uint16_t)0x3);
                else umma_commit(&empty_bar[s]);
            }
            if (PAIR) umma_commit_pair_mc(&acc_bar, (uint16_t)0x3);
            else umma_commit(&acc_bar);
            ++tile_it;
        }
    } else if (warp >= 2) {
        // ---------------- epilogue: one tile at a time
        const int q = warp & 3;
        uint32_t tile_it = 0;
        const uint32_t te_local = smem_u32(&tmem_empty_bar);
        const uint32_t te_leader = PAIR ? mapa_shared(te_local, 0u) : te_local;
        for (int t = group; t < ntiles; t += ngroups) {
            const TileRef tr = tiles[t];
            const TcArgs a = probs[tr.p].a;
            if (!live(a)) continue;
            const int bn = probs[tr.p].bn;
            const bool got = mbar_wait(&acc_bar, tile_it & 1u, deadline, &abort_flag, err);
            if (!__all_sync(0xffffffffu, got)) break;
            tc_fence_after();
            const int m0 = tr.mi * (PAIR ? 2 * BM : BM) + BM * (int)rank;
            const int row = m0 + 32 * q + lane;
            tc_epilogue_part3<BN>(a, tmem, q, row, tr.ni * bn, tr.z, a.ncls, true, 0, bn);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                if (PAIR) mbar_arrive_remote(te_leader);
                else mbar_arrive(&tmem_empty_bar);
            }
            ++tile_it;
        }
    }
    if (warp == 0 && lane == 0 && abort_flag) {
        const uint64_t now = globaltimer_ns();
        if (rank == 0) {
            const uint64_t until = now + 200000000ull;
            for (int g = issued - STAGES < 0 ? 0 : issued - STAGES; g < issued; ++g) {
                const uint32_t addr = smem_u32(&full_bar[g % STAGES]);
                const uint32_t ph = (uint32_t)((g / STAGES) & 1);
                while (!mbar_try_wait_cluster(addr, ph) && globaltimer_ns() < until) {
                }
            }
        } else {
            while (globaltimer_ns() < now + 1000000ull) {
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (PAIR) cluster_sync_all();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        if (PAIR) tmem_dealloc_pair(tmem, tmem_cols);
        else tmem_dealloc(tmem, tmem_cols);
    }
}

// ------------------------------------------------------------------ bounded-wait self-test
// One mbarrier wait that nothing completes, through the same bounded wait as
// the GEMM kernels' pipelines: it must give up at the deadline and report it.
__global__ void wait_probe_kernel(uint64_t limit_ns, int *err, int *status) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint64_t deadline = globaltimer_ns() + limit_ns;
        const bool ok = mbar_wait(&bar, 0u, deadline, &abort_flag, err);   // phase 0 never completes
        *status = ok ? OMM_OK : OMM_ERR_TIMEOUT;
    }
}

// ------------------------------------------------------------------ digit packing
// column-major source (rows x cols, ld_src) -> planes [ndig][cols][ldd], element
// (i, j) at j*ldd + i (the K-major layout when K runs along the rows).
__global__ void pack_cm_kernel(int64_t rows, int64_t cols, const double *__restrict__ src, int64_t ld_src,
                               __nv_bfloat16 *dst, int64_t ldd, int64_t plane, int ndig,
                               const DevState *state) {
    if (state != nullptr && *((volatile const int *)&state->done)) return;
    for (int64_t j = blockIdx.y; j < cols; j += gridDim.y)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows;
             i += (int64_t)gridDim.x * blockDim.x) {
            __nv_bfloat16 d1, d2, d3;
            split3_i(src[i + j * ld_src], d1, d2, d3);
            const int64_t o = j * ldd + i;
            dst[o] = d1;
            if (ndig > 1) dst[plane + o] = d2;
            if (ndig > 2) dst[2 * plane + o] = d3;
        }
}

// column-major source (rows x cols) -> planes [ndig][rows][ldd], element (i, j)
// at i*ldd + j (K-major when K runs along the columns); 32x32 smem transpose.
__global__ void pack_t_kernel(int64_t rows, int64_t cols, const double *__restrict__ src, int64_t ld_src,
                              __nv_bfloat16 *dst, int64_t ldd, int64_t plane, int ndig,
                              const DevState *state) {
    if (state != nullptr && *((volatile const int *)&state->done)) return;
    __shared__ double tile[32][33];
    const int64_t ti = (int64_t)blockIdx.x * 32, tj = (int64_t)blockIdx.y * 32;
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;   // 32 x 8 threads
    for (int r = ly; r < 32; r += 8) {
        const int64_t i = ti + lx, j = tj + r;
        tile[r][lx] = (i < rows && j < cols) ? src[i + j * ld_src] : 0.0;
    }
    __syncthreads();
    for (int r = ly; r < 32; r += 8) {
        const int64_t i = ti + r, j = tj + lx;
        if (i < rows && j < cols) {
            __nv_bfloat16 d1, d2, d3;
            split3_i(tile[lx][r], d1, d2, d3);
            const int64_t o = i * ldd + j;
            dst[o] = d1;
            if (ndig > 1) dst[plane + o] = d2;
            if (ndig > 2) dst[2 * plane + o] = d3;
        }
    }
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (fn == nullptr) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            set_error("cuTensorMapEncodeTiled entry point unavailable");
            return nullptr;
        }
        fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

template <int BN, int STAGES, int BKT>
int launch_tc(const CUtensorMap &ma, const CUtensorMap &mb, const TcArgs &a, int nbatch, cudaStream_t st) {
    const int smem = STAGES * (a.nA * BM * BKT * 2 + a.nB * BN * BKT * 2) + 1024;
    static int attr_bytes = 0;
    if (smem > attr_bytes) {
        OMM_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<BN, STAGES, BKT>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr_bytes = smem;
    }
    TcArgs b = a;
    const int nkb = (a.K + BKT - 1) / BKT;
    bool has_main = false, has_small = false;
    for (int p = 0; p < a.npairs; ++p) {
        if (a.pa[p] == 0 && a.pb[p] == 0) has_main = true; else has_small = true;
    }
    b.ncls = (has_main && has_small) ? 2 : 1;
    int kacc = 512 / (BN * b.ncls);
    while (kacc > 1 && kacc > nkb) kacc >>= 1;
    b.kacc = kacc;
    dim3 grid((unsigned)ceil_div(a.N, BN), (unsigned)ceil_div(a.M, BM), (unsigned)nbatch);
    tc_gemm_kernel<BN, STAGES, BKT><<<grid, 192, smem, st>>>(ma, mb, b);
    count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

template <int STAGES, int BKT>
int launch_tc_pair(const CUtensorMap &ma, const CUtensorMap &mb_half, const TcArgs &a, int nbatch,
                   cudaStream_t st) {
    const int smem = STAGES * (a.nA * BM * BKT * 2 + a.nB * 128 * BKT * 2) + 1024;
    static int attr_bytes = 0;
    if (smem > attr_bytes) {
        OMM_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_pair_kernel<STAGES, BKT>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr_bytes = smem;
    }
    TcArgs b = a;
    const int nkb = (a.K + BKT - 1) / BKT;
    bool has_main = false, has_small = false;
    for (int p = 0; p < a.npairs; ++p) {
        if (a.pa[p] == 0 && a.pb[p] == 0) has_main = true; else has_small = true;
    }
    b.ncls = (has_main && has_small) ? 2 : 1;
    int kacc = 512 / (256 * b.ncls);
    while (kacc > 1 && kacc > nkb) kacc >>= 1;
    b.kacc = kacc;
    dim3 grid((unsigned)(2 * ceil_div(a.N, 256)), (unsigned)ceil_div(a.M, 2 * BM), (unsigned)nbatch);
    tc_gemm_pair_kernel<STAGES, BKT><<<grid, kPairThreads, smem, st>>>(ma, mb_half, b);
    count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

template <bool PAIR>
int launch_list(const TileProblem *probs, const TileRef *tiles, int ntiles, int ctas, int nA, int nB,
                cudaStream_t st) {
    constexpr int BKT = 64;
    const int stage = nA * BM * BKT * 2 + nB * (PAIR ? 128 : 256) * BKT * 2;
    // as many stages as fit in 220 KB (three 64 KB pair stages; two 96 KB single stages)
    const int stages = (220 * 1024) / stage >= 3 ? 3 : 2;
    const int smem = stages * stage + 1024;
    auto kern = stages == 3 ? tc_gemm_list_kernel<PAIR, 3, BKT> : tc_gemm_list_kernel<PAIR, 2, BKT>;
    static int attr3 = 0, attr2 = 0;
    int &attr = stages == 3 ? attr3 : attr2;
    if (smem > attr) {
        OMM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr = smem;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ctas, 1, 1);
    cfg.blockDim = dim3(192, 1, 1);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cudaLaunchAttribute attr_c[1];
    attr_c[0].id = cudaLaunchAttributeClusterDimension;
    attr_c[0].val.clusterDim.x = PAIR ? 2 : 1;
    attr_c[0].val.clusterDim.y = 1;
    attr_c[0].val.clusterDim.z = 1;
    cfg.attrs = attr_c;
    cfg.numAttrs = 1;
    OMM_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, probs, tiles, ntiles));
    count_launch();
    return OMM_OK;
}

}  // namespace

void list_prepare(TcArgs &a) {
    bool has_main = false, has_small = false;
    for (int p = 0; p < a.npairs; ++p) {
        if (a.pa[p] == 0 && a.pb[p] == 0) has_main = true; else has_small = true;
    }
    a.ncls = (has_main && has_small) ? 2 : 1;
    a.kacc = 1;
}

int list_tile_width(int N, int mode) {
    const int q = mode == LIST_PAIR ? 32 : 16;   // the pair's half tile stays a multiple of 16 rows
    const int w = (int)ceil_div(N, q) * q;
    return w < 256 ? w : 256;
}

void list_tiles(int p, const TcArgs &a, int nbatch, int mode, int bn, std::vector<TileRef> &out) {
    const int tm = (int)ceil_div(a.M, mode == LIST_PAIR ? 2 * BM : BM);
    const int tn = (int)ceil_div(a.N, bn);
    for (int z = 0; z < nbatch; ++z)
        for (int mi = 0; mi < tm; ++mi)
            for (int ni = 0; ni < tn; ++ni) out.push_back(TileRef{p, z, mi, ni});
}

int gemm_list(const TileProblem *probs, const TileRef *tiles, int ntiles, int mode, int ctas, int nA, int nB,
              cudaStream_t st) {
    if (ntiles <= 0) return OMM_OK;
    if (nA < 1 || nB < 1 || nA + nB > 4 || ctas < 1) return OMM_ERR_ARG;
    if (mode == LIST_PAIR) {
        if (ctas & 1) return OMM_ERR_ARG;
        return launch_list<true>(probs, tiles, ntiles, ctas, nA, nB, st);
    }
    return launch_list<false>(probs, tiles, ntiles, ctas, nA, nB, st);
}

int make_digit_map(CUtensorMap *map, const __nv_bfloat16 *base, int64_t K, int64_t rows, int64_t ld,
                   int64_t plane_elems, int nplanes, int box_rows, int bk) {
    auto enc = encode_fn();
    if (enc == nullptr) return OMM_ERR_CUDA;
    if ((ld % 8) != 0 || (plane_elems % 8) != 0 || (((uintptr_t)base) & 15u) != 0) return OMM_ERR_ARG;
    if (K <= 0 || rows <= 0 || nplanes <= 0 || box_rows <= 0 || box_rows > 256) return OMM_ERR_ARG;
    cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)nplanes};
    cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)plane_elems * 2};
    if (bk != 64 && bk != 32) return OMM_ERR_ARG;
    cuuint32_t box[3] = {(cuuint32_t)bk, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    memset(map, 0, sizeof(*map));
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void *)base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE,
                     bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d): K=%lld rows=%lld ld=%lld planes=%d box_rows=%d",
                  (int)r, (long long)K, (long long)rows, (long long)ld, nplanes, box_rows);
        return OMM_ERR_CUDA;
    }
    return OMM_OK;
}

int gemm(const CUtensorMap &mapA, const CUtensorMap &mapB, const TcArgs &a, int nbatch, int bn,
         cudaStream_t st, const CUtensorMap *mapB_half) {
    if (a.M <= 0 || a.N <= 0 || a.K < 0 || a.nA < 1 || a.nA > 3 || a.nB < 1 || a.nB > 3) return OMM_ERR_ARG;
    if (a.npairs < 1 || a.npairs > 9 || nbatch < 1) return OMM_ERR_ARG;
    for (int p = 0; p < a.npairs; ++p)
        if (a.pa[p] >= a.nA || a.pb[p] >= a.nB) return OMM_ERR_ARG;
    // CTA pairs: 256 x 256 tiles with the B tile split between the two SMs; needs the
    // 64-wide K blocks and a B map whose box is 128 rows
    if (mapB_half != nullptr && a.bk == 64 && bn == 256) {
        if (a.nA + a.nB <= 3) return launch_tc_pair<4, 64>(mapA, *mapB_half, a, nbatch, st);   // 4 x 48 KB
        if (a.nA + a.nB <= 4) return launch_tc_pair<3, 64>(mapA, *mapB_half, a, nbatch, st);   // 3 x 64 KB
        return launch_tc_pair<2, 64>(mapA, *mapB_half, a, nbatch, st);                         // 2 x 96 KB
    }
    // The tensor maps decide the K-block width: 64 (128-byte swizzle) or 32 (64-byte).
    if (a.bk == 32) {
        if (bn == 256) return launch_tc<256, 3, 32>(mapA, mapB, a, nbatch, st);
        if (a.nA + a.nB <= 4) return launch_tc<128, 6, 32>(mapA, mapB, a, nbatch, st);
        return launch_tc<128, 4, 32>(mapA, mapB, a, nbatch, st);
    }
    if (bn == 256) {
        if (a.nA + 2 * a.nB <= 4) return launch_tc<256, 3, 64>(mapA, mapB, a, nbatch, st);
        if (a.nA + a.nB <= 4) return launch_tc<256, 2, 64>(mapA, mapB, a, nbatch, st);   // 2 x 96 KB stages
        return launch_tc<256, 1, 64>(mapA, mapB, a, nbatch, st);
    }
    if (a.nA + a.nB <= 4) return launch_tc<128, 3, 64>(mapA, mapB, a, nbatch, st);
    return launch_tc<128, 2, 64>(mapA, mapB, a, nbatch, st);
}

int pack_cm(int64_t rows, int64_t cols, const double *src, int64_t ld_src, __nv_bfloat16 *dst, int64_t ldd,
            int64_t plane, int ndig, const DevState *state, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return OMM_OK;
    dim3 grid((unsigned)ceil_div(rows, 256 * 2), (unsigned)(cols < 8192 ? cols : 8192));
    pack_cm_kernel<<<grid, 256, 0, st>>>(rows, cols, src, ld_src, dst, ldd, plane, ndig, state);
    count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

int pack_t(int64_t rows, int64_t cols, const double *src, int64_t ld_src, __nv_bfloat16 *dst, int64_t ldd,
           int64_t plane, int ndig, const DevState *state, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return OMM_OK;
    dim3 grid((unsigned)ceil_div(rows, 32), (unsigned)ceil_div(cols, 32));
    pack_t_kernel<<<grid, 256, 0, st>>>(rows, cols, src, ld_src, dst, ldd, plane, ndig, state);
    count_launch();
    OMM_CUDA_TRY(cudaGetLastError());
    return OMM_OK;
}

void pairs_for_digits(int ndig, TcArgs &a) {
    // digit pairs (p, q) with p + q <= ndig + 1 (1-based), smallest terms first
    int k = 0;
    for (int lvl = ndig + 1; lvl >= 2; --lvl)
        for (int p = 1; p <= ndig; ++p) {
            const int q = lvl - p;
            if (q < 1 || q > ndig) continue;
            a.pa[k] = (uint8_t)(p - 1);
            a.pb[k] = (uint8_t)(q - 1);
            ++k;
        }
    a.npairs = k;
    a.nA = ndig;
    a.nB = ndig;
}

void pairs_one_b(int ndig, TcArgs &a) {
    // B carries one digit: pairs (p, 1), p = ndig .. 1 (1-based), smallest terms first
    int k = 0;
    for (int p = ndig; p >= 1; --p) {
        a.pa[k] = (uint8_t)(p - 1);
        a.pb[k] = 0;
        ++k;
    }
    a.npairs = k;
    a.nA = ndig;
    a.nB = 1;
}

}  // namespace tc
}  // namespace omm

// ---------------------------------------------------------------- op-level entry
extern "C" int omm_selftest_bounded_wait(int64_t limit_ns, int32_t *status_out, void *stream) {
    using namespace omm;
    if (status_out == nullptr || limit_ns < 1000 || limit_ns > 10000000000ll) return OMM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int *d = nullptr;   // [0] error flag, [1] status
    OMM_CUDA_TRY(cudaMalloc(&d, 2 * sizeof(int)));
    int h[2] = {0, OMM_ERR_STATE};
    int rc = OMM_OK;
    if (cudaMemcpyAsync(d, h, sizeof(h), cudaMemcpyHostToDevice, st) != cudaSuccess) rc = OMM_ERR_CUDA;
    if (rc == OMM_OK) {
        tc::wait_probe_kernel<<<1, 32, 0, st>>>((uint64_t)limit_ns, d, d + 1);
        count_launch();
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = OMM_ERR_CUDA;
    }
    cudaFree(d);
    if (rc != OMM_OK) return rc;
    *status_out = h[1];
    return OMM_OK;
}

extern "C" int64_t omm_op_split_gemm_workspace_bytes(int64_t M, int64_t N, int64_t K, int32_t ndigits) {
    if (M < 0 || N < 0 || K < 0 || ndigits < 1 || ndigits > 3) return -1;
    const int64_t ldk = (K + 7) / 8 * 8;
    return (int64_t)ndigits * (M + N) * ldk * 2 + 1024;
}

extern "C" int omm_op_split_gemm(int32_t transA, int32_t transB, int64_t M, int64_t N, int64_t K,
                                 int32_t ndigits, double alpha, const double *A, int64_t lda,
                                 const double *B, int64_t ldb, double beta, const double *Cin,
                                 int64_t ldcin, double *C, int64_t ldc, void *workspace,
                                 int64_t workspace_bytes, void *stream) {
    using namespace omm;
    if (M <= 0 || N <= 0 || K <= 0 || ndigits < 1 || ndigits > 3) return OMM_ERR_ARG;
    if (M > (1 << 30) || N > (1 << 30) || K > (1 << 30)) return OMM_ERR_ARG;
    if (A == nullptr || B == nullptr || C == nullptr || workspace == nullptr) return OMM_ERR_ARG;
    if (lda < (transA ? K : M) || ldb < (transB ? N : K) || ldc < M) return OMM_ERR_ARG;
    if (beta != 0.0 && (Cin == nullptr || ldcin < M)) return OMM_ERR_ARG;
    if (workspace_bytes < omm_op_split_gemm_workspace_bytes(M, N, K, ndigits)) return OMM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t ldk = (K + 7) / 8 * 8;
    uintptr_t base = ((uintptr_t)workspace + 255) & ~(uintptr_t)255;
    __nv_bfloat16 *Ad = (__nv_bfloat16 *)base;
    __nv_bfloat16 *Bd = Ad + (int64_t)ndigits * M * ldk;
    if ((((uintptr_t)Bd) & 15u) != 0) return OMM_ERR_ARG;
    int rc;
    // op(A) is M x K: K-major rows of op(A)
    if (transA) rc = tc::pack_cm(K, M, A, lda, Ad, ldk, M * ldk, ndigits, nullptr, st);
    else rc = tc::pack_t(M, K, A, lda, Ad, ldk, M * ldk, ndigits, nullptr, st);
    if (rc) return rc;
    // op(B) is K x N: K-major rows are the columns of op(B)
    if (transB) rc = tc::pack_t(N, K, B, ldb, Bd, ldk, N * ldk, ndigits, nullptr, st);
    else rc = tc::pack_cm(K, N, B, ldb, Bd, ldk, N * ldk, ndigits, nullptr, st);
    if (rc) return rc;
    CUtensorMap ma, mb;
    const int bk = ndigits >= 2 ? 32 : 64;
    if ((rc = tc::make_digit_map(&ma, Ad, K, M, ldk, M * ldk, ndigits, 128, bk))) return rc;
    const int bn = N > 128 ? 256 : 128;
    if ((rc = tc::make_digit_map(&mb, Bd, K, N, ldk, N * ldk, ndigits, bn, bk))) return rc;
    tc::TcArgs a{};
    tc::pairs_for_digits(ndigits, a);
    a.bk = bk;
    a.M = (int)M;
    a.N = (int)N;
    a.K = (int)K;
    a.alpha = alpha;
    a.beta = beta;
    a.Cin = beta != 0.0 ? Cin : nullptr;
    a.ldcin = ldcin;
    a.C = C;
    a.ldc = ldc;
    a.err = nullptr;
    return tc::gemm(ma, mb, a, 1, bn, st);
}
