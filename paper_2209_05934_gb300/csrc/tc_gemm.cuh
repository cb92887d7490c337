// Split-BF16 tcgen05 GEMM: host-side interface inside the library.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include <vector>

#include "omm_internal.cuh"

namespace omm {
namespace tc {

// Arguments of one (optionally z-batched) split GEMM
//   C_z = alpha * sum_pairs A_{pa} B_{pb}^T + beta * Cin_z
// with A, B given by 3-D tensor maps over BF16 digit planes [plane][rows][ld];
// batch z reads A rows from z*a_row_step and B rows from z*b_row_step.
struct TcArgs {
    int M, N, K;
    int nA, nB;                  // digit planes loaded per operand
    int npairs;
    uint8_t pa[9], pb[9];        // digit pairs (0-based plane indices)
    int a_row0, b_row0;          // first row of the operand in its tensor map
    int a_row_step, b_row_step;  // row advance per batch index z
    double alpha, beta;
    const double *Cin;           // nullable
    int64_t ldcin, cin_step;
    double *C;                   // FP64 column-major output (or nullptr when C32 is set)
    float *C32;                  // FP32 column-major output: accumulate, scale and split in FP32
    int64_t ldc, c_step;
    __nv_bfloat16 *Dout;         // nullable: BF16 digits of C, planes [ndig][..][ldd]
    int64_t ldd, dplane, dout_step;
    int ndig;
    const DevState *state;       // nullable: return at once when state->done
    int *err;                    // nullable: set to 1 when a bounded wait times out
    int kacc;                    // set by the launcher: K-range accumulators in tensor memory
    int ncls;                    // set by the launcher: 2 = leading digit pair kept apart
    int bk;                      // K-block width of the tensor maps: 64 (128-byte swizzle) or 32
    int a_split_row;             // > 0: the A rows at and past this output row carry one digit (their
                                 // further planes are zero), so CTA-pair tiles that start there load
                                 // A's first plane only and skip the pairs of the others; 0: none
};

// One problem of a grouped (tile-list) launch: its tensor maps (device copies)
// and arguments.  Every problem of one launch has the same digit planes and
// 64-wide K blocks; K > 0.
struct TileProblem {   // CUtensorMap keeps the maps 64-byte aligned in arrays
    CUtensorMap mapA;        // A planes, 128-row box
    CUtensorMap mapB;        // B planes, box of bn rows (one CTA per tile) or bn/2 rows (CTA pairs)
    TcArgs a;                // kacc, ncls filled by list_prepare
    int bn;                  // output tile width: list_tile_width(N, mode)
};
// One output tile: problem p, batch z, row tile mi, column tile ni (256 columns;
// 128 rows per tile with one CTA, 256 with a CTA pair).
struct TileRef {
    int32_t p, z, mi, ni;
};
enum { LIST_SINGLE = 0, LIST_PAIR = 1 };

// Fill kacc / ncls of a problem for the tile-list kernels (one K range per class).
void list_prepare(TcArgs &a);
// Output tile width of a problem with N columns: N rounded up to 16 (32 for CTA
// pairs), at most 256.  The MMA's N is the tile width, so a narrow problem does
// no tensor work on columns it does not have; the width changes no result (every
// output element accumulates over K in the same order).
int list_tile_width(int N, int mode);
// Tiles of problem p in (z, mi, ni) order for the given mode and tile width.
void list_tiles(int p, const TcArgs &a, int nbatch, int mode, int bn, std::vector<TileRef> &out);
// One persistent launch over a tile list: `ctas` CTAs (a multiple of 2 with
// LIST_PAIR), each taking tiles ctas-apart (pairs: cluster-apart) in list order.
int gemm_list(const TileProblem *probs, const TileRef *tiles, int ntiles, int mode, int ctas, int nA, int nB,
              cudaStream_t st);

int make_digit_map(CUtensorMap *map, const __nv_bfloat16 *base, int64_t K, int64_t rows, int64_t ld,
                   int64_t plane_elems, int nplanes, int box_rows, int bk = 64);
// mapB_half: a map of the same B planes with a 128-row box; when given (and the
// maps use 64-wide K blocks and bn = 256), the GEMM runs on CTA pairs
// (tcgen05.mma.cta_group::2, 256 x 256 tiles, half the B tile per SM)
int gemm(const CUtensorMap &mapA, const CUtensorMap &mapB, const TcArgs &a, int nbatch, int bn,
         cudaStream_t st, const CUtensorMap *mapB_half = nullptr);
int pack_cm(int64_t rows, int64_t cols, const double *src, int64_t ld_src, __nv_bfloat16 *dst, int64_t ldd,
            int64_t plane, int ndig, const DevState *state, cudaStream_t st);
int pack_t(int64_t rows, int64_t cols, const double *src, int64_t ld_src, __nv_bfloat16 *dst, int64_t ldd,
           int64_t plane, int ndig, const DevState *state, cudaStream_t st);
void pairs_for_digits(int ndig, TcArgs &a);
// A with ndig digits, B with one: the pairs (p, 1), p = ndig .. 1, and nB = 1
void pairs_one_b(int ndig, TcArgs &a);

}  // namespace tc
}  // namespace omm
