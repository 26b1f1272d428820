// Launch interfaces of the per-level encode/decode kernels and the SIMT leaf GEMM.
#pragma once

#include <cuda_runtime.h>

#include "rbc_internal.h"

namespace rbc {

// One encode or decode pass over G consecutive levels (parents at depth `depth`).
//
// Column layouts.  A block of the recursion is nb_d x nb_d.  Plain layout: element (y, x) at
// column x.  Recursive padded layout (the intermediates): every leaf-sized column segment of
// m logical columns is stored in seg >= m physical columns (seg a multiple of 4), so every
// sub-block, at every level, starts 16-byte aligned; a block with n0^k segments per row is
// seg * n0^k physical columns wide and the sub-block column Lc of a grid starts at Lc times
// the sub-block's physical width.  Physical column x holds logical column
// (x / seg) * m + x % seg when x % seg < m (else padding, never read).
//
//   encode: X = parents (parent p at X + p*strideX, leading dim ldx), each an n0^G x n0^G grid
//           of nb x nb blocks, plain (plain = 1) or recursive with sub-block width xcol;
//           Y = outputs, output `path` of parent p at Y + (p*outs_per_parent + path)*strideY,
//           leading dim ldy, rows_out x cols_out physical positions written (padding
//           positions are zeros), split panels [hi | lo] (or [b0 | b1 | b2]) kpanel apart.  Positions x with
//           x % seg >= mval or rows y >= nb are padding.
//   decode: X = children (child `path` of parent p at X + (p*outs_per_parent + path)*strideX,
//           leading dim ldx), nb rows x xcol physical columns (padding as above); Y = parents
//           (p*strideY, leading dim ldy), plain (plain = 1) or recursive with sub-block
//           width xcol.
// Draw set of a node at relative depth j with heap id n: draw[dbase[j] + n - dfirst[j]]
// (per-node scope) or draw[depth + j] (per-level scope).
// Realization batches: with real_parents > 0 the parents of the launch belong to consecutive
// independent realizations, real_parents each; parent p is node node_first + p % real_parents
// of realization p / real_parents, whose draw sets start at draw[(p / real_parents) * real_draws].
struct PassArgs {
  const void* X;
  int64_t ldx, strideX;
  void* Y;
  int64_t ldy, strideY;
  int64_t nb;
  int64_t rows_out, cols_out;
  int64_t seg, mval;  // column segment pitch and its valid width (see above)
  int64_t xcol;       // physical width of an nb x nb sub-block in the recursive layout
  int plain;          // encode: X plain; decode: Y plain
  int64_t parents;
  int64_t outs_per_parent;
  int64_t node_first;
  int64_t real_parents;  // 0: all parents belong to one realization
  int64_t real_draws;
  int depth;
  int tensor;     // encode: 0 left operand (u^), 1 right operand (v^)
  int formula;    // rbc::BuiltinFormula of the plan's U, V, W (compiled-in one-level passes)
  int split;      // encode: extra panels written, 0 none, 1 [hi | lo], 2 [b0 | b1 | b2]
  int trans;      // encode, last pass: write each output transposed
  int vload;      // set by the launcher: input rows allow VEC-wide vector loads
  int vstore;     // set by the launcher: output rows allow VEC-wide vector stores
  int64_t kpanel;
  // encode, last pass of f16x3 leaves: power-of-two factor per leaf row (tensor 0: output row y)
  // or leaf column (tensor 1: output column x) applied before the split; null: none
  const float* lscale;
  int64_t dbase[kMaxLevels];
  int64_t dfirst[kMaxLevels];
};

int max_levels_per_pass(int n0);
// Children per node up to which an fp32 n0 = 2 encode pass covers three levels.
constexpr int kTop3MaxR = 8;
// Levels an fp32 encode pass covers for leaf size m, R children per node and leaf store type:
// two for Laderman's formula when m >= 32 (the first level held in shared memory,
// 128-position tiles); three for n0 = 2 with R <= kTop3MaxR unless the leaves are stored
// transposed (tf32); else max_levels_per_pass.
int max_encode_levels_per_pass(int n0, int R, int formula, int64_t m, int store);
// Levels an fp32 decode pass covers for leaf size m: two for Laderman's formula when m >= 32 (the
// lower level handed over in shared memory, 64-position tiles), else max_levels_per_pass.
int max_decode_levels_per_pass(int n0, int formula, int64_t m);
// g = 0 is the identity pass of L = 0 (conversion and padding of the single leaf).
cudaError_t launch_encode_pass(const Tables<double>& t, const PassArgs& a, int n0, int g, int io, int store,
                               cudaStream_t st);
cudaError_t launch_encode_pass(const Tables<float>& t, const PassArgs& a, int n0, int g, int io, int store,
                               cudaStream_t st);
cudaError_t launch_decode_pass(const Tables<double>& t, const PassArgs& a, int n0, int g, cudaStream_t st);
cudaError_t launch_decode_pass(const Tables<float>& t, const PassArgs& a, int n0, int g, cudaStream_t st);

// Leaf operand scales of the f16x3 mode.  amaxA[0 .. m) and amaxB[0 .. m) (zeroed by the caller)
// receive, as fp32 bit patterns, max |A[i][c]| over the rows i == r (mod m) of A and max
// |B[r][j]| over the columns j == c (mod m) of B (N x N fp32, leading dimensions lda, ldb); one
// launch.
cudaError_t launch_fold_absmax(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t N, int64_t m,
                               unsigned* amaxA, unsigned* amaxB, cudaStream_t st);
// scale[r] = 2^e with e the largest integer such that amax[r] * growth * 2^e < 2^15 (1 for a
// zero class or r >= m), inv[r] = 2^-e, for r < mp.
cudaError_t launch_leaf_scales(const unsigned* amax, int64_t m, int64_t mp, double growth, float* scale, float* inv,
                               cudaStream_t st);

// Batched leaf products M_leaf = S_leaf * T_leaf on the CUDA cores (fp32 or fp64 FMA).
struct SimtGemmArgs {
  const void* S;        // left operands [leaf][mp][K] row-major, leading dim lds
  const void* T;        // right operands [leaf][mp (k)][row length ldt >= mp (n)] row-major
  int64_t lds, ldt, strideS, strideT;
  int64_t K;            // inner dimension (multiple of the tile K)
  int64_t m;            // valid rows/cols of each leaf product
  int64_t mp;           // padded rows/cols (multiple of the tile)
  int64_t leaves;
  void* out;            // mode 0: M[leaf] (ldo, strideO); modes 1/2: C (ldo)
  int64_t ldo, strideO;
  int mode;             // 0: store M; 1: fused decode (atomic adds into zeroed C); 2: store C (L = 0)
};

int simt_tile(int io, int64_t m);  // padding granularity of the SIMT leaf path
// Padded size of a small leaf (exact-size product kernel), or 0 when m needs the tiled path.
int64_t simt_small_pad(int io, int64_t m);
cudaError_t launch_simt_gemm(const Tables<double>& t, const SimtGemmArgs& a, cudaStream_t st);
cudaError_t launch_simt_gemm(const Tables<float>& t, const SimtGemmArgs& a, cudaStream_t st);

}  // namespace rbc
