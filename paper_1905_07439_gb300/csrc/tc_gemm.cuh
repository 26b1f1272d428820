// Leaf products on the 5th-generation tensor cores (tcgen05 + TMEM + TMA) with the
// decode fused into the epilogue.
#pragma once

#include <cuda_runtime.h>

#include "rbc_internal.h"

namespace rbc {

struct TcGemmArgs {
  const void* S;   // left operands [leaf][mp][K], K-major, leaf storage type ([hi | lo] when split)
  const void* T;   // right operands [leaf][mp (k rows)][K (n, row length)], n contiguous
  int64_t K;       // row length of S and T^T (mp, or 2*mp for the split modes)
  int64_t m;       // valid rows/cols of each leaf product
  int64_t mp;      // padded rows/cols (multiple of the tile)
  int64_t leaves;
  void* C;         // fp32 output, zeroed unless direct
  int64_t ldc;
  int direct;      // 1: one leaf, plain stores (L = 0)
  int store_m;     // 1: store each leaf product to M (level-by-level decode follows)
  void* M;         // [leaf][mp][mp] fp32 when store_m, leaf products strideM elements apart
  int64_t strideM;
  int leaf;        // rbc_leaf_dtype
  int* status;     // device status word (RBC_ETIMEOUT on an expired wait)
  int stall;       // test hook: issue no operand copies (the bounded waits then expire)
  const float* rinv;  // f16x3: inverse scales of the rows of S and the columns of T (mp each,
  const float* cinv;  // powers of two), applied to every product entry; null otherwise
};

// One instance of a (possibly grouped) leaf-product launch, as the kernel reads it.
struct TcInst {
  int64_t m, mp, leaves, tile_begin;  // tile_begin: first global tile of this instance
  int nk, tiles_m, tiles_n, group_m, kpanel;
  int epi;     // 0: fused decode by reductions, 1: direct store (L = 0), 2: store M
  int vec_ok;  // 16-byte vector access to C allowed
  int pad_;
  float* C;
  int64_t ldc;
  float* M;
  int64_t ldm, strideM;
  const float* rinv;  // f16x3: inverse row / column scales (see TcGemmArgs)
  const float* cinv;
};

// A grouped launch: the leaf products of many instances (same leaf mode and tile width) in
// one persistent kernel.  insts and maps live in device memory; maps holds two 64-byte
// tensor maps (S, T) per instance.
struct TcGroupArgs {
  const TcInst* insts;
  const void* maps;
  int ninst;
  int64_t total_tiles;
  int leaf;
  int bn;
  int ctas;  // CTAs per SM: 1, or 2 for plain (not split) 128-wide tiles
  int* status;
};

int64_t tc_pad(int64_t m);
int tc_default_bn(int leaf, int64_t mp);
int tc_default_group(int leaf, int64_t mp, int64_t K);
// Fill the descriptor and the two tensor maps (host memory, 128 bytes) of one instance.
bool tc_prepare_instance(const TcGemmArgs& a, int bn, int group_m, int64_t tile_begin, TcInst* d, void* maps2);
int64_t tc_instance_tiles(const TcInst& d);
cudaError_t launch_tc_gemm(const Tables<float>& t, const TcGemmArgs& a, cudaStream_t st);
cudaError_t launch_tc_gemm_grouped(const TcGroupArgs& g, cudaStream_t st);

}  // namespace rbc
