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
  void* M;         // [leaf][mp][mp] fp32 when store_m
  int leaf;        // rbc_leaf_dtype
  int* status;     // device status word (RBC_ETIMEOUT on an expired wait)
};

int64_t tc_pad(int64_t m);
bool tc_supports_store_m();
cudaError_t launch_tc_gemm(const Tables<float>& t, const TcGemmArgs& a, cudaStream_t st);

}  // namespace rbc
