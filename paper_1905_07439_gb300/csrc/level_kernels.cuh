// Launch interfaces of the per-level encode/decode kernels and the SIMT leaf GEMM.
#pragma once

#include <cuda_runtime.h>

#include "rbc_internal.h"

namespace rbc {

struct EncodeArgs {
  const void* X;        // parents: parent p at X + p*strideX, leading dim ldx (elements)
  int64_t ldx, strideX;
  void* Y;              // children: child p*R + r at Y + (p*R + r)*strideY, leading dim ldy
  int64_t ldy, strideY;
  int64_t nb;           // child block size (valid rows = cols)
  int64_t rows_out;     // written output rows (>= nb; rows beyond nb are zero padding)
  int64_t cols_out;     // written output columns per panel (>= nb)
  int64_t parents;      // number of parent nodes in this launch
  int64_t node_first;   // heap id of parent 0
  int tensor;           // 0: left operand (u^), 1: right operand (v^)
  int trans;            // 1: write each child transposed
  int split;            // 0: plain; 1: split panels [hi | lo] (hi = round(x), lo = round(x - hi))
  int64_t kpanel;       // column offset between split panels
};

struct DecodeArgs {
  const void* M;        // children: child p*R + r at M + (p*R + r)*strideM, leading dim ldm
  int64_t ldm, strideM;
  void* P;              // parents: parent p at P + p*strideP, leading dim ldp
  int64_t ldp, strideP;
  int64_t nb;           // child block size
  int64_t parents;
  int64_t node_first;
};

cudaError_t launch_encode_level(const Tables<double>& t, const EncodeArgs& a, int n0, int io,
                                int store, cudaStream_t st);
cudaError_t launch_encode_level(const Tables<float>& t, const EncodeArgs& a, int n0, int io,
                                int store, cudaStream_t st);
cudaError_t launch_decode_level(const Tables<double>& t, const DecodeArgs& a, int n0, cudaStream_t st);
cudaError_t launch_decode_level(const Tables<float>& t, const DecodeArgs& a, int n0, cudaStream_t st);

// Batched leaf products M_leaf = S_leaf * T_leaf^T on the CUDA cores (fp32 or fp64 FMA).
struct SimtGemmArgs {
  const void* S;        // left operands [leaf][mp][K] row-major, leading dim lds
  const void* Tt;       // right operands stored transposed [leaf][mp][K], leading dim ldt
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
cudaError_t launch_simt_gemm(const Tables<double>& t, const SimtGemmArgs& a, cudaStream_t st);
cudaError_t launch_simt_gemm(const Tables<float>& t, const SimtGemmArgs& a, cudaStream_t st);

}  // namespace rbc
