// Per-level encode and decode kernels of the recursion (Section 2.1.1,
// Eq. recursive-random-formula), written for any formula size n0 <= 4, any R, any depth.
//
// Encode, one level: for every parent node p at depth d and every child r,
//     S_{p,r} = sum_{k,l} u^(p)_{klr} X_p[k, l]      (X_p split into n0 x n0 blocks),
// with u^ the randomized table of Prop. 10 computed in-kernel from the base tensor and the
// node's packed draw (both in the constant bank), so the randomization moves no data.
// One thread owns one position (y, x) of the child blocks: it reads the n0^2 parent
// entries at that position once and writes the R children (coalesced along x).
//
// Decode, one level: P_p[i, j] = sum_r w^(p)_{ijr} M_{p,r}, r sequential.
#include <cuda_runtime.h>

#include "convert.cuh"
#include "level_kernels.cuh"
#include "rbc_internal.h"

namespace rbc {

namespace {

constexpr int kTile = 32;
constexpr int kRowsPerThread = 4;  // block = 32 x 8 threads over a 32 x 32 tile

template <typename T>
__device__ __forceinline__ T load_in(const void* base, int64_t off) {
  return static_cast<const T*>(base)[off];
}

// Encode one level.  Tin/Tc: I/O element and arithmetic type; N0: formula block count
// per side (N0 == 1 is the identity used for L = 0); S: storage of the outputs.
template <typename Tin, typename Tc, int N0, int S>
__global__ void __launch_bounds__(256) encode_level_kernel(const __grid_constant__ Tables<Tc> t,
                                                           const EncodeArgs a) {
  using Tout = typename StoreType<S>::T;
  __shared__ Tc tile[kTile][kTile + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t x0 = (int64_t)blockIdx.x * kTile, y0 = (int64_t)blockIdx.y * kTile;
  const int R = (N0 == 1) ? 1 : t.R;
  const int n0 = N0;
  const int cs_row = a.tensor == 0 ? 0 : 1;  // u^: (pi1,s1) rows, (pi2,s2) cols
  const int cs_col = a.tensor == 0 ? 1 : 2;  // v^: (pi2,s2) rows, (pi3,s3) cols
  const Tc* base = a.tensor == 0 ? t.U : t.V;

  for (int64_t p = blockIdx.z; p < a.parents; p += gridDim.z) {
    // Randomized index maps of this node (uniform across the block).
    int prow[N0], pcol[N0];
    Tc srow[N0], scol[N0];
    if (N0 > 1) {
      const uint64_t w = t.draw[t.per_level ? 0 : (a.node_first + p - t.draw_base)];
#pragma unroll
      for (int j = 0; j < N0; ++j) {
        prow[j] = draw_perm(w, cs_row, j);
        pcol[j] = draw_perm(w, cs_col, j);
        srow[j] = (Tc)draw_sign(w, cs_row, j);
        scol[j] = (Tc)draw_sign(w, cs_col, j);
      }
    }
    // Gather the n0 x n0 parent entries of each owned position.
    Tc in[kRowsPerThread][N0][N0];
    const Tin* X = static_cast<const Tin*>(a.X) + p * a.strideX;
#pragma unroll
    for (int q = 0; q < kRowsPerThread; ++q) {
      const int64_t y = y0 + ty + q * 8, x = x0 + tx;
      const bool ok = y < a.nb && x < a.nb;
#pragma unroll
      for (int k = 0; k < N0; ++k)
#pragma unroll
        for (int l = 0; l < N0; ++l)
          in[q][k][l] = ok ? (Tc)X[(k * a.nb + y) * a.ldx + l * a.nb + x] : (Tc)0;
    }
    for (int r = 0; r < R; ++r) {
      Tc coef[N0][N0];
#pragma unroll
      for (int k = 0; k < N0; ++k)
#pragma unroll
        for (int l = 0; l < N0; ++l)
          coef[k][l] = (N0 == 1) ? (Tc)1
                                 : base[(prow[k] * n0 + pcol[l]) * t.R + r] * srow[k] * scol[l];
      Tc v[kRowsPerThread];
#pragma unroll
      for (int q = 0; q < kRowsPerThread; ++q) {
        Tc s = (Tc)0;
#pragma unroll
        for (int k = 0; k < N0; ++k)
#pragma unroll
          for (int l = 0; l < N0; ++l) s = s + coef[k][l] * in[q][k][l];
        v[q] = s;
      }
      Tout* Y = static_cast<Tout*>(a.Y) + (p * R + r) * a.strideY;
      if (a.trans) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kRowsPerThread; ++q) tile[ty + q * 8][tx] = v[q];
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kRowsPerThread; ++q) v[q] = tile[tx][ty + q * 8];
      }
      // Output position: (orow, ocol) = (y, x), or (x, y) when transposed.
      const int64_t orow0 = a.trans ? x0 : y0, ocol0 = a.trans ? y0 : x0;
#pragma unroll
      for (int q = 0; q < kRowsPerThread; ++q) {
        const int64_t orow = orow0 + ty + q * 8, ocol = ocol0 + tx;
        if (orow >= a.rows_out || ocol >= a.cols_out) continue;
        Tout* dst = Y + orow * a.ldy + ocol;
        if (a.split == 0) {
          dst[0] = to_store<S>((double)v[q]);
        } else {
          // split compensated leaves: x = hi + lo with hi = round(x), lo = round(x - hi),
          // stored as two panels [hi | lo] along the row
          const Tout hi = to_store<S>((double)v[q]);
          const Tout lo = to_store<S>((double)(v[q] - (Tc)from_store<S>(hi)));
          dst[0] = hi;
          dst[a.kpanel] = lo;
        }
      }
    }
  }
}

// Decode one level.  Tm: type of the children, To: type of the parents.
template <typename Tm, typename To, typename Tc, int N0>
__global__ void __launch_bounds__(256) decode_level_kernel(const __grid_constant__ Tables<Tc> t,
                                                           const DecodeArgs a) {
  const int64_t x = (int64_t)blockIdx.x * kTile + threadIdx.x;
  const int64_t ybase = (int64_t)blockIdx.y * kTile + threadIdx.y;
  const int R = t.R;
  for (int64_t p = blockIdx.z; p < a.parents; p += gridDim.z) {
    const uint64_t w = t.draw[t.per_level ? 0 : (a.node_first + p - t.draw_base)];
    int p1[N0], p3[N0];
    Tc s1[N0], s3[N0];
#pragma unroll
    for (int j = 0; j < N0; ++j) {
      p1[j] = draw_perm(w, 0, j);
      p3[j] = draw_perm(w, 2, j);
      s1[j] = (Tc)draw_sign(w, 0, j);
      s3[j] = (Tc)draw_sign(w, 2, j);
    }
#pragma unroll
    for (int q = 0; q < kRowsPerThread; ++q) {
      const int64_t y = ybase + q * 8;
      if (y >= a.nb || x >= a.nb) continue;
      Tc acc[N0][N0];
#pragma unroll
      for (int i = 0; i < N0; ++i)
#pragma unroll
        for (int j = 0; j < N0; ++j) acc[i][j] = (Tc)0;
      const Tm* M = static_cast<const Tm*>(a.M) + p * R * a.strideM;
      for (int r = 0; r < R; ++r) {
        const Tc mv = (Tc)M[r * a.strideM + y * a.ldm + x];
#pragma unroll
        for (int i = 0; i < N0; ++i)
#pragma unroll
          for (int j = 0; j < N0; ++j) {
            const Tc wv = t.scale * t.W[(p1[i] * N0 + p3[j]) * R + r] * s1[i] * s3[j];
            acc[i][j] = acc[i][j] + wv * mv;
          }
      }
      To* P = static_cast<To*>(a.P) + p * a.strideP;
#pragma unroll
      for (int i = 0; i < N0; ++i)
#pragma unroll
        for (int j = 0; j < N0; ++j) P[(i * a.nb + y) * a.ldp + j * a.nb + x] = (To)acc[i][j];
    }
  }
}

inline dim3 level_grid(int64_t rows, int64_t cols, int64_t parents) {
  const int64_t gz = parents < 65535 ? parents : 65535;
  return dim3((unsigned)((cols + kTile - 1) / kTile), (unsigned)((rows + kTile - 1) / kTile),
              (unsigned)gz);
}

template <typename Tin, typename Tc, int S>
cudaError_t launch_encode_n0(const Tables<Tc>& t, const EncodeArgs& a, int n0, cudaStream_t st) {
  // The grid spans the output extents, which cover the child blocks (padding written as 0).
  const int64_t span = a.rows_out > a.cols_out ? a.rows_out : a.cols_out;
  const dim3 grid = level_grid(span, span, a.parents), block(kTile, 8);
  switch (n0) {
    case 1: encode_level_kernel<Tin, Tc, 1, S><<<grid, block, 0, st>>>(t, a); break;
    case 2: encode_level_kernel<Tin, Tc, 2, S><<<grid, block, 0, st>>>(t, a); break;
    case 3: encode_level_kernel<Tin, Tc, 3, S><<<grid, block, 0, st>>>(t, a); break;
    case 4: encode_level_kernel<Tin, Tc, 4, S><<<grid, block, 0, st>>>(t, a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename Tm, typename To, typename Tc>
cudaError_t launch_decode_n0(const Tables<Tc>& t, const DecodeArgs& a, int n0, cudaStream_t st) {
  const dim3 grid = level_grid(a.nb, a.nb, a.parents), block(kTile, 8);
  switch (n0) {
    case 2: decode_level_kernel<Tm, To, Tc, 2><<<grid, block, 0, st>>>(t, a); break;
    case 3: decode_level_kernel<Tm, To, Tc, 3><<<grid, block, 0, st>>>(t, a); break;
    case 4: decode_level_kernel<Tm, To, Tc, 4><<<grid, block, 0, st>>>(t, a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_encode_level(const Tables<double>& t, const EncodeArgs& a, int n0, int io,
                                int store, cudaStream_t st) {
  if (io != RBC_IO_F64 || store != kStoreF64) return cudaErrorInvalidValue;
  return launch_encode_n0<double, double, kStoreF64>(t, a, n0, st);
}

cudaError_t launch_encode_level(const Tables<float>& t, const EncodeArgs& a, int n0, int io,
                                int store, cudaStream_t st) {
  if (io != RBC_IO_F32) return cudaErrorInvalidValue;
  switch (store) {
    case kStoreF32: return launch_encode_n0<float, float, kStoreF32>(t, a, n0, st);
    case kStoreTF32: return launch_encode_n0<float, float, kStoreTF32>(t, a, n0, st);
    case kStoreBF16: return launch_encode_n0<float, float, kStoreBF16>(t, a, n0, st);
    case kStoreF16: return launch_encode_n0<float, float, kStoreF16>(t, a, n0, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_decode_level(const Tables<double>& t, const DecodeArgs& a, int n0, cudaStream_t st) {
  return launch_decode_n0<double, double, double>(t, a, n0, st);
}

cudaError_t launch_decode_level(const Tables<float>& t, const DecodeArgs& a, int n0, cudaStream_t st) {
  return launch_decode_n0<float, float, float>(t, a, n0, st);
}

}  // namespace rbc
