// Encode and decode passes of the recursion (Section 2.1.1, Eq. recursive-random-formula),
// each pass covering G consecutive levels (G <= 3 for n0 = 2, G <= 2 for n0 = 3, G = 1 for
// n0 = 4) so that the intermediate operands of those levels never leave registers.
//
// Encode pass: one thread owns one position (y, x) of the output blocks.  It reads the
// n0^G x n0^G entries of its parent at that position, then walks the G-level subtree depth
// first: at a node, child r receives S_r = sum_{k,l} u^(node)_{klr} X[k, l] (sub-blocks of the
// node's input, l inner, k outer), and the leaves of the walk are written to the R^G output
// operands.  u^ is formed in-kernel from the base tensor and the node's packed draw, both in
// the constant bank (Prop. 10), so the randomization moves no data.
//
// Decode pass: the same walk in post-order.  A node's output block (i, j) is
// sum_r w^(node)_{ijr} M_r (r sequential), M_r the child's output at this position.
//
// Neighbouring threads own neighbouring x, so every load and store is coalesced.
#include <cuda_runtime.h>

#include "convert.cuh"
#include "level_kernels.cuh"
#include "rbc_internal.h"

namespace rbc {

namespace {

constexpr int kThreadsX = 128;

__host__ __device__ constexpr int cpow(int b, int e) { return e == 0 ? 1 : b * cpow(b, e - 1); }

template <typename Tc>
__device__ __forceinline__ uint64_t node_draw(const Tables<Tc>& t, const PassArgs& a, int rel_depth,
                                              int64_t node) {
  if (t.per_level) return t.draw[a.depth + rel_depth];
  return t.draw[a.dbase[rel_depth] + (node - a.dfirst[rel_depth])];
}

__device__ __forceinline__ int64_t heap_child(int64_t node, int r, int R) { return node * R + r + 1; }

// ------------------------------------------------------------------ encode walk
template <typename Tc, int N0, int G>
struct EncodeWalk {
  static constexpr int W = cpow(N0, G), WC = W / N0;
  template <class Emit>
  __device__ __forceinline__ static void go(const Tables<Tc>& t, const PassArgs& a, const Tc* base, int cr,
                                            int cc, int rel, int64_t node, int64_t path, const Tc (&in)[W * W],
                                            Emit& emit) {
    const uint64_t w = node_draw(t, a, rel, node);
    int prow[N0], pcol[N0];
    Tc srow[N0], scol[N0];
#pragma unroll
    for (int j = 0; j < N0; ++j) {
      prow[j] = draw_perm(w, cr, j);
      pcol[j] = draw_perm(w, cc, j);
      srow[j] = (Tc)draw_sign(w, cr, j);
      scol[j] = (Tc)draw_sign(w, cc, j);
    }
    const int R = t.R;
    for (int r = 0; r < R; ++r) {
      Tc cin[WC * WC];
#pragma unroll
      for (int e = 0; e < WC * WC; ++e) cin[e] = (Tc)0;
#pragma unroll
      for (int k = 0; k < N0; ++k)
#pragma unroll
        for (int l = 0; l < N0; ++l) {
          const Tc coef = base[(prow[k] * N0 + pcol[l]) * R + r] * srow[k] * scol[l];
          if (coef != (Tc)0) {
#pragma unroll
            for (int u = 0; u < WC; ++u)
#pragma unroll
              for (int v = 0; v < WC; ++v)
                cin[u * WC + v] = cin[u * WC + v] + coef * in[(k * WC + u) * W + (l * WC + v)];
          }
        }
      EncodeWalk<Tc, N0, G - 1>::go(t, a, base, cr, cc, rel + 1, heap_child(node, r, R), path * R + r, cin, emit);
    }
  }
};

template <typename Tc, int N0>
struct EncodeWalk<Tc, N0, 0> {
  template <class Emit>
  __device__ __forceinline__ static void go(const Tables<Tc>&, const PassArgs&, const Tc*, int, int, int,
                                            int64_t, int64_t path, const Tc (&in)[1], Emit& emit) {
    emit(path, in[0]);
  }
};

template <typename Tc, int S>
struct EncodeEmit {
  using Tout = typename StoreType<S>::T;
  Tout* Y;       // this parent's first output operand
  int64_t strideY, off, kpanel;
  int split;
  __device__ __forceinline__ void operator()(int64_t path, Tc v) {
    Tout* dst = Y + path * strideY + off;
    const Tout hi = to_store<S>((double)v);
    dst[0] = hi;
    if (split) dst[kpanel] = to_store<S>((double)(v - (Tc)from_store<S>(hi)));
  }
};

template <typename Tin, typename Tc, int N0, int G, int S>
__global__ void __launch_bounds__(kThreadsX) encode_pass_kernel(const __grid_constant__ Tables<Tc> t,
                                                                const PassArgs a) {
  constexpr int W = cpow(N0, G);
  using Tout = typename StoreType<S>::T;
  const int64_t x = (int64_t)blockIdx.x * kThreadsX + threadIdx.x;
  const int64_t y = blockIdx.y;
  if (x >= a.cols_out) return;
  const bool valid = y < a.nb && x < a.nb;
  const int cr = a.tensor == 0 ? 0 : 1;  // u^: (pi1, s1) rows, (pi2, s2) cols
  const int cc = a.tensor == 0 ? 1 : 2;  // v^: (pi2, s2) rows, (pi3, s3) cols
  const Tc* base = a.tensor == 0 ? t.U : t.V;
  const int64_t outs = a.outs_per_parent;
  for (int64_t p = blockIdx.z; p < a.parents; p += gridDim.z) {
    EncodeEmit<Tc, S> emit;
    emit.Y = static_cast<Tout*>(a.Y) + p * outs * a.strideY;
    emit.strideY = a.strideY;
    emit.off = y * a.ldy + x;
    emit.kpanel = a.kpanel;
    emit.split = a.split;
    if (!valid) {  // zero padding of the leaf operands
      for (int64_t q = 0; q < outs; ++q) emit(q, (Tc)0);
      continue;
    }
    const Tin* X = static_cast<const Tin*>(a.X) + p * a.strideX;
    Tc in[W * W];
#pragma unroll
    for (int k = 0; k < W; ++k)
#pragma unroll
      for (int l = 0; l < W; ++l) in[k * W + l] = (Tc)X[(k * a.nb + y) * a.ldx + l * a.nb + x];
    EncodeWalk<Tc, N0, G>::go(t, a, base, cr, cc, 0, a.node_first + p, 0, in, emit);
  }
}

// ------------------------------------------------------------------ decode walk
template <typename Tc, int N0, int G>
struct DecodeWalk {
  static constexpr int W = cpow(N0, G), WC = W / N0;
  template <class Fetch>
  __device__ __forceinline__ static void go(const Tables<Tc>& t, const PassArgs& a, int rel, int64_t node,
                                            int64_t path, Tc (&out)[W * W], Fetch& fetch) {
    const uint64_t w = node_draw(t, a, rel, node);
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
    for (int e = 0; e < W * W; ++e) out[e] = (Tc)0;
    const int R = t.R;
    for (int r = 0; r < R; ++r) {
      Tc cout[WC * WC];
      DecodeWalk<Tc, N0, G - 1>::go(t, a, rel + 1, heap_child(node, r, R), path * R + r, cout, fetch);
#pragma unroll
      for (int i = 0; i < N0; ++i)
#pragma unroll
        for (int j = 0; j < N0; ++j) {
          const Tc wv = t.scale * t.W[(p1[i] * N0 + p3[j]) * R + r] * s1[i] * s3[j];
          if (wv != (Tc)0) {
#pragma unroll
            for (int u = 0; u < WC; ++u)
#pragma unroll
              for (int v = 0; v < WC; ++v)
                out[(i * WC + u) * W + (j * WC + v)] = out[(i * WC + u) * W + (j * WC + v)] + wv * cout[u * WC + v];
          }
        }
    }
  }
};

template <typename Tc, int N0>
struct DecodeWalk<Tc, N0, 0> {
  template <class Fetch>
  __device__ __forceinline__ static void go(const Tables<Tc>&, const PassArgs&, int, int64_t, int64_t path,
                                            Tc (&out)[1], Fetch& fetch) {
    out[0] = fetch(path);
  }
};

template <typename Tm, typename To, typename Tc, int N0, int G>
__global__ void __launch_bounds__(kThreadsX) decode_pass_kernel(const __grid_constant__ Tables<Tc> t,
                                                                const PassArgs a) {
  constexpr int W = cpow(N0, G);
  const int64_t x = (int64_t)blockIdx.x * kThreadsX + threadIdx.x;
  const int64_t y = blockIdx.y;
  if (x >= a.nb || y >= a.nb) return;
  for (int64_t p = blockIdx.z; p < a.parents; p += gridDim.z) {
    const Tm* M = static_cast<const Tm*>(a.X) + p * a.outs_per_parent * a.strideX;
    const int64_t off = y * a.ldx + x;
    const int64_t sM = a.strideX;
    auto fetch = [M, off, sM](int64_t path) -> Tc { return (Tc)M[path * sM + off]; };
    Tc out[W * W];
    DecodeWalk<Tc, N0, G>::go(t, a, 0, a.node_first + p, 0, out, fetch);
    To* P = static_cast<To*>(a.Y) + p * a.strideY;
#pragma unroll
    for (int k = 0; k < W; ++k)
#pragma unroll
      for (int l = 0; l < W; ++l) P[(k * a.nb + y) * a.ldy + l * a.nb + x] = (To)out[k * W + l];
  }
}

inline dim3 pass_grid(int64_t rows, int64_t cols, int64_t parents) {
  const int64_t gz = parents < 65535 ? parents : 65535;
  return dim3((unsigned)((cols + kThreadsX - 1) / kThreadsX), (unsigned)rows, (unsigned)gz);
}

template <typename Tin, typename Tc, int S, int N0>
cudaError_t enc_g(const Tables<Tc>& t, const PassArgs& a, int g, cudaStream_t st) {
  const dim3 grid = pass_grid(a.rows_out, a.cols_out, a.parents);
  switch (g) {
    case 1: encode_pass_kernel<Tin, Tc, N0, 1, S><<<grid, kThreadsX, 0, st>>>(t, a); break;
    case 2:
      if constexpr (N0 <= 3) {
        encode_pass_kernel<Tin, Tc, N0, 2, S><<<grid, kThreadsX, 0, st>>>(t, a);
        break;
      }
      return cudaErrorInvalidValue;
    case 3:
      if constexpr (N0 == 2) {
        encode_pass_kernel<Tin, Tc, N0, 3, S><<<grid, kThreadsX, 0, st>>>(t, a);
        break;
      }
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename Tin, typename Tc, int S>
cudaError_t enc_n0(const Tables<Tc>& t, const PassArgs& a, int n0, int g, cudaStream_t st) {
  switch (n0) {
    case 2: return enc_g<Tin, Tc, S, 2>(t, a, g, st);
    case 3: return enc_g<Tin, Tc, S, 3>(t, a, g, st);
    case 4: return enc_g<Tin, Tc, S, 4>(t, a, g, st);
  }
  return cudaErrorInvalidValue;
}

template <typename Tm, typename To, typename Tc, int N0>
cudaError_t dec_g(const Tables<Tc>& t, const PassArgs& a, int g, cudaStream_t st) {
  const dim3 grid = pass_grid(a.nb, a.nb, a.parents);
  switch (g) {
    case 1: decode_pass_kernel<Tm, To, Tc, N0, 1><<<grid, kThreadsX, 0, st>>>(t, a); break;
    case 2:
      if constexpr (N0 <= 3) {
        decode_pass_kernel<Tm, To, Tc, N0, 2><<<grid, kThreadsX, 0, st>>>(t, a);
        break;
      }
      return cudaErrorInvalidValue;
    case 3:
      if constexpr (N0 == 2) {
        decode_pass_kernel<Tm, To, Tc, N0, 3><<<grid, kThreadsX, 0, st>>>(t, a);
        break;
      }
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename Tm, typename To, typename Tc>
cudaError_t dec_n0(const Tables<Tc>& t, const PassArgs& a, int n0, int g, cudaStream_t st) {
  switch (n0) {
    case 2: return dec_g<Tm, To, Tc, 2>(t, a, g, st);
    case 3: return dec_g<Tm, To, Tc, 3>(t, a, g, st);
    case 4: return dec_g<Tm, To, Tc, 4>(t, a, g, st);
  }
  return cudaErrorInvalidValue;
}

// Identity "encode" of the single leaf when L = 0: conversion, padding and split panels.
template <typename Tin, int S>
__global__ void __launch_bounds__(kThreadsX) copy_leaf_kernel(const PassArgs a) {
  using Tout = typename StoreType<S>::T;
  const int64_t x = (int64_t)blockIdx.x * kThreadsX + threadIdx.x;
  const int64_t y = blockIdx.y;
  if (x >= a.cols_out) return;
  const Tin* X = static_cast<const Tin*>(a.X);
  const double v = (y < a.nb && x < a.nb) ? (double)X[y * a.ldx + x] : 0.0;
  Tout* dst = static_cast<Tout*>(a.Y) + y * a.ldy + x;
  const Tout hi = to_store<S>(v);
  dst[0] = hi;
  if (a.split) dst[a.kpanel] = to_store<S>(v - from_store<S>(hi));
}

}  // namespace

int max_levels_per_pass(int n0) { return n0 == 2 ? 3 : (n0 == 3 ? 2 : 1); }

cudaError_t launch_encode_pass(const Tables<double>& t, const PassArgs& a, int n0, int g, int io, int store,
                               cudaStream_t st) {
  if (io != RBC_IO_F64 || store != kStoreF64) return cudaErrorInvalidValue;
  if (g == 0) {
    copy_leaf_kernel<double, kStoreF64><<<pass_grid(a.rows_out, a.cols_out, 1), kThreadsX, 0, st>>>(a);
    return cudaGetLastError();
  }
  return enc_n0<double, double, kStoreF64>(t, a, n0, g, st);
}

cudaError_t launch_encode_pass(const Tables<float>& t, const PassArgs& a, int n0, int g, int io, int store,
                               cudaStream_t st) {
  if (io != RBC_IO_F32) return cudaErrorInvalidValue;
  if (g == 0) {
    const dim3 grid = pass_grid(a.rows_out, a.cols_out, 1);
    switch (store) {
      case kStoreF32: copy_leaf_kernel<float, kStoreF32><<<grid, kThreadsX, 0, st>>>(a); break;
      case kStoreTF32: copy_leaf_kernel<float, kStoreTF32><<<grid, kThreadsX, 0, st>>>(a); break;
      case kStoreBF16: copy_leaf_kernel<float, kStoreBF16><<<grid, kThreadsX, 0, st>>>(a); break;
      case kStoreF16: copy_leaf_kernel<float, kStoreF16><<<grid, kThreadsX, 0, st>>>(a); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  switch (store) {
    case kStoreF32: return enc_n0<float, float, kStoreF32>(t, a, n0, g, st);
    case kStoreTF32: return enc_n0<float, float, kStoreTF32>(t, a, n0, g, st);
    case kStoreBF16: return enc_n0<float, float, kStoreBF16>(t, a, n0, g, st);
    case kStoreF16: return enc_n0<float, float, kStoreF16>(t, a, n0, g, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_decode_pass(const Tables<double>& t, const PassArgs& a, int n0, int g, cudaStream_t st) {
  return dec_n0<double, double, double>(t, a, n0, g, st);
}

cudaError_t launch_decode_pass(const Tables<float>& t, const PassArgs& a, int n0, int g, cudaStream_t st) {
  return dec_n0<float, float, float>(t, a, n0, g, st);
}

}  // namespace rbc
