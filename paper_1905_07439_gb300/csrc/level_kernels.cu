// Encode and decode passes of the recursion (Section 2.1.1, Eq. recursive-random-formula).
// Each pass covers G consecutive levels (G <= 2 for n0 = 2, G = 1 for n0 >= 3, see
// max_levels_per_pass), so that the intermediate operands of those levels never leave
// registers.  fp32 encodes go deeper: up to four levels for n0 = 2 (encode_top_kernel) and two
// for Laderman's formula (encode_deep_kernel).
//
// Table-driven passes (any formula): at the start of every parent, the CTA expands the
// randomized tables of the parent's G-level subtree into shared memory (Prop. 10:
// u^_klr = u_{pi1(k) pi2(l) r} s1(k) s2(l), likewise v^, w^), from the base tensors and the
// nodes' packed draws, both held in the constant bank.  The randomization therefore moves no
// operand data, and the inner loops read each coefficient row with 16-byte broadcast loads.
//
// Encode pass: a thread owns VEC adjacent positions (y, x..x+VEC-1) of the output blocks. It
// reads the n0^G x n0^G entries of its parent at those positions, then walks the subtree
// depth first: at a node, child r receives S_r = sum_{k,l} u^(node)_{klr} X[k, l] (sub-blocks
// of the node's input, l inner, k outer), and the leaves of the walk are the R^G outputs.
//
// Decode pass: the same walk in post-order.  A node's output block (i, j) is
// sum_r w^(node)_{ijr} M_r (r sequential), M_r the child's output at these positions; the
// children of a bottom node are loaded several at a time so that their loads overlap.
//
// One-level passes of the built-in formulas (formulas.h) have the formula's sparsity compiled
// in and apply the node's signed permutation to the operands (encode_fixed_kernel,
// decode_fixed_kernel); one-level fp32 decodes of other n0 >= 3 formulas use nonzero lists
// (decode_sparse_kernel).  fp32 encodes of Laderman's formula cover two levels per pass, the
// first level held in shared memory (encode_deep_kernel); fp32 two-level decodes of Strassen's
// formula hand the lower level to the upper one through shared memory (decode_deep_kernel).
//
// Intermediates use the padded column layout of level_kernels.cuh with zero padding, so the
// passes that read them take the branch-free vector variant (FAST) whatever m is.
// Neighbouring threads own neighbouring positions: every load and store is coalesced.
#include <cuda_runtime.h>

#include <cstring>

#include <type_traits>

#include "convert.cuh"
#include "formulas.h"
#include "level_kernels.cuh"
#include "rbc_internal.h"

namespace rbc {

namespace {

constexpr int kThreadsX = 128;

__host__ __device__ constexpr int cpow(int b, int e) { return e == 0 ? 1 : b * cpow(b, e - 1); }

// Positions per thread when the layout allows vector access: keeps the per-thread working
// set (about VEC * 1.33 * n0^(2G) values) within the register file.
template <typename Tc, int N0, int G>
struct Vec {
  static constexpr int n = cpow(N0, 2 * G);
  static constexpr int value = sizeof(Tc) == 8 ? (n >= 64 ? 1 : (n >= 16 ? 2 : 4)) : (n >= 64 ? 2 : 4);
};

template <typename T, int VEC>
__device__ __forceinline__ void load_vec(T (&dst)[VEC], const T* src) {
  if constexpr (VEC * sizeof(T) == 16) {
    const int4 r = *reinterpret_cast<const int4*>(src);
    memcpy(dst, &r, 16);
  } else if constexpr (VEC * sizeof(T) == 8) {
    const int2 r = *reinterpret_cast<const int2*>(src);
    memcpy(dst, &r, 8);
  } else {
#pragma unroll
    for (int v = 0; v < VEC; ++v) dst[v] = src[v];
  }
}

template <typename T, int VEC>
__device__ __forceinline__ void store_vec(T* dst, const T (&x)[VEC]) {
  if constexpr (VEC * sizeof(T) == 16) {
    int4 r;
    memcpy(&r, x, 16);
    *reinterpret_cast<int4*>(dst) = r;
  } else if constexpr (VEC * sizeof(T) == 8) {
    int2 r;
    memcpy(&r, x, 8);
    *reinterpret_cast<int2*>(dst) = r;
  } else if constexpr (VEC * sizeof(T) == 4) {
    int r;
    memcpy(&r, x, 4);
    *reinterpret_cast<int*>(dst) = r;
  } else {
#pragma unroll
    for (int v = 0; v < VEC; ++v) dst[v] = x[v];
  }
}

// Number of nodes of a G-level subtree with R children per node: sum_{j<G} R^j.
__host__ __device__ inline int subtree_nodes(int R, int G) {
  int s = 0, p = 1;
  for (int j = 0; j < G; ++j) {
    s += p;
    p *= R;
  }
  return s;
}
// Coefficient rows of one child (n0^2 entries) padded to a multiple of 4 entries, so that a
// row loads as 16-byte vectors.
__host__ __device__ constexpr int coef_stride(int n0) { return (n0 * n0 + 3) / 4 * 4; }

// Local id of the node at relative depth j with path prefix q: sum_{i<j} R^i + q.
__device__ __forceinline__ int local_id(int R, int j, int q) { return subtree_nodes(R, j) + q; }

// Expand coefficient rows of the subtree under launch parent p (at depth a.depth) into
// coef[(row * R + r) * coef_stride(n0) + a * n0 + b] for tensor `which` (0 u^, 1 v^, 2 w^),
// row = 0 .. rows-1 holding the node with local id local_of(row); the row padding holds zeros.
template <typename Tc, class Map>
__device__ void expand_rows(const Tables<Tc>& t, const PassArgs& a, int rows, int which, int64_t p, Tc* coef,
                            Map local_of) {
  int64_t real = 0, hp = a.node_first + p;
  if (a.real_parents > 0) {
    real = p / a.real_parents;
    hp = a.node_first + (p - real * a.real_parents);
  }
  const uint64_t* draws = t.draw + real * a.real_draws;
  const int R = t.R, n0 = t.n0, nn = n0 * n0, ns = coef_stride(n0);
  const int total = rows * R * ns;
  const Tc* base = which == 0 ? t.U : (which == 1 ? t.V : t.W);
  const int cr = which == 1 ? 1 : 0;  // row stream: pi1/s1 (u^, w^) or pi2/s2 (v^)
  const int cc = which == 0 ? 1 : 2;  // column stream: pi2/s2 (u^) or pi3/s3 (v^, w^)
  const Tc sc = which == 2 ? t.scale : (Tc)1;
  const int nthreads = blockDim.x * blockDim.y;
  for (int e = threadIdx.y * blockDim.x + threadIdx.x; e < total; e += nthreads) {
    const int row = e / (R * ns);
    const int rem = e - row * R * ns;
    const int local = local_of(row);
    const int r = rem / ns, ab = rem - r * ns, ra = ab / n0, cb = ab - ra * n0;
    if (ab >= nn) {
      coef[e] = (Tc)0;
      continue;
    }
    int j = 0, start = 0, width = 1;
    while (local >= start + width) {
      start += width;
      width *= R;
      ++j;
    }
    int64_t rj = 1;
    for (int i = 0; i < j; ++i) rj *= R;
    const int64_t heap = hp * rj + (int64_t)local;  // descendant of hp: hp*R^j + sum_{i<j} R^i + q
    const uint64_t w = t.per_level ? draws[a.depth + j] : draws[a.dbase[j] + (heap - a.dfirst[j])];
    const Tc v = base[(draw_perm(w, cr, ra) * n0 + draw_perm(w, cc, cb)) * R + r];
    coef[e] = sc * v * (Tc)draw_sign(w, cr, ra) * (Tc)draw_sign(w, cc, cb);
  }
}

// All rows of the G-level subtree under launch parent p, row = local id.
struct IdentityRows {
  __device__ __forceinline__ int operator()(int row) const { return row; }
};
template <typename Tc>
__device__ void expand_subtree(const Tables<Tc>& t, const PassArgs& a, int G, int which, int64_t p, Tc* coef) {
  expand_rows(t, a, subtree_nodes(t.R, G), which, p, coef, IdentityRows{});
}

// One child's coefficient row from shared memory, as 16-byte vectors.
template <typename Tc, int N0>
__device__ __forceinline__ void load_coefs(Tc (&c)[coef_stride(N0)], const Tc* src) {
  constexpr int NS = coef_stride(N0);
  if constexpr (sizeof(Tc) == 4) {
#pragma unroll
    for (int i = 0; i < NS / 4; ++i) {
      const float4 v = reinterpret_cast<const float4*>(src)[i];
      memcpy(&c[4 * i], &v, 16);
    }
  } else {
#pragma unroll
    for (int i = 0; i < NS / 2; ++i) {
      const double2 v = reinterpret_cast<const double2*>(src)[i];
      memcpy(&c[2 * i], &v, 16);
    }
  }
}

// Zero coefficients are skipped in fp64 (its FMA pipe is the scarce resource); fp32 passes
// run the dense, branch-free form, which measured faster.
template <typename Tc>
__device__ __forceinline__ bool use_coef(Tc c) {
  return sizeof(Tc) == 4 || c != (Tc)0;
}

// ------------------------------------------------------------------ encode walk
template <typename Tc, int N0, int G, int VEC>
struct EncodeWalk {
  static constexpr int W = cpow(N0, G), WC = W / N0;
  template <class Emit>
  __device__ __forceinline__ static void go(const Tc* coef, int R, int j, int q, int64_t path,
                                            const Tc (&in)[W * W][VEC], Emit& emit) {
    constexpr int NS = coef_stride(N0);
    const Tc* row = coef + (size_t)local_id(R, j, q) * R * NS;
    for (int r = 0; r < R; ++r) {
      Tc c[NS];
      load_coefs<Tc, N0>(c, row + r * NS);
      Tc cin[WC * WC][VEC];
#pragma unroll
      for (int e = 0; e < WC * WC; ++e)
#pragma unroll
        for (int v = 0; v < VEC; ++v) cin[e][v] = (Tc)0;
#pragma unroll
      for (int k = 0; k < N0; ++k)
#pragma unroll
        for (int l = 0; l < N0; ++l) {
          const Tc cf = c[k * N0 + l];
          if (use_coef(cf)) {
#pragma unroll
            for (int u = 0; u < WC; ++u)
#pragma unroll
              for (int w = 0; w < WC; ++w)
#pragma unroll
                for (int v = 0; v < VEC; ++v)
                  cin[u * WC + w][v] = cin[u * WC + w][v] + cf * in[(k * WC + u) * W + (l * WC + w)][v];
          }
        }
      EncodeWalk<Tc, N0, G - 1, VEC>::go(coef, R, j + 1, q * R + r, path * R + r, cin, emit);
    }
  }
};

template <typename Tc, int N0, int VEC>
struct EncodeWalk<Tc, N0, 0, VEC> {
  template <class Emit>
  __device__ __forceinline__ static void go(const Tc*, int, int, int, int64_t path, const Tc (&in)[1][VEC],
                                            Emit& emit) {
    emit(path, in[0]);
  }
};

// Store VEC adjacent outputs: one vector store when aligned and complete, else element by
// element up to the output width.
template <typename T, int VEC>
__device__ __forceinline__ void store_some(T* dst, const T (&x)[VEC], bool vec, int64_t avail) {
  if (vec && avail >= VEC) {
    store_vec<T, VEC>(dst, x);
  } else {
#pragma unroll
    for (int v = 0; v < VEC; ++v)
      if (v < avail) dst[v] = x[v];
  }
}

// Two fp32 values rounded to a 16-bit leaf format (nearest even) with one instruction, and back.
template <int S> struct Pair2;
template <> struct Pair2<kStoreBF16> {
  using T = __nv_bfloat162;
  static __device__ __forceinline__ T cvt(float a, float b) { return __floats2bfloat162_rn(a, b); }
  static __device__ __forceinline__ float2 back(T v) { return __bfloat1622float2(v); }
};
template <> struct Pair2<kStoreF16> {
  using T = __half2;
  static __device__ __forceinline__ T cvt(float a, float b) { return __floats2half2_rn(a, b); }
  static __device__ __forceinline__ float2 back(T v) { return __half22float2(v); }
};

template <typename Tc, int S, int VEC>
struct EncodeEmitV {
  using Tout = typename StoreType<S>::T;
  Tout* Y;
  int64_t strideY, off, kpanel, avail;
  int split;
  bool vec;
  bool scaled = false;  // f16x3 leaves: multiply by sc (powers of two) before the split
  Tc sc[VEC];
  // Leaf operand scale of positions (y, x .. x + VEC - 1) of the last encode pass.
  __device__ __forceinline__ void set_scale(const PassArgs& a, int64_t y, int64_t x) {
    if (!a.lscale) return;
    scaled = true;
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      const int64_t i = a.tensor == 0 ? y : min(x + v, a.cols_out - 1);
      sc[v] = (Tc)a.lscale[i];
    }
  }
  __device__ __forceinline__ void operator()(int64_t path, const Tc (&val_in)[VEC]) {
    Tc val[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) val[v] = scaled ? val_in[v] * sc[v] : val_in[v];
    Tout* dst = Y + path * strideY + off;
    if constexpr ((S == kStoreBF16 || S == kStoreF16) && sizeof(Tc) == 4 && VEC % 2 == 0) {
      using P = Pair2<S>;
      typename P::T h2[VEC / 2];
      Tout hi[VEC];
#pragma unroll
      for (int i = 0; i < VEC / 2; ++i) h2[i] = P::cvt(val[2 * i], val[2 * i + 1]);
      memcpy(hi, h2, sizeof(hi));
      store_some<Tout, VEC>(dst, hi, vec, avail);
      if (split) {
        // remainders x - b0 (and x - b0 - b1) are exact in fp32: each piece keeps the
        // leading 8 significant bits of what is left
        float rem[VEC];
        typename P::T l2[VEC / 2];
        Tout lo[VEC];
#pragma unroll
        for (int i = 0; i < VEC / 2; ++i) {
          const float2 h = P::back(h2[i]);
          rem[2 * i] = val[2 * i] - h.x;
          rem[2 * i + 1] = val[2 * i + 1] - h.y;
          if constexpr (S == kStoreF16)  // f16x3: the low piece is kept as 2^11 (x - h0)
            l2[i] = P::cvt(kF16LoScale * rem[2 * i], kF16LoScale * rem[2 * i + 1]);
          else
            l2[i] = P::cvt(rem[2 * i], rem[2 * i + 1]);
        }
        memcpy(lo, l2, sizeof(lo));
        store_some<Tout, VEC>(dst + kpanel, lo, vec, avail);
        if (S != kStoreF16 && split > 1) {
          typename P::T t2[VEC / 2];
          Tout lo2[VEC];
#pragma unroll
          for (int i = 0; i < VEC / 2; ++i) {
            const float2 l = P::back(l2[i]);
            t2[i] = P::cvt(rem[2 * i] - l.x, rem[2 * i + 1] - l.y);
          }
          memcpy(lo2, t2, sizeof(lo2));
          store_some<Tout, VEC>(dst + 2 * kpanel, lo2, vec, avail);
        }
      }
    } else {
      Tout hi[VEC];
#pragma unroll
      for (int v = 0; v < VEC; ++v) hi[v] = to_store<S>((double)val[v]);
      store_some<Tout, VEC>(dst, hi, vec, avail);
      if (split) {
        Tc rem[VEC];
        Tout lo[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          rem[v] = val[v] - (Tc)from_store<S>(hi[v]);
          lo[v] = to_store<S>(S == kStoreF16 ? (double)kF16LoScale * (double)rem[v] : (double)rem[v]);
        }
        store_some<Tout, VEC>(dst + kpanel, lo, vec, avail);
        if (S != kStoreF16 && split > 1) {
#pragma unroll
          for (int v = 0; v < VEC; ++v) lo[v] = to_store<S>((double)(rem[v] - (Tc)from_store<S>(lo[v])));
          store_some<Tout, VEC>(dst + 2 * kpanel, lo, vec, avail);
        }
      }
    }
  }
};

// Physical column x of a padded layout -> logical column (valid when x % seg < m).
__device__ __forceinline__ int64_t logical_col(int64_t x, int64_t seg, int64_t m) {
  const int64_t s = x / seg;
  return s * m + (x - s * seg);
}

// Grid: x over the physical positions of the output blocks taken row after row (rows of
// cols_out rounded up to VEC, so that a thread's VEC positions share a row and a column
// segment), z over parents.  Small blocks thus fill whole CTAs.  Padding positions encode
// zeros.
// FAST: every access of the launch is aligned and complete (vector loads and stores, and
// whole vectors of valid positions), so there are no per-element checks.
template <typename Tin, typename Tc, int N0, int G, int S, int VEC, bool FAST>
__global__ void __launch_bounds__(kThreadsX) encode_pass_kernel(const __grid_constant__ Tables<Tc> t,
                                                                const PassArgs a) {
  constexpr int W = cpow(N0, G);
  using Tout = typename StoreType<S>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Tc* coef = reinterpret_cast<Tc*>(smem_raw);
  const int64_t colsv = (a.cols_out + VEC - 1) / VEC * VEC;
  const int64_t pos = ((int64_t)blockIdx.x * kThreadsX + threadIdx.x) * VEC;
  const int64_t y = pos / colsv, x = pos - y * colsv;
  const bool inside = y < a.rows_out && x < a.cols_out;
  const int64_t outs = a.outs_per_parent;
  const int64_t xs = x % a.seg;                      // position inside its column segment
  const int64_t avail_in = a.mval - xs;              // valid positions from x on
  // source column offset of this position inside a sub-block
  const int64_t xsrc = a.plain ? logical_col(x, a.seg, a.mval) : x;
  const int64_t colstep = a.plain ? a.nb : a.xcol;   // sub-block column pitch in X
  for (int64_t p = blockIdx.z; p < a.parents; p += gridDim.z) {
    __syncthreads();  // the previous parent's readers are done with the tables
    expand_subtree(t, a, G, a.tensor, p, coef);
    __syncthreads();
    if (!inside) continue;
    EncodeEmitV<Tc, S, VEC> emit;
    emit.Y = static_cast<Tout*>(a.Y) + p * outs * a.strideY;
    emit.strideY = a.strideY;
    emit.off = y * a.ldy + x;
    emit.kpanel = a.kpanel;
    emit.split = a.split;
    emit.vec = FAST || a.vstore != 0;
    emit.avail = FAST ? VEC : a.cols_out - x;
    emit.set_scale(a, y, x);
    if (y >= a.nb || avail_in <= 0) {  // padding only: zero outputs
      Tc z[VEC];
#pragma unroll
      for (int v = 0; v < VEC; ++v) z[v] = (Tc)0;
      for (int64_t q = 0; q < outs; ++q) emit(q, z);
      continue;
    }
    const Tin* X = static_cast<const Tin*>(a.X) + p * a.strideX;
    const bool full = FAST || (a.vload && avail_in >= VEC);
    Tc in[W * W][VEC];
#pragma unroll
    for (int k = 0; k < W; ++k)
#pragma unroll
      for (int l = 0; l < W; ++l) {
        const Tin* src = X + (k * a.nb + y) * a.ldx + l * colstep + xsrc;
        Tin raw[VEC];
        if (full) {
          load_vec<Tin, VEC>(raw, src);
        } else {
#pragma unroll
          for (int v = 0; v < VEC; ++v) raw[v] = (v < avail_in) ? src[v] : (Tin)0;
        }
#pragma unroll
        for (int v = 0; v < VEC; ++v) in[k * W + l][v] = (Tc)raw[v];
      }
    EncodeWalk<Tc, N0, G, VEC>::go(coef, t.R, 0, 0, 0, in, emit);
  }
}

// Encode passes of TOP + 2 levels for n0 = 2 (fp32 arithmetic, R <= kTop3MaxR).  The first TOP
// levels (1 or 2) are split over the CTAs: CTA (tile, t) forms the node with path t at depth
// TOP at its positions straight from the parent's 2^(TOP+2) x 2^(TOP+2) blocks (the u^
// coefficients on the path are the same for the whole CTA, so zero terms load nothing), then
// walks the two levels below that node in registers like the two-level pass.  The R^TOP CTAs of
// one position tile are neighbours in the grid, so the parent's rows come from DRAM once and
// are re-read from L2: no intermediate of those levels is written or read.
// Shared tables (compact rows): 0 the node t, 1..R its children, R+1 the root, R+2 (TOP = 2)
// the first-level node on t's path.
template <int TOP>
struct TopRows {
  int R, t;
  __device__ __forceinline__ int operator()(int row) const {
    if (row == 0) return subtree_nodes(R, TOP) + t;
    if (row <= R) return subtree_nodes(R, TOP + 1) + t * R + (row - 1);
    if (row == R + 1) return 0;
    return 1 + t / R;  // TOP == 2: first-level node r1 of t = r1 * R + r2
  }
};
__host__ __device__ constexpr int top_rows(int R, int TOP) { return R + 1 + TOP; }

template <typename Tin, typename Tc, int S, int TOP, int VEC, bool FAST>
__global__ void __launch_bounds__(kThreadsX) encode_top_kernel(const __grid_constant__ Tables<Tc> t,
                                                               const PassArgs a) {
  constexpr int N0 = 2, WC = 4, NS = coef_stride(N0);
  using Tout = typename StoreType<S>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Tc* coef = reinterpret_cast<Tc*>(smem_raw);
  const int R = t.R;
  const int RT = TOP == 1 ? R : R * R;
  const int tp = (int)(blockIdx.x % (unsigned)RT);  // path of the first TOP levels
  const int64_t tile = blockIdx.x / (unsigned)RT;
  const int64_t colsv = (a.cols_out + VEC - 1) / VEC * VEC;
  const int64_t pos = (tile * kThreadsX + threadIdx.x) * VEC;
  const int64_t y = pos / colsv, x = pos - y * colsv;
  const bool inside = y < a.rows_out && x < a.cols_out;
  const int64_t outs = a.outs_per_parent;
  const int64_t xs = x % a.seg;
  const int64_t avail_in = a.mval - xs;
  const int64_t xsrc = a.plain ? logical_col(x, a.seg, a.mval) : x;
  const int64_t colstep = a.plain ? a.nb : a.xcol;
  for (int64_t p = blockIdx.z; p < a.parents; p += gridDim.z) {
    __syncthreads();
    expand_rows(t, a, top_rows(R, TOP), a.tensor, p, coef, TopRows<TOP>{R, tp});
    __syncthreads();
    if (!inside) continue;
    EncodeEmitV<Tc, S, VEC> emit;
    emit.Y = static_cast<Tout*>(a.Y) + p * outs * a.strideY;
    emit.strideY = a.strideY;
    emit.off = y * a.ldy + x;
    emit.kpanel = a.kpanel;
    emit.split = a.split;
    emit.vec = FAST || a.vstore != 0;
    emit.avail = FAST ? VEC : a.cols_out - x;
    emit.set_scale(a, y, x);
    if (y >= a.nb || avail_in <= 0) {  // padding only: zero outputs of the node's subtree
      Tc z[VEC];
#pragma unroll
      for (int v = 0; v < VEC; ++v) z[v] = (Tc)0;
      for (int64_t q = (int64_t)tp * R * R; q < (int64_t)(tp + 1) * R * R; ++q) emit(q, z);
      continue;
    }
    const Tin* X = static_cast<const Tin*>(a.X) + p * a.strideX;
    const bool full = FAST || (a.vload && avail_in >= VEC);
    Tc c1[NS], c2[NS];
    load_coefs<Tc, N0>(c1, coef + ((size_t)(R + 1) * R + (TOP == 1 ? tp : tp / R)) * NS);
    if constexpr (TOP == 2) load_coefs<Tc, N0>(c2, coef + ((size_t)(R + 2) * R + tp % R) * NS);
    Tc cin[WC * WC][VEC];
#pragma unroll
    for (int e = 0; e < WC * WC; ++e)
#pragma unroll
      for (int v = 0; v < VEC; ++v) cin[e][v] = (Tc)0;
    // quadrant (k, l) of the parent, and with TOP = 2 quadrant (k2, l2) inside it; a rolled
    // loop (16 vector loads in flight per term) keeps the register count of the two-level walk
#pragma unroll 1
    for (int kl = 0; kl < (TOP == 1 ? 4 : 16); ++kl) {
      const int k = TOP == 1 ? kl >> 1 : kl >> 3, l = TOP == 1 ? kl & 1 : (kl >> 2) & 1;
      const int k2 = TOP == 1 ? 0 : (kl >> 1) & 1, l2 = TOP == 1 ? 0 : kl & 1;
      const Tc cf = TOP == 1 ? c1[k * 2 + l] : c1[k * 2 + l] * c2[k2 * 2 + l2];
      if (cf == (Tc)0) continue;
      const int rb = TOP == 1 ? k * WC : k * 2 * WC + k2 * WC, cb = TOP == 1 ? l * WC : l * 2 * WC + l2 * WC;
#pragma unroll
      for (int u = 0; u < WC; ++u)
#pragma unroll
        for (int w = 0; w < WC; ++w) {
          const Tin* src = X + ((rb + u) * a.nb + y) * a.ldx + (cb + w) * colstep + xsrc;
          Tin raw[VEC];
          if (full) {
            load_vec<Tin, VEC>(raw, src);
          } else {
#pragma unroll
            for (int v = 0; v < VEC; ++v) raw[v] = (v < avail_in) ? src[v] : (Tin)0;
          }
#pragma unroll
          for (int v = 0; v < VEC; ++v) cin[u * WC + w][v] = cin[u * WC + w][v] + cf * (Tc)raw[v];
        }
    }
    // compact rows 0 (the node) and 1..R (its children) are the local ids of a two-level walk
    EncodeWalk<Tc, N0, 2, VEC>::go(coef, R, 0, 0, tp, cin, emit);
  }
}

// Final encode pass writing each output transposed (T^T, rows n, K contiguous), for tensor-core
// kinds that take both operands K-major.  The CTA owns 32 (x) x 8 (y) positions; every
// output goes through a double-buffered shared tile so that each warp stores runs of 8
// consecutive elements of a transposed row.  All threads walk the subtree (padding positions
// on zeros) so that every thread reaches the same barriers.
template <typename Tc, int S>
struct TransposedEmit {
  using Tout = typename StoreType<S>::T;
  Tc (*tile)[32][9];
  Tout* Y;
  int64_t strideY, ldy, kpanel, x0, y0;
  int split, tx, ty, tid, buf;
  __device__ __forceinline__ void operator()(int64_t path, const Tc (&val)[1]) {
    tile[buf][tx][ty] = val[0];
    __syncthreads();
    const int r = tid >> 3, c = tid & 7;
    const Tc w = tile[buf][r][c];
    Tout* dst = Y + path * strideY + (x0 + r) * ldy + (y0 + c);
    const Tout hi = to_store<S>((double)w);
    dst[0] = hi;
    if (split) {
      const Tc rem = w - (Tc)from_store<S>(hi);
      const Tout lo = to_store<S>((double)rem);
      dst[kpanel] = lo;
      if (split > 1) dst[2 * kpanel] = to_store<S>((double)(rem - (Tc)from_store<S>(lo)));
    }
    buf ^= 1;
  }
};

template <typename Tin, typename Tc, int N0, int G, int S>
__global__ void __launch_bounds__(256) encode_pass_trans_kernel(const __grid_constant__ Tables<Tc> t,
                                                               const PassArgs a) {
  constexpr int W = cpow(N0, G);
  using Tout = typename StoreType<S>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Tc* coef = reinterpret_cast<Tc*>(smem_raw);
  __shared__ Tc tile[2][32][9];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t x0 = (int64_t)blockIdx.x * 32, y0 = (int64_t)blockIdx.y * 8;
  const int64_t x = x0 + tx, y = y0 + ty;
  const bool valid = y < a.nb && x < a.mval;  // the final pass: one segment per leaf row
  const int64_t colstep = a.plain ? a.nb : a.xcol;
  for (int64_t p = blockIdx.z; p < a.parents; p += gridDim.z) {
    __syncthreads();
    expand_subtree(t, a, G, a.tensor, p, coef);
    __syncthreads();
    TransposedEmit<Tc, S> emit;
    emit.tile = tile;
    emit.Y = static_cast<Tout*>(a.Y) + p * a.outs_per_parent * a.strideY;
    emit.strideY = a.strideY;
    emit.ldy = a.ldy;
    emit.kpanel = a.kpanel;
    emit.x0 = x0;
    emit.y0 = y0;
    emit.split = a.split;
    emit.tx = tx;
    emit.ty = ty;
    emit.tid = ty * 32 + tx;
    emit.buf = 0;
    const Tin* X = static_cast<const Tin*>(a.X) + p * a.strideX;
    Tc in[W * W][1];
#pragma unroll
    for (int k = 0; k < W; ++k)
#pragma unroll
      for (int l = 0; l < W; ++l)
        in[k * W + l][0] = valid ? (Tc)X[(k * a.nb + y) * a.ldx + l * colstep + x] : (Tc)0;
    EncodeWalk<Tc, N0, G, 1>::go(coef, t.R, 0, 0, 0, in, emit);
  }
}

// ------------------------------------------------------------------ decode walk
template <typename Tc, int N0, int G, int VEC>
struct DecodeWalk {
  static constexpr int W = cpow(N0, G), WC = W / N0;
  template <class Fetch>
  __device__ __forceinline__ static void go(const Tc* coef, int R, int j, int q, int64_t path,
                                            Tc (&out)[W * W][VEC], Fetch& fetch) {
    constexpr int NS = coef_stride(N0);
    const Tc* row = coef + (size_t)local_id(R, j, q) * R * NS;
#pragma unroll
    for (int e = 0; e < W * W; ++e)
#pragma unroll
      for (int v = 0; v < VEC; ++v) out[e][v] = (Tc)0;
    for (int r = 0; r < R; ++r) {
      Tc cout[WC * WC][VEC];
      DecodeWalk<Tc, N0, G - 1, VEC>::go(coef, R, j + 1, q * R + r, path * R + r, cout, fetch);
      Tc c[NS];
      load_coefs<Tc, N0>(c, row + r * NS);
#pragma unroll
      for (int i = 0; i < N0; ++i)
#pragma unroll
        for (int jj = 0; jj < N0; ++jj) {
          const Tc wv = c[i * N0 + jj];
          if (use_coef(wv)) {
#pragma unroll
            for (int u = 0; u < WC; ++u)
#pragma unroll
              for (int w = 0; w < WC; ++w)
#pragma unroll
                for (int v = 0; v < VEC; ++v)
                  out[(i * WC + u) * W + (jj * WC + w)][v] =
                      out[(i * WC + u) * W + (jj * WC + w)][v] + wv * cout[u * WC + w][v];
          }
        }
    }
  }
};

// Bottom node: its R children are leaves of the walk; they are loaded eight at a time.
template <typename Tc, int N0, int VEC>
struct DecodeWalk<Tc, N0, 1, VEC> {
  static constexpr int W = N0;
  template <class Fetch>
  __device__ __forceinline__ static void go(const Tc* coef, int R, int j, int q, int64_t path,
                                            Tc (&out)[W * W][VEC], Fetch& fetch) {
    constexpr int NS = coef_stride(N0);
    const Tc* row = coef + (size_t)local_id(R, j, q) * R * NS;
#pragma unroll
    for (int e = 0; e < W * W; ++e)
#pragma unroll
      for (int v = 0; v < VEC; ++v) out[e][v] = (Tc)0;
    constexpr int B = 8;
    for (int r0 = 0; r0 < R; r0 += B) {
      Tc m[B][VEC];
#pragma unroll
      for (int b = 0; b < B; ++b)
        if (r0 + b < R) fetch(path * R + r0 + b, m[b]);
#pragma unroll
      for (int b = 0; b < B; ++b) {
        if (r0 + b < R) {
          Tc c[NS];
          load_coefs<Tc, N0>(c, row + (r0 + b) * NS);
#pragma unroll
          for (int e = 0; e < N0 * N0; ++e) {
            const Tc wv = c[e];
            if (use_coef(wv)) {
#pragma unroll
              for (int v = 0; v < VEC; ++v) out[e][v] = out[e][v] + wv * m[b][v];
            }
          }
        }
      }
    }
  }
};

template <typename Tm, typename Tc, int VEC>
struct DecodeFetch {
  const Tm* M;
  int64_t strideM, off, avail;
  bool vec;
  __device__ __forceinline__ void operator()(int64_t path, Tc (&dst)[VEC]) const {
    const Tm* src = M + path * strideM + off;
    Tm raw[VEC];
    if (vec && avail >= VEC) {
      load_vec<Tm, VEC>(raw, src);
    } else {
#pragma unroll
      for (int v = 0; v < VEC; ++v) raw[v] = v < avail ? src[v] : (Tm)0;
    }
#pragma unroll
    for (int v = 0; v < VEC; ++v) dst[v] = (Tc)raw[v];
  }
};

template <typename Tm, typename To, typename Tc, int N0, int G, int VEC, bool FAST>
__global__ void __launch_bounds__(kThreadsX) decode_pass_kernel(const __grid_constant__ Tables<Tc> t,
                                                                const PassArgs a) {
  constexpr int W = cpow(N0, G);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Tc* coef = reinterpret_cast<Tc*>(smem_raw);
  const int64_t colsv = (a.xcol + VEC - 1) / VEC * VEC;  // physical width of a child
  const int64_t pos = ((int64_t)blockIdx.x * kThreadsX + threadIdx.x) * VEC;
  const int64_t y = pos / colsv, x = pos - y * colsv;
  const int64_t xs = x % a.seg, avail = a.mval - xs;
  const bool valid = y < a.nb && x < a.xcol && avail > 0;
  // destination column inside a sub-block of the parent, and the sub-block column pitch
  const int64_t xdst = a.plain ? logical_col(x, a.seg, a.mval) : x;
  const int64_t colstep = a.plain ? a.nb : a.xcol;
  // recursive parents take whole vectors (padding lanes hold zeros and are never read)
  const int64_t avail_st = FAST ? VEC : (a.plain ? avail : VEC);
  for (int64_t p = blockIdx.z; p < a.parents; p += gridDim.z) {
    __syncthreads();
    expand_subtree(t, a, G, 2, p, coef);
    __syncthreads();
    if (!valid) continue;
    DecodeFetch<Tm, Tc, VEC> fetch;
    fetch.M = static_cast<const Tm*>(a.X) + p * a.outs_per_parent * a.strideX;
    fetch.strideM = a.strideX;
    fetch.off = y * a.ldx + x;
    fetch.avail = FAST ? VEC : avail;
    fetch.vec = FAST || a.vload != 0;
    Tc out[W * W][VEC];
    DecodeWalk<Tc, N0, G, VEC>::go(coef, t.R, 0, 0, 0, out, fetch);
    To* P = static_cast<To*>(a.Y) + p * a.strideY;
    const bool vs = FAST || a.vstore != 0;
#pragma unroll
    for (int k = 0; k < W; ++k)
#pragma unroll
      for (int l = 0; l < W; ++l) {
        To o[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) o[v] = (To)out[k * W + l][v];
        store_some<To, VEC>(P + (k * a.nb + y) * a.ldy + l * colstep + xdst, o, vs, avail_st);
      }
  }
}

// ------------------------------------------------------------------ sparse one-level decode
// One-level fp32 decode passes of formulas with n0 >= 3 (Laderman: 51 of 207 coefficients of
// W are nonzero).  Each child's nonzero coefficients are listed once per parent, in (i, j)
// order, and a thread's output accumulators sit in shared memory, where the lists index them.
// Every output sums over the children in the same order as the dense walk, without its zero
// terms, so the results are the same.  (The same scheme for the encode measured slower than
// the dense register walk, which keeps the encode dense.)
//
// Shared memory: [coef: R x NS][count: R][pairs: R x NN (entry, coefficient bits)]
//                [stage: NN x kThreadsX x VEC floats].
struct SparseSmem {
  size_t cnt, pairs, stage, total;
  __host__ __device__ SparseSmem(int R, int n0, int vec) {
    const int nn = n0 * n0, ns = coef_stride(n0);
    cnt = (size_t)R * ns * sizeof(float);                       // a multiple of 16 (ns % 4 == 0)
    pairs = cnt + ((size_t)R * sizeof(int) + 15) / 16 * 16;
    stage = pairs + ((size_t)R * nn * sizeof(int2) + 15) / 16 * 16;
    total = stage + (size_t)nn * kThreadsX * vec * sizeof(float);
  }
};

// Count and list the nonzero coefficients of every child (one-level subtree: node 0).
__device__ __forceinline__ void build_lists(const float* coef, int R, int n0, int* cnt, int2* pairs) {
  const int nn = n0 * n0, ns = coef_stride(n0);
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    int n = 0;
    for (int e = 0; e < nn; ++e) {
      const float c = coef[r * ns + e];
      if (c != 0.f) pairs[r * nn + n++] = make_int2(e, __float_as_int(c));
    }
    cnt[r] = n;
  }
}

template <int VEC>
__device__ __forceinline__ void stage_store(float* p, const float (&x)[VEC]) {
  store_vec<float, VEC>(p, x);
}
template <int VEC>
__device__ __forceinline__ void stage_load(float (&x)[VEC], const float* p) {
  load_vec<float, VEC>(x, p);
}

template <int N0, int VEC, bool FAST>
__global__ void __launch_bounds__(kThreadsX) decode_sparse_kernel(const __grid_constant__ Tables<float> t,
                                                                  const PassArgs a) {
  constexpr int NN = N0 * N0;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int R = t.R;
  const SparseSmem lay(R, N0, VEC);
  float* coef = reinterpret_cast<float*>(smem_raw);
  int* cnt = reinterpret_cast<int*>(smem_raw + lay.cnt);
  const int2* pairs = reinterpret_cast<const int2*>(smem_raw + lay.pairs);
  float* stage = reinterpret_cast<float*>(smem_raw + lay.stage) + threadIdx.x * VEC;
  const int64_t colsv = (a.xcol + VEC - 1) / VEC * VEC;
  const int64_t pos = ((int64_t)blockIdx.x * kThreadsX + threadIdx.x) * VEC;
  const int64_t y = pos / colsv, x = pos - y * colsv;
  const int64_t xs = x % a.seg, avail = a.mval - xs;
  const bool valid = y < a.nb && x < a.xcol && avail > 0;
  const int64_t xdst = a.plain ? logical_col(x, a.seg, a.mval) : x;
  const int64_t colstep = a.plain ? a.nb : a.xcol;
  const int64_t avail_st = FAST ? VEC : (a.plain ? avail : VEC);
  for (int64_t p = blockIdx.z; p < a.parents; p += gridDim.z) {
    __syncthreads();
    expand_subtree(t, a, 1, 2, p, coef);
    __syncthreads();
    build_lists(coef, R, N0, cnt, const_cast<int2*>(pairs));
    __syncthreads();
    if (!valid) continue;
    DecodeFetch<float, float, VEC> fetch;
    fetch.M = static_cast<const float*>(a.X) + p * a.outs_per_parent * a.strideX;
    fetch.strideM = a.strideX;
    fetch.off = y * a.ldx + x;
    fetch.avail = FAST ? VEC : avail;
    fetch.vec = FAST || a.vload != 0;
    {
      float z[VEC];
#pragma unroll
      for (int v = 0; v < VEC; ++v) z[v] = 0.f;
#pragma unroll
      for (int e = 0; e < NN; ++e) stage_store<VEC>(stage + e * kThreadsX * VEC, z);
    }
    constexpr int B = 4;  // children loaded together (8 spilled registers and measured slower)
    for (int r0 = 0; r0 < R; r0 += B) {
      float m[B][VEC];
#pragma unroll
      for (int b = 0; b < B; ++b)
        if (r0 + b < R) fetch(r0 + b, m[b]);
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int r = r0 + b, n = r < R ? cnt[r] : 0;
        for (int i = 0; i < n; ++i) {
          const int2 pr = pairs[r * NN + i];
          const float c = __int_as_float(pr.y);
          float* sp = stage + pr.x * kThreadsX * VEC;
          float acc[VEC];
          stage_load<VEC>(acc, sp);
#pragma unroll
          for (int v = 0; v < VEC; ++v) acc[v] = acc[v] + c * m[b][v];
          stage_store<VEC>(sp, acc);
        }
      }
    }
    float* P = static_cast<float*>(a.Y) + p * a.strideY;
    const bool vs = FAST || a.vstore != 0;
#pragma unroll
    for (int k = 0; k < N0; ++k)
#pragma unroll
      for (int l = 0; l < N0; ++l) {
        float o[VEC];
        stage_load<VEC>(o, stage + (k * N0 + l) * kThreadsX * VEC);
        store_some<float, VEC>(P + (k * a.nb + y) * a.ldy + l * colstep + xdst, o, vs, avail_st);
      }
  }
}

// ------------------------------------------------------------------ built-in formulas, one level
// One-level passes of the built-in formulas (Strassen, Laderman).  The node's signed
// permutations act on the operands, and the base formula's sparsity is compiled in:
//   S_r = sum_{k,l} u_{pi1(k) pi2(l) r} s1(k) s2(l) A_kl
//       = sum_{(k',l'): u_{k'l'r} != 0} u_{k'l'r} [s1(k) s2(l) A_kl]_{k = pi1^-1(k'), l = pi2^-1(l')}
// (likewise T_r with pi2, pi3, s2, s3), so a thread loads the sub-blocks in permuted order with
// their signs and adds the formula's nonzero terms; and
//   C_ij = scale s1(i) s3(j) D_{pi1(i) pi3(j)},   D_{i'j'} = sum_r w_{i'j'r} M_r,
// so the decode sums the nonzero terms of D (children in order) and stores D_{i'j'} into block
// (pi1^-1(i'), pi3^-1(j')).  No coefficient table is expanded and no zero term is evaluated.

template <int I, int N, class Fn>
__device__ __forceinline__ void static_for(Fn&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

// Draw set of launch parent p (the root of its one-level subtree).
template <typename Tc>
__device__ __forceinline__ uint64_t parent_draw(const Tables<Tc>& t, const PassArgs& a, int64_t p) {
  int64_t real = 0, hp = a.node_first + p;
  if (a.real_parents > 0) {
    real = p / a.real_parents;
    hp = a.node_first + (p - real * a.real_parents);
  }
  const uint64_t* draws = t.draw + real * a.real_draws;
  return t.per_level ? draws[a.depth] : draws[a.dbase[0] + (hp - a.dfirst[0])];
}

// inv[k'] = pi_c^-1(k') and sg[k'] = s_c(pi_c^-1(k')) of stream c of a draw set.
template <typename Tc, int N0>
__device__ __forceinline__ void inverse_stream(uint64_t w, int c, int (&inv)[N0], Tc (&sg)[N0]) {
#pragma unroll
  for (int kp = 0; kp < N0; ++kp) {
    int src = 0;
#pragma unroll
    for (int j = 0; j < N0; ++j)
      if (draw_perm(w, c, j) == kp) src = j;
    inv[kp] = src;
    sg[kp] = (Tc)draw_sign(w, c, src);
  }
}

template <typename Tin, typename Tc, class F, int TENSOR, int S, int VEC, bool FAST>
__global__ void __launch_bounds__(kThreadsX) encode_fixed_kernel(const __grid_constant__ Tables<Tc> t,
                                                                 const PassArgs a) {
  constexpr int N0 = F::n0, R = F::R, NN = N0 * N0;
  constexpr int CR = TENSOR == 1 ? 1 : 0, CC = TENSOR == 0 ? 1 : 2;  // row / column streams
  using Tout = typename StoreType<S>::T;
  const int64_t colsv = (a.cols_out + VEC - 1) / VEC * VEC;
  const int64_t pos = ((int64_t)blockIdx.x * kThreadsX + threadIdx.x) * VEC;
  const int64_t y = pos / colsv, x = pos - y * colsv;
  if (y >= a.rows_out || x >= a.cols_out) return;
  const int64_t outs = a.outs_per_parent;
  const int64_t xs = x % a.seg;
  const int64_t avail_in = a.mval - xs;
  const int64_t xsrc = a.plain ? logical_col(x, a.seg, a.mval) : x;
  const int64_t colstep = a.plain ? a.nb : a.xcol;
  const bool padding = y >= a.nb || avail_in <= 0;
  const bool full = FAST || (a.vload && avail_in >= VEC);
  for (int64_t p = blockIdx.z; p < a.parents; p += gridDim.z) {
    EncodeEmitV<Tc, S, VEC> emit;
    emit.Y = static_cast<Tout*>(a.Y) + p * outs * a.strideY;
    emit.strideY = a.strideY;
    emit.off = y * a.ldy + x;
    emit.kpanel = a.kpanel;
    emit.split = a.split;
    emit.vec = FAST || a.vstore != 0;
    emit.avail = FAST ? VEC : a.cols_out - x;
    emit.set_scale(a, y, x);
    if (padding) {  // zero outputs
      Tc z[VEC];
#pragma unroll
      for (int v = 0; v < VEC; ++v) z[v] = (Tc)0;
      for (int64_t q = 0; q < outs; ++q) emit(q, z);
      continue;
    }
    const uint64_t w = parent_draw(t, a, p);
    int ir[N0], ic[N0];
    Tc sr[N0], sc[N0];
    inverse_stream<Tc, N0>(w, CR, ir, sr);
    inverse_stream<Tc, N0>(w, CC, ic, sc);
    const Tin* X = static_cast<const Tin*>(a.X) + p * a.strideX;
    Tc in[NN][VEC];  // in[k' n0 + l'] = s s' X(pi^-1(k'), pi'^-1(l'))
#pragma unroll
    for (int kp = 0; kp < N0; ++kp)
#pragma unroll
      for (int lp = 0; lp < N0; ++lp) {
        const Tin* src = X + (ir[kp] * a.nb + y) * a.ldx + ic[lp] * colstep + xsrc;
        Tin raw[VEC];
        if (full) {
          load_vec<Tin, VEC>(raw, src);
        } else {
#pragma unroll
          for (int v = 0; v < VEC; ++v) raw[v] = (v < avail_in) ? src[v] : (Tin)0;
        }
        const Tc sg = sr[kp] * sc[lp];
#pragma unroll
        for (int v = 0; v < VEC; ++v) in[kp * N0 + lp][v] = sg * (Tc)raw[v];
      }
    static_for<0, R>([&](auto rr) {
      constexpr int r = decltype(rr)::value;
      Tc acc[VEC];
#pragma unroll
      for (int v = 0; v < VEC; ++v) acc[v] = (Tc)0;
      static_for<0, NN>([&](auto ee) {
        constexpr int e = decltype(ee)::value;
        constexpr int c = TENSOR == 0 ? F::U[e * R + r] : F::V[e * R + r];
        if constexpr (c != 0) {
#pragma unroll
          for (int v = 0; v < VEC; ++v) acc[v] = acc[v] + (Tc)c * in[e][v];
        }
      });
      emit(r, acc);
    });
  }
}

template <typename Tc, class F, int VEC, bool FAST>
__global__ void __launch_bounds__(kThreadsX) decode_fixed_kernel(const __grid_constant__ Tables<Tc> t,
                                                                 const PassArgs a) {
  constexpr int N0 = F::n0, R = F::R, NN = N0 * N0, B = 4;
  const int64_t colsv = (a.xcol + VEC - 1) / VEC * VEC;
  const int64_t pos = ((int64_t)blockIdx.x * kThreadsX + threadIdx.x) * VEC;
  const int64_t y = pos / colsv, x = pos - y * colsv;
  const int64_t xs = x % a.seg, avail = a.mval - xs;
  if (!(y < a.nb && x < a.xcol && avail > 0)) return;
  const int64_t xdst = a.plain ? logical_col(x, a.seg, a.mval) : x;
  const int64_t colstep = a.plain ? a.nb : a.xcol;
  const int64_t avail_st = FAST ? VEC : (a.plain ? avail : VEC);
  const bool vs = FAST || a.vstore != 0;
  for (int64_t p = blockIdx.z; p < a.parents; p += gridDim.z) {
    DecodeFetch<Tc, Tc, VEC> fetch;
    fetch.M = static_cast<const Tc*>(a.X) + p * a.outs_per_parent * a.strideX;
    fetch.strideM = a.strideX;
    fetch.off = y * a.ldx + x;
    fetch.avail = FAST ? VEC : avail;
    fetch.vec = FAST || a.vload != 0;
    Tc D[NN][VEC];
#pragma unroll
    for (int e = 0; e < NN; ++e)
#pragma unroll
      for (int v = 0; v < VEC; ++v) D[e][v] = (Tc)0;
    static_for<0, (R + B - 1) / B>([&](auto gg) {
      constexpr int r0 = decltype(gg)::value * B;
      Tc m[B][VEC];
      static_for<0, B>([&](auto bb) {
        constexpr int b = decltype(bb)::value;
        if constexpr (r0 + b < R) fetch(r0 + b, m[b]);
      });
      static_for<0, B>([&](auto bb) {
        constexpr int b = decltype(bb)::value;
        if constexpr (r0 + b < R) {
          static_for<0, NN>([&](auto ee) {
            constexpr int e = decltype(ee)::value;
            constexpr int c = F::W[e * R + r0 + b];
            if constexpr (c != 0) {
#pragma unroll
              for (int v = 0; v < VEC; ++v) D[e][v] = D[e][v] + (Tc)c * m[b][v];
            }
          });
        }
      });
    });
    const uint64_t w = parent_draw(t, a, p);
    int ir[N0], ic[N0];
    Tc sr[N0], sc[N0];
    inverse_stream<Tc, N0>(w, 0, ir, sr);
    inverse_stream<Tc, N0>(w, 2, ic, sc);
    Tc* P = static_cast<Tc*>(a.Y) + p * a.strideY;
#pragma unroll
    for (int ip = 0; ip < N0; ++ip)
#pragma unroll
      for (int jp = 0; jp < N0; ++jp) {
        const Tc f = t.scale * sr[ip] * sc[jp];
        Tc o[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) o[v] = f * D[ip * N0 + jp][v];
        store_some<Tc, VEC>(P + (ir[ip] * a.nb + y) * a.ldy + ic[jp] * colstep + xdst, o, vs, avail_st);
      }
  }
}

// ------------------------------------------------------------------ built-in formulas, two levels
// Two-level encode pass of a built-in formula with the intermediate level in shared memory.  A
// CTA owns kDeepPos consecutive output positions of one output row y, for one parent:
//   phase 1: thread (tau, g) -- tau = (k2, l2) one of the n0^2 sub-blocks of the second level,
//            g a group of four positions -- loads the n0^2 first-level blocks (k1, l1) at
//            sub-block tau (in the order of the parent's signed permutations, as the one-level
//            pass does), forms every first-level child S_r1 = sum u_{k'l'r1} [...] and writes it
//            to shared memory;
//   phase 2: thread (r1, g) reads the n0^2 sub-blocks of child r1 at its positions (in the order
//            of r1's own signed permutations) and forms the R grandchildren (r1, r2), the
//            outputs, stored in the leaf type.
// The first level's result never leaves the SM, so the pass moves the bytes of one level's
// input and the second level's output only.  Terms are the formula's nonzeros in the
// one-level passes' order.
constexpr int kDeepPos = 128;  // output positions per CTA (32 groups of four)

// Draw set of the node at relative depth j in {0, 1} below launch parent p with path q.
template <typename Tc>
__device__ __forceinline__ uint64_t subtree_draw(const Tables<Tc>& t, const PassArgs& a, int64_t p, int j, int q) {
  int64_t real = 0, hp = a.node_first + p;
  if (a.real_parents > 0) {
    real = p / a.real_parents;
    hp = a.node_first + (p - real * a.real_parents);
  }
  const uint64_t* draws = t.draw + real * a.real_draws;
  if (t.per_level) return draws[a.depth + j];
  const int64_t heap = j == 0 ? hp : hp * t.R + 1 + q;  // child q of hp: hp R + q + 1
  return draws[a.dbase[j] + (heap - a.dfirst[j])];
}

template <typename Tin, class F, int TENSOR, int S>
__global__ void __launch_bounds__(F::n0 * F::n0 * (kDeepPos / 4))
    encode_deep_kernel(const __grid_constant__ Tables<float> t, const PassArgs a) {
  constexpr int N0 = F::n0, R = F::R, NN = N0 * N0, VEC = 4, G = kDeepPos / VEC, THREADS = NN * G;
  constexpr int CR = TENSOR == 1 ? 1 : 0, CC = TENSOR == 0 ? 1 : 2;  // row / column streams
  using Tout = typename StoreType<S>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* inter = reinterpret_cast<float*>(smem_raw);  // [r1][tau][position]
  const int tid = threadIdx.x;
  const int64_t y = blockIdx.y, x0 = (int64_t)blockIdx.x * kDeepPos;
  const int64_t outs = a.outs_per_parent;  // R^2
  const int64_t colstep = a.plain ? a.nb : a.xcol;
  for (int64_t p = blockIdx.z; p < a.parents; p += gridDim.z) {
    Tout* Yp = static_cast<Tout*>(a.Y) + p * outs * a.strideY;
    auto emitter = [&](int64_t x) {
      EncodeEmitV<float, S, VEC> e;
      e.Y = Yp;
      e.strideY = a.strideY;
      e.off = y * a.ldy + x;
      e.kpanel = a.kpanel;
      e.split = a.split;
      e.vec = a.vstore != 0;
      e.avail = a.cols_out - x;
      e.set_scale(a, y, x);
      return e;
    };
    if (y >= a.nb) {  // a padding row of every output: zeros
      const float z[VEC] = {};
      for (int item = tid; item < R * G; item += THREADS) {
        const int r1 = item / G, g = item - r1 * G;
        const int64_t x = x0 + g * VEC;
        if (x >= a.cols_out) continue;
        EncodeEmitV<float, S, VEC> emit = emitter(x);
        for (int r2 = 0; r2 < R; ++r2) emit(r1 * R + r2, z);
      }
      continue;
    }
    // ---- phase 1: first level into shared memory
    {
      const int tau = tid / G, g = tid - tau * G;
      const int k2 = tau / N0, l2 = tau - k2 * N0;
      const int64_t x = x0 + g * VEC;
      const int64_t xs = x % a.seg, avail_in = a.mval - xs;
      float in[NN][VEC];
      if (x < a.cols_out && avail_in > 0) {
        const uint64_t w = subtree_draw(t, a, p, 0, 0);
        int ir[N0], ic[N0];
        float sr[N0], sc[N0];
        inverse_stream<float, N0>(w, CR, ir, sr);
        inverse_stream<float, N0>(w, CC, ic, sc);
        const Tin* X = static_cast<const Tin*>(a.X) + p * a.strideX;
        const int64_t xsrc = a.plain ? logical_col(x, a.seg, a.mval) : x;
        const bool full = a.vload && avail_in >= VEC;
#pragma unroll
        for (int kp = 0; kp < N0; ++kp)
#pragma unroll
          for (int lp = 0; lp < N0; ++lp) {
            const Tin* src = X + ((ir[kp] * N0 + k2) * a.nb + y) * a.ldx + (ic[lp] * N0 + l2) * colstep + xsrc;
            Tin raw[VEC];
            if (full) {
              load_vec<Tin, VEC>(raw, src);
            } else {
#pragma unroll
              for (int v = 0; v < VEC; ++v) raw[v] = (v < avail_in) ? src[v] : (Tin)0;
            }
            const float sg = sr[kp] * sc[lp];
#pragma unroll
            for (int v = 0; v < VEC; ++v) in[kp * N0 + lp][v] = sg * (float)raw[v];
          }
      } else {
#pragma unroll
        for (int e = 0; e < NN; ++e)
#pragma unroll
          for (int v = 0; v < VEC; ++v) in[e][v] = 0.f;
      }
      static_for<0, R>([&](auto rr) {
        constexpr int r = decltype(rr)::value;
        float acc[VEC] = {};
        static_for<0, NN>([&](auto ee) {
          constexpr int e = decltype(ee)::value;
          constexpr int c = TENSOR == 0 ? F::U[e * R + r] : F::V[e * R + r];
          if constexpr (c != 0) {
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[v] = acc[v] + (float)c * in[e][v];
          }
        });
        *reinterpret_cast<float4*>(inter + ((size_t)(r * NN + tau) * kDeepPos + g * VEC)) =
            make_float4(acc[0], acc[1], acc[2], acc[3]);
      });
    }
    __syncthreads();
    // ---- phase 2: second level from shared memory to the outputs
    for (int item = tid; item < R * G; item += THREADS) {
      const int r1 = item / G, g = item - r1 * G;
      const int64_t x = x0 + g * VEC;
      if (x >= a.cols_out) continue;
      const uint64_t w = subtree_draw(t, a, p, 1, r1);
      int ir[N0], ic[N0];
      float sr[N0], sc[N0];
      inverse_stream<float, N0>(w, CR, ir, sr);
      inverse_stream<float, N0>(w, CC, ic, sc);
      float in[NN][VEC];
#pragma unroll
      for (int kp = 0; kp < N0; ++kp)
#pragma unroll
        for (int lp = 0; lp < N0; ++lp) {
          const float4 v4 = *reinterpret_cast<const float4*>(
              inter + ((size_t)(r1 * NN + ir[kp] * N0 + ic[lp]) * kDeepPos + g * VEC));
          const float sg = sr[kp] * sc[lp];
          in[kp * N0 + lp][0] = sg * v4.x;
          in[kp * N0 + lp][1] = sg * v4.y;
          in[kp * N0 + lp][2] = sg * v4.z;
          in[kp * N0 + lp][3] = sg * v4.w;
        }
      EncodeEmitV<float, S, VEC> emit = emitter(x);
      static_for<0, R>([&](auto rr) {
        constexpr int r = decltype(rr)::value;
        float acc[VEC] = {};
        static_for<0, NN>([&](auto ee) {
          constexpr int e = decltype(ee)::value;
          constexpr int c = TENSOR == 0 ? F::U[e * R + r] : F::V[e * R + r];
          if constexpr (c != 0) {
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[v] = acc[v] + (float)c * in[e][v];
          }
        });
        emit(r1 * R + r, acc);
      });
    }
    __syncthreads();  // shared memory is reused by the next parent
  }
}

// Two-level decode pass of a built-in formula with the lower level handed over in shared memory.
// A CTA owns POS consecutive positions of one child row y, for one parent:
//   phase 1: item (r1, g) loads the R grandchildren (r1, r2) at its four positions (all R loads
//            in flight at once), forms child r1's n0^2 blocks D_{i'j'} = sum_r2 w_{i'j'r2} M_(r1, r2)
//            (r2 in order) and writes each, scaled and signed by r1's draws, to its sub-block
//            (pi1^-1(i'), pi3^-1(j')) in shared memory;
//   phase 2: item (tau, g) -- tau one of the n0^2 sub-blocks -- forms the parent's blocks
//            sum_r1 w_{i'j'r1} child_r1[tau] (r1 in order) and stores them.
// Small per-thread state (one child's R loads, n0^2 sums) keeps many CTAs, and so many loads, in
// flight per SM.  The sums run over the formula's nonzeros in the one-level passes' order.
template <class F, int POS>
__global__ void __launch_bounds__(kThreadsX) decode_deep_kernel(const __grid_constant__ Tables<float> t,
                                                                const PassArgs a) {
  constexpr int N0 = F::n0, R = F::R, NN = N0 * N0, VEC = 4, G = POS / VEC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* inter = reinterpret_cast<float*>(smem_raw);  // [r1][tau][position]
  const int tid = threadIdx.x;
  const int64_t y = blockIdx.y, x0 = (int64_t)blockIdx.x * POS;
  const int64_t colstep = a.plain ? a.nb : a.xcol;
  for (int64_t p = blockIdx.z; p < a.parents; p += gridDim.z) {
    // ---- phase 1: the lower level of each child r1 into shared memory
    for (int item = tid; item < R * G; item += kThreadsX) {
      const int r1 = item / G, g = item - r1 * G;
      const int64_t x = x0 + g * VEC;
      const int64_t xs = x % a.seg, avail = a.mval - xs;
      if (x >= a.xcol || avail <= 0) continue;
      DecodeFetch<float, float, VEC> fetch;
      fetch.M = static_cast<const float*>(a.X) + (p * a.outs_per_parent + (int64_t)r1 * R) * a.strideX;
      fetch.strideM = a.strideX;
      fetch.off = y * a.ldx + x;
      fetch.avail = avail;
      fetch.vec = a.vload != 0;
      float m[R][VEC];
      static_for<0, R>([&](auto rr) { fetch(decltype(rr)::value, m[decltype(rr)::value]); });
      float D[NN][VEC] = {};
      static_for<0, R>([&](auto rr) {
        constexpr int r = decltype(rr)::value;
        static_for<0, NN>([&](auto ee) {
          constexpr int e = decltype(ee)::value;
          constexpr int c = F::W[e * R + r];
          if constexpr (c != 0) {
#pragma unroll
            for (int v = 0; v < VEC; ++v) D[e][v] = D[e][v] + (float)c * m[r][v];
          }
        });
      });
      const uint64_t w = subtree_draw(t, a, p, 1, r1);
      int ir[N0], ic[N0];
      float sr[N0], sc[N0];
      inverse_stream<float, N0>(w, 0, ir, sr);
      inverse_stream<float, N0>(w, 2, ic, sc);
#pragma unroll
      for (int ip = 0; ip < N0; ++ip)
#pragma unroll
        for (int jp = 0; jp < N0; ++jp) {
          const float f = t.scale * sr[ip] * sc[jp];
          const int e = ip * N0 + jp;
          *reinterpret_cast<float4*>(inter + ((size_t)(r1 * NN + ir[ip] * N0 + ic[jp]) * POS + g * VEC)) =
              make_float4(f * D[e][0], f * D[e][1], f * D[e][2], f * D[e][3]);
        }
    }
    __syncthreads();
    // ---- phase 2: the parent's level from shared memory
    for (int item = tid; item < NN * G; item += kThreadsX) {
      const int tau = item / G, g = item - tau * G;
      const int i2 = tau / N0, j2 = tau - i2 * N0;
      const int64_t x = x0 + g * VEC;
      const int64_t xs = x % a.seg, avail = a.mval - xs;
      if (x >= a.xcol || avail <= 0) continue;
      float D[NN][VEC] = {};
      static_for<0, R>([&](auto rr) {
        constexpr int r = decltype(rr)::value;
        const float4 v4 = *reinterpret_cast<const float4*>(inter + ((size_t)(r * NN + tau) * POS + g * VEC));
        const float mv[VEC] = {v4.x, v4.y, v4.z, v4.w};
        static_for<0, NN>([&](auto ee) {
          constexpr int e = decltype(ee)::value;
          constexpr int c = F::W[e * R + r];
          if constexpr (c != 0) {
#pragma unroll
            for (int v = 0; v < VEC; ++v) D[e][v] = D[e][v] + (float)c * mv[v];
          }
        });
      });
      const uint64_t w = subtree_draw(t, a, p, 0, 0);
      int ir[N0], ic[N0];
      float sr[N0], sc[N0];
      inverse_stream<float, N0>(w, 0, ir, sr);
      inverse_stream<float, N0>(w, 2, ic, sc);
      float* P = static_cast<float*>(a.Y) + p * a.strideY;
      const int64_t xdst = a.plain ? logical_col(x, a.seg, a.mval) : x;
      const int64_t avail_st = a.plain ? avail : VEC;
      const bool vs = a.vstore != 0;
#pragma unroll
      for (int ip = 0; ip < N0; ++ip)
#pragma unroll
        for (int jp = 0; jp < N0; ++jp) {
          const float f = t.scale * sr[ip] * sc[jp];
          float o[VEC];
#pragma unroll
          for (int v = 0; v < VEC; ++v) o[v] = f * D[ip * N0 + jp][v];
          store_some<float, VEC>(P + ((ir[ip] * N0 + i2) * a.nb + y) * a.ldy + (ic[jp] * N0 + j2) * colstep + xdst,
                                 o, vs, avail_st);
        }
    }
    __syncthreads();  // shared memory is reused by the next parent
  }
}

inline dim3 pass_grid(int64_t rows, int64_t cols, int64_t parents, int vec) {
  const int64_t gz = parents < 65535 ? parents : 65535;
  const int64_t span = (int64_t)kThreadsX * vec;
  const int64_t positions = rows * ((cols + vec - 1) / vec * vec);
  return dim3((unsigned)((positions + span - 1) / span), 1, (unsigned)gz);
}

template <typename K>
cudaError_t prep(K kern, size_t smem) {
  if (smem > 48 * 1024) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

inline bool aligned(const void* p, size_t bytes) { return ((uintptr_t)p % bytes) == 0; }

template <typename Tin, typename Tc, int S, int N0, int G>
cudaError_t enc_one(const Tables<Tc>& t, const PassArgs& a_in, cudaStream_t st) {
  using Tout = typename StoreType<S>::T;
  const size_t smem = (size_t)subtree_nodes(t.R, G) * t.R * coef_stride(N0) * sizeof(Tc);
  if (a_in.trans) {
    if (a_in.rows_out % 8 || a_in.cols_out % 32 || a_in.rows_out != a_in.cols_out) return cudaErrorInvalidValue;
    const int64_t gz = a_in.parents < 65535 ? a_in.parents : 65535;
    const dim3 grid((unsigned)(a_in.cols_out / 32), (unsigned)(a_in.rows_out / 8), (unsigned)gz), block(32, 8);
    auto kern = encode_pass_trans_kernel<Tin, Tc, N0, G, S>;
    cudaError_t e = prep(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, block, smem, st>>>(t, a_in);
    return cudaGetLastError();
  }
  constexpr int VEC = Vec<Tc, N0, G>::value;
  PassArgs a = a_in;
  if (a.seg <= 0 || a.seg % 4 || a.mval <= 0 || a.mval > a.seg) return cudaErrorInvalidValue;
  // a plain input's columns are aligned when every segment starts aligned (or there is one)
  const bool xalign = a.plain ? (a.nb % VEC == 0 && (a.mval % VEC == 0 || a.cols_out <= a.seg)) : a.xcol % VEC == 0;
  a.vload = xalign && a.ldx % VEC == 0 && a.strideX % VEC == 0 && aligned(a.X, VEC * sizeof(Tin));
  a.vstore = a.ldy % VEC == 0 && a.strideY % VEC == 0 && a.kpanel % VEC == 0 && aligned(a.Y, VEC * sizeof(Tout));
  // The passes write zeros into every padding column of the intermediates, so whole vectors
  // read from a padded-layout input are exact even where they run past the valid columns.
  const bool fast = a.vload && a.vstore && a.cols_out % VEC == 0 && (a.plain ? a.mval % VEC == 0 : true);
  if constexpr (G == 2 && N0 == 3 && std::is_same_v<Tc, float>) {
    if (a.formula == LadermanFormula::id) {
      using F = LadermanFormula;
      constexpr int threads = F::n0 * F::n0 * (kDeepPos / 4);
      const size_t smem_deep = (size_t)F::R * F::n0 * F::n0 * kDeepPos * sizeof(float);
      const int64_t gz = a.parents < 65535 ? a.parents : 65535;
      if (a.rows_out > 65535) return cudaErrorInvalidValue;
      const dim3 grid((unsigned)((a.cols_out + kDeepPos - 1) / kDeepPos), (unsigned)a.rows_out, (unsigned)gz);
      // four positions per thread: alignment for 16-byte loads and 4-element stores
      const bool x4 = a.plain ? (a.nb % 4 == 0 && (a.mval % 4 == 0 || a.cols_out <= a.seg)) : a.xcol % 4 == 0;
      a.vload = x4 && a.ldx % 4 == 0 && a.strideX % 4 == 0 && aligned(a.X, 4 * sizeof(Tin));
      a.vstore = a.ldy % 4 == 0 && a.strideY % 4 == 0 && a.kpanel % 4 == 0 && aligned(a.Y, 4 * sizeof(Tout));
      auto kern = a.tensor == 0 ? encode_deep_kernel<Tin, F, 0, S> : encode_deep_kernel<Tin, F, 1, S>;
      cudaError_t e = prep(kern, smem_deep);
      if (e != cudaSuccess) return e;
      kern<<<grid, threads, smem_deep, st>>>(t, a);
      return cudaGetLastError();
    }
  }
  if constexpr (G == 1 && (N0 == 2 || N0 == 3)) {
    using F = std::conditional_t<N0 == 2, StrassenFormula, LadermanFormula>;
    if (a.formula == F::id) {
      const dim3 grid = pass_grid(a.rows_out, a.cols_out, a.parents, VEC);
      if (a.tensor == 0) {
        if (fast) encode_fixed_kernel<Tin, Tc, F, 0, S, VEC, true><<<grid, kThreadsX, 0, st>>>(t, a);
        else encode_fixed_kernel<Tin, Tc, F, 0, S, VEC, false><<<grid, kThreadsX, 0, st>>>(t, a);
      } else {
        if (fast) encode_fixed_kernel<Tin, Tc, F, 1, S, VEC, true><<<grid, kThreadsX, 0, st>>>(t, a);
        else encode_fixed_kernel<Tin, Tc, F, 1, S, VEC, false><<<grid, kThreadsX, 0, st>>>(t, a);
      }
      return cudaGetLastError();
    }
  }
  auto kern = fast ? encode_pass_kernel<Tin, Tc, N0, G, S, VEC, true> : encode_pass_kernel<Tin, Tc, N0, G, S, VEC, false>;
  cudaError_t e = prep(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<pass_grid(a.rows_out, a.cols_out, a.parents, VEC), kThreadsX, smem, st>>>(t, a);
  return cudaGetLastError();
}

// Passes of TOP + 2 levels for n0 = 2 in fp32 (encode_top_kernel): four positions per thread, as
// in the two-level pass.
template <typename Tin, int S, int TOP>
cudaError_t enc_top(const Tables<float>& t, const PassArgs& a_in, cudaStream_t st) {
  using Tout = typename StoreType<S>::T;
  constexpr int N0 = 2, VEC = Vec<float, 2, 2>::value;
  if (a_in.trans || t.R > kTop3MaxR) return cudaErrorInvalidValue;
  PassArgs a = a_in;
  if (a.seg <= 0 || a.seg % 4 || a.mval <= 0 || a.mval > a.seg) return cudaErrorInvalidValue;
  const int RT = TOP == 1 ? t.R : t.R * t.R;
  const size_t smem = (size_t)top_rows(t.R, TOP) * t.R * coef_stride(N0) * sizeof(float);
  const bool xalign = a.plain ? (a.nb % VEC == 0 && (a.mval % VEC == 0 || a.cols_out <= a.seg)) : a.xcol % VEC == 0;
  a.vload = xalign && a.ldx % VEC == 0 && a.strideX % VEC == 0 && aligned(a.X, VEC * sizeof(Tin));
  a.vstore = a.ldy % VEC == 0 && a.strideY % VEC == 0 && a.kpanel % VEC == 0 && aligned(a.Y, VEC * sizeof(Tout));
  const bool fast = a.vload && a.vstore && a.cols_out % VEC == 0 && (a.plain ? a.mval % VEC == 0 : true);
  dim3 grid = pass_grid(a.rows_out, a.cols_out, a.parents, VEC);
  if ((uint64_t)grid.x * (uint64_t)RT > 0x7fffffffull) return cudaErrorInvalidValue;
  grid.x *= (unsigned)RT;
  auto kern = fast ? encode_top_kernel<Tin, float, S, TOP, VEC, true> : encode_top_kernel<Tin, float, S, TOP, VEC, false>;
  cudaError_t e = prep(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreadsX, smem, st>>>(t, a);
  return cudaGetLastError();
}

template <typename Tin, typename Tc, int S, int N0>
cudaError_t enc_g(const Tables<Tc>& t, const PassArgs& a, int g, cudaStream_t st) {
  switch (g) {
    case 1: return enc_one<Tin, Tc, S, N0, 1>(t, a, st);
    case 2:
      if constexpr (N0 <= 3) return enc_one<Tin, Tc, S, N0, 2>(t, a, st);
      break;
    case 3:
      if constexpr (N0 == 2 && std::is_same_v<Tc, float>) return enc_top<Tin, S, 1>(t, a, st);
      break;
    case 4:
      if constexpr (N0 == 2 && std::is_same_v<Tc, float>) return enc_top<Tin, S, 2>(t, a, st);
      break;
  }
  return cudaErrorInvalidValue;
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

template <typename Tm, typename To, typename Tc, int N0, int G>
cudaError_t dec_one(const Tables<Tc>& t, const PassArgs& a_in, cudaStream_t st) {
  constexpr int VEC = Vec<Tc, N0, G>::value;
  const size_t smem = (size_t)subtree_nodes(t.R, G) * t.R * coef_stride(N0) * sizeof(Tc);
  PassArgs a = a_in;
  if (a.seg <= 0 || a.seg % 4 || a.mval <= 0 || a.mval > a.seg || a.xcol % a.seg) return cudaErrorInvalidValue;
  const bool yalign = a.plain ? (a.nb % VEC == 0 && (a.mval % VEC == 0 || a.xcol <= a.seg)) : true;
  a.vload = a.ldx % VEC == 0 && a.strideX % VEC == 0 && aligned(a.X, VEC * sizeof(Tm));
  a.vstore = yalign && a.ldy % VEC == 0 && a.strideY % VEC == 0 && aligned(a.Y, VEC * sizeof(To));
  // Children (leaf products and padded-layout intermediates) hold zeros in their padding
  // columns, so whole-vector loads are exact; a padded-layout parent takes whole-vector
  // stores, a plain one (C) only complete vectors.
  const bool fast = a.vload && a.vstore && (a.plain ? a.mval % VEC == 0 : true);
  if constexpr (G == 2 && (N0 == 2 || N0 == 3) && std::is_same_v<Tc, float> && std::is_same_v<Tm, float> &&
                std::is_same_v<To, float>) {
    using F = std::conditional_t<N0 == 2, StrassenFormula, LadermanFormula>;
    if (a.formula == F::id) {
      constexpr int POS = N0 == 2 ? 128 : 64;  // positions per CTA (shared memory R n0^2 POS floats)
      const size_t smem_deep = (size_t)F::R * F::n0 * F::n0 * POS * sizeof(float);
      const int64_t gz = a.parents < 65535 ? a.parents : 65535;
      if (a.nb > 65535) return cudaErrorInvalidValue;
      const dim3 grid((unsigned)((a.xcol + POS - 1) / POS), (unsigned)a.nb, (unsigned)gz);
      // four positions per thread: alignment for 16-byte loads and stores
      const bool y4 = a.plain ? (a.nb % 4 == 0 && (a.mval % 4 == 0 || a.xcol <= a.seg)) : true;
      a.vload = a.ldx % 4 == 0 && a.strideX % 4 == 0 && aligned(a.X, 16);
      a.vstore = y4 && a.ldy % 4 == 0 && a.strideY % 4 == 0 && aligned(a.Y, 16);
      auto kern = decode_deep_kernel<F, POS>;
      cudaError_t e = prep(kern, smem_deep);
      if (e != cudaSuccess) return e;
      kern<<<grid, kThreadsX, smem_deep, st>>>(t, a);
      return cudaGetLastError();
    }
  }
  if constexpr (G == 1 && (N0 == 2 || N0 == 3) && std::is_same_v<Tm, Tc> && std::is_same_v<To, Tc>) {
    using F = std::conditional_t<N0 == 2, StrassenFormula, LadermanFormula>;
    if (a.formula == F::id) {
      const dim3 grid = pass_grid(a.nb, a.xcol, a.parents, VEC);
      if (fast) decode_fixed_kernel<Tc, F, VEC, true><<<grid, kThreadsX, 0, st>>>(t, a);
      else decode_fixed_kernel<Tc, F, VEC, false><<<grid, kThreadsX, 0, st>>>(t, a);
      return cudaGetLastError();
    }
  }
  if constexpr (sizeof(Tc) == 4 && sizeof(Tm) == 4 && sizeof(To) == 4 && G == 1 && N0 >= 3) {
    const SparseSmem lay(t.R, N0, VEC);
    auto kern = fast ? decode_sparse_kernel<N0, VEC, true> : decode_sparse_kernel<N0, VEC, false>;
    cudaError_t e = prep(kern, lay.total);
    if (e != cudaSuccess) return e;
    kern<<<pass_grid(a.nb, a.xcol, a.parents, VEC), kThreadsX, lay.total, st>>>(t, a);
    return cudaGetLastError();
  }
  auto kern = fast ? decode_pass_kernel<Tm, To, Tc, N0, G, VEC, true> : decode_pass_kernel<Tm, To, Tc, N0, G, VEC, false>;
  cudaError_t e = prep(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<pass_grid(a.nb, a.xcol, a.parents, VEC), kThreadsX, smem, st>>>(t, a);
  return cudaGetLastError();
}

template <typename Tm, typename To, typename Tc, int N0>
cudaError_t dec_g(const Tables<Tc>& t, const PassArgs& a, int g, cudaStream_t st) {
  switch (g) {
    case 1: return dec_one<Tm, To, Tc, N0, 1>(t, a, st);
    case 2:
      if constexpr (N0 <= 3) return dec_one<Tm, To, Tc, N0, 2>(t, a, st);
      break;
    case 3:
      if constexpr (N0 == 2) return dec_one<Tm, To, Tc, N0, 3>(t, a, st);
      break;
  }
  return cudaErrorInvalidValue;
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

// Identity "encode" of the single leaf when L = 0: conversion, padding and split panels
// (output position (y, x), or (x, y) when a.trans: then the block is read down columns).
template <typename Tin, int S>
__global__ void __launch_bounds__(kThreadsX) copy_leaf_kernel(const PassArgs a) {
  using Tout = typename StoreType<S>::T;
  const int64_t pos = (int64_t)blockIdx.x * kThreadsX + threadIdx.x;  // row after row
  const int64_t y = pos / a.cols_out, x = pos - y * a.cols_out;
  if (y >= a.rows_out) return;
  const Tin* X = static_cast<const Tin*>(a.X);
  const int64_t sy = a.trans ? x : y, sx = a.trans ? y : x;  // source entry
  double v = (sy < a.nb && sx < a.nb) ? (double)X[sy * a.ldx + sx] : 0.0;
  if (a.lscale) v *= (double)a.lscale[a.tensor == 0 ? y : x];  // f16x3: a power of two, exact
  Tout* dst = static_cast<Tout*>(a.Y) + y * a.ldy + x;
  const Tout hi = to_store<S>(v);
  dst[0] = hi;
  if (a.split) {
    // v holds an fp32 value: the remainders below are exact
    const double rem = v - from_store<S>(hi);
    if (S == kStoreF16) {  // f16x3: the low piece is kept as 2^11 (x - h0)
      dst[a.kpanel] = to_store<S>((double)kF16LoScale * rem);
      return;
    }
    const Tout lo = to_store<S>(rem);
    dst[a.kpanel] = lo;
    if (a.split > 1) dst[2 * a.kpanel] = to_store<S>(rem - from_store<S>(lo));
  }
}

}  // namespace

namespace {

// ------------------------------------------------------------------ f16x3 leaf operand scales
// Largest |entry| of each class of rows of A (rows i == r mod m, over all columns) and of each
// class of columns of B (columns j == c mod m, over all rows), N x N fp32, as fp32 bit patterns
// (non-negative floats order like their bits) gathered with atomicMax; blockIdx.z = 0 takes A,
// 1 takes B.  A CTA covers 32 rows x 1024 columns; with V4 every thread reads 16-byte vectors
// (8 per row of A, 32 rows of 4 columns of B), all loads of a thread issued before any max.
constexpr int kAmaxRows = 32, kAmaxCols = 1024;
template <bool V4>
__global__ void __launch_bounds__(256) fold_absmax_kernel(const float* __restrict__ A, int64_t lda,
                                                          const float* __restrict__ B, int64_t ldb, int64_t N,
                                                          int64_t m, unsigned* __restrict__ amaxA,
                                                          unsigned* __restrict__ amaxB) {
  const int64_t r0 = (int64_t)blockIdx.y * kAmaxRows, c0 = (int64_t)blockIdx.x * kAmaxCols;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (blockIdx.z == 0) {
    // warp w: rows r0 + w + 8 i; lanes stride the columns
#pragma unroll 1
    for (int rr = warp; rr < kAmaxRows; rr += 8) {
      const int64_t r = r0 + rr;
      if (r >= N) break;
      const float* row = A + r * lda;
      float mx = 0.f;
      if constexpr (V4) {
        float4 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int64_t c = c0 + 4 * (lane + 32 * q);
          v[q] = c < N ? *reinterpret_cast<const float4*>(row + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
          mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v[q].x), fabsf(v[q].y)), fmaxf(fabsf(v[q].z), fabsf(v[q].w))));
      } else {
        for (int64_t c = c0 + lane; c < c0 + kAmaxCols && c < N; c += 32) mx = fmaxf(mx, fabsf(row[c]));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0 && mx > 0.f) atomicMax(amaxA + r % m, __float_as_uint(mx));
    }
  } else {
    if constexpr (V4) {
      // thread t: columns c0 + 4t .. c0 + 4t + 3 over the CTA's 32 rows
      const int64_t c = c0 + 4 * threadIdx.x;
      if (c >= N) return;
      float4 mx = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 8
      for (int rr = 0; rr < kAmaxRows; ++rr) {
        const int64_t r = r0 + rr;
        if (r >= N) break;
        const float4 v = *reinterpret_cast<const float4*>(B + r * ldb + c);
        mx = make_float4(fmaxf(mx.x, fabsf(v.x)), fmaxf(mx.y, fabsf(v.y)), fmaxf(mx.z, fabsf(v.z)),
                         fmaxf(mx.w, fabsf(v.w)));
      }
      const float e[4] = {mx.x, mx.y, mx.z, mx.w};
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (e[q] > 0.f) atomicMax(amaxB + (c + q) % m, __float_as_uint(e[q]));
    } else {
      for (int64_t c = c0 + threadIdx.x; c < c0 + kAmaxCols && c < N; c += 256) {
        float mx = 0.f;
        for (int64_t r = r0; r < r0 + kAmaxRows && r < N; ++r) mx = fmaxf(mx, fabsf(B[r * ldb + c]));
        if (mx > 0.f) atomicMax(amaxB + c % m, __float_as_uint(mx));
      }
    }
  }
}

__global__ void leaf_scales_kernel(const unsigned* __restrict__ amax, int64_t m, int64_t mp, double growth,
                                   float* __restrict__ scale, float* __restrict__ inv) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= mp) return;
  int e = 0;
  if (r < m) {
    // in fp64: the largest fp32 entries times the growth bound stay finite
    const double t = (double)__uint_as_float(amax[r]) * growth;
    if (t > 0.0) {
      int ex;
      frexp(t, &ex);  // t < 2^ex
      e = min(max(15 - ex, -126), 126);  // 2^e and 2^-e are normal fp32 numbers
    }
  }
  scale[r] = ldexpf(1.f, e);
  inv[r] = ldexpf(1.f, -e);
}

}  // namespace

cudaError_t launch_fold_absmax(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t N, int64_t m,
                               unsigned* amaxA, unsigned* amaxB, cudaStream_t st) {
  if (N <= 0 || m <= 0 || lda < N || ldb < N) return cudaErrorInvalidValue;
  const int64_t gy = (N + kAmaxRows - 1) / kAmaxRows, gx = (N + kAmaxCols - 1) / kAmaxCols;
  if (gy > 65535) return cudaErrorInvalidValue;
  // 16-byte vectors when every row starts aligned and N is a multiple of 4
  const bool v4 = N % 4 == 0 && lda % 4 == 0 && ldb % 4 == 0 && ((uintptr_t)A % 16) == 0 && ((uintptr_t)B % 16) == 0;
  const dim3 grid((unsigned)gx, (unsigned)gy, 2);
  if (v4) fold_absmax_kernel<true><<<grid, 256, 0, st>>>(A, lda, B, ldb, N, m, amaxA, amaxB);
  else fold_absmax_kernel<false><<<grid, 256, 0, st>>>(A, lda, B, ldb, N, m, amaxA, amaxB);
  return cudaGetLastError();
}

cudaError_t launch_leaf_scales(const unsigned* amax, int64_t m, int64_t mp, double growth, float* scale, float* inv,
                               cudaStream_t st) {
  if (mp <= 0 || m > mp) return cudaErrorInvalidValue;
  leaf_scales_kernel<<<(unsigned)((mp + 255) / 256), 256, 0, st>>>(amax, m, mp, growth, scale, inv);
  return cudaGetLastError();
}

// Levels per pass of the register walks: two for n0 = 2 (16 values per position); one for
// n0 = 3 and 4.  Walks holding 64 or more values per position (three levels of n0 = 2, two of
// n0 = 3) need about 220 registers, run at low occupancy, and measured slower than an extra
// pass over an intermediate; the deeper fp32 encodes below split their top levels over CTAs or
// hand them over in shared memory instead.
int max_levels_per_pass(int n0) { return n0 == 2 ? 2 : 1; }
int max_decode_levels_per_pass(int n0, int formula, int64_t m) {
  // Laderman's formula: two levels (the lower handed over in shared memory), when the child rows
  // fill the 64-position tiles reasonably (m >= 32)
  if (formula == kFormulaLaderman && m >= 32) return 2;
  return max_levels_per_pass(n0);
}

int max_encode_levels_per_pass(int n0, int R, int formula, int64_t m, int store) {
  // Laderman's formula: two levels (the first in shared memory), when the leaf rows fill the
  // 128-position tiles reasonably (m >= 32)
  if (formula == kFormulaLaderman && m >= 32) return 2;
  // n0 = 2: four levels, the first two split over the CTAs (encode_top_kernel), for up to
  // kTop3MaxR children; not for the transposed final pass of tf32 leaves
  if (n0 == 2 && R <= kTop3MaxR && store != kStoreTF32) return 4;
  return max_levels_per_pass(n0);
}


cudaError_t launch_encode_pass(const Tables<double>& t, const PassArgs& a, int n0, int g, int io, int store,
                               cudaStream_t st) {
  if (io != RBC_IO_F64 || store != kStoreF64) return cudaErrorInvalidValue;
  if (g == 0) {
    copy_leaf_kernel<double, kStoreF64><<<pass_grid(a.rows_out, a.cols_out, 1, 1), kThreadsX, 0, st>>>(a);
    return cudaGetLastError();
  }
  return enc_n0<double, double, kStoreF64>(t, a, n0, g, st);
}

cudaError_t launch_encode_pass(const Tables<float>& t, const PassArgs& a, int n0, int g, int io, int store,
                               cudaStream_t st) {
  if (io != RBC_IO_F32) return cudaErrorInvalidValue;
  if (g == 0) {
    const dim3 grid = pass_grid(a.rows_out, a.cols_out, 1, 1);
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
