// rbc_matmul: orchestration of one randomized recursive product C = F^(L)(A, B)
// (Section 2.1.1, Eq. recursive-random-formula) on one stream:
//   encode A and B level by level (root first) into the leaf operands,
//   run the R^L leaf products, and decode (fused into the leaf epilogue, or level by level).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <memory>
#include <vector>

#include "convert.cuh"
#include "level_kernels.cuh"
#include "matmul_internal.h"
#include "rbc_internal.h"
#include "tc_gemm.cuh"

namespace rbc {
namespace detail {

thread_local int64_t g_launches = 0;  // kernels launched by the current call


bool is_tc_leaf(int leaf) {
  return leaf == RBC_LEAF_TF32 || leaf == RBC_LEAF_BF16 || leaf == RBC_LEAF_F16 ||
         leaf == RBC_LEAF_3XBF16 || leaf == RBC_LEAF_3XTF32 || leaf == RBC_LEAF_BF16X6 || leaf == RBC_LEAF_F16X3;
}

int leaf_panels(int leaf) {
  if (leaf == RBC_LEAF_BF16X6) return 3;
  return (leaf == RBC_LEAF_3XBF16 || leaf == RBC_LEAF_3XTF32 || leaf == RBC_LEAF_F16X3) ? 2 : 1;
}

int leaf_store(int leaf) {
  switch (leaf) {
    case RBC_LEAF_F64: return kStoreF64;
    case RBC_LEAF_F32: return kStoreF32;
    case RBC_LEAF_TF32:
    case RBC_LEAF_3XTF32: return kStoreTF32;
    case RBC_LEAF_BF16:
    case RBC_LEAF_3XBF16:
    case RBC_LEAF_BF16X6: return kStoreBF16;
    case RBC_LEAF_F16:
    case RBC_LEAF_F16X3: return kStoreF16;
  }
  return -1;
}

size_t store_bytes(int s) { return s == kStoreF64 ? 8 : (s == kStoreBF16 || s == kStoreF16) ? 2 : 4; }

Passes plan_passes(int L, int g) {
  Passes ps;
  if (L == 0) return ps;
  const int k = (L + g - 1) / g;
  int depth = 0;
  for (int i = 0; i < k; ++i) {
    ps.g[i] = i == 0 ? L - (k - 1) * g : g;
    ps.top[i] = depth;
    depth += ps.g[i];
  }
  ps.count = k;
  return ps;
}

// Contributions per C element of the fused decode: (sum_r nnz(W_::r) / n0^2)^L.
double fused_contributions(const rbc_plan_s* p) {
  int nnz = 0;
  for (double w : p->W) nnz += w != 0.0;
  double per = (double)nnz / (p->n0 * p->n0), c = 1.0;
  for (int d = 0; d < p->L; ++d) c *= per;
  return c;
}

rbc_status make_layout(const rbc_plan_s* p, int64_t N, int io, int leaf, int decode_req, Layout* lo,
                       int64_t reals) {
  if (!p) return fail(RBC_EINVAL, "null plan");
  if (reals < 1) return fail(RBC_EINVAL, "realization count must be positive");
  if (reals > 1 && (p->L == 0 || decode_req != 2))
    return fail(RBC_EINVAL, "realization batches need L >= 1 and staged decode");
  if (io != RBC_IO_F32 && io != RBC_IO_F64) return fail(RBC_EINVAL, "bad io dtype");
  if (leaf < RBC_LEAF_F64 || leaf > RBC_LEAF_F16X3) return fail(RBC_EINVAL, "bad leaf dtype");
  if (io == RBC_IO_F64 && leaf != RBC_LEAF_F64)
    return fail(RBC_EUNSUPPORTED, "fp64 I/O supports the fp64 leaf mode only");
  if (io == RBC_IO_F32 && leaf == RBC_LEAF_F64)
    return fail(RBC_EUNSUPPORTED, "fp64 leaves with fp32 I/O are not implemented");
  const int64_t blocks = ipow(p->n0, p->L);
  if (N <= 0 || N % blocks) return fail(RBC_EINVAL, "N must be a positive multiple of n0^L");
  const int L = p->L, R = p->R, n0 = p->n0;
  if (n0 * n0 * R > kMaxCoef) return fail(RBC_EUNSUPPORTED, "n0*n0*R exceeds the kernel table size (256)");
  lo->m = N / blocks;
  lo->es_io = io == RBC_IO_F64 ? 8 : 4;
  lo->es_acc = lo->es_io;
  lo->store = leaf_store(leaf);
  lo->es_leaf = store_bytes(lo->store);
  lo->split = leaf_panels(leaf) - 1;  // extra panels of a split leaf operand
  // Small SIMT leaves take the exact-size product kernel, which stores M (staged decode) or
  // C (L = 0); an explicitly fused decode keeps the tiled kernel.
  const int64_t small = is_tc_leaf(leaf) || (decode_req == 1 && L > 0) ? 0 : simt_small_pad(io, lo->m);
  if (is_tc_leaf(leaf)) {
    lo->mp = tc_pad(lo->m);
  } else if (small) {
    lo->mp = small;
  } else {
    const int tile = simt_tile(io, lo->m);
    lo->mp = (lo->m + tile - 1) / tile * tile;
  }
  lo->K = lo->mp * (1 + lo->split);
  lo->seg = seg_pitch(lo->m);
  lo->passes = plan_passes(L, io == RBC_IO_F32 ? max_encode_levels_per_pass(n0, R, p->builtin, lo->m, lo->store) : max_levels_per_pass(n0));
  lo->dpasses = plan_passes(L, io == RBC_IO_F32 ? max_decode_levels_per_pass(n0, p->builtin, lo->m) : max_levels_per_pass(n0));
  const bool fused_ok = p->scope == RBC_DRAW_PER_LEVEL || p->draw_count <= kMaxDraws;
  if (decode_req == 1 && !fused_ok) return fail(RBC_EUNSUPPORTED, "fused decode needs <= 1024 draw sets");
  if (decode_req == 0) {
    // Fused scatter costs one read-modify-write of C per contribution; it pays only when C
    // stays in L2 and few leaves feed each element.
    const double c_bytes = (double)N * N * lo->es_io;
    lo->decode = (fused_ok && !small && L <= 1 && c_bytes <= 64.0 * (1 << 20) && fused_contributions(p) <= 4.0)
                     ? 1 : 2;
  } else {
    lo->decode = decode_req;
  }
  if (L == 0) lo->decode = 1;
  size_t off = kStatusBytes;  // device status word(s) first
  for (int i = 1; i < lo->passes.count; ++i) {
    const int d = lo->passes.top[i];
    const int64_t nd = lo->m * ipow(n0, L - d), wd = lo->seg * ipow(n0, L - d);
    const size_t bytes = align256((size_t)(reals * ipow(R, d)) * nd * wd * lo->es_io);
    lo->encA[d] = off;
    off += bytes;
    lo->encB[d] = off;
    off += bytes;
  }
  if (leaf == RBC_LEAF_F16X3) {  // leaf operand scales: amax S, T (bits), scale S, T, inverse S, T
    lo->scales = off;
    off += align256(6 * (size_t)lo->mp * sizeof(float));
  }
  const int64_t leaves = reals * ipow(R, L);
  const size_t leaf_bytes = align256((size_t)leaves * lo->mp * lo->K * lo->es_leaf);
  lo->leafS = off;
  off += leaf_bytes;
  lo->leafT = off;
  off += leaf_bytes;
  lo->mstride = lo->mp * lo->mp;
  if (lo->decode == 2 && L > 0) {
    lo->M = off;
    off += align256((size_t)leaves * lo->mstride * lo->es_acc);
    for (int i = 1; i < lo->dpasses.count; ++i) {
      const int d = lo->dpasses.top[i];
      const int64_t nd = lo->m * ipow(n0, L - d), wd = lo->seg * ipow(n0, L - d);
      lo->dec[d] = off;
      off += align256((size_t)(reals * ipow(R, d)) * nd * wd * lo->es_acc);
    }
  }
  lo->total = off;
  return RBC_OK;
}

template <typename T>
struct TablesBox {
  std::unique_ptr<Tables<T>> t{new Tables<T>()};
};

// Parents per launch so that the subtree draws of a chunk fit the kernel table.
int64_t pass_chunk(const rbc_plan_s* p, int g, int64_t parents) {
  if (p->scope == RBC_DRAW_PER_LEVEL) return parents;
  int64_t per = 0;
  for (int j = 0; j < g; ++j) per += ipow(p->R, j);
  const int64_t c = kMaxDraws / per;
  return c < 1 ? 1 : c;
}

// Draw sets one realization needs for parents [c0, c0 + cnt) at depth d and their subtrees
// over g levels (per-node scope), or all of its levels (per-level scope).
int64_t launch_draws(const rbc_plan_s* p, int g, int64_t cnt) {
  if (p->scope == RBC_DRAW_PER_LEVEL) return p->draw_count;
  int64_t n = 0;
  for (int j = 0; j < g; ++j) n += cnt * ipow(p->R, j);
  return n;
}

// Every launch of the pass at depth d over g levels: f(k0, kc, c0, cnt) covers realizations
// [k0, k0 + kc) and, in each, parents [c0, c0 + cnt).  When the draw sets of a whole
// realization fit the kernel table, as many realizations as fit share a launch; otherwise
// one realization at a time, its parents chunked.
template <class F>
rbc_status for_each_launch(const Reals& rs, int d, int g, F&& f) {
  const rbc_plan_s* p = rs.plan;
  const int64_t P = ipow(p->R, d);
  const int64_t D = launch_draws(p, g, P);
  if (D <= kMaxDraws) {
    const int64_t rc = D > 0 ? std::max<int64_t>(1, kMaxDraws / D) : rs.count;
    for (int64_t k0 = 0; k0 < rs.count; k0 += rc) {
      const rbc_status s = f(k0, std::min(rc, rs.count - k0), (int64_t)0, P);
      if (s != RBC_OK) return s;
    }
    return RBC_OK;
  }
  const int64_t chunk = pass_chunk(p, g, P);
  for (int64_t k = 0; k < rs.count; ++k)
    for (int64_t c0 = 0; c0 < P; c0 += chunk) {
      const rbc_status s = f(k, (int64_t)1, c0, std::min(chunk, P - c0));
      if (s != RBC_OK) return s;
    }
  return RBC_OK;
}

// Tables of one launch: base tensors of the formula and, realization after realization, the
// draw sets of parents [c0, c0 + cnt) at depth d with their g-level subtrees.
template <typename T>
rbc_status launch_tables(const Reals& rs, int d, int g, int64_t k0, int64_t kc, int64_t c0, int64_t cnt, PassArgs* a,
                         Tables<T>& tab) {
  const rbc_plan_s* p = rs.plan;
  rbc_status s = fill_tables(p, 0, 0, &tab);
  if (s != RBC_OK) return s;
  a->depth = d;
  a->node_first = depth_start(p->R, d) + c0;
  a->real_parents = cnt;
  int64_t first[kMaxLevels], count[kMaxLevels], nr = 0, per = 0;
  if (p->scope == RBC_DRAW_PER_LEVEL) {
    first[0] = 0;
    count[0] = p->draw_count;
    nr = 1;
    per = p->draw_count;
  } else {
    for (int j = 0; j < g; ++j) {
      const int64_t rj = ipow(p->R, j);
      first[j] = depth_start(p->R, d + j) + c0 * rj;
      count[j] = cnt * rj;
      a->dfirst[j] = first[j];
      a->dbase[j] = per;
      per += count[j];
    }
    nr = g;
  }
  if (kc * per > kMaxDraws) return fail(RBC_EUNSUPPORTED, "one launch needs more than 1024 draw sets");
  a->real_draws = per;
  int64_t o = 0;
  for (int64_t k = 0; k < kc; ++k) {
    const uint64_t* q = rs.draws + (k0 + k) * p->draw_count;
    for (int i = 0; i < nr; ++i)
      for (int64_t e = 0; e < count[i]; ++e) tab.draw[o++] = q[first[i] + e];
  }
  return RBC_OK;
}

// f16x3 leaf operand scales in the workspace: [amax S | amax T | scale S | scale T | inverse S |
// inverse T], mp entries each.
const float* leaf_scale(const Layout& lo, char* ws, int tensor) {
  return lo.scales ? reinterpret_cast<const float*>(ws + lo.scales) + (2 + tensor) * lo.mp : nullptr;
}
const float* leaf_inverse(const Layout& lo, char* ws, int tensor) {
  return lo.scales ? reinterpret_cast<const float*>(ws + lo.scales) + (4 + tensor) * lo.mp : nullptr;
}

// Growth bound of the leaf operand entries over the recursion: (max_r sum_{k,l} |u_klr|)^L for
// the left operand (V for the right); the signed permutations keep each column's magnitudes.
double leaf_growth(const rbc_plan_s* p, int tensor) {
  const std::vector<double>& X = tensor == 0 ? p->U : p->V;
  double g = 0;
  for (int r = 0; r < p->R; ++r) {
    double c = 0;
    for (int e = 0; e < p->n0 * p->n0; ++e) c += std::fabs(X[(size_t)e * p->R + r]);
    g = std::max(g, c);
  }
  double t = 1;
  for (int d = 0; d < p->L; ++d) t *= g;
  return t;
}

// The f16x3 scales of one call: the largest |entry| of each class of rows of A and of columns of
// B congruent mod m (the rows of S and columns of T they feed), then the power of two per class
// that keeps the grown entries below 2^15.
rbc_status leaf_scales(const rbc_plan_s* p, const Layout& lo, const void* A, int64_t lda, const void* B,
                       int64_t ldb, int64_t N, char* ws, cudaStream_t st) {
  if (!lo.scales) return RBC_OK;
  unsigned* amax = reinterpret_cast<unsigned*>(ws + lo.scales);
  float* f = reinterpret_cast<float*>(ws + lo.scales);
  cudaError_t e = cudaMemsetAsync(amax, 0, 2 * (size_t)lo.mp * sizeof(unsigned), st);
  if (e == cudaSuccess)
    e = launch_fold_absmax(static_cast<const float*>(A), lda, static_cast<const float*>(B), ldb, N, lo.m, amax,
                           amax + lo.mp, st);
  for (int tensor = 0; tensor < 2 && e == cudaSuccess; ++tensor)
    e = launch_leaf_scales(amax + tensor * lo.mp, lo.m, lo.mp, std::min(leaf_growth(p, tensor), 1e300),
                           f + (2 + tensor) * lo.mp, f + (4 + tensor) * lo.mp, st);
  g_launches += 3;
  return e == cudaSuccess ? RBC_OK : fail(RBC_ECUDA, cudaGetErrorString(e));
}

// Encode one operand through all passes into the leaf operand buffer (row-major, K-major
// rows of length lo.K, zero padded to mp, split panels [hi | lo]).
template <typename T>
rbc_status encode_operand(const Reals& rs, const Layout& lo, int io, int tensor, const void* X, int64_t ldx,
                          char* ws, Tables<T>& tab, cudaStream_t st) {
  const rbc_plan_s* p = rs.plan;
  const int L = p->L, R = p->R, n0 = p->n0;
  const size_t* enc = tensor == 0 ? lo.encA : lo.encB;
  char* leafbuf = ws + (tensor == 0 ? lo.leafS : lo.leafT);
  if (L == 0) {
    PassArgs a{};
    a.X = X;
    a.ldx = ldx;
    a.Y = leafbuf;
    a.ldy = lo.K;
    a.nb = lo.m;
    a.rows_out = lo.mp;
    a.cols_out = lo.mp;
    a.parents = 1;
    a.outs_per_parent = 1;
    a.split = lo.split;
    a.kpanel = lo.mp;
    a.trans = tensor == 1 && lo.store == kStoreTF32;
    a.seg = lo.mp;
    a.mval = lo.m;
    a.plain = 1;
    a.tensor = tensor;
    a.lscale = leaf_scale(lo, ws, tensor);
    cudaError_t e = launch_encode_pass(tab, a, n0, 0, io, lo.store, st);
    ++g_launches;
    return e == cudaSuccess ? RBC_OK : fail(RBC_ECUDA, cudaGetErrorString(e));
  }
  for (int i = 0; i < lo.passes.count; ++i) {
    const int d = lo.passes.top[i], g = lo.passes.g[i];
    const bool last = i + 1 == lo.passes.count;
    const int64_t n_par = lo.m * ipow(n0, L - d), nb = lo.m * ipow(n0, L - d - g);
    const int64_t w_par = lo.seg * ipow(n0, L - d), w_nb = lo.seg * ipow(n0, L - d - g);  // physical widths
    const int64_t P = ipow(R, d), outs = ipow(R, g);
    rbc_status s = for_each_launch(rs, d, g, [&](int64_t k0, int64_t kc, int64_t c0, int64_t cnt) {
      PassArgs a{};
      rbc_status s2 = launch_tables(rs, d, g, k0, kc, c0, cnt, &a, tab);
      if (s2 != RBC_OK) return s2;
      a.formula = p->builtin;
      const int64_t first = k0 * P + c0;  // first parent of the launch, realization-major
      if (d == 0) {  // the caller's matrix, plain layout
        a.X = X;
        a.ldx = ldx;
        a.strideX = 0;
        a.plain = 1;
      } else {
        a.X = ws + enc[d] + (size_t)first * n_par * w_par * lo.es_io;
        a.ldx = w_par;
        a.strideX = n_par * w_par;
      }
      a.xcol = w_nb;
      a.mval = lo.m;
      if (last) {
        a.Y = leafbuf + (size_t)first * outs * lo.mp * lo.K * lo.es_leaf;
        a.ldy = lo.K;
        a.strideY = lo.mp * lo.K;
        a.rows_out = lo.mp;
        a.cols_out = lo.mp;
        a.split = lo.split;
        a.kpanel = lo.mp;
        a.seg = lo.mp;  // one segment per leaf row
        // tf32 tensor-core leaves take T K-major: write T^T
        a.trans = tensor == 1 && lo.store == kStoreTF32;
        a.lscale = leaf_scale(lo, ws, tensor);
      } else {
        a.Y = ws + enc[d + g] + (size_t)first * outs * nb * w_nb * lo.es_io;
        a.ldy = w_nb;
        a.strideY = nb * w_nb;
        a.rows_out = nb;
        a.cols_out = w_nb;
        a.seg = lo.seg;
      }
      a.nb = nb;
      a.parents = kc * cnt;
      a.outs_per_parent = outs;
      a.tensor = tensor;
      const int store = last ? lo.store : (io == RBC_IO_F64 ? kStoreF64 : kStoreF32);
      cudaError_t e = launch_encode_pass(tab, a, n0, g, io, store, st);
      ++g_launches;
      return e == cudaSuccess ? RBC_OK : fail(RBC_ECUDA, cudaGetErrorString(e));
    });
    if (s != RBC_OK) return s;
  }
  return RBC_OK;
}

// Staged decode: passes from the leaves up to C (realization k's output at C + k * strideC).
template <typename T>
rbc_status decode_passes(const Reals& rs, const Layout& lo, void* C, int64_t ldc, char* ws, Tables<T>& tab,
                         cudaStream_t st) {
  const rbc_plan_s* p = rs.plan;
  const int L = p->L, R = p->R, n0 = p->n0;
  for (int i = lo.dpasses.count - 1; i >= 0; --i) {
    const int d = lo.dpasses.top[i], g = lo.dpasses.g[i];
    const bool bottom = i + 1 == lo.dpasses.count;
    const int64_t n_par = lo.m * ipow(n0, L - d), nb = lo.m * ipow(n0, L - d - g);
    const int64_t w_par = lo.seg * ipow(n0, L - d), w_nb = lo.seg * ipow(n0, L - d - g);  // physical widths
    const int64_t P = ipow(R, d), outs = ipow(R, g);
    rbc_status s = for_each_launch(rs, d, g, [&](int64_t k0, int64_t kc, int64_t c0, int64_t cnt) {
      PassArgs a{};
      rbc_status s2 = launch_tables(rs, d, g, k0, kc, c0, cnt, &a, tab);
      if (s2 != RBC_OK) return s2;
      a.formula = p->builtin;
      const int64_t first = k0 * P + c0;
      if (bottom) {  // leaf products: rows of mp >= seg columns
        a.X = ws + lo.M + (size_t)first * outs * lo.mstride * lo.es_acc;
        a.ldx = lo.mp;
        a.strideX = lo.mstride;
      } else {
        a.X = ws + lo.dec[d + g] + (size_t)first * outs * nb * w_nb * lo.es_acc;
        a.ldx = w_nb;
        a.strideX = nb * w_nb;
      }
      a.xcol = w_nb;
      a.seg = lo.seg;
      a.mval = lo.m;
      if (d == 0) {  // one parent per realization: the caller's C, plain layout
        a.Y = static_cast<char*>(C) + (size_t)k0 * rs.strideC * lo.es_io;
        a.ldy = ldc;
        a.strideY = rs.strideC;
        a.plain = 1;
      } else {
        a.Y = ws + lo.dec[d] + (size_t)first * n_par * w_par * lo.es_acc;
        a.ldy = w_par;
        a.strideY = n_par * w_par;
      }
      a.nb = nb;
      a.parents = kc * cnt;
      a.outs_per_parent = outs;
      cudaError_t e = launch_decode_pass(tab, a, n0, g, st);
      ++g_launches;
      return e == cudaSuccess ? RBC_OK : fail(RBC_ECUDA, cudaGetErrorString(e));
    });
    if (s != RBC_OK) return s;
  }
  return RBC_OK;
}

inline void mark(const rbc_matmul_opts* o, int i, cudaStream_t st) {
  if (o && o->events[i]) cudaEventRecord(static_cast<cudaEvent_t>(o->events[i]), st);
}

template <typename T>
rbc_status run(const Reals& rs, const Layout& lo, const void* A, const void* B, void* C, int64_t N,
               int64_t lda, int64_t ldb, int64_t ldc, int io, int leaf, char* ws, cudaStream_t st,
               const rbc_matmul_opts* opts) {
  static thread_local TablesBox<T> box;
  Tables<T>& tab = *box.t;
  const rbc_plan_s* p = rs.plan;
  mark(opts, 0, st);
  rbc_status s = RBC_OK;
  if (lo.scales) {
    if constexpr (sizeof(T) != 4) return fail(RBC_EUNSUPPORTED, "f16x3 leaves need fp32 I/O");
    s = leaf_scales(p, lo, A, lda, B, ldb, N, ws, st);
    if (s != RBC_OK) return s;
  }
  s = encode_operand<T>(rs, lo, io, 0, A, lda, ws, tab, st);
  if (s != RBC_OK) return s;
  s = encode_operand<T>(rs, lo, io, 1, B, ldb, ws, tab, st);
  if (s != RBC_OK) return s;
  const int L = p->L;
  const int64_t leaves = rs.count * ipow(p->R, L);
  const bool fused = lo.decode == 1 || L == 0;
  if (fused && L > 0) {
    cudaError_t e = cudaMemset2DAsync(C, (size_t)ldc * lo.es_io, 0, (size_t)N * lo.es_io, (size_t)N, st);
    if (e != cudaSuccess) return fail(RBC_ECUDA, cudaGetErrorString(e));
  }
  mark(opts, 1, st);
  if (fused) {
    s = fill_tables(p, 0, p->draw_count, &tab);
  } else {
    s = fill_tables(p, 0, 0, &tab);
  }
  if (s != RBC_OK) return s;
  if (is_tc_leaf(leaf)) {
    TcGemmArgs g{};
    g.S = ws + lo.leafS;
    g.T = ws + lo.leafT;
    g.K = lo.K;
    g.m = lo.m;
    g.mp = lo.mp;
    g.leaves = leaves;
    g.C = C;
    g.ldc = ldc;
    g.direct = L == 0;
    g.store_m = !fused;
    g.M = fused ? nullptr : ws + lo.M;
    g.strideM = lo.mstride;
    g.leaf = leaf;
    g.status = reinterpret_cast<int*>(ws);
    g.stall = opts ? opts->stall_leaf_copies : 0;
    g.rinv = leaf_inverse(lo, ws, 0);
    g.cinv = leaf_inverse(lo, ws, 1);
    if constexpr (sizeof(T) == 4) {
      cudaError_t e = launch_tc_gemm(tab, g, st);
      ++g_launches;
      if (e != cudaSuccess) return fail(RBC_ECUDA, cudaGetErrorString(e));
    } else {
      return fail(RBC_EUNSUPPORTED, "tensor-core leaves need fp32 I/O");
    }
  } else {
    SimtGemmArgs g{};
    g.S = ws + lo.leafS;
    g.T = ws + lo.leafT;
    g.lds = lo.K;
    g.ldt = lo.K;
    g.strideS = lo.mp * lo.K;
    g.strideT = lo.mp * lo.K;
    g.K = lo.K;
    g.m = lo.m;
    g.mp = lo.mp;
    g.leaves = leaves;
    if (fused) {
      g.out = C;
      g.ldo = ldc;
      g.mode = L == 0 ? 2 : 1;
    } else {
      g.out = ws + lo.M;
      g.ldo = lo.mp;
      g.strideO = lo.mstride;
      g.mode = 0;
    }
    cudaError_t e = launch_simt_gemm(tab, g, st);
    ++g_launches;
    if (e != cudaSuccess) return fail(RBC_ECUDA, cudaGetErrorString(e));
  }
  mark(opts, 2, st);
  if (!fused) {
    s = decode_passes<T>(rs, lo, C, ldc, ws, tab, st);
    if (s != RBC_OK) return s;
  }
  mark(opts, 3, st);
  return RBC_OK;
}

template rbc_status encode_operand<float>(const Reals&, const Layout&, int, int, const void*, int64_t, char*,
                                          Tables<float>&, cudaStream_t);
template rbc_status decode_passes<float>(const Reals&, const Layout&, void*, int64_t, char*, Tables<float>&,
                                         cudaStream_t);

}  // namespace detail
}  // namespace rbc

using namespace rbc;
using namespace rbc::detail;

extern "C" {

size_t rbc_workspace_size_ex(rbc_plan_t plan, int64_t N, int io, int leaf, const rbc_matmul_opts* o) {
  Layout lo;
  if (make_layout(plan, N, io, leaf, o ? o->decode : 0, &lo) != RBC_OK) return 0;
  return lo.total;
}

size_t rbc_workspace_size(rbc_plan_t plan, int64_t N, int io, int leaf) {
  return rbc_workspace_size_ex(plan, N, io, leaf, nullptr);
}

rbc_status rbc_matmul_ex(rbc_plan_t plan, const void* A, const void* B, void* C, int64_t N,
                         int64_t lda, int64_t ldb, int64_t ldc, int io, int leaf, void* workspace,
                         size_t ws_bytes, void* stream, rbc_matmul_opts* opts) {
  if (!plan || !A || !B || !C) return fail(RBC_EINVAL, "null argument");
  if (opts && (opts->decode < 0 || opts->decode > 2)) return fail(RBC_EINVAL, "bad decode option");
  if (opts && opts->stall_leaf_copies && !is_tc_leaf(leaf))
    return fail(RBC_EINVAL, "the stall test hook applies to tensor-core leaf modes");
  Layout lo;
  rbc_status s = make_layout(plan, N, io, leaf, opts ? opts->decode : 0, &lo);
  if (s != RBC_OK) return s;
  if (lda < N || ldb < N || ldc < N) return fail(RBC_EINVAL, "leading dimension smaller than N");
  if (lo.total > 0 && (!workspace || ((uintptr_t)workspace & 255)))
    return fail(RBC_EINVAL, "workspace must be a 256-byte aligned device pointer");
  if (ws_bytes < lo.total) return fail(RBC_ENOMEM, "workspace too small");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  g_launches = 0;
  {
    cudaError_t e = cudaMemsetAsync(ws, 0, sizeof(int), st);  // clear the status word
    if (e != cudaSuccess) return fail(RBC_ECUDA, cudaGetErrorString(e));
  }
  const Reals rs{plan, plan->packed.data(), 1, 0};
  if (io == RBC_IO_F64)
    s = run<double>(rs, lo, A, B, C, N, lda, ldb, ldc, io, leaf, ws, st, opts);
  else
    s = run<float>(rs, lo, A, B, C, N, lda, ldb, ldc, io, leaf, ws, st, opts);
  if (opts) opts->launches = g_launches;
  return s;
}

size_t rbc_realizations_workspace_size(rbc_plan_t plan, int64_t N, int io, int leaf, int64_t count) {
  if (!plan || count < 1) return 0;
  Layout lo;
  if (plan->L == 0) return make_layout(plan, N, io, leaf, 0, &lo) == RBC_OK ? lo.total : 0;
  if (make_layout(plan, N, io, leaf, 2, &lo, count) != RBC_OK) return 0;
  return lo.total;
}

rbc_status rbc_matmul_realizations(rbc_plan_t plan, const uint64_t* seeds, int64_t count, const void* A,
                                   const void* B, void* C, int64_t N, int64_t lda, int64_t ldb, int64_t ldc,
                                   int64_t strideC, int io, int leaf, void* workspace, size_t ws_bytes,
                                   void* stream) {
  if (!plan || !seeds || count < 1 || !A || !B || !C)
    return fail(RBC_EINVAL, "null argument or empty realization list");
  if (lda < N || ldb < N || ldc < N) return fail(RBC_EINVAL, "leading dimension smaller than N");
  if (count > 1 && strideC < ldc * N) return fail(RBC_EINVAL, "strideC smaller than ldc * N: outputs overlap");
  if (!workspace || ((uintptr_t)workspace & 255))
    return fail(RBC_EINVAL, "workspace must be a 256-byte aligned device pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t es = io == RBC_IO_F64 ? 8 : 4;
  if (plan->L == 0) {  // the standard product: no draws, every realization is the same
    for (int64_t k = 0; k < count; ++k) {
      rbc_status s = rbc_matmul_ex(plan, A, B, static_cast<char*>(C) + (size_t)k * strideC * es, N, lda, ldb, ldc,
                                   io, leaf, workspace, ws_bytes, stream, nullptr);
      if (s != RBC_OK) return s;
    }
    return RBC_OK;
  }
  Layout one;
  rbc_status s = make_layout(plan, N, io, leaf, 2, &one, 1);
  if (s != RBC_OK) return s;
  if (ws_bytes < one.total) return fail(RBC_ENOMEM, "workspace smaller than one realization needs");
  // The largest batch whose layout fits: a batch of b needs at most kStatusBytes + b * (one
  // realization's bytes beyond the status words).
  const size_t per = one.total - kStatusBytes;
  const int64_t batch = (int64_t)std::min<size_t>((size_t)count, (ws_bytes - kStatusBytes) / per);
  Layout lo;
  s = make_layout(plan, N, io, leaf, 2, &lo, batch);
  if (s != RBC_OK) return s;
  std::vector<uint64_t> draws;
  try {
    draws.resize((size_t)(batch * plan->draw_count));
  } catch (...) {
    return fail(RBC_ENOMEM, "out of host memory for the draws of a batch");
  }
  char* ws = static_cast<char*>(workspace);
  cudaError_t e = cudaMemsetAsync(ws, 0, sizeof(int), st);
  if (e != cudaSuccess) return fail(RBC_ECUDA, cudaGetErrorString(e));
  for (int64_t k0 = 0; k0 < count; k0 += batch) {
    const int64_t kc = std::min(batch, count - k0);
    Layout lk;
    if (kc != batch) {
      s = make_layout(plan, N, io, leaf, 2, &lk, kc);
      if (s != RBC_OK) return s;
    }
    for (int64_t k = 0; k < kc; ++k) packed_draws(plan, seeds[k0 + k], draws.data() + k * plan->draw_count);
    const Reals rs{plan, draws.data(), kc, strideC};
    void* Ck = static_cast<char*>(C) + (size_t)k0 * strideC * es;
    const Layout& l = kc == batch ? lo : lk;
    s = io == RBC_IO_F64 ? run<double>(rs, l, A, B, Ck, N, lda, ldb, ldc, io, leaf, ws, st, nullptr)
                         : run<float>(rs, l, A, B, Ck, N, lda, ldb, ldc, io, leaf, ws, st, nullptr);
    if (s != RBC_OK) return s;
  }
  return RBC_OK;
}

rbc_status rbc_workspace_check(void* workspace, void* stream, int* device_status) {
  if (!workspace || !device_status) return fail(RBC_EINVAL, "null argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, workspace, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemsetAsync(workspace, 0, sizeof(int), st);
  if (e != cudaSuccess) return fail(RBC_ECUDA, cudaGetErrorString(e));
  *device_status = v;
  return v == 0 ? RBC_OK : fail((rbc_status)v, "a kernel of a previous call reported an error");
}

rbc_status rbc_matmul(rbc_plan_t plan, const void* A, const void* B, void* C, int64_t N, int64_t lda,
                      int64_t ldb, int64_t ldc, int io, int leaf, void* workspace, size_t ws_bytes,
                      void* stream) {
  return rbc_matmul_ex(plan, A, B, C, N, lda, ldb, ldc, io, leaf, workspace, ws_bytes, stream, nullptr);
}

}  // extern "C"
