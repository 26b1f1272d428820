// Pieces of rbc_matmul shared with the grouped batch: workspace layout and the encode /
// decode pass sequences of one product.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "rbc_internal.h"

namespace rbc {
namespace detail {

constexpr size_t kStatusBytes = 256;  // device status word(s) at the start of a workspace

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
// Column segment pitch of the intermediates' recursive padded layout: the leaf width m
// rounded up to 4 elements, so that every sub-block of every level starts 16-byte aligned.
inline int64_t seg_pitch(int64_t m) { return (m + 3) / 4 * 4; }

extern thread_local int64_t g_launches;

// Grouping of the L levels into passes, root first: [L - (k-1)*g, g, ..., g] with g the most
// levels one pass holds in registers; the small pass sits at the root, where intermediates
// are smallest ((R/n0^2)^depth N^2 elements).
struct Passes {
  int count = 0;
  int g[kMaxLevels] = {};
  int top[kMaxLevels] = {};  // depth of the parents of each pass
};

struct Layout {
  int64_t m = 0, mp = 0, K = 0;
  int64_t seg = 0;  // seg_pitch(m): an intermediate block at depth d is m n0^(L-d) rows x seg n0^(L-d) columns
  int store = 0, decode = 0;  // decode: 1 fused, 2 staged passes
  int split = 0;              // extra panels of the leaf operands: 0 plain, 1 [hi | lo], 2 [b0 | b1 | b2]
  size_t es_io = 0, es_acc = 0, es_leaf = 0;
  Passes passes;   // encode passes, root first
  Passes dpasses;  // decode passes (the same levels may be grouped differently)
  size_t encA[kMaxLevels + 1] = {}, encB[kMaxLevels + 1] = {};  // intermediates at depth d
  size_t leafS = 0, leafT = 0, M = 0, dec[kMaxLevels + 1] = {};
  size_t scales = 0;    // f16x3: leaf operand scales (0: none)
  int64_t mstride = 0;  // elements from one leaf product to the next in M (mp^2)
  size_t total = 0;
};

// Independent realizations of one plan's computation computed together, differing only in
// their draws: realization k's draw sets (plan->draw_count words, heap or level order) are
// at draws + k * plan->draw_count.  Their intermediates sit realization-major in one
// workspace; output k is C + k * strideC.
struct Reals {
  const rbc_plan_s* plan = nullptr;
  const uint64_t* draws = nullptr;
  int64_t count = 1;
  int64_t strideC = 0;  // elements
};

bool is_tc_leaf(int leaf);
int leaf_panels(int leaf);  // stored panels per leaf operand: 1, 2 (split modes, f16x3) or 3 (bf16x6)
// f16x3 leaf operand scales of a layout (null for other modes): scale (encode) and inverse
// (leaf epilogue) of the rows of S (tensor 0) or the columns of T (tensor 1), in workspace ws.
const float* leaf_scale(const Layout& lo, char* ws, int tensor);
const float* leaf_inverse(const Layout& lo, char* ws, int tensor);
// Compute the f16x3 scales of one product (A, B: N x N fp32, device) into ws; RBC_OK when the
// layout has none.
rbc_status leaf_scales(const rbc_plan_s* p, const Layout& lo, const void* A, int64_t lda, const void* B,
                       int64_t ldb, int64_t N, char* ws, cudaStream_t st);
Passes plan_passes(int L, int g);  // passes of at most g levels
// reals > 1: the layout of that many realizations (staged decode only).
rbc_status make_layout(const rbc_plan_s* p, int64_t N, int io, int leaf, int decode_req, Layout* lo,
                       int64_t reals = 1);

template <typename T>
rbc_status encode_operand(const Reals& rs, const Layout& lo, int io, int tensor, const void* X, int64_t ldx,
                          char* ws, Tables<T>& tab, cudaStream_t st);
template <typename T>
rbc_status decode_passes(const Reals& rs, const Layout& lo, void* C, int64_t ldc, char* ws, Tables<T>& tab,
                         cudaStream_t st);
template <typename T>
inline rbc_status encode_operand(const rbc_plan_s* p, const Layout& lo, int io, int tensor, const void* X,
                                 int64_t ldx, char* ws, Tables<T>& tab, cudaStream_t st) {
  const Reals rs{p, p->packed.data(), 1, 0};
  return encode_operand<T>(rs, lo, io, tensor, X, ldx, ws, tab, st);
}
template <typename T>
inline rbc_status decode_passes(const rbc_plan_s* p, const Layout& lo, void* C, int64_t ldc, char* ws,
                                Tables<T>& tab, cudaStream_t st) {
  const Reals rs{p, p->packed.data(), 1, 0};
  return decode_passes<T>(rs, lo, C, ldc, ws, tab, st);
}

}  // namespace detail
}  // namespace rbc
