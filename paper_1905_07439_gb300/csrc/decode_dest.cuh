// Fused decode bookkeeping: the C blocks a leaf product contributes to.
//
// Unrolling the decode of Eq. recursive-random-formula over L levels, leaf
// rho = (r_1, ..., r_L) (r_1 at the root) contributes to C block (I, J) with
// I = (i_1 ... i_L), J = (j_1 ... j_L) in base n0 (root digit most significant) and
// coefficient prod_d w^(node_d)_{i_d j_d r_d}, node_1 the root and node_{d+1} the child r_d
// of node_d.  Only the nonzeros of each level's slice are listed; the list of one leaf is
// the product of its per-level lists.
#pragma once

#include <cstdint>

#include "rbc_internal.h"

namespace rbc {

template <typename T>
struct DestList {
  int cnt[kMaxLevels];
  int8_t i[kMaxLevels][kMaxN0 * kMaxN0];
  int8_t j[kMaxLevels][kMaxN0 * kMaxN0];
  T c[kMaxLevels][kMaxN0 * kMaxN0];
  int total;
};

// Build the per-level nonzero lists of `leaf` (one thread).  The tables must hold every
// draw set of the tree from the root on (draw[heap id], or draw[depth] per level).
template <typename T>
__device__ inline void build_dest_list(const Tables<T>& t, int64_t leaf, DestList<T>& d) {
  const int L = t.L, R = t.R, n0 = t.n0;
  int digit[kMaxLevels];
  int64_t rem = leaf;
  for (int q = L - 1; q >= 0; --q) {
    digit[q] = (int)(rem % R);
    rem /= R;
  }
  int64_t node = 0;
  int total = 1;
  for (int q = 0; q < L; ++q) {
    const uint64_t w = t.draw[t.per_level ? q : node];
    const int r = digit[q];
    int c = 0;
    for (int i = 0; i < n0; ++i)
      for (int j = 0; j < n0; ++j) {
        const T wv = t.W[(draw_perm(w, 0, i) * n0 + draw_perm(w, 2, j)) * R + r];
        if (wv != (T)0) {
          d.i[q][c] = (int8_t)i;
          d.j[q][c] = (int8_t)j;
          d.c[q][c] = t.scale * wv * (T)draw_sign(w, 0, i) * (T)draw_sign(w, 2, j);
          ++c;
        }
      }
    d.cnt[q] = c;
    total *= c;
    node = node * R + r + 1;
  }
  d.total = total;
}

// Destination number `idx` of the list: block row I, block column J and coefficient.
template <typename T>
__device__ __forceinline__ T dest_at(const DestList<T>& d, int idx, int n0, int L, int64_t* I,
                                     int64_t* J) {
  int64_t bi = 0, bj = 0, mul = 1;
  T coef = (T)1;
  for (int q = L - 1; q >= 0; --q) {
    const int e = idx % d.cnt[q];
    idx /= d.cnt[q];
    bi += mul * d.i[q][e];
    bj += mul * d.j[q][e];
    coef = coef * d.c[q][e];
    mul *= n0;
  }
  *I = bi;
  *J = bj;
  return coef;
}

}  // namespace rbc
