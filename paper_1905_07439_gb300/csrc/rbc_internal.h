// Internal declarations of librbc: plan object, kernel coefficient tables, launch helpers.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/rbc.h"

namespace rbc {

// Limits of the coefficient tables carried in kernel parameters (the constant bank):
// base tensors of n0*n0*R entries and one packed 64-bit word per draw set.
constexpr int kMaxN0 = 4;
constexpr int kMaxCoef = 256;   // n0*n0*R
constexpr int kMaxDraws = 1024; // draw sets visible to one launch
constexpr int kMaxLevels = 8;

// Packed draw set: pi_{c+1}(j) in bits [8c + 2j, 8c + 2j + 2), c = 0..2, j < n0 <= 4;
// s_{c+1}(j) = -1 iff bit 32 + 8c + j is set.
inline uint64_t pack_draw(const int pi[3][kMaxN0], const int s[3][kMaxN0], int n0) {
  uint64_t w = 0;
  for (int c = 0; c < 3; ++c)
    for (int j = 0; j < n0; ++j) {
      w |= (uint64_t)(pi[c][j] & 3) << (8 * c + 2 * j);
      if (s[c][j] < 0) w |= 1ull << (32 + 8 * c + j);
    }
  return w;
}

// Per-launch coefficient tables: base U, V, W in the arithmetic type of the launch, the
// packed draws of the nodes the launch touches, and the rescale (1-kappa)^-1.
template <typename T>
struct Tables {
  T U[kMaxCoef];
  T V[kMaxCoef];
  T W[kMaxCoef];
  uint64_t draw[kMaxDraws];
  T scale;
  int n0, R, L;
  int per_level;      // 1: one draw set per depth; 0: one per node (the launch's PassArgs locate them)
};

#if defined(__CUDACC__)
__host__ __device__ __forceinline__ int draw_perm(uint64_t w, int c, int j) {
  return (int)((w >> (8 * c + 2 * j)) & 3u);
}
__host__ __device__ __forceinline__ int draw_sign(uint64_t w, int c, int j) {
  return ((w >> (32 + 8 * c + j)) & 1u) ? -1 : 1;
}
#endif

}  // namespace rbc

struct rbc_plan_s {
  int R = 0, n0 = 0, L = 0, mode = 0, scope = 0, rescale = -1;
  int builtin = 0;  // rbc::BuiltinFormula of U, V, W
  uint64_t seed = 0;
  std::vector<double> U, V, W;
  double kappa = 0, tau = 0, gamma = 0, scale = 1;
  int64_t draw_count = 0;
  std::vector<uint64_t> packed;   // one word per draw set
  std::vector<int8_t> perms;      // [draw][3][n0]
  std::vector<int8_t> signs;      // [draw][3][n0]
};

namespace rbc {

// Thread-local last error text (rbc_last_error).
void set_error(const std::string& msg);
rbc_status fail(rbc_status st, const std::string& msg);

// Heap id of the first node at depth d: (R^d - 1)/(R - 1) (= d when R = 1).
inline int64_t depth_start(int R, int d) {
  if (R == 1) return d;
  int64_t s = 0, p = 1;
  for (int i = 0; i < d; ++i) { s += p; p *= R; }
  return s;
}
inline int64_t ipow(int64_t b, int e) {
  int64_t r = 1;
  while (e-- > 0) r *= b;
  return r;
}

// The packed draw sets of plan p's computation under another seed (p->draw_count words).
void packed_draws(const rbc_plan_s* p, uint64_t seed, uint64_t* out);

// Fill the tables of a launch touching draw sets [key_first, key_first + count).
template <typename T>
rbc_status fill_tables(const rbc_plan_s* p, int64_t key_first, int64_t count, Tables<T>* t);

}  // namespace rbc
