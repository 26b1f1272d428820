// Host side of a plan: validation, formula constants (kappa, tau, Gamma) and the
// counter-based random draws of every recursion node (Section 2.1, Section 2.1.1).
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>

#include "formulas.h"
#include "rbc_internal.h"

namespace rbc {

// The built-in formula that U, V, W equal exactly, if any.
template <class F>
static bool equals_formula(const rbc_plan_s* p) {
  if (p->n0 != F::n0 || p->R != F::R) return false;
  for (int e = 0; e < F::n0 * F::n0 * F::R; ++e)
    if (p->U[e] != (double)F::U[e] || p->V[e] != (double)F::V[e] || p->W[e] != (double)F::W[e]) return false;
  return true;
}
static int builtin_formula(const rbc_plan_s* p) {
  if (equals_formula<StrassenFormula>(p)) return kFormulaStrassen;
  if (equals_formula<LadermanFormula>(p)) return kFormulaLaderman;
  return kFormulaGeneric;
}

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
rbc_status fail(rbc_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

// SplitMix64 output function (Steele, Lea & Flood, 2014).
static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

static inline uint64_t stream_word(uint64_t seed, uint64_t key, uint64_t c) {
  return mix64(seed + kGolden * (1ull + 8ull * key + c));
}

// Uniform permutation by Fisher-Yates driven by the stream word (see rbc.h).
static void draw_permutation(uint64_t w, int n0, int* p) {
  for (int j = 0; j < n0; ++j) p[j] = j;
  for (int i = n0 - 1; i >= 1; --i) {
    const uint64_t x = mix64(w + (uint64_t)i);
    const int j = (int)(((unsigned __int128)x * (unsigned __int128)(i + 1)) >> 64);
    const int t = p[i];
    p[i] = p[j];
    p[j] = t;
  }
}

static void draw_set(const rbc_plan_s* pl, uint64_t seed, uint64_t key, int pi[3][kMaxN0], int s[3][kMaxN0]) {
  const bool perm = pl->mode == RBC_RAND_FULL || pl->mode == RBC_RAND_PERM;
  const bool sign = pl->mode == RBC_RAND_FULL || pl->mode == RBC_RAND_SIGN;
  for (int c = 0; c < 3; ++c) {
    if (perm) {
      draw_permutation(stream_word(seed, key, (uint64_t)c), pl->n0, pi[c]);
    } else {
      for (int j = 0; j < pl->n0; ++j) pi[c][j] = j;
    }
    const uint64_t w = stream_word(seed, key, (uint64_t)(3 + c));
    for (int j = 0; j < pl->n0; ++j) s[c][j] = (sign && ((w >> j) & 1u)) ? -1 : 1;
  }
}

// kappa of Eq. epsilon-def, sequential in (i, j, l, r).
static double formula_kappa(const rbc_plan_s* p) {
  const int n = p->n0, R = p->R;
  double acc = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int l = 0; l < n; ++l) {
        double s = 0.0;
        for (int r = 0; r < R; ++r)
          s += p->U[(i * n + l) * R + r] * p->V[(l * n + j) * R + r] * p->W[(i * n + j) * R + r];
        acc += 1.0 - s;
      }
  return acc / (double)(n * n * n);
}

// ||Y - X|| over [n]^6 (Def. ABC).
static double formula_tau(const rbc_plan_s* p) {
  const int n = p->n0, R = p->R;
  double acc = 0.0;
  for (int k = 0; k < n; ++k)
    for (int l = 0; l < n; ++l)
      for (int k2 = 0; k2 < n; ++k2)
        for (int l2 = 0; l2 < n; ++l2)
          for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
              double y = 0.0;
              for (int r = 0; r < R; ++r)
                y += p->U[(k * n + l) * R + r] * p->V[(k2 * n + l2) * R + r] *
                     p->W[(i * n + j) * R + r];
              const double x = (k == i && l2 == j && l == k2) ? 1.0 : 0.0;
              acc += (y - x) * (y - x);
            }
  return std::sqrt(acc);
}

// Eq. square-root-of-sum.
static double formula_gamma(const rbc_plan_s* p) {
  const int n2 = p->n0 * p->n0, R = p->R;
  double acc = 0.0;
  for (int r = 0; r < R; ++r) {
    double u = 0, v = 0, w = 0;
    for (int e = 0; e < n2; ++e) {
      u += p->U[e * R + r] * p->U[e * R + r];
      v += p->V[e * R + r] * p->V[e * R + r];
      w += p->W[e * R + r] * p->W[e * R + r];
    }
    acc += u * v * w;
  }
  return std::sqrt(acc);
}

void packed_draws(const rbc_plan_s* p, uint64_t seed, uint64_t* out) {
  if (seed == p->seed) {
    for (int64_t key = 0; key < p->draw_count; ++key) out[key] = p->packed[key];
    return;
  }
  for (int64_t key = 0; key < p->draw_count; ++key) {
    int pi[3][kMaxN0], s[3][kMaxN0];
    draw_set(p, seed, (uint64_t)key, pi, s);
    out[key] = pack_draw(pi, s, p->n0);
  }
}

template <typename T>
rbc_status fill_tables(const rbc_plan_s* p, int64_t key_first, int64_t count, Tables<T>* t) {
  const int nc = p->n0 * p->n0 * p->R;
  if (nc > kMaxCoef)
    return fail(RBC_EUNSUPPORTED, "n0*n0*R exceeds the kernel table size (256)");
  if (count > kMaxDraws)
    return fail(RBC_EUNSUPPORTED, "recursion tree has more draw sets than one launch holds (1024)");
  if (key_first < 0 || key_first + count > p->draw_count)
    return fail(RBC_EINVAL, "draw range out of bounds");
  for (int e = 0; e < nc; ++e) {
    t->U[e] = (T)p->U[e];
    t->V[e] = (T)p->V[e];
    t->W[e] = (T)p->W[e];
  }
  for (int64_t i = 0; i < count; ++i) t->draw[i] = p->packed[key_first + i];
  t->scale = (T)p->scale;
  t->n0 = p->n0;
  t->R = p->R;
  t->L = p->L;
  t->per_level = p->scope == RBC_DRAW_PER_LEVEL;
  return RBC_OK;
}
template rbc_status fill_tables<float>(const rbc_plan_s*, int64_t, int64_t, Tables<float>*);

template rbc_status fill_tables<double>(const rbc_plan_s*, int64_t, int64_t, Tables<double>*);

}  // namespace rbc

using namespace rbc;

extern "C" {

rbc_status rbc_plan_create_ex(const rbc_plan_desc* d, rbc_plan_t* out) {
  if (!d || !out || !d->U || !d->V || !d->W) return fail(RBC_EINVAL, "null argument");
  *out = nullptr;
  if (d->n0 < 2 || d->n0 > kMaxN0) return fail(RBC_EINVAL, "n0 must be in [2, 4]");
  if (d->R < 1 || d->R > 4096) return fail(RBC_EINVAL, "R must be in [1, 4096]");
  if (d->levels < 0 || d->levels > kMaxLevels) return fail(RBC_EINVAL, "levels must be in [0, 8]");
  if (d->rand_mode < RBC_RAND_FULL || d->rand_mode > RBC_RAND_NONE)
    return fail(RBC_EINVAL, "bad rand_mode");
  if (d->draw_scope != RBC_DRAW_PER_NODE && d->draw_scope != RBC_DRAW_PER_LEVEL)
    return fail(RBC_EINVAL, "bad draw_scope");
  if (d->rescale_kappa < -1 || d->rescale_kappa > 1) return fail(RBC_EINVAL, "bad rescale_kappa");
  int64_t draws = d->draw_scope == RBC_DRAW_PER_LEVEL ? d->levels : depth_start(d->R, d->levels);
  if (draws > (int64_t)1 << 24) return fail(RBC_EINVAL, "recursion tree too large");

  rbc_plan_s* p = new (std::nothrow) rbc_plan_s();
  if (!p) return fail(RBC_ENOMEM, "out of host memory");
  const size_t nc = (size_t)d->n0 * d->n0 * d->R;
  p->R = d->R;
  p->n0 = d->n0;
  p->L = d->levels;
  p->mode = d->rand_mode;
  p->scope = d->draw_scope;
  p->rescale = d->rescale_kappa;
  p->seed = d->seed;
  p->U.assign(d->U, d->U + nc);
  p->V.assign(d->V, d->V + nc);
  p->W.assign(d->W, d->W + nc);
  for (size_t e = 0; e < nc; ++e)
    if (!std::isfinite(p->U[e]) || !std::isfinite(p->V[e]) || !std::isfinite(p->W[e])) {
      delete p;
      return fail(RBC_EINVAL, "non-finite coefficient");
    }
  p->kappa = formula_kappa(p);
  if (p->kappa == 1.0) {
    delete p;
    return fail(RBC_EKAPPA, "kappa == 1: the randomized formula is undefined");
  }
  p->tau = formula_tau(p);
  p->builtin = builtin_formula(p);
  p->gamma = formula_gamma(p);
  const bool rescale = d->rescale_kappa == -1 ? d->rand_mode != RBC_RAND_NONE : d->rescale_kappa == 1;
  p->scale = rescale ? 1.0 / (1.0 - p->kappa) : 1.0;
  p->draw_count = draws;
  try {
    p->packed.resize((size_t)draws);
    p->perms.resize((size_t)draws * 3 * d->n0);
    p->signs.resize((size_t)draws * 3 * d->n0);
  } catch (...) {
    delete p;
    return fail(RBC_ENOMEM, "out of host memory for draws");
  }
  for (int64_t key = 0; key < draws; ++key) {
    int pi[3][kMaxN0], s[3][kMaxN0];
    draw_set(p, p->seed, (uint64_t)key, pi, s);
    p->packed[key] = pack_draw(pi, s, d->n0);
    for (int c = 0; c < 3; ++c)
      for (int j = 0; j < d->n0; ++j) {
        p->perms[(key * 3 + c) * d->n0 + j] = (int8_t)pi[c][j];
        p->signs[(key * 3 + c) * d->n0 + j] = (int8_t)s[c][j];
      }
  }
  *out = p;
  return RBC_OK;
}

rbc_status rbc_plan_create(const double* U, const double* V, const double* W, int R, int n0,
                           int levels, uint64_t seed, rbc_plan_t* out) {
  rbc_plan_desc d;
  d.U = U;
  d.V = V;
  d.W = W;
  d.R = R;
  d.n0 = n0;
  d.levels = levels;
  d.seed = seed;
  d.rand_mode = RBC_RAND_FULL;
  d.draw_scope = RBC_DRAW_PER_NODE;
  d.rescale_kappa = -1;
  return rbc_plan_create_ex(&d, out);
}

void rbc_plan_destroy(rbc_plan_t plan) { delete plan; }

rbc_status rbc_plan_query(rbc_plan_t p, rbc_plan_info* info) {
  if (!p || !info) return fail(RBC_EINVAL, "null argument");
  info->R = p->R;
  info->n0 = p->n0;
  info->levels = p->L;
  info->rand_mode = p->mode;
  info->draw_scope = p->scope;
  info->draw_count = p->draw_count;
  info->leaf_count = ipow(p->R, p->L);
  info->kappa = p->kappa;
  info->tau = p->tau;
  info->gamma = p->gamma;
  info->scale = p->scale;
  info->seed = p->seed;
  info->builtin_formula = p->builtin;
  return RBC_OK;
}

rbc_status rbc_plan_draws(rbc_plan_t p, int64_t first, int64_t count, int8_t* perms, int8_t* signs) {
  if (!p || (count > 0 && (!perms || !signs))) return fail(RBC_EINVAL, "null argument");
  if (first < 0 || count < 0 || first + count > p->draw_count)
    return fail(RBC_EINVAL, "draw range out of bounds");
  const size_t w = (size_t)3 * p->n0;
  std::memcpy(perms, p->perms.data() + first * w, (size_t)count * w);
  std::memcpy(signs, p->signs.data() + first * w, (size_t)count * w);
  return RBC_OK;
}

rbc_status rbc_plan_tables(rbc_plan_t p, int64_t key, double* Uh, double* Vh, double* Wh) {
  if (!p || !Uh || !Vh || !Wh) return fail(RBC_EINVAL, "null argument");
  if (key < 0 || key >= p->draw_count) return fail(RBC_EINVAL, "draw index out of bounds");
  const int n = p->n0, R = p->R;
  const int8_t* pi = p->perms.data() + key * 3 * n;
  const int8_t* s = p->signs.data() + key * 3 * n;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b)
      for (int r = 0; r < R; ++r) {
        const int e = (a * n + b) * R + r;
        Uh[e] = p->U[(pi[0 * n + a] * n + pi[1 * n + b]) * R + r] * s[0 * n + a] * s[1 * n + b];
        Vh[e] = p->V[(pi[1 * n + a] * n + pi[2 * n + b]) * R + r] * s[1 * n + a] * s[2 * n + b];
        Wh[e] = p->scale * s[0 * n + a] * s[2 * n + b] * p->W[(pi[0 * n + a] * n + pi[2 * n + b]) * R + r];
      }
  return RBC_OK;
}

const char* rbc_status_string(rbc_status s) {
  switch (s) {
    case RBC_OK: return "ok";
    case RBC_EINVAL: return "invalid argument";
    case RBC_ENOMEM: return "out of memory / workspace too small";
    case RBC_ECUDA: return "CUDA error";
    case RBC_ETIMEOUT: return "device wait timed out";
    case RBC_EBUSY: return "busy";
    case RBC_EKAPPA: return "kappa == 1";
    case RBC_EUNSUPPORTED: return "unsupported combination";
  }
  return "unknown status";
}

const char* rbc_last_error(void) { return g_last_error.c_str(); }

int rbc_version(void) { return 201; }

}  // extern "C"
