// Leaf products F^(0)(S, T) = S T (Section 2.1.1) on the CUDA cores, batched over all R^L
// leaves, for the fp64 and fp32 leaf modes (the tensor cores have no fp32-input or fast
// fp64 path).  Optional fused decode: the epilogue scatters the leaf's tile into every C
// block (I, J) with coefficient prod_d w^(node_d)_{i_d j_d r_d} (Eq. recursive-random-formula
// unrolled over the levels), by atomic adds into a zeroed C.
#include <cuda_runtime.h>

#include <cstring>

#include "decode_dest.cuh"
#include "level_kernels.cuh"

namespace rbc {

namespace {

// E elements as 16-byte vectors when they fill whole vectors (the address is then 16-byte
// aligned by construction), else one by one.
template <typename T, int E>
__device__ __forceinline__ void load_vec(T (&dst)[E], const T* src) {
  if constexpr (E * sizeof(T) % 16 == 0) {
#pragma unroll
    for (int q = 0; q < (int)(E * sizeof(T) / 16); ++q) {
      const int4 v = reinterpret_cast<const int4*>(src)[q];
      memcpy(reinterpret_cast<char*>(dst) + 16 * q, &v, 16);
    }
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) dst[e] = src[e];
  }
}

template <typename T, int E>
__device__ __forceinline__ void store_vec(T* dst, const T (&x)[E]) {
  if constexpr (E * sizeof(T) % 16 == 0) {
#pragma unroll
    for (int q = 0; q < (int)(E * sizeof(T) / 16); ++q) {
      int4 v;
      memcpy(&v, reinterpret_cast<const char*>(x) + 16 * q, 16);
      reinterpret_cast<int4*>(dst)[q] = v;
    }
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) dst[e] = x[e];
  }
}

// Micro-tile of a thread: TM rows and TN columns of the CTA tile, taken as two halves of
// contiguous rows (columns), one in each half of the tile, so that each half is read from
// shared memory (and written out) as one vector.
template <int H, int HALF>
__device__ __forceinline__ int micro_index(int t, int i) {
  return i < H ? t * H + i : HALF + t * H + (i - H);
}

// MODE (compiled in, so that each variant holds only its own epilogue): 0 store the product
// to M, 1 fused decode into C, 2 store C (L = 0).  CTAs of 128 threads are sized for three per
// SM (at most 170 registers a thread): the fp32 64 x 128 tiles with 8 x 8 micro-tiles measured
// 52.6 TFLOP/s on the leaves of randomized Strassen (n = 8192, L = 1..4), Laderman (n = 6561,
// L = 1..3) and perturbed Strassen (n = 4096, L = 1..3), against 49.0 for 128 x 128 tiles of 256
// threads at one CTA per SM.
template <typename T, int BM, int BN, int BK, int TM, int TN, int MODE>
__global__ void __launch_bounds__((BM / TM) * (BN / TN), (BM / TM) * (BN / TN) == 128 ? 3 : 1)
    simt_gemm_kernel(const __grid_constant__ Tables<T> t, const SimtGemmArgs a) {
  constexpr int TX = BN / TN, TY = BM / TM, NT = TX * TY;
  constexpr int HM = TM / 2, HN = TN / 2;  // contiguous rows / columns per half
  constexpr int EA = BM * BK / NT, EB = BN * BK / NT;
  static_assert(BK % EA == 0 && BN % EB == 0 && (BN / EB) * BK == NT, "tile/thread mismatch");
  constexpr int KA = BK / EA;   // threads per row of the S tile (BM rows x BK)
  constexpr int KB = BN / EB;   // threads per row of the T tile (BK rows x BN)
  __shared__ __align__(16) T As[2][BK][BM];
  __shared__ __align__(16) T Bs[2][BK][BN];
  __shared__ DestList<T> dl;

  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int64_t row0 = (int64_t)blockIdx.y * BM, col0 = (int64_t)blockIdx.x * BN;
  const int ar = tid / KA, ak = (tid % KA) * EA;
  const int bk = tid / KB, bn = (tid % KB) * EB;
  const int nk = (int)(a.K / BK);

  for (int64_t leaf = blockIdx.z; leaf < a.leaves; leaf += gridDim.z) {
    const T* S = static_cast<const T*>(a.S) + leaf * a.strideS + (row0 + ar) * a.lds + ak;
    const T* Tp = static_cast<const T*>(a.T) + leaf * a.strideT + (int64_t)bk * a.ldt + col0 + bn;
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = (T)0;

    T ra[EA], rb[EB];
    load_vec<T, EA>(ra, S);
    load_vec<T, EB>(rb, Tp);
    __syncthreads();  // previous leaf's readers are done with buffer 0
#pragma unroll
    for (int e = 0; e < EA; ++e) As[0][ak + e][ar] = ra[e];
#pragma unroll
    for (int e = 0; e < EB; ++e) Bs[0][bk][bn + e] = rb[e];
    __syncthreads();
    for (int kt = 0; kt < nk; ++kt) {
      const int buf = kt & 1;
      if (kt + 1 < nk) {
        load_vec<T, EA>(ra, S + (int64_t)(kt + 1) * BK);
        load_vec<T, EB>(rb, Tp + (int64_t)(kt + 1) * BK * a.ldt);
      }
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T av[TM], bv[TN];
        load_vec<T, HM>(*reinterpret_cast<T(*)[HM]>(av), &As[buf][kk][ty * HM]);
        load_vec<T, HM>(*reinterpret_cast<T(*)[HM]>(av + HM), &As[buf][kk][BM / 2 + ty * HM]);
        load_vec<T, HN>(*reinterpret_cast<T(*)[HN]>(bv), &Bs[buf][kk][tx * HN]);
        load_vec<T, HN>(*reinterpret_cast<T(*)[HN]>(bv + HN), &Bs[buf][kk][BN / 2 + tx * HN]);
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
      }
      if (kt + 1 < nk) {
#pragma unroll
        for (int e = 0; e < EA; ++e) As[buf ^ 1][ak + e][ar] = ra[e];
#pragma unroll
        for (int e = 0; e < EB; ++e) Bs[buf ^ 1][bk][bn + e] = rb[e];
      }
      __syncthreads();
    }

    if constexpr (MODE == 0) {
      T* M = static_cast<T*>(a.out) + leaf * a.strideO;
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        T* row = M + (row0 + micro_index<HM, BM / 2>(ty, i)) * a.ldo + col0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          T part[HN];
#pragma unroll
          for (int j = 0; j < HN; ++j) part[j] = acc[i][h * HN + j];
          store_vec<T, HN>(row + micro_index<HN, BN / 2>(tx, h * HN), part);
        }
      }
    } else if constexpr (MODE == 2) {
      T* C = static_cast<T*>(a.out);
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          const int64_t r = row0 + micro_index<HM, BM / 2>(ty, i), c = col0 + micro_index<HN, BN / 2>(tx, j);
          if (r < a.m && c < a.m) C[r * a.ldo + c] = acc[i][j];
        }
    } else {
      if (tid == 0) build_dest_list(t, leaf, dl);
      __syncthreads();
      T* C = static_cast<T*>(a.out);
      for (int d = 0; d < dl.total; ++d) {
        int64_t I, J;
        const T coef = dest_at(dl, d, t.n0, t.L, &I, &J);
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) {
            const int64_t r = row0 + micro_index<HM, BM / 2>(ty, i), c = col0 + micro_index<HN, BN / 2>(tx, j);
            if (r < a.m && c < a.m) atomicAdd(C + (I * a.m + r) * a.ldo + J * a.m + c, coef * acc[i][j]);
          }
      }
      __syncthreads();  // dl is rebuilt for the next leaf
    }
  }
}

// Small leaves (mp < 32, a multiple of 4): every product exactly m x m x m (the padding of
// S and T is zero and is skipped).  A CTA stages the S and T operands of `nl` consecutive
// leaves (contiguous ranges of the leaf buffers) in shared memory; each thread computes 2 x 2
// output blocks of the first 2 ceil(m/2) rows and columns, summing over k in order as the
// tiled kernel does.  Modes 0 (store M, its padding rows and columns set to zero like the
// tiled kernels' products of zero-padded operands) and 2 (store C, L = 0).
constexpr int kSmallThreads = 128;

template <typename T>
__global__ void __launch_bounds__(kSmallThreads) simt_small_gemm_kernel(const SimtGemmArgs a, int nl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int mp = (int)a.mp, mv = (int)a.m, hb = (mv + 1) / 2, units = hb * hb;
  const int per = mp * mp;  // elements of one leaf operand (lds = ldt = mp)
  T* sS = reinterpret_cast<T*>(smem_raw);
  T* sT = sS + (size_t)nl * per;
  const int64_t groups = (a.leaves + nl - 1) / nl;
  for (int64_t g = blockIdx.x; g < groups; g += gridDim.x) {
    const int64_t l0 = g * nl;
    const int cnt = (int)(a.leaves - l0 < nl ? a.leaves - l0 : nl);
    const T* S = static_cast<const T*>(a.S) + l0 * a.strideS;
    const T* Tg = static_cast<const T*>(a.T) + l0 * a.strideT;
    __syncthreads();  // the previous group's readers are done
    for (int e = threadIdx.x; e < cnt * per; e += kSmallThreads) {
      sS[e] = S[e];
      sT[e] = Tg[e];
    }
    __syncthreads();
    if (a.mode == 0) {  // zero padding of M beyond the computed 2 ceil(m/2) rows and columns
      const int mc = 2 * hb;
      for (int e = threadIdx.x; e < cnt * per; e += kSmallThreads) {
        const int lf = e / per, rc = e - lf * per, r = rc / mp, c = rc - r * mp;
        if (r >= mc || c >= mc) static_cast<T*>(a.out)[(l0 + lf) * a.strideO + r * a.ldo + c] = (T)0;
      }
    }
    for (int u = threadIdx.x; u < cnt * units; u += kSmallThreads) {
      const int lf = u / units, rem = u - lf * units, bi = rem / hb, bj = rem - bi * hb;
      const T* sr = sS + lf * per + 2 * bi * mp;
      const T* tc = sT + lf * per + 2 * bj;
      T c00 = (T)0, c01 = (T)0, c10 = (T)0, c11 = (T)0;
      for (int k = 0; k < mv; ++k) {
        const T s0 = sr[k], s1 = sr[mp + k], t0 = tc[k * mp], t1 = tc[k * mp + 1];
        c00 = fma(s0, t0, c00);
        c01 = fma(s0, t1, c01);
        c10 = fma(s1, t0, c10);
        c11 = fma(s1, t1, c11);
      }
      const int64_t r = 2 * bi, c = 2 * bj;
      if (a.mode == 0) {
        T* M = static_cast<T*>(a.out) + (l0 + lf) * a.strideO + r * a.ldo + c;
        M[0] = c00;
        M[1] = c01;
        M[a.ldo] = c10;
        M[a.ldo + 1] = c11;
      } else {
        T* C = static_cast<T*>(a.out) + r * a.ldo + c;
        const bool r1 = r + 1 < a.m, c1 = c + 1 < a.m;
        if (r < a.m && c < a.m) C[0] = c00;
        if (r < a.m && c1) C[1] = c01;
        if (r1 && c < a.m) C[a.ldo] = c10;
        if (r1 && c1) C[a.ldo + 1] = c11;
      }
    }
  }
}

template <typename T>
cudaError_t launch_small(const SimtGemmArgs& a, cudaStream_t st) {
  const int64_t per = a.mp * a.mp;
  if (a.mp % 4 || a.mp >= 32 || a.m > a.mp || a.K != a.mp || a.lds != a.mp || a.ldt != a.mp || a.strideS != per ||
      a.strideT != per || a.mode == 1 || (a.mode == 0 && (a.ldo != a.mp || a.strideO < per)))
    return cudaErrorInvalidValue;
  const int units = (int)((a.m + 1) / 2 * ((a.m + 1) / 2));
  // about two output blocks per thread, within 48 KB of shared memory
  int nl = (2 * kSmallThreads + units - 1) / units;
  const int fit = (int)((48 * 1024) / (2 * per * sizeof(T)));
  nl = nl < fit ? nl : fit;
  if (nl < 1) nl = 1;
  const int64_t groups = (a.leaves + nl - 1) / nl;
  const int64_t grid = groups < 152 * 16 ? groups : 152 * 16;
  const size_t smem = (size_t)2 * nl * per * sizeof(T);
  simt_small_gemm_kernel<T><<<(unsigned)grid, kSmallThreads, smem, st>>>(a, nl);
  return cudaGetLastError();
}

template <typename T, int BM, int BN, int BK, int TM, int TN>
cudaError_t launch_tile(const Tables<T>& t, const SimtGemmArgs& a, cudaStream_t st) {
  if (a.mp % BM || a.mp % BN || a.K % BK) return cudaErrorInvalidValue;
  const int64_t gz = a.leaves < 65535 ? a.leaves : 65535;
  const dim3 grid((unsigned)(a.mp / BN), (unsigned)(a.mp / BM), (unsigned)gz);
  constexpr int NT = (BM / TM) * (BN / TN);
  switch (a.mode) {
    case 0: simt_gemm_kernel<T, BM, BN, BK, TM, TN, 0><<<grid, NT, 0, st>>>(t, a); break;
    case 1: simt_gemm_kernel<T, BM, BN, BK, TM, TN, 1><<<grid, NT, 0, st>>>(t, a); break;
    case 2: simt_gemm_kernel<T, BM, BN, BK, TM, TN, 2><<<grid, NT, 0, st>>>(t, a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

// The large tile wherever it pads m to no more than the small tile plus 1/8.
int simt_tile(int io, int64_t m) {
  const int64_t big = io == RBC_IO_F32 ? 128 : 64;
  const int64_t pb = (m + big - 1) / big * big, ps = (m + 31) / 32 * 32;
  return m >= big && pb * 8 <= ps * 9 ? (int)big : 32;
}

int64_t simt_small_pad(int io, int64_t m) {
  (void)io;
  const int64_t mp = (m + 3) / 4 * 4;  // rows of whole 16-byte vectors for the pass kernels
  return mp < 32 ? mp : 0;
}

cudaError_t launch_simt_gemm(const Tables<float>& t, const SimtGemmArgs& a, cudaStream_t st) {
  if (a.mp < 32) return launch_small<float>(a, st);
  if (simt_tile(RBC_IO_F32, a.m) == 128) return launch_tile<float, 64, 128, 8, 8, 8>(t, a, st);
  return launch_tile<float, 32, 32, 8, 2, 2>(t, a, st);
}

cudaError_t launch_simt_gemm(const Tables<double>& t, const SimtGemmArgs& a, cudaStream_t st) {
  if (a.mp < 32) return launch_small<double>(a, st);
  if (simt_tile(RBC_IO_F64, a.m) == 64) return launch_tile<double, 64, 64, 8, 4, 4>(t, a, st);
  return launch_tile<double, 32, 32, 8, 2, 2>(t, a, st);
}

}  // namespace rbc
