// Frobenius reductions in fp64 for the relative errors of Section 3
// (||C - C_ref|| / ||C_ref||).  Two kernels: fixed-size grid of per-block partial sums in
// a fixed order, then one warp summing the partials in a fixed order, so repeated calls
// give bit-identical results.
#include <cuda_runtime.h>

#include "rbc_internal.h"

namespace rbc {
namespace {

constexpr int kNormBlocks = 304;  // 2 x 152 SMs
constexpr int kNormThreads = 256;

template <typename TX, typename TY>
__global__ void __launch_bounds__(kNormThreads)
    norm_partial_kernel(const TX* X, const TY* Y, int64_t rows, int64_t cols, int64_t ldx,
                        int64_t ldy, double* work) {
  double d2 = 0.0, y2 = 0.0;
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e - r * cols;
    const double x = (double)X[r * ldx + c];
    if (Y) {
      const double y = (double)Y[r * ldy + c];
      d2 += (x - y) * (x - y);
      y2 += y * y;
    } else {
      d2 += x * x;
    }
  }
  __shared__ double sd[kNormThreads / 32], sy[kNormThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    d2 += __shfl_down_sync(0xffffffffu, d2, o);
    y2 += __shfl_down_sync(0xffffffffu, y2, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sd[wid] = d2;
    sy[wid] = y2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kNormThreads / 32; ++w) {
      a += sd[w];
      b += sy[w];
    }
    work[2 * blockIdx.x] = a;
    work[2 * blockIdx.x + 1] = b;
  }
}

__global__ void norm_final_kernel(const double* work, int nblocks, double* out) {
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += 32) {
    a += work[2 * i];
    b += work[2 * i + 1];
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if (threadIdx.x == 0) {
    out[0] = a;
    out[1] = b;
  }
}

template <typename TX, typename TY>
cudaError_t launch_norms(const void* X, const void* Y, int64_t rows, int64_t cols, int64_t ldx,
                         int64_t ldy, double* out, double* work, cudaStream_t st) {
  norm_partial_kernel<TX, TY><<<kNormBlocks, kNormThreads, 0, st>>>(
      static_cast<const TX*>(X), static_cast<const TY*>(Y), rows, cols, ldx, ldy, work);
  norm_final_kernel<<<1, 32, 0, st>>>(work, kNormBlocks, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- realization errors
// Errors of K realizations against a reference (Section 3).  Each CTA owns kErrPer elements
// (kErrEpt per thread, strided by the block size so that loads coalesce) and writes one
// partial sum of squared differences per realization (EACH) or per prefix length (AVERAGE:
// running sums of the realizations in fp64, the average formed as sum / n).  A final CTA
// sums the partials of every realization in CTA order.
constexpr int kErrThreads = 256, kErrEpt = 4, kErrPer = kErrThreads * kErrEpt;

__device__ __forceinline__ double block_sum(double v, double* sm) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sm[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kErrThreads / 32; ++w) s += sm[w];
  return s;  // valid in thread 0
}

template <typename TC>
__global__ void __launch_bounds__(kErrThreads)
    err_each_kernel(const TC* C, int64_t K, int64_t N, int64_t ldc, int64_t strideC, const double* Ref,
                    int64_t ldr, double* part, int64_t nblk) {
  __shared__ double sm[2][kErrThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kErrPer + threadIdx.x, total = N * N;
  int it = 0;
  for (int64_t k = blockIdx.y; k < K; k += gridDim.y, ++it) {
    double d2 = 0.0;
#pragma unroll
    for (int v = 0; v < kErrEpt; ++v) {
      const int64_t e = base + (int64_t)v * kErrThreads;
      if (e < total) {
        const int64_t r = e / N, c = e - r * N;
        const double d = (double)C[k * strideC + r * ldc + c] - Ref[r * ldr + c];
        d2 += d * d;
      }
    }
    const double s = block_sum(d2, sm[it & 1]);
    if (threadIdx.x == 0) part[k * nblk + blockIdx.x] = s;
  }
}

// Error of the running average, in segments of `seg` realizations so that the sequential
// scan over K runs in parallel: (1) per element, the sum of each segment; (2) per element,
// the exclusive prefix of the segment sums, in segment order; (3) per segment, the running
// sums continued from the prefix, one squared-error partial per realization and CTA.
template <typename TC>
__global__ void __launch_bounds__(kErrThreads)
    err_segsum_kernel(const TC* C, int64_t K, int64_t N, int64_t ldc, int64_t strideC, int64_t seg, double* segsum) {
  const int64_t total = N * N, base = (int64_t)blockIdx.x * kErrPer + threadIdx.x;
  const int64_t n0 = (int64_t)blockIdx.y * seg, n1 = n0 + seg < K ? n0 + seg : K;
#pragma unroll
  for (int v = 0; v < kErrEpt; ++v) {
    const int64_t e = base + (int64_t)v * kErrThreads;
    if (e >= total) continue;
    const int64_t r = e / N, c = e - r * N;
    double sum = 0.0;
    for (int64_t n = n0; n < n1; ++n) sum += (double)C[n * strideC + r * ldc + c];
    segsum[(int64_t)blockIdx.y * total + e] = sum;
  }
}

__global__ void __launch_bounds__(kErrThreads) err_prefix_kernel(int64_t total, int64_t nseg, double* segsum) {
  const int64_t e = (int64_t)blockIdx.x * kErrThreads + threadIdx.x;
  if (e >= total) return;
  double run = 0.0;
  for (int64_t s = 0; s < nseg; ++s) {
    const double t = segsum[s * total + e];
    segsum[s * total + e] = run;
    run += t;
  }
}

template <typename TC>
__global__ void __launch_bounds__(kErrThreads)
    err_average_kernel(const TC* C, int64_t K, int64_t N, int64_t ldc, int64_t strideC, const double* Ref,
                       int64_t ldr, int64_t seg, const double* prefix, double* part, int64_t nblk) {
  __shared__ double sm[2][kErrThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kErrPer + threadIdx.x, total = N * N;
  const int64_t n0 = (int64_t)blockIdx.y * seg, n1 = n0 + seg < K ? n0 + seg : K;
  int64_t off[kErrEpt];
  double ref[kErrEpt], sum[kErrEpt];
  TC next[kErrEpt];
#pragma unroll
  for (int v = 0; v < kErrEpt; ++v) {
    const int64_t e = base + (int64_t)v * kErrThreads;
    const bool in = e < total;
    const int64_t r = in ? e / N : 0, c = in ? e - r * N : 0;
    off[v] = in ? r * ldc + c : -1;
    ref[v] = in ? Ref[r * ldr + c] : 0.0;
    sum[v] = in ? prefix[(int64_t)blockIdx.y * total + e] : 0.0;
    next[v] = (off[v] >= 0 && n0 < n1) ? C[n0 * strideC + off[v]] : (TC)0;
  }
  for (int64_t n = n0; n < n1; ++n) {
    TC cur[kErrEpt];
#pragma unroll
    for (int v = 0; v < kErrEpt; ++v) {
      cur[v] = next[v];
      // prefetch realization n + 1 while this one is reduced
      next[v] = (off[v] >= 0 && n + 1 < n1) ? C[(n + 1) * strideC + off[v]] : (TC)0;
    }
    const double inv = 1.0 / (double)(n + 1);
    double d2 = 0.0;
#pragma unroll
    for (int v = 0; v < kErrEpt; ++v) {
      if (off[v] < 0) continue;
      sum[v] += (double)cur[v];
      const double d = sum[v] * inv - ref[v];
      d2 += d * d;
    }
    const double s = block_sum(d2, sm[n & 1]);
    if (threadIdx.x == 0) part[n * nblk + blockIdx.x] = s;
  }
}

// err[k] = sqrt(sum_b part[k][b]) / ||Ref||, ||Ref||^2 from the norm partials in CTA order.
__global__ void __launch_bounds__(kErrThreads)
    err_final_kernel(const double* part, int64_t K, int64_t nblk, const double* ref_part, int nref, double* err) {
  __shared__ double sm[kErrThreads / 32];
  __shared__ double ref2;
  double a = 0.0;
  for (int i = threadIdx.x; i < nref; i += kErrThreads) a += ref_part[2 * i];
  const double s = block_sum(a, sm);
  if (threadIdx.x == 0) ref2 = s;
  __syncthreads();
  const double rn = sqrt(ref2);
  for (int64_t k = threadIdx.x; k < K; k += kErrThreads) {
    double t = 0.0;
    for (int64_t b = 0; b < nblk; ++b) t += part[k * nblk + b];
    err[k] = sqrt(t) / rn;
  }
}

inline int64_t err_blocks(int64_t N) { return (N * N + kErrPer - 1) / kErrPer; }
// Segments of the running-average scan: 32 realizations each, at most 2^25 segment sums.
inline int64_t err_segments(int64_t K, int64_t N) {
  const int64_t want = (K + 31) / 32, cap = (int64_t)1 << 25;
  const int64_t fit = N * N > 0 ? cap / (N * N) : want;
  int64_t n = want < fit ? want : fit;
  if (n > 65535) n = 65535;  // grid y
  return n < 1 ? 1 : n;
}

}  // namespace
}  // namespace rbc

using namespace rbc;

extern "C" size_t rbc_realization_errors_work_size(int64_t K, int64_t N) {
  if (K < 0 || N < 0) return 0;
  return sizeof(double) * ((size_t)K * (size_t)err_blocks(N) + 2 * kNormBlocks +
                            (size_t)err_segments(K, N) * (size_t)(N * N));
}

extern "C" rbc_status rbc_realization_errors(const void* C, int ct, int64_t K, int64_t N, int64_t ldc,
                                             int64_t strideC, const double* Ref, int64_t ldr, int mode, double* err,
                                             void* work, size_t work_bytes, void* stream) {
  if (!C || !Ref || !err || !work) return fail(RBC_EINVAL, "null argument");
  if (K < 1 || N < 1 || ldc < N || ldr < N || (K > 1 && strideC < ldc * N))
    return fail(RBC_EINVAL, "bad shape: K, N >= 1, ldc, ldr >= N, strideC >= ldc * N");
  if (ct != RBC_IO_F32 && ct != RBC_IO_F64) return fail(RBC_EINVAL, "bad dtype");
  if (mode != RBC_ERR_EACH && mode != RBC_ERR_AVERAGE) return fail(RBC_EINVAL, "bad error mode");
  if (work_bytes < rbc_realization_errors_work_size(K, N)) return fail(RBC_ENOMEM, "error workspace too small");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t nblk = err_blocks(N);
  if (nblk > 0x7fffffff) return fail(RBC_EINVAL, "N too large");
  double* part = static_cast<double*>(work);
  double* ref_part = part + K * nblk;
  norm_partial_kernel<double, double><<<kNormBlocks, kNormThreads, 0, st>>>(Ref, (const double*)nullptr, N, N, ldr,
                                                                             0, ref_part);
  if (mode == RBC_ERR_EACH) {
    const dim3 grid((unsigned)nblk, (unsigned)(K < 65535 ? K : 65535));
    if (ct == RBC_IO_F32)
      err_each_kernel<float><<<grid, kErrThreads, 0, st>>>(static_cast<const float*>(C), K, N, ldc, strideC, Ref,
                                                           ldr, part, nblk);
    else
      err_each_kernel<double><<<grid, kErrThreads, 0, st>>>(static_cast<const double*>(C), K, N, ldc, strideC,
                                                            Ref, ldr, part, nblk);
  } else {
    const int64_t nseg = err_segments(K, N), seg = (K + nseg - 1) / nseg;
    double* segsum = ref_part + 2 * kNormBlocks;
    const dim3 grid((unsigned)nblk, (unsigned)nseg);
    const unsigned pgrid = (unsigned)((N * N + kErrThreads - 1) / kErrThreads);
    if (ct == RBC_IO_F32) {
      const float* Cf = static_cast<const float*>(C);
      err_segsum_kernel<float><<<grid, kErrThreads, 0, st>>>(Cf, K, N, ldc, strideC, seg, segsum);
      err_prefix_kernel<<<pgrid, kErrThreads, 0, st>>>(N * N, nseg, segsum);
      err_average_kernel<float><<<grid, kErrThreads, 0, st>>>(Cf, K, N, ldc, strideC, Ref, ldr, seg, segsum, part,
                                                              nblk);
    } else {
      const double* Cd = static_cast<const double*>(C);
      err_segsum_kernel<double><<<grid, kErrThreads, 0, st>>>(Cd, K, N, ldc, strideC, seg, segsum);
      err_prefix_kernel<<<pgrid, kErrThreads, 0, st>>>(N * N, nseg, segsum);
      err_average_kernel<double><<<grid, kErrThreads, 0, st>>>(Cd, K, N, ldc, strideC, Ref, ldr, seg, segsum, part,
                                                               nblk);
    }
  }
  err_final_kernel<<<1, kErrThreads, 0, st>>>(part, K, nblk, ref_part, kNormBlocks, err);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RBC_OK : fail(RBC_ECUDA, cudaGetErrorString(e));
}

extern "C" size_t rbc_norms_work_size(void) { return sizeof(double) * 2 * kNormBlocks; }

extern "C" rbc_status rbc_norms(const void* X, const void* Y, int64_t rows, int64_t cols,
                                int64_t ldx, int64_t ldy, int xt, int yt, double* out, void* work,
                                size_t work_bytes, void* stream) {
  if (!X || !out || !work) return fail(RBC_EINVAL, "null argument");
  if (rows < 0 || cols < 0 || ldx < cols || (Y && ldy < cols)) return fail(RBC_EINVAL, "bad shape");
  if (work_bytes < rbc_norms_work_size()) return fail(RBC_ENOMEM, "norm workspace too small");
  if ((xt != RBC_IO_F32 && xt != RBC_IO_F64) || (Y && yt != RBC_IO_F32 && yt != RBC_IO_F64))
    return fail(RBC_EINVAL, "bad dtype");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* w = static_cast<double*>(work);
  cudaError_t e;
  if (!Y) yt = xt;
  if (xt == RBC_IO_F32 && yt == RBC_IO_F32)
    e = launch_norms<float, float>(X, Y, rows, cols, ldx, ldy, out, w, st);
  else if (xt == RBC_IO_F32)
    e = launch_norms<float, double>(X, Y, rows, cols, ldx, ldy, out, w, st);
  else if (yt == RBC_IO_F32)
    e = launch_norms<double, float>(X, Y, rows, cols, ldx, ldy, out, w, st);
  else
    e = launch_norms<double, double>(X, Y, rows, cols, ldx, ldy, out, w, st);
  if (e != cudaSuccess) return fail(RBC_ECUDA, cudaGetErrorString(e));
  return RBC_OK;
}
