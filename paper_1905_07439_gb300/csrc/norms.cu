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

}  // namespace
}  // namespace rbc

using namespace rbc;

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
