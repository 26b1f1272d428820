// rbc_matmul_static: the same product as rbc_matmul, with its scratch taken from a fixed
// array that lives in the library's own device memory instead of a caller-provided
// workspace.
//
// Who needs this: callers that cannot obtain device memory at the point where they multiply
// -- code that runs while another component owns the whole device heap (a framework that
// reserves all free memory for its caching allocator up front), programs certified to
// allocate only during start-up, and code paths where an allocation failure cannot be
// handled.  They still pass A, B and C; everything else comes from the array below.
//
// The array is a file-scope __device__ object: every GPU that loads this library holds
// kStaticScratchBytes of it until the process exits.  Host code must not use the symbol
// itself as a pointer (on the host it is only a stand-in for the device object); the
// device address is looked up once per device with cudaGetSymbolAddress and cached for the
// life of the process (a device reset after the first call would leave it stale).  The
// status word of the bounded device waits sits at the start of the array, like at the start
// of a workspace; rbc_static_scratch_check reads and clears it.
#include <cuda_runtime.h>

#include <mutex>

#include "rbc_internal.h"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)64 << 20;  // 64 MiB

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up on first use).
rbc_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rbc::fail(RBC_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return rbc::fail(RBC_EUNSUPPORTED, "device ordinal above 63");
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return rbc::fail(RBC_ECUDA, cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return RBC_OK;
}

}  // namespace

extern "C" {

size_t rbc_static_scratch_bytes(void) { return kStaticScratchBytes; }

rbc_status rbc_matmul_static(rbc_plan_t plan, const void* A, const void* B, void* C, int64_t N, int64_t lda,
                             int64_t ldb, int64_t ldc, int io_dtype, int leaf_dtype, void* stream) {
  if (!plan || !A || !B || !C) return rbc::fail(RBC_EINVAL, "null argument");
  const size_t need = rbc_workspace_size(plan, N, io_dtype, leaf_dtype);
  if (need == 0) {
    // invalid combination: let the regular entry point report the precise reason
    return rbc_matmul(plan, A, B, C, N, lda, ldb, ldc, io_dtype, leaf_dtype, nullptr, 0, stream);
  }
  if (need > kStaticScratchBytes)
    return rbc::fail(RBC_ENOMEM, "product needs " + std::to_string(need) +
                                     " bytes of scratch; the static scratch holds 67108864 (64 MiB)");
  void* scratch = nullptr;
  rbc_status s = scratch_address(&scratch);
  if (s != RBC_OK) return s;
  return rbc_matmul(plan, A, B, C, N, lda, ldb, ldc, io_dtype, leaf_dtype, scratch, kStaticScratchBytes, stream);
}

void* rbc_static_scratch_ptr(void) {
  void* scratch = nullptr;
  return scratch_address(&scratch) == RBC_OK ? scratch : nullptr;
}

rbc_status rbc_static_scratch_check(void* stream, int* device_status) {
  if (!device_status) return rbc::fail(RBC_EINVAL, "null argument");
  void* scratch = nullptr;
  rbc_status s = scratch_address(&scratch);
  if (s != RBC_OK) return s;
  return rbc_workspace_check(scratch, stream, device_status);
}

}  // extern "C"
