// Leaf storage formats and the conversions the encode kernels apply when they write
// leaf operands (Section 2.1.1: leaves F^(0) are standard products in the leaf type).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>

namespace rbc {

enum LeafStore : int { kStoreF64 = 0, kStoreF32 = 1, kStoreTF32 = 2, kStoreBF16 = 3, kStoreF16 = 4 };

// The low fp16 piece of a split (f16x3 leaves) is stored multiplied by 2^11, so that it stays a
// normal fp16 number whenever the high piece is one (the remainder is at most 2^-11 of the
// value); the leaf kernel scales the cross-term products back by 2^-11.
constexpr float kF16LoScale = 2048.f;

// Round-to-nearest-even of an fp32 value to 10 explicit significand bits (tf32), kept in
// an fp32 container with the low 13 bits zero.  Integer arithmetic on the bit pattern;
// finite inputs only (the caller's data are finite).
__device__ __forceinline__ float round_tf32(float x) {
  uint32_t b = __float_as_uint(x);
  b = (b + 0xFFFu + ((b >> 13) & 1u)) & 0xFFFFE000u;
  return __uint_as_float(b);
}

template <int S> struct StoreType;
template <> struct StoreType<kStoreF64> { using T = double; };
template <> struct StoreType<kStoreF32> { using T = float; };
template <> struct StoreType<kStoreTF32> { using T = float; };
template <> struct StoreType<kStoreBF16> { using T = __nv_bfloat16; };
template <> struct StoreType<kStoreF16> { using T = __half; };

template <int S> __device__ __forceinline__ typename StoreType<S>::T to_store(double v);
template <> __device__ __forceinline__ double to_store<kStoreF64>(double v) { return v; }
template <> __device__ __forceinline__ float to_store<kStoreF32>(double v) { return (float)v; }
template <> __device__ __forceinline__ float to_store<kStoreTF32>(double v) { return round_tf32((float)v); }
template <> __device__ __forceinline__ __nv_bfloat16 to_store<kStoreBF16>(double v) {
  return __float2bfloat16_rn((float)v);
}
template <> __device__ __forceinline__ __half to_store<kStoreF16>(double v) {
  return __float2half_rn((float)v);
}

template <int S> __device__ __forceinline__ double from_store(typename StoreType<S>::T v);
template <> __device__ __forceinline__ double from_store<kStoreF64>(double v) { return v; }
template <> __device__ __forceinline__ double from_store<kStoreF32>(float v) { return v; }
template <> __device__ __forceinline__ double from_store<kStoreTF32>(float v) { return v; }
template <> __device__ __forceinline__ double from_store<kStoreBF16>(__nv_bfloat16 v) {
  return (double)__bfloat162float(v);
}
template <> __device__ __forceinline__ double from_store<kStoreF16>(__half v) {
  return (double)__half2float(v);
}

}  // namespace rbc
