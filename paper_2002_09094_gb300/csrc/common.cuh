// Shared helpers of the libivfkm CUDA sources (sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#define IVF_FULL_MASK 0xffffffffu

namespace ivfk {

// Kernel launches counted process-wide (ivf_launch_count).
void note_launch();

// Error propagation inside host code: return the first failing cudaError_t.
#define IVF_CU(expr)                      \
  do {                                    \
    cudaError_t e__ = (expr);             \
    if (e__ != cudaSuccess) return e__;   \
  } while (0)

#define IVF_LAUNCH_CHECK()                \
  do {                                    \
    ::ivfk::note_launch();                \
    cudaError_t e__ = cudaGetLastError(); \
    if (e__ != cudaSuccess) return e__;   \
  } while (0)

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// FP32 bits -> the same value as FP64, from the IEEE 754 binary32 and
// binary64 layouts: for a normal number the sign is kept, the exponent is
// rebased from bias 127 to bias 1023 and the 23 fraction bits move to the
// top of the 52.  Integer operations only (FP64 conversions issue at the low
// FP64 rate of this part); zero, subnormal, infinite and NaN inputs take the
// hardware conversion.  Exact, like the conversion it replaces.
__device__ __forceinline__ double f32_bits_to_f64(uint32_t b) {
  const uint32_t e = (b >> 23) & 0xFFu;
  if (e == 0u || e == 0xFFu) return (double)__uint_as_float(b);
  const uint64_t d = ((uint64_t)(b >> 31) << 63) | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(b & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)d);
}

// Stored value -> float (storage types of the assignment stream).
__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(__half x) { return __half2float(x); }
__device__ __forceinline__ float to_f32(__nv_bfloat16 x) { return __bfloat162float(x); }

template <typename T>
__device__ __forceinline__ T from_f64(double x);
template <>
__device__ __forceinline__ float from_f64<float>(double x) { return __double2float_rn(x); }
template <>
__device__ __forceinline__ __half from_f64<__half>(double x) { return __float2half_rn(__double2float_rn(x)); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f64<__nv_bfloat16>(double x) {
  return __float2bfloat16_rn(__double2float_rn(x));
}

template <typename T>
__device__ __forceinline__ T from_f32(float x);
template <>
__device__ __forceinline__ float from_f32<float>(float x) { return x; }
template <>
__device__ __forceinline__ __half from_f32<__half>(float x) { return __float2half_rn(x); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

// Number of bits needed to hold values in [0, n).
inline int bits_for(int64_t n) {
  int b = 0;
  while (b < 63 && (int64_t(1) << b) < n) ++b;
  return b < 1 ? 1 : b;
}

}  // namespace ivfk
