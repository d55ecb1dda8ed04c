// common.cuh -- shared device helpers of libidl (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/idl.h"

namespace idl {

// Process-wide count of kernel launches made by this library (idl_launch_count).
void count_launch();

// ----------------------------------------------------------------------------
// Status word: kernels record the first error they see (atomicCAS from OK).
// ----------------------------------------------------------------------------
__device__ __forceinline__ void set_status(int* status, int code) {
  if (status) atomicCAS(status, IDL_OK, code);
}

// ----------------------------------------------------------------------------
// Counter-based draws (SplitMix64 finaliser; Steele, Lea & Flood 2014).
//   u(seed, tag, i) = mix64(base(seed, tag) + (i + 1) * GAMMA)
//   base(seed, tag) = mix64(seed ^ tag * C_TAG)
// ----------------------------------------------------------------------------
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kTagMul = 0xD1B54A32D192ED03ull;
enum : uint32_t { kTagBucket = 1, kTagSign = 2, kTagPerm = 3, kTagGauss = 4, kTagGaussId = 5, kTagErrStart = 6,
                  kTagModeBucket = 16, kTagModeSign = 32, kTagGaussMode = 48 };
constexpr int kFeistelRounds = 4;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t stream_base(uint64_t seed, uint32_t tag) {
  return mix64(seed ^ (uint64_t(tag) * kTagMul));
}
__host__ __device__ __forceinline__ uint64_t stream_at(uint64_t base, uint64_t i) {
  return mix64(base + (i + 1) * kGamma);
}
// floor(u * L / 2^64)  (multiply-shift, Lemire 2019)
__device__ __forceinline__ uint32_t bounded(uint64_t u, uint64_t L) {
  return uint32_t(__umul64hi(u, L));
}

// ----------------------------------------------------------------------------
// Small utilities
// ----------------------------------------------------------------------------
__host__ __device__ __forceinline__ int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ int64_t round_up(int64_t a, int64_t b) { return cdiv(a, b) * b; }

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double2; };  // 16-byte vector of doubles

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace idl
