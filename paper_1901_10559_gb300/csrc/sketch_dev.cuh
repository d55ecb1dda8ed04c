// sketch_dev.cuh -- device bodies of the CountSketch kernels, shared by the
// single-problem kernels (countsketch.cu) and the batched ones (batch.cu).
#pragma once

#include "common.cuh"

namespace idl {

template <typename T> __device__ __forceinline__ typename Vec4<T>::type ldcs_vec(const T* p);
template <> __device__ __forceinline__ float4 ldcs_vec<float>(const float* p) { return __ldcs((const float4*)p); }
template <> __device__ __forceinline__ double2 ldcs_vec<double>(const double* p) { return __ldcs((const double2*)p); }

__device__ __forceinline__ void vadd(float4& a, const float4& v, bool neg) {
  if (neg) { a.x -= v.x; a.y -= v.y; a.z -= v.z; a.w -= v.w; }
  else     { a.x += v.x; a.y += v.y; a.z += v.z; a.w += v.w; }
}
__device__ __forceinline__ void vadd(double2& a, const double2& v, bool neg) {
  if (neg) { a.x -= v.x; a.y -= v.y; } else { a.x += v.x; a.y += v.y; }
}

// One block of the dense CountSketch: bucket b, column tile `tile` (blockDim.x
// vectors of 16 bytes): Y[b, cols] = sum over the bucket's rows i of s[i] A[i, cols]
// (accum: added to Y's current values -- the sketch of a further block of rows).
template <typename T, bool VEC>
__device__ __forceinline__ void cs_dense_block(const T* __restrict__ A, int64_t lda, int64_t R,
                                               const int8_t* __restrict__ s, const int32_t* __restrict__ ptr,
                                               const int32_t* __restrict__ rows, T* __restrict__ Y, int64_t ldy,
                                               int64_t b, int tile, bool accum = false) {
  using V = typename Vec4<T>::type;
  constexpr int W = 16 / sizeof(T);  // elements per vector
  const int64_t c0 = ((int64_t)tile * blockDim.x + threadIdx.x) * W;
  if (c0 >= R) return;
  const int a0 = ptr[b], a1 = ptr[b + 1];
  T* yrow = Y + b * ldy + c0;
  if (VEC && c0 + W <= R) {
    V acc;
    if constexpr (W == 4) acc = make_float4(0.f, 0.f, 0.f, 0.f); else acc = make_double2(0.0, 0.0);
    const T* Ab = A + c0;                      // column c0 of row 0
    int j = a0;
    for (; j + 4 <= a1; j += 4) {
      const int r0 = rows[j], r1 = rows[j + 1], r2 = rows[j + 2], r3 = rows[j + 3];
      const V v0 = ldcs_vec<T>(Ab + (int64_t)r0 * lda);
      const V v1 = ldcs_vec<T>(Ab + (int64_t)r1 * lda);
      const V v2 = ldcs_vec<T>(Ab + (int64_t)r2 * lda);
      const V v3 = ldcs_vec<T>(Ab + (int64_t)r3 * lda);
      const bool n0 = s[r0] < 0, n1 = s[r1] < 0, n2 = s[r2] < 0, n3 = s[r3] < 0;
      vadd(acc, v0, n0);
      vadd(acc, v1, n1);
      vadd(acc, v2, n2);
      vadd(acc, v3, n3);
    }
    for (; j < a1; ++j) {
      const int r = rows[j];
      vadd(acc, ldcs_vec<T>(Ab + (int64_t)r * lda), s[r] < 0);
    }
    if (accum) vadd(acc, *(const V*)yrow, false);
    *(V*)yrow = acc;
  } else {
    const int w = (int)((R - c0) < W ? (R - c0) : W);
    T acc[W];
#pragma unroll
    for (int q = 0; q < W; ++q) acc[q] = T(0);
    for (int j = a0; j < a1; ++j) {
      const int r = rows[j];
      const bool neg = s[r] < 0;
      const T* ap = A + (int64_t)r * lda + c0;
#pragma unroll
      for (int q = 0; q < W; ++q)
        if (q < w) acc[q] += neg ? -ap[q] : ap[q];
    }
#pragma unroll
    for (int q = 0; q < W; ++q)
      if (q < w) yrow[q] = accum ? yrow[q] + acc[q] : acc[q];
  }
}

}  // namespace idl
