// tsketch_dev.cuh -- device body of the TensorSketch kernel, shared by the
// single-problem kernel (tensorsketch.cu) and the batched one (batch.cu).
#pragma once

#include "common.cuh"

namespace idl {

constexpr int kTsMaxModes = 8;
constexpr int kTsThreads = 1024;

struct TsArgs {
  const float* F[kTsMaxModes];
  const int32_t* h[kTsMaxModes];
  const int8_t* s[kTsMaxModes];
  int64_t ldf[kTsMaxModes];
  int dims[kTsMaxModes];
  int N;
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In-place radix-2 DIT FFT of z (bit-reversed input, natural-order output).
// tw: per-stage twiddles, stage half-length hl at offset hl: exp(-i pi k / hl).
__device__ __forceinline__ void fft_inplace(float2* z, const float2* tw, int L, bool inverse) {
  for (int hl = 1; hl < L; hl <<= 1) {
    for (int b = threadIdx.x; b < (L >> 1); b += blockDim.x) {
      const int k = b & (hl - 1);
      const int i = ((b - k) << 1) + k;
      const int j = i + hl;
      float2 w = tw[hl + k];
      if (inverse) w.y = -w.y;
      const float2 t = cmul(w, z[j]);
      const float2 u = z[i];
      z[i] = make_float2(u.x + t.x, u.y + t.y);
      z[j] = make_float2(u.x - t.x, u.y - t.y);
    }
    __syncthreads();
  }
}

// One block: columns r0 and r0 + 1.  sm: (2 L + 2 (L/2 + 1)) float2 of shared memory.
__device__ __forceinline__ void tensorsketch_block(const TsArgs& a, int64_t R, int L, int logL,
                                                   const double* __restrict__ lambda, float* __restrict__ Y,
                                                   int64_t ldy, int64_t r0, float2* sm) {
  float2* z = sm;                    // L
  float2* tw = z + L;                // L (per-stage tables, offset 1..L-1)
  float2* P0 = tw + L;               // L/2 + 1
  float2* P1 = P0 + (L / 2 + 1);     // L/2 + 1
  const bool two = r0 + 1 < R;
  for (int q = threadIdx.x; q < L; q += blockDim.x) {
    if (q == 0) { tw[0] = make_float2(1.f, 0.f); continue; }
    const int hl = 1 << (31 - __clz(q));         // stage of this slot
    const int k = q - hl;
    float sv, cv;
    sincospif(-(float)k / (float)hl, &sv, &cv);
    tw[q] = make_float2(cv, sv);
  }
  for (int f = threadIdx.x; f <= L / 2; f += blockDim.x) { P0[f] = make_float2(1.f, 0.f); P1[f] = make_float2(1.f, 0.f); }
  const int shift = 32 - logL;
  for (int n = 0; n < a.N; ++n) {
    for (int q = threadIdx.x; q < L; q += blockDim.x) z[q] = make_float2(0.f, 0.f);
    __syncthreads();
    const float* f0 = a.F[n] + r0 * a.ldf[n];
    const float* f1 = f0 + a.ldf[n];
    const int In = a.dims[n];
    for (int i = threadIdx.x; i < In; i += blockDim.x) {
      const unsigned hv = (unsigned)a.h[n][i];
      if (hv >= (unsigned)L) continue;               // caller-supplied map out of range: entry skipped
      const int pos = (int)(__brev(hv) >> shift);
      const float sg = a.s[n][i] < 0 ? -1.f : 1.f;
      atomicAdd(&z[pos].x, sg * f0[i]);
      if (two) atomicAdd(&z[pos].y, sg * f1[i]);
    }
    __syncthreads();
    fft_inplace(z, tw, L, false);
    for (int f = threadIdx.x; f <= L / 2; f += blockDim.x) {
      const float2 zf = z[f];
      const float2 zc = z[(L - f) & (L - 1)];
      const float2 c0 = make_float2(0.5f * (zf.x + zc.x), 0.5f * (zf.y - zc.y));   // (Z + conj Zc)/2
      const float2 c1 = make_float2(0.5f * (zf.y + zc.y), -0.5f * (zf.x - zc.x));  // (Z - conj Zc)/2i
      P0[f] = cmul(P0[f], c0);
      P1[f] = cmul(P1[f], c1);
    }
    __syncthreads();
  }
  // W = P0 + i P1 over the full spectrum (mirror: P[L-f] = conj P[f]), bit-reversed
  for (int f = threadIdx.x; f < L; f += blockDim.x) {
    float2 p0, p1;
    if (f <= L / 2) { p0 = P0[f]; p1 = P1[f]; }
    else { p0 = P0[L - f]; p0.y = -p0.y; p1 = P1[L - f]; p1.y = -p1.y; }
    const int pos = (int)(__brev((unsigned)f) >> shift);
    z[pos] = make_float2(p0.x - p1.y, p0.y + p1.x);
  }
  __syncthreads();
  fft_inplace(z, tw, L, true);
  const float s0 = (float)(lambda[r0] / (double)L);
  const float s1 = two ? (float)(lambda[r0 + 1] / (double)L) : 0.f;
  for (int l = threadIdx.x; l < L; l += blockDim.x) {
    const float2 v = z[l];
    Y[(int64_t)l * ldy + r0] = v.x * s0;
    if (two) Y[(int64_t)l * ldy + r0 + 1] = v.y * s1;
  }
}

}  // namespace idl
