// tsolve_dev.cuh -- device bodies of T = inv(R11) R12 (FP64) and of the
// s-value update, shared by cpqr.cu and batch.cu.
#pragma once

#include "common.cuh"

namespace idl {

// rest[pos] = r for the non-skeleton columns r, ascending (sJ: the K pivots in shared memory)
__device__ __forceinline__ void rest_elem(int r, const int32_t* sJ, int K, int R, int32_t* __restrict__ rest) {
  int less = 0;
  bool piv = false;
  for (int q = 0; q < K; ++q) {
    const int j = sJ[q];
    if (j < 0 || j >= R) continue;               // invalid pivots (flagged upstream) are ignored
    less += j < r;
    piv |= j == r;
  }
  const int pos = r - less;
  if (!piv && pos >= 0 && pos < R - K) rest[pos] = r;
}

constexpr int kSolveMaxK = 128;
constexpr int kRinvWarps = 4;

// inv(R11) in FP64, R11 = rows 0..K-1 of the pivot columns in pivot order
// (upper triangular).  One warp per column j of the inverse: column-oriented
// back substitution of R11 x = e_j (x_i = b_i / u_ii, then b_k -= u_ki x_i for
// k < i, lanes over k), with the K reciprocals 1/u_ii formed once.  Launched
// with kRinvWarps warps per block (columns spread over the SMs' FP64 units;
// every thread of the block helps stage R11).  Output Rinv: K x K row-major,
// zero below the diagonal.
template <typename T>
__device__ __forceinline__ void rinv_block(const T* __restrict__ Y, int ld, int K, int R, const int32_t* __restrict__ J,
                                          double* __restrict__ Rinv, int blk, int nblk, double* U) {
  // U: K x (K+1) doubles of shared memory; its column K holds 1/u_ii
  const int KP = K + 1;
#pragma unroll 4
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    const int j = e / K, i = e - j * K;                              // column j (pivot j), row i
    const int jj = J[j];
    U[i * KP + j] = (i <= j && jj >= 0 && jj < R) ? (double)Y[(int64_t)jj * ld + i] : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < K; i += blockDim.x) U[i * KP + K] = 1.0 / U[i * KP + i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  for (int j = blk * nw + (threadIdx.x >> 5); j < K; j += nblk * nw) {
    double b[kSolveMaxK / 32];                                        // b_k for k = lane + 32 q
#pragma unroll
    for (int q = 0; q < kSolveMaxK / 32; ++q) b[q] = (lane + 32 * q == j) ? 1.0 : 0.0;
    for (int i = j; i >= 0; --i) {
      // owner lane of row i holds b_i
      const int q = i >> 5;
      double bi = 0.0;
#pragma unroll
      for (int qq = 0; qq < kSolveMaxK / 32; ++qq)
        if (qq == q) bi = b[qq];
      bi = __shfl_sync(0xffffffffu, bi, i & 31);
      const double xi = bi * U[i * KP + K];
#pragma unroll
      for (int qq = 0; qq < kSolveMaxK / 32; ++qq) {
        const int k = lane + 32 * qq;
        if (k == i) b[qq] = xi;
        else if (k < i) b[qq] -= U[k * KP + i] * xi;
      }
    }
#pragma unroll
    for (int q = 0; q < kSolveMaxK / 32; ++q) {
      const int k = lane + 32 * q;
      if (k < K) Rinv[(int64_t)k * K + j] = (k <= j) ? b[q] : 0.0;
    }
  }
}

// T[:, c] = inv(R11) R12[:, c] for the non-skeleton columns c, FP64.  A block owns
// 64 columns; inv(R11) and the block's R12 rows sit in shared memory; every
// thread forms whole dot products (no sequential dependence between outputs).
constexpr int kTNB = 64;
// FP32 sketches: R12 holds FP32 values, so T = inv(R11) R12 is accumulated
// in double-float arithmetic on the FP32 pipes: inv(R11) = a_hi + a_lo
// (two floats), a_hi b exactly by an FMA (p + e), a_lo b rounded, sums by
// TwoSum (Knuth) into a (hi, lo) pair -- about 48 significant bits, far
// below the FP32 sketch's own rounding, at a fraction of the FP64 pipes' cost.
constexpr int kTNBdf = 32;                 // columns per block of the double-float product
__device__ __forceinline__ void tgemm_block_df(const float* __restrict__ Y, int ld, int K, int R,
                                              const double* __restrict__ Rinv, const int32_t* __restrict__ rest,
                                              int nrest, double* __restrict__ Tout, int blk, float* sh) {
  float* Ah = sh;                          // K x K
  float* Al = Ah + K * K;                  // K x K
  float* B = Al + K * K;                   // K x (kTNBdf + 1)
  const int BP = kTNBdf + 1;
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    const double a = Rinv[e];
    const float h = (float)a;
    Ah[e] = h;
    Al[e] = (float)(a - (double)h);
  }
  const int cb = blk * kTNBdf;
  for (int e = threadIdx.x; e < K * kTNBdf; e += blockDim.x) {
    const int cc = e / K, i = e - cc * K;
    const int c = cb + cc;
    const int r = (c < nrest) ? rest[c] : -1;
    B[i * BP + cc] = (r >= 0 && r < R) ? Y[(int64_t)r * ld + i] : 0.f;
  }
  __syncthreads();
  const int cc = threadIdx.x & (kTNBdf - 1);
  const int c = cb + cc;
  for (int i = threadIdx.x >> 5; i < K; i += blockDim.x >> 5) {
    float sh_ = 0.f, sl = 0.f;
    for (int k = i; k < K; ++k) {
      const float ah = Ah[i * K + k], al = Al[i * K + k], b = B[k * BP + cc];
      const float p = ah * b;
      const float e = fmaf(ah, b, -p);                 // ah b = p + e exactly
      const float q = fmaf(al, b, e);
      const float t = sh_ + p;                         // TwoSum(sh_, p)
      const float bp = t - sh_;
      const float err = (sh_ - (t - bp)) + (p - bp);
      sh_ = t;
      sl += err + q;
    }
    if (c < nrest) Tout[(int64_t)i * nrest + c] = (double)sh_ + (double)sl;
  }
}

template <typename T>
__device__ __forceinline__ void tgemm_block(const T* __restrict__ Y, int ld, int K, int R,
                                           const double* __restrict__ Rinv, const int32_t* __restrict__ rest,
                                           int nrest, double* __restrict__ Tout, int blk, double* sh) {
  double* Ri = sh;                         // K x K
  double* B = sh + K * K;                  // K x (kTNB + 1)
  const int BP = kTNB + 1;
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) Ri[e] = Rinv[e];
  const int cb = blk * kTNB;
  for (int e = threadIdx.x; e < K * kTNB; e += blockDim.x) {
    const int cc = e / K, i = e - cc * K;
    const int c = cb + cc;
    const int r = (c < nrest) ? rest[c] : -1;
    B[i * BP + cc] = (r >= 0 && r < R) ? (double)Y[(int64_t)r * ld + i] : 0.0;
  }
  __syncthreads();
  // thread -> (column cc = tid % 64, rows i = tid / 64 + 4 q)
  const int cc = threadIdx.x & (kTNB - 1);
  const int c = cb + cc;
  for (int i = threadIdx.x >> 6; i < K; i += blockDim.x >> 6) {
    double acc0 = 0.0, acc1 = 0.0;
    int k = i;
    for (; k + 1 < K; k += 2) {
      acc0 = fma(Ri[i * K + k], B[k * BP + cc], acc0);
      acc1 = fma(Ri[i * K + k + 1], B[(k + 1) * BP + cc], acc1);
    }
    if (k < K) acc0 = fma(Ri[i * K + k], B[k * BP + cc], acc0);
    if (c < nrest) Tout[(int64_t)i * nrest + c] = acc0 + acc1;
  }
}

// lambda_hat_k = lambda_{J_k} (1 + sum_c T_kc)  (Algorithm 3); one block per k
__device__ __forceinline__ void lambda_hat_block(const double* __restrict__ lam, const int32_t* __restrict__ J,
                                                 const double* __restrict__ Tm, int nrest, int K,
                                                 double* __restrict__ out, int k) {
  __shared__ double part[32];
  double s = 0.0;
  for (int c = threadIdx.x; c < nrest; c += blockDim.x) s += Tm[(int64_t)k * nrest + c];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) {
      const int j = J[k];
      out[k] = (j >= 0 && j < nrest + K) ? lam[j] * (1.0 + s) : 0.0;
    }
  }
  __syncthreads();
}

}  // namespace idl
