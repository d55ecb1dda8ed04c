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
constexpr int kRinvWarps = 4;        // FP64 inverse (FP64 pipes: spread over SMs)
constexpr int kRinvWarpsDf = 8;      // double-float inverse (FP32 pipes: more threads stage R11)

// inv(R11) in FP64, R11 = rows 0..K-1 of the pivot columns in pivot order
// (upper triangular).  One warp per column j of the inverse: column-oriented
// back substitution of R11 x = e_j (x_i = b_i / u_ii, then b_k -= u_ki x_i for
// k < i, lanes over k; only the 32-row chunks that still hold rows k < i are
// touched), with the K reciprocals 1/u_ii formed once.  Launched with kRinvWarps
// warps per block: GB300's FP64 pipe retires about two lanes per clock per SM,
// so the columns are spread over as many SMs as possible.  Output Rinv: K x K
// row-major, zero below the diagonal; Rsplit (optional): the same as FP32 pairs,
// hi = fl(x) in [0, K^2), lo = fl(x - hi) in [K^2, 2 K^2) -- the operand of the
// double-float product, split once here instead of in every product block.
template <typename T>
__device__ __forceinline__ void rinv_block(const T* __restrict__ Y, int ld, int K, int R, const int32_t* __restrict__ J,
                                          double* __restrict__ Rinv, int blk, int nblk, double* U,
                                          float* __restrict__ Rsplit = nullptr) {
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
        if (qq > q) break;                                            // rows k <= i only
        const int k = lane + 32 * qq;
        if (k == i) b[qq] = xi;
        else if (k < i) b[qq] -= U[k * KP + i] * xi;
      }
    }
#pragma unroll
    for (int q = 0; q < kSolveMaxK / 32; ++q) {
      const int k = lane + 32 * q;
      if (k < K) {
        const double x = (k <= j) ? b[q] : 0.0;
        Rinv[(int64_t)k * K + j] = x;
        if (Rsplit) {
          const float h = (float)x;
          Rsplit[k * K + j] = h;
          Rsplit[K * K + k * K + j] = (float)(x - (double)h);
        }
      }
    }
  }
}

// Double-float helpers: a value is an unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi) / 2 (Dekker 1971; Knuth's TwoSum), about 48 significant bits.
__device__ __forceinline__ void df_fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}
// (bh, bl) -= u * (xh, xl), u a float
__device__ __forceinline__ void df_sub_mul(float& bh, float& bl, float u, float xh, float xl) {
  const float p = u * xh;
  const float pe = fmaf(u, xh, -p) + u * xl;       // u x = p + pe (pe rounded)
  const float t = bh - p;                          // TwoSum(bh, -p)
  const float bv = t - bh;
  const float err = (bh - (t - bv)) + (-p - bv);
  df_fast_two_sum(t, err + (bl - pe), bh, bl);
}

// inv(R11) for FP32 sketches, in double-float arithmetic on the FP32 pipes
// (GB300's FP64 pipe adds about a microsecond of latency per step of the
// sequential back substitution: 29 us for K = 50 in FP64).  Same recurrence as
// rinv_block, with R11's entries exact FP32 values, 1/u_ii as a double-float
// (r = fl(1/u) + fl((1 - u fl(1/u)) fl(1/u))), x_i = b_i r_i, b_k -= u_ki x_i.
// Output: Rsplit as rinv_block's (hi in [0, K^2), lo in [K^2, 2 K^2)).  U: K x (K + 2)
// floats of shared memory (columns K, K+1: the reciprocal's hi and lo), then K
// ints (the pivots, staged first so that the gather of R11 issues its loads
// without waiting on J).
__device__ __forceinline__ void rinv_block_df(const float* __restrict__ Y, int ld, int K, int R,
                                             const int32_t* __restrict__ J, float* __restrict__ Rsplit, int blk,
                                             int nblk, float* U) {
  const int KP = K + 2;
  int* sJ = reinterpret_cast<int*>(U + K * KP);
  for (int q = threadIdx.x; q < K; q += blockDim.x) sJ[q] = J[q];
  __syncthreads();
#pragma unroll 8
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    const int j = e / K, i = e - j * K;
    const int jj = sJ[j];
    U[i * KP + j] = (i <= j && jj >= 0 && jj < R) ? Y[(int64_t)jj * ld + i] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    const float u = U[i * KP + i];
    const float rh = 1.f / u;
    U[i * KP + K] = rh;
    U[i * KP + K + 1] = fmaf(-u, rh, 1.f) * rh;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  for (int j = blk * nw + (threadIdx.x >> 5); j < K; j += nblk * nw) {
    float bh[kSolveMaxK / 32], bl[kSolveMaxK / 32];                  // b_k for k = lane + 32 q
#pragma unroll
    for (int q = 0; q < kSolveMaxK / 32; ++q) { bh[q] = (lane + 32 * q == j) ? 1.f : 0.f; bl[q] = 0.f; }
    for (int i = j; i >= 0; --i) {
      const int q = i >> 5;
      float ih = 0.f, il = 0.f;
#pragma unroll
      for (int qq = 0; qq < kSolveMaxK / 32; ++qq)
        if (qq == q) { ih = bh[qq]; il = bl[qq]; }
      ih = __shfl_sync(0xffffffffu, ih, i & 31);
      il = __shfl_sync(0xffffffffu, il, i & 31);
      // x_i = b_i * r_i (double-float product)
      const float rh = U[i * KP + K], rl = U[i * KP + K + 1];
      const float p = ih * rh;
      float xh, xl;
      df_fast_two_sum(p, fmaf(ih, rh, -p) + (ih * rl + il * rh), xh, xl);
#pragma unroll
      for (int qq = 0; qq < kSolveMaxK / 32; ++qq) {
        if (qq > q) break;                                            // rows k <= i only
        const int k = lane + 32 * qq;
        if (k == i) { bh[qq] = xh; bl[qq] = xl; }
        else if (k < i) df_sub_mul(bh[qq], bl[qq], U[k * KP + i], xh, xl);
      }
    }
#pragma unroll
    for (int q = 0; q < kSolveMaxK / 32; ++q) {
      const int k = lane + 32 * q;
      if (k < K) {
        Rsplit[k * K + j] = (k <= j) ? bh[q] : 0.f;
        Rsplit[K * K + k * K + j] = (k <= j) ? bl[q] : 0.f;
      }
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
constexpr int kTNBdf = 64;                 // columns per block of the double-float product

// (sh, sl) += (ah + al) b in double-float: ah b = p + e exactly (FMA), al b rounded,
// p added by TwoSum (Knuth), the small terms into sl.
__device__ __forceinline__ void df_acc(float& sh, float& sl, float ah, float al, float b) {
  const float p = ah * b;
  const float e = fmaf(ah, b, -p);
  const float q = fmaf(al, b, e);
  const float t = sh + p;
  const float bp = t - sh;
  const float err = (sh - (t - bp)) + (p - bp);
  sh = t;
  sl += err + q;
}

// Rsplit: inv(R11) as FP32 pairs (rinv_block's split output).  Block: kTNBdf
// non-skeleton columns, 256 threads; thread -> one row i (i = tid / 16 + 16 r) and
// four adjacent columns, so one (hi, lo) load of inv(R11) and one 16-byte load of
// R12 feed four independent double-float chains.  sh: tgemm_df_floats(K) floats
// (B starts on a 16-byte boundary for its float4 reads, whatever K's parity).
__host__ __device__ constexpr int tgemm_df_b_off(int K) { return (2 * K * K + 3) & ~3; }
__host__ __device__ constexpr int tgemm_df_floats(int K) { return tgemm_df_b_off(K) + K * (kTNBdf + 4) + kTNBdf; }
__device__ __forceinline__ void tgemm_block_df(const float* __restrict__ Y, int ld, int K, int R,
                                              const float* __restrict__ Rsplit, const int32_t* __restrict__ rest,
                                              int nrest, double* __restrict__ Tout, int blk, float* sh) {
  float2* A2 = reinterpret_cast<float2*>(sh);          // K x K (hi, lo)
  float* B = sh + tgemm_df_b_off(K);                   // K x BP, 16-byte aligned
  constexpr int BP = kTNBdf + 4;
  int* sr = reinterpret_cast<int*>(B + K * BP);        // the block's columns of A
  const int cb = blk * kTNBdf;
  // the column list first, so that the gather below issues independent loads
  if (threadIdx.x < kTNBdf) {
    const int c = cb + threadIdx.x;
    const int r = c < nrest ? rest[c] : -1;
    sr[threadIdx.x] = (r >= 0 && r < R) ? r : -1;
  }
#pragma unroll 4
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) A2[e] = make_float2(Rsplit[e], Rsplit[K * K + e]);
  __syncthreads();
#pragma unroll 4
  for (int e = threadIdx.x; e < K * kTNBdf; e += blockDim.x) {
    const int cc = e / K, i = e - cc * K;
    const int r = sr[cc];
    B[i * BP + cc] = r >= 0 ? Y[(int64_t)r * ld + i] : 0.f;
  }
  __syncthreads();
  const int cg = threadIdx.x & 15;
  const int c0 = cb + 4 * cg;
  for (int i = threadIdx.x >> 4; i < K; i += 16) {
    float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f, h3 = 0.f, l3 = 0.f;
    for (int k = i; k < K; ++k) {
      const float2 a = A2[i * K + k];
      const float4 b = *reinterpret_cast<const float4*>(B + k * BP + 4 * cg);
      df_acc(h0, l0, a.x, a.y, b.x);
      df_acc(h1, l1, a.x, a.y, b.y);
      df_acc(h2, l2, a.x, a.y, b.z);
      df_acc(h3, l3, a.x, a.y, b.w);
    }
    double* trow = Tout + (int64_t)i * nrest;
    if (c0 < nrest) trow[c0] = (double)h0 + (double)l0;
    if (c0 + 1 < nrest) trow[c0 + 1] = (double)h1 + (double)l1;
    if (c0 + 2 < nrest) trow[c0 + 2] = (double)h2 + (double)l2;
    if (c0 + 3 < nrest) trow[c0 + 3] = (double)h3 + (double)l3;
  }
}

template <typename T>
__device__ __forceinline__ void tgemm_block(const T* __restrict__ Y, int ld, int K, int R,
                                           const double* __restrict__ Rinv, const int32_t* __restrict__ rest,
                                           int nrest, double* __restrict__ Tout, int blk, double* sh) {
  double* Ri = sh;                         // K x K
  double* B = sh + K * K;                  // K x (kTNB + 1)
  const int BP = kTNB + 1;
  int* sr = reinterpret_cast<int*>(B + K * BP);   // the block's columns of A (kTNB ints)
  const int cb = blk * kTNB;
  if (threadIdx.x < kTNB) {
    const int c = cb + threadIdx.x;
    const int r = c < nrest ? rest[c] : -1;
    sr[threadIdx.x] = (r >= 0 && r < R) ? r : -1;
  }
#pragma unroll 4
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) Ri[e] = Rinv[e];
  __syncthreads();
#pragma unroll 4
  for (int e = threadIdx.x; e < K * kTNB; e += blockDim.x) {
    const int cc = e / K, i = e - cc * K;
    const int r = sr[cc];
    B[i * BP + cc] = r >= 0 ? (double)Y[(int64_t)r * ld + i] : 0.0;
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
