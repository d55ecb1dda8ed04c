// gaussian.cu -- the Gaussian stage Y2 = Omega Y1 (Sec. 1.2.1) on CUDA cores.
//
// Output is column-major (Y2 = (Y1^T Omega^T)^T, one contiguous column of m2
// values per original column r), which is the layout the QR stage reads.
//
// This file holds the FP64 path (CUDA cores) and a CUDA-core FP32 path kept
// for comparison; FP32 data go to the tcgen05 path of gaussian_tc.cu by
// default.  Split-K over m1 with a second pass that sums the partial products
// in a fixed order.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace idl {

constexpr int kGBN = 64;     // columns r per block
constexpr int kGBK = 32;     // m1 per smem stage
constexpr int kGThreads = 256;

// Y1 tile: kGBK x kGBN; Omega^T tile: kGBK x MP (MP = m2 rounded to 16).
// Thread (ty, tx): tx in [0,16) owns 4 columns, ty in [0,16) owns rows ty + 16q.
template <typename T, int MQ>
__global__ void __launch_bounds__(kGThreads) gauss_simt_kernel(const T* __restrict__ Om, int m2, int64_t m1,
                                                               const T* __restrict__ Y1, int64_t R, int64_t ldy1,
                                                               int64_t kchunk, T* __restrict__ part, int MP,
                                                               int rbf16) {
  __shared__ T ys[kGBK][kGBN];
  __shared__ T os[kGBK][16 * MQ + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t r0 = (int64_t)blockIdx.x * kGBN;
  const int64_t k0 = (int64_t)blockIdx.y * kchunk;
  const int64_t k1 = min(m1, k0 + kchunk);
  T acc[MQ][4];
#pragma unroll
  for (int q = 0; q < MQ; ++q)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[q][c] = T(0);
  for (int64_t kb = k0; kb < k1; kb += kGBK) {
    for (int e = threadIdx.x; e < kGBK * kGBN; e += kGThreads) {
      const int kk = e / kGBN, cc = e % kGBN;
      const int64_t k = kb + kk, r = r0 + cc;
      T y = (k < k1 && r < R) ? Y1[k * ldy1 + r] : T(0);
      if (rbf16) y = (T)__bfloat162float(__float2bfloat16_rn((float)y));
      ys[kk][cc] = y;
    }
    for (int e = threadIdx.x; e < kGBK * 16 * MQ; e += kGThreads) {
      const int j = e / kGBK, kk = e % kGBK;
      const int64_t k = kb + kk;
      T o = (k < k1 && j < m2) ? Om[(int64_t)j * m1 + k] : T(0);
      if (rbf16) o = (T)__bfloat162float(__float2bfloat16_rn((float)o));
      os[kk][j] = o;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kGBK; ++kk) {
      T y[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) y[c] = ys[kk][tx * 4 + c];
#pragma unroll
      for (int q = 0; q < MQ; ++q) {
        const T o = os[kk][ty + 16 * q];
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[q][c] = fma(o, y[c], acc[q][c]);
      }
    }
    __syncthreads();
  }
  // part layout: [split][R][MP]
  T* pp = part + (int64_t)blockIdx.y * R * MP;
#pragma unroll
  for (int q = 0; q < MQ; ++q) {
    const int j = ty + 16 * q;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t r = r0 + tx * 4 + c;
      if (r < R && j < MP) pp[r * MP + j] = acc[q][c];
    }
  }
}

template <typename T>
__global__ void gauss_reduce_kernel(const T* __restrict__ part, int splits, int64_t R, int MP, int m2,
                                    T* __restrict__ Y2, int64_t ldy2) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= R * m2) return;
  const int64_t r = e / m2;
  const int j = (int)(e - r * m2);
  T s = T(0);
  for (int q = 0; q < splits; ++q) s += part[(int64_t)q * R * MP + r * MP + j];
  Y2[r * ldy2 + j] = s;
}

int launch_gaussian_reduce(idl_ctx* ctx, const float* part, int splits, int64_t R, int MP, int64_t m2, float* Y2,
                           int64_t ldy2) {
  const int64_t n = R * m2;
  gauss_reduce_kernel<float><<<(unsigned)cdiv(n, 256), 256, 0, ctx->stream>>>(part, splits, R, MP, (int)m2, Y2, ldy2),
      idl::count_launch();
  return cuda_check(ctx, cudaGetLastError(), "gaussian reduce");
}

// Omega (FP64) -> working precision copy
__global__ void omega_to_f32_kernel(const double* __restrict__ Om, int64_t n, float* __restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < n) out[e] = (float)Om[e];
}

template <typename T, int MQ>
static void launch_simt(idl_ctx* ctx, const T* Om, int m2, int64_t m1, const T* Y1, int64_t R, int64_t ldy1,
                        T* part, int splits, int64_t kchunk, int MP, int rbf16) {
  dim3 grid((unsigned)cdiv(R, kGBN), (unsigned)splits);
  gauss_simt_kernel<T, MQ><<<grid, kGThreads, 0, ctx->stream>>>(Om, m2, m1, Y1, R, ldy1, kchunk, part, MP, rbf16), idl::count_launch();
}

template <typename T>
static int simt_impl(idl_ctx* ctx, const T* Om, int64_t m2, int64_t m1, const T* Y1, int64_t R, int64_t ldy1, T* Y2,
                     int64_t ldy2, int rbf16) {
  const int MQ = (int)cdiv(m2, 16);
  const int MP = MQ * 16;
  const int64_t nbx = cdiv(R, kGBN);
  int64_t splits = cdiv(2 * ctx->num_sms, nbx);
  const int64_t maxs = cdiv(m1, kGBK);
  if (splits > maxs) splits = maxs;
  if (splits < 1) splits = 1;
  if (splits > 1024) splits = 1024;
  const int64_t kchunk = round_up(cdiv(m1, splits), kGBK);
  splits = cdiv(m1, kchunk);
  T* part = (T*)ws_get(ctx, kWsPart, sizeof(T) * (size_t)(splits * R * MP));
  if (!part) return IDL_ENOMEM;
  // static shared memory bounds the Omega tile: m2 <= 256 in FP32, m2 <= 112 in FP64
  if (sizeof(T) == 8 && MQ > 7) return fail(ctx, IDL_ELIMIT, "gaussian: FP64 path needs m2 <= 112");
  switch (MQ) {
#define CASE(q) case q: launch_simt<T, q>(ctx, Om, (int)m2, m1, Y1, R, ldy1, part, (int)splits, kchunk, MP, rbf16); break;
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7)
#undef CASE
#define CASE(q) case q: if constexpr (sizeof(T) == 4) launch_simt<T, q>(ctx, Om, (int)m2, m1, Y1, R, ldy1, part, (int)splits, kchunk, MP, rbf16); break;
    CASE(8) CASE(9) CASE(10) CASE(11) CASE(12) CASE(13) CASE(14) CASE(15) CASE(16)
#undef CASE
    default: return fail(ctx, IDL_ELIMIT, "gaussian: m2 > 256");
  }
  const int64_t n = R * m2;
  gauss_reduce_kernel<T><<<(unsigned)cdiv(n, 256), 256, 0, ctx->stream>>>(part, (int)splits, R, MP, (int)m2, Y2, ldy2), idl::count_launch();
  return cuda_check(ctx, cudaGetLastError(), "gaussian simt");
}

int launch_gaussian(idl_ctx* ctx, const double* Omega, int64_t m2, int64_t m1, const void* Y1, int64_t R, int64_t ldy1,
                    int dtype, int precision, void* Y2, int64_t ldy2) {
  if (m2 > 256) return fail(ctx, IDL_ELIMIT, "gaussian: m2 > 256");
  if (dtype == IDL_F64)
    return simt_impl<double>(ctx, Omega, m2, m1, (const double*)Y1, R, ldy1, (double*)Y2, ldy2, 0);
  if (!ctx->gemm_simt)
    return launch_gaussian_tc(ctx, Omega, m2, m1, (const float*)Y1, R, ldy1, false, precision, (float*)Y2, ldy2);
  // CUDA-core path (kept for comparison): FP32 FMA, or bf16-rounded operands for IDL_PREC_BF16
  float* om32 = (float*)ws_get(ctx, kWsOmegaConv, sizeof(float) * (size_t)(m2 * m1));
  if (!om32) return IDL_ENOMEM;
  omega_to_f32_kernel<<<(unsigned)cdiv(m2 * m1, 256), 256, 0, ctx->stream>>>(Omega, m2 * m1, om32), idl::count_launch();
  return simt_impl<float>(ctx, om32, m2, m1, (const float*)Y1, R, ldy1, (float*)Y2, ldy2,
                          precision == IDL_PREC_BF16 ? 1 : 0);
}

}  // namespace idl

// ---------------------------------------------------------------------------
// Khatri-Rao Gaussian sketch of a CP tensor (Eq. G-matrix): the per-mode products
// G_n = Omega^(n)T A^(n) (L x R, from the Gaussian stage) multiplied entrywise
// and scaled by the s-values, y_lr = lambda_r prod_n G_n[l, r].
// ---------------------------------------------------------------------------
namespace idl {

__global__ void kr_product_kernel(const float* __restrict__ G, int N, int64_t L, int64_t R,
                                  const double* __restrict__ lambda, float* __restrict__ Y) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= L * R) return;
  const int64_t r = e / L;
  float v = (float)lambda[r];
  for (int n = 0; n < N; ++n) v *= G[(int64_t)n * L * R + e];
  Y[e] = v;
}

int launch_kr_product(idl_ctx* ctx, const float* G, int N, int64_t L, int64_t R, const double* lambda, float* Y) {
  const int64_t n = L * R;
  if (n <= 0) return IDL_OK;
  kr_product_kernel<<<(unsigned)cdiv(n, 256), 256, 0, ctx->stream>>>(G, N, L, R, lambda, Y), count_launch();
  return cuda_check(ctx, cudaGetLastError(), "khatri-rao product");
}

}  // namespace idl

// ---------------------------------------------------------------------------
// Y2 (+)= Yp for column-major m x R sketches (ld of Y2: ldy2; Yp packed, ld m):
// the partial sketches of row blocks add up to the sketch of all rows.
// ---------------------------------------------------------------------------
namespace idl {

template <typename T>
__global__ void add_sketch_kernel(const T* __restrict__ Yp, int64_t m, int64_t R, T* __restrict__ Y2, int64_t ldy2,
                                  int accumulate) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m * R) return;
  const int64_t r = e / m, j = e - r * m;
  T* y = Y2 + r * ldy2 + j;
  *y = accumulate ? *y + Yp[e] : Yp[e];
}

int launch_add_sketch(idl_ctx* ctx, const void* Yp, int64_t m, int64_t R, int dtype, void* Y2, int64_t ldy2,
                      int accumulate) {
  const unsigned blocks = (unsigned)cdiv(m * R, 256);
  if (m * R <= 0) return IDL_OK;
  if (dtype == IDL_F32)
    add_sketch_kernel<float><<<blocks, 256, 0, ctx->stream>>>((const float*)Yp, m, R, (float*)Y2, ldy2, accumulate);
  else
    add_sketch_kernel<double><<<blocks, 256, 0, ctx->stream>>>((const double*)Yp, m, R, (double*)Y2, ldy2, accumulate);
  count_launch();
  return cuda_check(ctx, cudaGetLastError(), "add sketch");
}

}  // namespace idl
