// tensorsketch.cu -- TensorSketch of the Khatri-Rao matrix of CP factors,
// Y = T M with M = (Khatri-Rao of A^(1..N)) diag(lambda), never forming M
// (Sec. 1.3, Eq. TA-formula; the sketch step of Algorithm 3):
//   Y[:, r] = lambda_r * IFFT( prod_n FFT( S^(n) a^(n)_r ) ).
//
// One block per pair of columns (r, r+1): the two columns' CountSketches of
// each mode are packed into one complex vector, transformed by a register-
// blocked Stockham FFT (radix 16), separated by Hermitian symmetry and
// multiplied into the running spectra; one inverse FFT gives both columns
// (tsketch_dev.cuh).  N modes cost N + 1 complex FFTs per pair of columns.
// FP32 arithmetic.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "tsketch_dev.cuh"
#include "tsketch8k_dev.cuh"

namespace idl {

__global__ void __launch_bounds__(kTsMaxThreads, 1) tensorsketch_kernel(const __grid_constant__ TsArgs a, int64_t R, int L, int logL,
                                                                     const double* __restrict__ lambda,
                                                                     float* __restrict__ Y, int64_t ldy, bool cm,
                                                                     const float2* __restrict__ tw) {
  extern __shared__ __align__(16) float2 sm[];
  tensorsketch_block(a, R, L, logL, lambda, Y, ldy, cm, (int64_t)blockIdx.x * 2, tw, sm);
}

// L = 8192: persistent blocks, one per SM, pairs of columns in turn (tsketch8k_dev.cuh)
__global__ void __launch_bounds__(ts8::kT, 1) tensorsketch8k_kernel(const __grid_constant__ TsArgs a, int64_t R,
                                                                     const double* __restrict__ lambda,
                                                                     float* __restrict__ Y, int64_t ldy, bool cm,
                                                                     const float2* __restrict__ tab) {
  extern __shared__ __align__(16) float2 sm[];
  float2 *z, *tw1, *tw2;
  ts8::block_setup(sm, tab, &z, &tw1, &tw2);
  const int64_t npairs = (R + 1) / 2;
  ts8::Pre pre;
  for (int64_t q = blockIdx.x; q < npairs; q += gridDim.x) {
    ts8::load_mode(a, 0, 2 * q, 2 * q + 1 < R, pre);
    ts8::pair_body(a, R, 2 * q, lambda, Y, ldy, cm, pre, z, tw1, tw2);
  }
}

__global__ void ts_twiddle_kernel(float2* tw) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < kTsTwEntries) ts::twiddle_entry(e, tw);
}

__global__ void ts8_table_kernel(float2* tab) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < ts8::kTw1 + ts8::kTw2) tab[e] = ts8::table_entry(e);
}

// The twiddle table of the L = 8192 kernels (built once per context, on its stream).
const float2* ts8_twiddles(idl_ctx* ctx) {
  if (!ctx->ts8_tw) {
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(float2) * (ts8::kTw1 + ts8::kTw2)) != cudaSuccess) {
      (void)cudaGetLastError();
      ctx->err = "twiddle table allocation failed";
      return nullptr;
    }
    ts8_table_kernel<<<(unsigned)cdiv(ts8::kTw1 + ts8::kTw2, 256), 256, 0, ctx->stream>>>((float2*)p),
        idl::count_launch();
    if (cudaGetLastError() != cudaSuccess) { cudaFree(p); ctx->err = "twiddle table build failed"; return nullptr; }
    ctx->ts8_tw = p;
  }
  return (const float2*)ctx->ts8_tw;
}

// The FFT twiddle table of the context (built once, on the context's stream).
const float2* ts_twiddles(idl_ctx* ctx) {
  if (!ctx->ts_tw) {
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(float2) * kTsTwEntries) != cudaSuccess) {
      (void)cudaGetLastError();
      ctx->err = "twiddle table allocation failed";
      return nullptr;
    }
    ts_twiddle_kernel<<<(unsigned)cdiv(kTsTwEntries, 256), 256, 0, ctx->stream>>>((float2*)p), idl::count_launch();
    if (cudaGetLastError() != cudaSuccess) { cudaFree(p); ctx->err = "twiddle table build failed"; return nullptr; }
    ctx->ts_tw = p;
  }
  return (const float2*)ctx->ts_tw;
}

int launch_tensorsketch(idl_ctx* ctx, int N, const int64_t* dims, int64_t R, const void* const* factors,
                        const int64_t* ldf, const double* lambda, const int32_t* const* hs, const int8_t* const* ss,
                        int64_t L, float* Y, int64_t ldy, bool colmajor) {
  if (N < 1 || N > kTsMaxModes) return fail(ctx, IDL_EINVAL, "tensorsketch: need 1 <= N <= 8");
  if (L < 16 || L > 8192 || (L & (L - 1))) return fail(ctx, IDL_ELIMIT, "tensorsketch: L must be a power of two in [16, 8192]");
  TsArgs a = {};
  a.N = N;
  for (int n = 0; n < N; ++n) {
    a.F[n] = (const float*)factors[n];
    a.h[n] = hs[n];
    a.s[n] = ss[n];
    a.ldf[n] = ldf[n];
    a.dims[n] = (int)dims[n];
  }
  if (L == ts8::kL) {
    cudaError_t e = ensure_smem(ctx, (const void*)tensorsketch8k_kernel, ts8::kSmemBytes);
    if (e != cudaSuccess) return cuda_check(ctx, e, "tensorsketch attribute");
    const float2* tab = ts8_twiddles(ctx);
    if (!tab) return IDL_ENOMEM;
    const int64_t grid = std::min<int64_t>((R + 1) / 2, ctx->num_sms);
    tensorsketch8k_kernel<<<(unsigned)grid, ts8::kT, ts8::kSmemBytes, ctx->stream>>>(a, R, lambda, Y, ldy, colmajor,
                                                                                      tab),
        idl::count_launch();
    return cuda_check(ctx, cudaGetLastError(), "tensorsketch");
  }
  int logL = 0;
  while ((1LL << logL) < L) ++logL;
  const size_t smem = ts_smem_bytes((int)L);
  cudaError_t e = ensure_smem(ctx, (const void*)tensorsketch_kernel, smem);
  if (e != cudaSuccess) return cuda_check(ctx, e, "tensorsketch attribute");
  const float2* tw = ts_twiddles(ctx);
  if (!tw) return IDL_ENOMEM;
  tensorsketch_kernel<<<(unsigned)cdiv(R, 2), ts_threads((int)L), smem, ctx->stream>>>(a, R, (int)L, logL, lambda, Y,
                                                                                      ldy, colmajor, tw),
      idl::count_launch();
  return cuda_check(ctx, cudaGetLastError(), "tensorsketch");
}

}  // namespace idl
