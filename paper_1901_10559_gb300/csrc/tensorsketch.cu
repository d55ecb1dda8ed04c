// tensorsketch.cu -- TensorSketch of the Khatri-Rao matrix of CP factors,
// Y = T M with M = (Khatri-Rao of A^(1..N)) diag(lambda), never forming M
// (Sec. 1.3, Eq. TA-formula; Algorithm 3 line 5):
//   Y[:, r] = lambda_r * IFFT( prod_n FFT( S^(n) a^(n)_r ) ).
//
// One block per pair of columns (r, r+1), everything in shared memory:
//   * per mode n, the two columns' CountSketches are packed as the real and
//     imaginary parts of one complex length-L vector z (scatter with shared
//     atomics into bit-reversed positions), transformed by one in-place radix-2
//     FFT, and separated by Hermitian symmetry:
//        C_r[f] = (Z[f] + conj Z[-f]) / 2,   C_{r+1}[f] = (Z[f] - conj Z[-f]) / 2i;
//   * the spectra are multiplied into P_r, P_{r+1} (f = 0..L/2; the rest is
//     the conjugate mirror of a real signal's spectrum);
//   * one inverse FFT of P_r + i P_{r+1} gives both real columns at once.
// N modes cost N + 1 complex FFTs per pair of columns.  Twiddles are stored per
// stage (stage with half-length h at offset h) so a stage reads them with
// unit stride.  FP32 arithmetic.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"
#include "tsketch_dev.cuh"

namespace idl {

__global__ void __launch_bounds__(kTsThreads, 1) tensorsketch_kernel(TsArgs a, int64_t R, int L, int logL,
                                                                     const double* __restrict__ lambda,
                                                                     float* __restrict__ Y, int64_t ldy) {
  extern __shared__ __align__(16) float2 sm[];
  tensorsketch_block(a, R, L, logL, lambda, Y, ldy, (int64_t)blockIdx.x * 2, sm);
}

int launch_tensorsketch(idl_ctx* ctx, int N, const int64_t* dims, int64_t R, const void* const* factors,
                        const int64_t* ldf, const double* lambda, const int32_t* const* hs, const int8_t* const* ss,
                        int64_t L, float* Y, int64_t ldy) {
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
  int logL = 0;
  while ((1LL << logL) < L) ++logL;
  const size_t smem = sizeof(float2) * (size_t)(2 * L + 2 * (L / 2 + 1));
  cudaError_t e = cudaFuncSetAttribute(tensorsketch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_check(ctx, e, "tensorsketch attribute");
  tensorsketch_kernel<<<(unsigned)cdiv(R, 2), kTsThreads, smem, ctx->stream>>>(a, R, (int)L, logL, lambda, Y, ldy), idl::count_launch();
  return cuda_check(ctx, cudaGetLastError(), "tensorsketch");
}

}  // namespace idl
