// errest.cu -- the ID error estimate of the paper's experiments (Sec. 6, the
// randomized spectral-norm estimate of Woolfe et al. Sec. 3.4), on the device:
//   ||A - A_J P||_2 / ||A||_2
// by the power method on E^T E, E = A - A_J P, and on A^T A, each from a
// counter-based Gaussian start vector (tag 6; seed and seed + 1), FP64 vectors
// and FP64 accumulation of the products with A's entries.
//
// One step x -> E^T E x without forming E:
//   w = x - scatter_J(P x)      w[J_k] = -sum_c T_kc x[rest_c], w[rest_c] = x[rest_c]
//   y = A w                     (one pass over A)
//   u = A^T y                   (one pass over A)
//   x' = u - P^T u_J            x'[J_k] = 0, x'[rest_c] = u[rest_c] - sum_k T_kc u[J_k]
// then est = sqrt(||x'||), x = x' / ||x'||.  The loop runs without a host round
// trip (the norm stays on the device).
#include <cuda_runtime.h>

#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace idl {

__global__ void err_rest_kernel(const int32_t* __restrict__ J, int K, int R, int32_t* __restrict__ rest) {
  extern __shared__ int32_t sJ[];
  for (int q = threadIdx.x; q < K; q += blockDim.x) sJ[q] = J[q];
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  int less = 0;
  bool piv = false;
  for (int q = 0; q < K; ++q) {
    const int j = sJ[q];
    less += j < r;
    piv |= j == r;
  }
  if (!piv && r - less < R - K) rest[r - less] = r;
}

// w = x - scatter_J(P x): warps 0..K-1 write w[J_k]; the other threads copy x[rest_c]
__global__ void err_w_kernel(const double* __restrict__ x, const int32_t* __restrict__ J,
                             const double* __restrict__ T, const int32_t* __restrict__ rest, int K, int R,
                             double* __restrict__ w) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int nr = R - K;
  const int64_t warp = g >> 5;
  const int lane = threadIdx.x & 31;
  if (warp < K) {
    double acc = 0.0;
    const double* t = T + warp * (int64_t)nr;
    for (int c = lane; c < nr; c += 32) acc += t[c] * x[rest[c]];
    acc = warp_sum(acc);
    if (lane == 0) w[J[warp]] = -acc;
    return;
  }
  const int64_t c = g - 32LL * K;
  if (c < nr) w[rest[c]] = x[rest[c]];
}

// y = A w: one warp per row
template <typename T>
__global__ void err_gemv_kernel(const T* __restrict__ A, int64_t I, int64_t R, int64_t lda,
                                const double* __restrict__ w, double* __restrict__ y) {
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= I) return;
  const T* a = A + row * lda;
  double acc = 0.0;
  for (int64_t c = lane; c < R; c += 32) acc += (double)a[c] * w[c];
  acc = warp_sum(acc);
  if (lane == 0) y[row] = acc;
}

// u += A^T y over a block of rows: thread = column of a 256-column tile
template <typename T>
__global__ void err_gemvt_kernel(const T* __restrict__ A, int64_t I, int64_t R, int64_t lda,
                                 const double* __restrict__ y, int rows_per_block, double* __restrict__ u) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t i0 = (int64_t)blockIdx.y * rows_per_block;
  const int64_t i1 = i0 + rows_per_block < I ? i0 + rows_per_block : I;
  if (c >= R) return;
  double acc = 0.0;
  for (int64_t i = i0; i < i1; ++i) acc += (double)A[i * lda + c] * y[i];
  atomicAdd(u + c, acc);
}

// CSR forms: y = A w (warp per row); u += A^T y (thread per row, atomics per nonzero)
template <typename T>
__global__ void err_gemv_csr_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                    const T* __restrict__ v, int64_t I, int64_t R, const double* __restrict__ w,
                                    double* __restrict__ y) {
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= I) return;
  double acc = 0.0;
  for (int64_t q = rp[row] + lane; q < rp[row + 1]; q += 32) {
    const int c = ci[q];
    if (c >= 0 && c < R) acc += (double)v[q] * w[c];
  }
  acc = warp_sum(acc);
  if (lane == 0) y[row] = acc;
}

template <typename T>
__global__ void err_gemvt_csr_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                     const T* __restrict__ v, int64_t I, int64_t R, const double* __restrict__ y,
                                     double* __restrict__ u) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= I) return;
  const double yr = y[row];
  for (int64_t q = rp[row]; q < rp[row + 1]; ++q) {
    const int c = ci[q];
    if (c >= 0 && c < R) atomicAdd(u + c, (double)v[q] * yr);
  }
}

// x' = u - P^T u_J
__global__ void err_ptu_kernel(const double* __restrict__ u, const int32_t* __restrict__ J,
                               const double* __restrict__ T, const int32_t* __restrict__ rest, int K, int R,
                               double* __restrict__ x) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int nr = R - K;
  if (g < K) { x[J[g]] = 0.0; return; }
  const int64_t c = g - K;
  if (c >= nr) return;
  double acc = u[rest[c]];
  for (int k = 0; k < K; ++k) acc -= T[(int64_t)k * nr + c] * u[J[k]];
  x[rest[c]] = acc;
}

// nrm[0] = ||x||_2 (one block); nrm[1] = sqrt(nrm[0]) is the running estimate
__global__ void err_norm_kernel(const double* __restrict__ x, int64_t n, double* __restrict__ nrm) {
  __shared__ double part[32];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += x[i] * x[i];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) { nrm[0] = sqrt(t); nrm[1] = sqrt(sqrt(t)); }
  }
}

__global__ void err_scale_kernel(double* __restrict__ x, int64_t n, const double* __restrict__ nrm) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const double d = nrm[0];
  if (i < n) x[i] = d > 0.0 ? x[i] / d : 0.0;
}

namespace {

struct ErrOp {
  // dense or CSR A
  const void* A = nullptr;
  int64_t lda = 0;
  const int64_t* rp = nullptr;
  const int32_t* ci = nullptr;
  const void* vals = nullptr;
  int dtype = IDL_F32;
  int64_t I = 0, R = 0;
};

template <typename T>
void apply_ata(const ErrOp& op, const double* w, double* y, double* u, cudaStream_t st, int num_sms) {
  const int64_t I = op.I, R = op.R;
  cudaMemsetAsync(u, 0, sizeof(double) * (size_t)R, st);
  if (op.A) {
    err_gemv_kernel<T><<<(unsigned)cdiv(I * 32, 256), 256, 0, st>>>((const T*)op.A, I, R, op.lda, w, y), count_launch();
    const int64_t tiles = cdiv(R, 256);
    int64_t chunks = cdiv(4LL * num_sms, tiles);
    if (chunks < 1) chunks = 1;
    if (chunks > I) chunks = I;
    const int rpb = (int)cdiv(I, chunks);
    dim3 grid((unsigned)tiles, (unsigned)cdiv(I, rpb));
    err_gemvt_kernel<T><<<grid, 256, 0, st>>>((const T*)op.A, I, R, op.lda, y, rpb, u), count_launch();
  } else {
    err_gemv_csr_kernel<T><<<(unsigned)cdiv(I * 32, 256), 256, 0, st>>>(op.rp, op.ci, (const T*)op.vals, I, R, w, y),
        count_launch();
    err_gemvt_csr_kernel<T><<<(unsigned)cdiv(I, 256), 256, 0, st>>>(op.rp, op.ci, (const T*)op.vals, I, R, y, u),
        count_launch();
  }
}

// est = power-method estimate of ||E||_2 (with_p) or ||A||_2, left in nrm[1]
int power(idl_ctx* ctx, const ErrOp& op, bool with_p, const int32_t* J, const double* T, const int32_t* rest,
          int K, int iters, uint64_t seed, double* x, double* w, double* y, double* u, double* nrm) {
  cudaStream_t st = ctx->stream;
  const int64_t R = op.R;
  cudaError_t e = launch_draw_gaussian_tag(st, seed, kTagErrStart, 1, R, x);
  if (e != cudaSuccess) return cuda_check(ctx, e, "error estimate start");
  err_norm_kernel<<<1, 1024, 0, st>>>(x, R, nrm), count_launch();
  err_scale_kernel<<<(unsigned)cdiv(R, 256), 256, 0, st>>>(x, R, nrm), count_launch();
  const unsigned wblocks = (unsigned)cdiv(32LL * K + (R - K), 256);
  for (int it = 0; it < iters; ++it) {
    const double* win = x;
    if (with_p) {
      err_w_kernel<<<wblocks, 256, 0, st>>>(x, J, T, rest, K, (int)R, w), count_launch();
      win = w;
    }
    if (op.dtype == IDL_F64) apply_ata<double>(op, win, y, u, st, ctx->num_sms);
    else apply_ata<float>(op, win, y, u, st, ctx->num_sms);
    const double* xn = u;
    if (with_p) {
      err_ptu_kernel<<<(unsigned)cdiv(R, 256), 256, 0, st>>>(u, J, T, rest, K, (int)R, w), count_launch();
      xn = w;
    }
    err_norm_kernel<<<1, 1024, 0, st>>>(xn, R, nrm), count_launch();
    cudaMemcpyAsync(x, xn, sizeof(double) * (size_t)R, cudaMemcpyDeviceToDevice, st);
    err_scale_kernel<<<(unsigned)cdiv(R, 256), 256, 0, st>>>(x, R, nrm), count_launch();
  }
  return cuda_check(ctx, cudaGetLastError(), "error estimate");
}

int id_error_run(idl_ctx* ctx, const ErrOp& op, const int32_t* J, const double* T, int64_t K, int iters,
                 uint64_t seed, double* err) {
  const int64_t R = op.R;
  double* x = (double*)ws_get(ctx, kWsErrVec, sizeof(double) * (size_t)(3 * R + op.I + 4));
  int32_t* rest = (int32_t*)ws_get(ctx, kWsRest, sizeof(int32_t) * (size_t)R);
  if (!x || !rest) return IDL_ENOMEM;
  double* w = x + R;
  double* u = w + R;
  double* y = u + R;
  double* nrm = y + op.I;
  err_rest_kernel<<<(unsigned)cdiv(R, 256), 256, sizeof(int32_t) * (size_t)K, ctx->stream>>>(J, (int)K, (int)R, rest),
      count_launch();
  double h[2] = {0.0, 0.0};
  int rc = power(ctx, op, true, J, T, rest, (int)K, iters, seed, x, w, y, u, nrm);
  if (rc != IDL_OK) return rc;
  cudaError_t e = cudaMemcpyAsync(&h[0], nrm + 1, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  if (e != cudaSuccess) return cuda_check(ctx, e, "error estimate readback");
  rc = power(ctx, op, false, J, T, rest, (int)K, iters, seed + 1, x, w, y, u, nrm);
  if (rc != IDL_OK) return rc;
  e = cudaMemcpyAsync(&h[1], nrm + 1, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_check(ctx, e, "error estimate readback");
  *err = h[1] > 0.0 ? h[0] / h[1] : 0.0;
  return IDL_OK;
}

}  // namespace
}  // namespace idl

namespace idl {

int launch_id_error_dense(idl_ctx* ctx, const void* A, int64_t I, int64_t R, int64_t lda, int dtype,
                          const int32_t* J, const double* T, int64_t K, int iters, uint64_t seed, double* err) {
  ErrOp op;
  op.A = A;
  op.lda = lda;
  op.dtype = dtype;
  op.I = I;
  op.R = R;
  return id_error_run(ctx, op, J, T, K, iters, seed, err);
}

int launch_id_error_csr(idl_ctx* ctx, const int64_t* rowptr, const int32_t* colidx, const void* vals, int64_t I,
                        int64_t R, int dtype, const int32_t* J, const double* T, int64_t K, int iters, uint64_t seed,
                        double* err) {
  ErrOp op;
  op.rp = rowptr;
  op.ci = colidx;
  op.vals = vals;
  op.dtype = dtype;
  op.I = I;
  op.R = R;
  return id_error_run(ctx, op, J, T, K, iters, seed, err);
}

}  // namespace idl
