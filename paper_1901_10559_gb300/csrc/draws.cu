// draws.cu -- the sketching operators' random maps and the bucket offsets of Phi.
//
// Draws (Sec. 1.3; Remark 2 and Sec. 7.2; Sec. 1.2.1), counter-based so every
// element is drawn independently by one thread:
//   plain CountSketch   h(i) = bounded(u(seed, 1, i), L),  s(i) = sign(u(seed, 2, i))
//   modified (Remark 2) h~(i) = pi(i) if pi(i) < L else bounded(u(seed, 1, i), L),
//                       pi = 4-round Feistel permutation of [0, 2^w) (Luby-Rackoff),
//                       restricted to [I] by cycle walking (Black-Rogaway 2002)
//   Gaussian Omega      Box-Muller on pairs of the row-major flat index
//   TensorSketch        h_n(i) = bounded(u(seed, 16+n, i), L), s_n(i) = sign(u(seed, 32+n, i))
//
// Bucket offsets: rows grouped by h (a counting sort): histogram, exclusive
// scan, atomic scatter, then every bucket's rows are put in ascending order by
// a rank sort, so the segmented sums of the CountSketch have a fixed order.
#include <cuda_runtime.h>

#include "common.cuh"
#include "draws_dev.cuh"
#include "internal.h"

namespace idl {

__global__ void draw_countsketch_kernel(CsDrawArgs a, int64_t I, int64_t L, int modified, int32_t* __restrict__ h,
                                        int8_t* __restrict__ s, int* status) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < I) cs_draw_elem(i, a, I, L, modified, h, s, status);
}

cudaError_t launch_draw_countsketch(cudaStream_t st, uint64_t seed, int64_t I, int64_t L, int modified,
                                    int32_t* h, int8_t* s, int* status) {
  if (I <= 0) return cudaSuccess;
  const CsDrawArgs a = make_cs_draw_args(seed, I);
  const int threads = 256;
  draw_countsketch_kernel<<<(unsigned)cdiv(I, threads), threads, 0, st>>>(a, I, L, modified, h, s, status),
      idl::count_launch();
  return cudaGetLastError();
}

// rows i0 .. i0 + n - 1 of an I-row CountSketch (the draws of the whole matrix)
__global__ void draw_countsketch_range_kernel(CsDrawArgs a, int64_t I, int64_t i0, int64_t n, int64_t L, int modified,
                                              int32_t* __restrict__ h, int8_t* __restrict__ s, int* status) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r < n) cs_draw_value(i0 + r, a, I, L, modified, h + r, s + r, status);
}

cudaError_t launch_draw_countsketch_range(cudaStream_t st, uint64_t seed, int64_t I, int64_t i0, int64_t n, int64_t L,
                                          int modified, int32_t* h, int8_t* s, int* status) {
  if (n <= 0) return cudaSuccess;
  const CsDrawArgs a = make_cs_draw_args(seed, I);
  draw_countsketch_range_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(a, I, i0, n, L, modified, h, s, status),
      idl::count_launch();
  return cudaGetLastError();
}

// One thread per Box-Muller pair (flat indices 2p, 2p+1): one log and one
// sincospi per pair.
__global__ void draw_gaussian_kernel(uint64_t base, int64_t n, double* __restrict__ Om) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (2 * p < n) gauss_pair(p, base, n, Om);
}

cudaError_t launch_draw_gaussian_tag(cudaStream_t st, uint64_t seed, uint32_t tag, int64_t m2, int64_t m1,
                                     double* Omega) {
  int64_t n = m2 * m1;
  if (n <= 0) return cudaSuccess;
  int threads = 256;
  draw_gaussian_kernel<<<(unsigned)cdiv(cdiv(n, 2), threads), threads, 0, st>>>(stream_base(seed, tag), n, Omega),
      idl::count_launch();
  return cudaGetLastError();
}

cudaError_t launch_draw_gaussian(cudaStream_t st, uint64_t seed, int64_t m2, int64_t m1, double* Omega) {
  return launch_draw_gaussian_tag(st, seed, kTagGauss, m2, m1, Omega);
}

__global__ void draw_gaussian_f32_kernel(uint64_t base, int64_t n, double* __restrict__ Om) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (2 * p < n) gauss_pair_f32(p, base, n, Om);
}

cudaError_t launch_draw_gaussian_f32(cudaStream_t st, uint64_t seed, int64_t m2, int64_t m1, double* Omega) {
  int64_t n = m2 * m1;
  if (n <= 0) return cudaSuccess;
  draw_gaussian_f32_kernel<<<(unsigned)cdiv(cdiv(n, 2), 256), 256, 0, st>>>(stream_base(seed, kTagGauss), n, Omega),
      idl::count_launch();
  return cudaGetLastError();
}

__global__ void draw_mode_kernel(uint64_t hb, uint64_t sb, int64_t In, int64_t L, int32_t* __restrict__ h,
                                 int8_t* __restrict__ s) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < In) mode_elem(i, hb, sb, L, h, s);
}

cudaError_t launch_draw_mode(cudaStream_t st, uint64_t seed, int n, int64_t In, int64_t L, int32_t* h,
                             int8_t* s) {
  if (In <= 0) return cudaSuccess;
  int threads = 256;
  draw_mode_kernel<<<(unsigned)cdiv(In, threads), threads, 0, st>>>(
      stream_base(seed, kTagModeBucket + n), stream_base(seed, kTagModeSign + n), In, L, h, s), idl::count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Bucket offsets
// ---------------------------------------------------------------------------
__global__ void bucket_hist_kernel(const int32_t* __restrict__ h, int64_t I, int64_t L, int32_t* __restrict__ cnt,
                                   int* status) {
  extern __shared__ int32_t sh[];
  bucket_hist_body(h, I, L, cnt, status, blockIdx.x, gridDim.x, sh);
}

__global__ void bucket_scan_kernel(const int32_t* cnt, int64_t L, int32_t* __restrict__ ptr, int32_t* cursor) {
  bucket_scan_body(cnt, L, ptr, cursor);
}

__global__ void bucket_scatter_kernel(const int32_t* __restrict__ h, int64_t I, int64_t L,
                                      int32_t* __restrict__ cursor, int32_t* __restrict__ row_list) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < I) bucket_scatter_elem(i, h, L, cursor, row_list);
}

__global__ void bucket_sort_warp_kernel(const int32_t* __restrict__ ptr, int64_t L, int32_t* __restrict__ row_list,
                                        int32_t* __restrict__ big, int32_t* __restrict__ nbig) {
  extern __shared__ int32_t sh[];
  const int wid = threadIdx.x >> 5;
  const int64_t b = blockIdx.x * (int64_t)(blockDim.x >> 5) + wid;
  if (b < L) bucket_sort_warp_body(ptr, b, row_list, big, nbig, sh + wid * kWarpSortCap);
}

__global__ void bucket_sort_block_kernel(const int32_t* __restrict__ ptr, int32_t* __restrict__ row_list,
                                         const int32_t* __restrict__ big, const int32_t* __restrict__ nbig,
                                         const int32_t* __restrict__ h, int64_t I) {
  extern __shared__ int32_t seg[];
  const int count = *nbig;
  for (int q = blockIdx.x; q < count; q += gridDim.x) bucket_sort_block_body(ptr, big[q], row_list, seg, h, I);
}

__global__ void __launch_bounds__(256) stable_count_kernel(const int32_t* __restrict__ h, int64_t I, int L,
                                                           int32_t* __restrict__ cnt, int* status) {
  extern __shared__ int32_t shc[];
  stable_count_block(h, I, L, blockIdx.x, cnt, status, shc);
}

__global__ void stable_prefix_kernel(int32_t* __restrict__ cnt, int64_t nblk, int L, int32_t* __restrict__ tot) {
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);           // one warp per bucket
  if (b < L) {
    const int32_t t = stable_prefix_bucket(cnt, nblk, L, b);
    if ((threadIdx.x & 31) == 0) tot[b] = t;
  }
}

__global__ void __launch_bounds__(256) stable_scatter_kernel(const int32_t* __restrict__ h, int64_t I, int L,
                                                             const int32_t* __restrict__ ptr,
                                                             const int32_t* __restrict__ cnt,
                                                             int32_t* __restrict__ row_list) {
  extern __shared__ int32_t shc[];
  stable_scatter_block(h, I, L, blockIdx.x, ptr, cnt, row_list, shc);
}

// Stable counting sort (see draws_dev.cuh): no per-bucket sort pass.
static int stable_bucket_offsets(idl_ctx* ctx, const int32_t* h, int64_t I, int64_t L, int32_t* bucket_ptr,
                                 int32_t* row_list) {
  cudaStream_t st = ctx->stream;
  const int W = stable_warps(L);
  const int64_t nblk = cdiv(I, (int64_t)W * kStableSub);
  int32_t* cnt = (int32_t*)ws_get(ctx, kWsCursor, sizeof(int32_t) * (size_t)(nblk * L + L + 1));
  if (!cnt) return IDL_ENOMEM;
  int32_t* tot = cnt + nblk * L;
  const size_t sm = sizeof(int32_t) * (size_t)W * L;
  cudaError_t e = ensure_smem(ctx, (const void*)stable_count_kernel, sm);
  if (e == cudaSuccess) e = ensure_smem(ctx, (const void*)stable_scatter_kernel, sm);
  if (e != cudaSuccess) return cuda_check(ctx, e, "bucket attribute");
  stable_count_kernel<<<(unsigned)nblk, 32 * W, sm, st>>>(h, I, (int)L, cnt, ctx->d_status), idl::count_launch();
  stable_prefix_kernel<<<(unsigned)cdiv(L, 8), 256, 0, st>>>(cnt, nblk, (int)L, tot), idl::count_launch();
  bucket_scan_kernel<<<1, 1024, 0, st>>>(tot, L, bucket_ptr, tot), idl::count_launch();
  stable_scatter_kernel<<<(unsigned)nblk, 32 * W, sm, st>>>(h, I, (int)L, bucket_ptr, cnt, row_list),
      idl::count_launch();
  return cuda_check(ctx, cudaGetLastError(), "bucket offsets");
}

int launch_bucket_offsets(idl_ctx* ctx, const int32_t* h, int64_t I, int64_t L, int32_t* bucket_ptr,
                          int32_t* row_list) {
  if (I > 0 && L <= kStableMaxL) return stable_bucket_offsets(ctx, h, I, L, bucket_ptr, row_list);
  cudaStream_t st = ctx->stream;
  int32_t* cursor = (int32_t*)ws_get(ctx, kWsCursor, sizeof(int32_t) * (size_t)(L + 1));
  int32_t* big = (int32_t*)ws_get(ctx, kWsBig, sizeof(int32_t) * (size_t)(L + 1));
  if (!cursor || !big) return IDL_ENOMEM;
  int32_t* nbig = big + L;
  cudaError_t e = cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (size_t)L, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(nbig, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return cuda_check(ctx, e, "bucket memset");
  {
    int threads = 512;
    int64_t blocks = cdiv(I, threads * 8);
    if (blocks > 4 * ctx->num_sms) blocks = 4 * ctx->num_sms;
    if (blocks < 1) blocks = 1;
    size_t sm = L <= kHistSmem ? sizeof(int32_t) * (size_t)L : 0;
    bucket_hist_kernel<<<(unsigned)blocks, threads, sm, st>>>(h, I, L, cursor, ctx->d_status), idl::count_launch();
  }
  bucket_scan_kernel<<<1, 1024, 0, st>>>(cursor, L, bucket_ptr, cursor), idl::count_launch();
  if (I > 0) bucket_scatter_kernel<<<(unsigned)cdiv(I, 256), 256, 0, st>>>(h, I, L, cursor, row_list), idl::count_launch();
  {
    int warps = 8;
    bucket_sort_warp_kernel<<<(unsigned)cdiv(L, warps), warps * 32, sizeof(int32_t) * warps * kWarpSortCap, st>>>(
        bucket_ptr, L, row_list, big, nbig), idl::count_launch();
    bucket_sort_block_kernel<<<64, 512, sizeof(int32_t) * kBlockSortCap, st>>>(bucket_ptr, row_list, big, nbig, h, I),
        idl::count_launch();
  }
  return cuda_check(ctx, cudaGetLastError(), "bucket offsets");
}

}  // namespace idl
