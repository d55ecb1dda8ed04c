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
#include "internal.h"

namespace idl {

struct FeistelKeys { uint64_t k[kFeistelRounds]; };

__device__ __forceinline__ uint64_t feistel(uint64_t x, int half, uint64_t mask, const FeistelKeys& K) {
  uint64_t l = x >> half, r = x & mask;
#pragma unroll
  for (int j = 0; j < kFeistelRounds; ++j) {
    uint64_t f = mix64(K.k[j] ^ r) & mask;
    uint64_t nl = r;
    r = l ^ f;
    l = nl;
  }
  return (l << half) | r;
}

__global__ void draw_countsketch_kernel(uint64_t bucket_base, uint64_t sign_base, int64_t I, int64_t L,
                                        int modified, int half, uint64_t mask, FeistelKeys keys,
                                        int32_t* __restrict__ h, int8_t* __restrict__ s, int* status) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= I) return;
  uint32_t x = bounded(stream_at(bucket_base, (uint64_t)i), (uint64_t)L);
  uint32_t hv = x;
  if (modified) {
    uint64_t y = feistel((uint64_t)i, half, mask, keys);
    // Cycle walking ends: i lies on a finite cycle of the bijection on [0, 2^w)
    // and i < I.  The cap only guards against corrupted arguments.
    int walks = 0;
    while (y >= (uint64_t)I && walks < (1 << 22)) { y = feistel(y, half, mask, keys); ++walks; }
    if (y >= (uint64_t)I) { set_status(status, IDL_ETIMEOUT); y = 0; }
    if (y < (uint64_t)L) hv = (uint32_t)y;
  }
  h[i] = (int32_t)hv;
  s[i] = (stream_at(sign_base, (uint64_t)i) >> 63) ? (int8_t)-1 : (int8_t)1;
}

static int feistel_width(int64_t I) {
  int w = 1;
  while (w < 62 && ((int64_t)1 << w) < I) ++w;
  if (w & 1) ++w;
  return w < 2 ? 2 : w;
}

cudaError_t launch_draw_countsketch(cudaStream_t st, uint64_t seed, int64_t I, int64_t L, int modified,
                                    int32_t* h, int8_t* s, int* status) {
  if (I <= 0) return cudaSuccess;
  FeistelKeys keys;
  uint64_t pb = stream_base(seed, kTagPerm);
  for (int r = 0; r < kFeistelRounds; ++r) keys.k[r] = stream_at(pb, (uint64_t)r);
  int w = feistel_width(I);
  int half = w / 2;
  uint64_t mask = (1ull << half) - 1;
  int threads = 256;
  int64_t blocks = cdiv(I, threads);
  draw_countsketch_kernel<<<(unsigned)blocks, threads, 0, st>>>(
      stream_base(seed, kTagBucket), stream_base(seed, kTagSign), I, L, modified, half, mask, keys, h, s, status), idl::count_launch();
  return cudaGetLastError();
}

// One thread per Box-Muller pair (flat indices 2p, 2p+1): one log and one
// sincospi per pair.  cos(2 pi u2) is evaluated as cospi(2 u2) (exact argument).
__global__ void draw_gaussian_kernel(uint64_t base, int64_t n, double* __restrict__ Om) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (2 * p >= n) return;
  const uint64_t a = stream_at(base, 2 * (uint64_t)p);
  const uint64_t c = stream_at(base, 2 * (uint64_t)p + 1);
  const double u1 = ((double)(a >> 11) + 1.0) * 0x1.0p-53;   // (0, 1]
  const double u2 = (double)(c >> 11) * 0x1.0p-53;           // [0, 1)
  const double rho = sqrt(-2.0 * log(u1));
  double sv, cv;
  sincospi(2.0 * u2, &sv, &cv);
  Om[2 * p] = rho * cv;
  if (2 * p + 1 < n) Om[2 * p + 1] = rho * sv;
}

cudaError_t launch_draw_gaussian(cudaStream_t st, uint64_t seed, int64_t m2, int64_t m1, double* Omega) {
  int64_t n = m2 * m1;
  if (n <= 0) return cudaSuccess;
  int threads = 256;
  draw_gaussian_kernel<<<(unsigned)cdiv(cdiv(n, 2), threads), threads, 0, st>>>(stream_base(seed, kTagGauss), n, Omega), idl::count_launch();
  return cudaGetLastError();
}

__global__ void draw_mode_kernel(uint64_t hb, uint64_t sb, int64_t In, int64_t L, int32_t* __restrict__ h,
                                 int8_t* __restrict__ s) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= In) return;
  h[i] = (int32_t)bounded(stream_at(hb, (uint64_t)i), (uint64_t)L);
  s[i] = (stream_at(sb, (uint64_t)i) >> 63) ? (int8_t)-1 : (int8_t)1;
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
constexpr int kHistSmem = 12288;  // buckets histogrammed in shared memory first

__global__ void bucket_hist_kernel(const int32_t* __restrict__ h, int64_t I, int64_t L, int32_t* __restrict__ cnt,
                                   int* status) {
  extern __shared__ int32_t sh[];
  const bool local = L <= kHistSmem;
  if (local) {
    for (int64_t b = threadIdx.x; b < L; b += blockDim.x) sh[b] = 0;
    __syncthreads();
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < I; i += (int64_t)gridDim.x * blockDim.x) {
    const int b = h[i];
    if (b < 0 || (int64_t)b >= L) { set_status(status, IDL_EDATA); continue; }   // caller-supplied h out of range
    if (local) atomicAdd(&sh[b], 1); else atomicAdd(&cnt[b], 1);
  }
  if (local) {
    __syncthreads();
    for (int64_t b = threadIdx.x; b < L; b += blockDim.x)
      if (sh[b]) atomicAdd(&cnt[b], sh[b]);
  }
}

// Single-block exclusive scan of cnt[0..L) into ptr[0..L] (and the scatter cursor).
// cnt and cursor may alias: each thread reads cnt[b] before it writes cursor[b].
__global__ void bucket_scan_kernel(const int32_t* cnt, int64_t L, int32_t* __restrict__ ptr, int32_t* cursor) {
  __shared__ int32_t warp_tot[32];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t base = 0; base < L; base += blockDim.x) {
    int64_t b = base + threadIdx.x;
    int32_t v = b < L ? cnt[b] : 0;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int32_t t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      if (lane < nw) warp_tot[lane] = t;  // inclusive warp prefix
    }
    __syncthreads();
    int32_t excl = carry + (wid ? warp_tot[wid - 1] : 0) + x - v;
    if (b < L) { ptr[b] = excl; cursor[b] = excl; }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) ptr[L] = carry;
}

__global__ void bucket_scatter_kernel(const int32_t* __restrict__ h, int64_t I, int64_t L,
                                      int32_t* __restrict__ cursor, int32_t* __restrict__ row_list) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= I) return;
  const int b = h[i];
  if (b < 0 || (int64_t)b >= L) return;        // flagged by the histogram pass
  int pos = atomicAdd(&cursor[b], 1);
  row_list[pos] = (int32_t)i;
}

constexpr int kWarpSortCap = 1024;   // rows per bucket sorted by one warp
constexpr int kBlockSortCap = 12288; // rows per bucket sorted by one block

// One warp per bucket: rank sort (rows are distinct, so rank = #smaller).
__global__ void bucket_sort_warp_kernel(const int32_t* __restrict__ ptr, int64_t L, int32_t* __restrict__ row_list,
                                        int32_t* __restrict__ big, int32_t* __restrict__ nbig) {
  extern __shared__ int32_t sh[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t b = blockIdx.x * (int64_t)(blockDim.x >> 5) + wid;
  if (b >= L) return;
  int32_t* seg = sh + wid * kWarpSortCap;
  int a0 = ptr[b], n = ptr[b + 1] - a0;
  if (n <= 1) return;
  if (n > kWarpSortCap) {
    if (lane == 0) big[atomicAdd(nbig, 1)] = (int32_t)b;
    return;
  }
  for (int j = lane; j < n; j += 32) seg[j] = row_list[a0 + j];
  __syncwarp();
  for (int j = lane; j < n; j += 32) {
    int x = seg[j], rank = 0;
    for (int t = 0; t < n; ++t) rank += seg[t] < x;
    row_list[a0 + rank] = x;
  }
}

__global__ void bucket_sort_block_kernel(const int32_t* __restrict__ ptr, int32_t* __restrict__ row_list,
                                         const int32_t* __restrict__ big, const int32_t* __restrict__ nbig) {
  extern __shared__ int32_t seg[];
  const int count = *nbig;
  for (int q = blockIdx.x; q < count; q += gridDim.x) {
    int b = big[q];
    int a0 = ptr[b], n = ptr[b + 1] - a0;
    if (n > kBlockSortCap) continue;    // left in arrival order (documented)
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) seg[j] = row_list[a0 + j];
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      int x = seg[j], rank = 0;
      for (int t = 0; t < n; ++t) rank += seg[t] < x;
      row_list[a0 + rank] = x;
    }
  }
}

int launch_bucket_offsets(idl_ctx* ctx, const int32_t* h, int64_t I, int64_t L, int32_t* bucket_ptr,
                          int32_t* row_list) {
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
    bucket_sort_block_kernel<<<64, 512, sizeof(int32_t) * kBlockSortCap, st>>>(bucket_ptr, row_list, big, nbig), idl::count_launch();
  }
  return cuda_check(ctx, cudaGetLastError(), "bucket offsets");
}

}  // namespace idl
