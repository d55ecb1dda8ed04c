// countsketch.cu -- Y1 = S A for dense and CSR A (Sec. 1.3; Algorithm 2 line 4).
//
// Both kernels are segmented reductions over the bucket offsets (one bucket
// = one output row of Y1): every row of A is read once, every row of Y1 is
// written once with plain coalesced stores, and nothing goes through global
// atomics, so HBM traffic is the algorithmic minimum
//   bytes(A) + bytes(h-ordered row list, signs) + bytes(Y1).
//
// Dense: block = (bucket, 1024-column tile); each thread owns one 16-byte
//   vector of columns and accumulates the bucket's rows (ascending row order,
//   so the summation order is fixed) with streaming (evict-first) loads, four
//   rows in flight per thread.
// CSR:   block = bucket; the bucket's output row lives in shared memory.  Rows
//   are taken in batches of blockDim; their nonzeros are flattened (a block
//   scan of row lengths, then a binary search per nonzero), so long and short
//   rows both give coalesced colidx/vals loads and full lanes.  Nonzeros are
//   added with shared-memory atomics.  Rows too wide for shared memory use
//   the same kernel with global atomics on the (pre-zeroed) output row.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace idl {

// ----------------------------------------------------------------------------
// dense
// ----------------------------------------------------------------------------
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

template <typename T, bool VEC>
__global__ void __launch_bounds__(256) cs_dense_kernel(const T* __restrict__ A, int64_t lda, int64_t R,
                                                       const int8_t* __restrict__ s,
                                                       const int32_t* __restrict__ ptr,
                                                       const int32_t* __restrict__ rows, T* __restrict__ Y,
                                                       int64_t ldy, int ntiles) {
  using V = typename Vec4<T>::type;
  constexpr int W = 16 / sizeof(T);  // elements per vector
  const int64_t b = blockIdx.x / ntiles;
  const int tile = blockIdx.x % ntiles;
  const int64_t c0 = ((int64_t)tile * blockDim.x + threadIdx.x) * W;
  if (c0 >= R) return;
  const int a0 = ptr[b], a1 = ptr[b + 1];
  T* yrow = Y + b * ldy + c0;
  if (VEC && c0 + W <= R) {
    V acc;
    if constexpr (W == 4) acc = make_float4(0.f, 0.f, 0.f, 0.f); else acc = make_double2(0.0, 0.0);
    int j = a0;
    for (; j + 4 <= a1; j += 4) {
      const int r0 = rows[j], r1 = rows[j + 1], r2 = rows[j + 2], r3 = rows[j + 3];
      const V v0 = ldcs_vec<T>(A + (int64_t)r0 * lda + c0);
      const V v1 = ldcs_vec<T>(A + (int64_t)r1 * lda + c0);
      const V v2 = ldcs_vec<T>(A + (int64_t)r2 * lda + c0);
      const V v3 = ldcs_vec<T>(A + (int64_t)r3 * lda + c0);
      vadd(acc, v0, s[r0] < 0);
      vadd(acc, v1, s[r1] < 0);
      vadd(acc, v2, s[r2] < 0);
      vadd(acc, v3, s[r3] < 0);
    }
    for (; j < a1; ++j) {
      const int r = rows[j];
      vadd(acc, ldcs_vec<T>(A + (int64_t)r * lda + c0), s[r] < 0);
    }
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
      if (q < w) yrow[q] = acc[q];
  }
}

template <typename T>
static int dense_impl(idl_ctx* ctx, const T* A, int64_t R, int64_t lda, const int8_t* s, const int32_t* ptr,
                      const int32_t* rows, int64_t L, T* Y, int64_t ldy) {
  constexpr int W = 16 / sizeof(T);
  const int threads = 256;
  const int64_t tile_cols = (int64_t)threads * W;
  const int ntiles = (int)cdiv(R, tile_cols);
  const int64_t blocks = L * ntiles;
  if (blocks > 0x7fffffffLL) return fail(ctx, IDL_ELIMIT, "countsketch: too many blocks");
  const bool vec = ((uintptr_t)A % 16 == 0) && ((uintptr_t)Y % 16 == 0) && ((lda * sizeof(T)) % 16 == 0) &&
                   ((ldy * sizeof(T)) % 16 == 0);
  if (vec)
    cs_dense_kernel<T, true><<<(unsigned)blocks, threads, 0, ctx->stream>>>(A, lda, R, s, ptr, rows, Y, ldy, ntiles), idl::count_launch();
  else
    cs_dense_kernel<T, false><<<(unsigned)blocks, threads, 0, ctx->stream>>>(A, lda, R, s, ptr, rows, Y, ldy, ntiles), idl::count_launch();
  return cuda_check(ctx, cudaGetLastError(), "countsketch dense");
}

int launch_countsketch_dense(idl_ctx* ctx, const void* A, int64_t I, int64_t R, int64_t lda, int dtype,
                             const int8_t* s, const int32_t* bucket_ptr, const int32_t* row_list, int64_t L,
                             void* Y1, int64_t ldy) {
  (void)I;
  if (dtype == IDL_F32)
    return dense_impl<float>(ctx, (const float*)A, R, lda, s, bucket_ptr, row_list, L, (float*)Y1, ldy);
  return dense_impl<double>(ctx, (const double*)A, R, lda, s, bucket_ptr, row_list, L, (double*)Y1, ldy);
}

// ----------------------------------------------------------------------------
// CSR
// ----------------------------------------------------------------------------
constexpr int kCsrThreads = 512;

// Block-wide exclusive scan of one int per thread; returns the exclusive prefix,
// writes the block total to *total.  scratch: >= 32 ints of shared memory.
__device__ __forceinline__ int block_excl_scan(int v, int* scratch, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) scratch[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int t = lane < nw ? scratch[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) scratch[lane] = t;
  }
  __syncthreads();
  const int excl = (wid ? scratch[wid - 1] : 0) + x - v;
  *total = scratch[nw - 1];
  __syncthreads();
  return excl;
}

template <typename T, bool SMEM>
__global__ void __launch_bounds__(kCsrThreads) cs_csr_kernel(const int64_t* __restrict__ rowptr,
                                                              const int32_t* __restrict__ colidx,
                                                              const T* __restrict__ vals, int64_t R, int64_t nnz,
                                                              const int8_t* __restrict__ s,
                                                              const int32_t* __restrict__ ptr,
                                                              const int32_t* __restrict__ rows, T* __restrict__ Y,
                                                              int64_t ldy, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // layout: [bbeg int64 x B][bstart int x (B+1)][bneg int x B][scan scratch 32][acc T x R]
  int64_t* bbeg = (int64_t*)smem_raw;
  int* bstart = (int*)(bbeg + kCsrThreads);
  int* bneg = bstart + kCsrThreads + 1;
  int* scratch = bneg + kCsrThreads;
  T* acc = (T*)(smem_raw + round_up((int64_t)(sizeof(int64_t) * kCsrThreads + sizeof(int) * (3 * kCsrThreads + 1 + 32)), 16));
  const int64_t b = blockIdx.x;
  T* yrow = Y + b * ldy;
  T* out = SMEM ? acc : yrow;
  if (SMEM) {
    for (int64_t c = threadIdx.x; c < R; c += blockDim.x) acc[c] = T(0);
  }
  __syncthreads();
  const int a0 = ptr[b], a1 = ptr[b + 1];
  for (int base = a0; base < a1; base += kCsrThreads) {
    const int n = min(kCsrThreads, a1 - base);
    int len = 0;
    int64_t beg = 0;
    int neg = 0;
    if ((int)threadIdx.x < n) {
      const int r = rows[base + threadIdx.x];
      beg = rowptr[r];
      const int64_t end = rowptr[r + 1];
      if (beg < 0 || end < beg || end > nnz) {
        set_status(status, IDL_EDATA);
      } else {
        len = (int)(end - beg);
      }
      neg = s[r] < 0;
    }
    int total;
    const int excl = block_excl_scan(len, scratch, &total);
    if ((int)threadIdx.x < n) { bbeg[threadIdx.x] = beg; bstart[threadIdx.x] = excl; bneg[threadIdx.x] = neg; }
    if (threadIdx.x == 0) bstart[n] = total;
    __syncthreads();
    for (int p = threadIdx.x; p < total; p += blockDim.x) {
      // largest t with bstart[t] <= p (rows with len 0 share a start; take the last)
      int lo = 0, hi = n - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bstart[mid] <= p) lo = mid; else hi = mid - 1;
      }
      const int64_t q = bbeg[lo] + (p - bstart[lo]);
      const int c = __ldcs(colidx + q);
      T v = __ldcs(vals + q);
      if (c < 0 || (int64_t)c >= R) { set_status(status, IDL_EDATA); continue; }
      if (bneg[lo]) v = -v;
      atomicAdd(out + c, v);
    }
    __syncthreads();
  }
  if (SMEM) {
    for (int64_t c = threadIdx.x; c < R; c += blockDim.x) yrow[c] = acc[c];
  }
}

static size_t csr_smem_header() {
  return (size_t)round_up((int64_t)(sizeof(int64_t) * kCsrThreads + sizeof(int) * (3 * kCsrThreads + 1 + 32)), 16);
}

template <typename T>
static int csr_impl(idl_ctx* ctx, const int64_t* rowptr, const int32_t* colidx, const T* vals, int64_t R, int64_t nnz,
                    const int8_t* s, const int32_t* ptr, const int32_t* rows, int64_t L, T* Y, int64_t ldy) {
  const size_t head = csr_smem_header();
  const size_t want = head + sizeof(T) * (size_t)R;
  if (L > 0x7fffffffLL) return fail(ctx, IDL_ELIMIT, "countsketch csr: too many buckets");
  // a batch of kCsrThreads rows is flattened with int offsets: bound the row width
  if (R > 4000000) return fail(ctx, IDL_ELIMIT, "countsketch csr: R > 4e6");
  if (want <= (size_t)ctx->smem_optin) {
    auto k = cs_csr_kernel<T, true>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)want);
    if (e != cudaSuccess) return cuda_check(ctx, e, "csr smem attribute");
    k<<<(unsigned)L, kCsrThreads, want, ctx->stream>>>(rowptr, colidx, vals, R, nnz, s, ptr, rows, Y, ldy,
                                                       ctx->d_status), idl::count_launch();
  } else {
    cudaError_t e = cudaMemset2DAsync(Y, ldy * sizeof(T), 0, R * sizeof(T), L, ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "csr zero");
    cs_csr_kernel<T, false><<<(unsigned)L, kCsrThreads, head, ctx->stream>>>(rowptr, colidx, vals, R, nnz, s, ptr,
                                                                              rows, Y, ldy, ctx->d_status), idl::count_launch();
  }
  return cuda_check(ctx, cudaGetLastError(), "countsketch csr");
}

int launch_countsketch_csr(idl_ctx* ctx, const int64_t* rowptr, const int32_t* colidx, const void* vals, int64_t I,
                           int64_t R, int64_t nnz, int dtype, const int8_t* s, const int32_t* bucket_ptr,
                           const int32_t* row_list, int64_t L, void* Y1, int64_t ldy) {
  (void)I;
  if (dtype == IDL_F32)
    return csr_impl<float>(ctx, rowptr, colidx, (const float*)vals, R, nnz, s, bucket_ptr, row_list, L, (float*)Y1, ldy);
  return csr_impl<double>(ctx, rowptr, colidx, (const double*)vals, R, nnz, s, bucket_ptr, row_list, L, (double*)Y1,
                          ldy);
}

}  // namespace idl
