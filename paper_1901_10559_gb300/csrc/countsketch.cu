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
//   are taken in batches of blockDim.  Short rows' nonzeros are flattened (a
//   block scan of their lengths and a row-id table), so loads stay coalesced
//   and lanes full, with four nonzeros in flight per thread; rows of >= 256
//   nonzeros are streamed by the whole block with 16-byte colidx/vals loads,
//   two in flight per thread.  Nonzeros are added with shared-memory atomics.
//   Rows too wide for shared memory use the same kernel with global atomics
//   on the (pre-zeroed) output row.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"
#include "sketch_dev.cuh"

namespace idl {

// ----------------------------------------------------------------------------
// dense
// ----------------------------------------------------------------------------
template <typename T, bool VEC>
__global__ void __launch_bounds__(256) cs_dense_kernel(const T* __restrict__ A, int64_t lda, int64_t R,
                                                       const int8_t* __restrict__ s,
                                                       const int32_t* __restrict__ ptr,
                                                       const int32_t* __restrict__ rows, T* __restrict__ Y,
                                                       int64_t ldy, int ntiles) {
  cs_dense_block<T, VEC>(A, lda, R, s, ptr, rows, Y, ldy, blockIdx.x / ntiles, blockIdx.x % ntiles);
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

constexpr int kLongRow = 256;     // rows at least this long are streamed by the whole block, vectorised
constexpr int kRowIdCap = 8192;   // short-row nonzeros expanded to a row-id table per batch
constexpr int kShortUnroll = 4;   // short-row nonzeros in flight per thread

template <typename T> struct CsrVec;
template <> struct CsrVec<float> { using V = float4; using C = int4; static constexpr int W = 4; };
template <> struct CsrVec<double> { using V = double2; using C = int2; static constexpr int W = 2; };

template <typename T>
__device__ __forceinline__ void csr_add(T* out, int64_t R, int c, T v, bool neg, int* status) {
  if (c < 0 || (int64_t)c >= R) { set_status(status, IDL_EDATA); return; }
  atomicAdd(out + c, neg ? -v : v);
}

// largest t in [0, n) with start[t] <= p  (rows of zero length share a start with the next row)
__device__ __forceinline__ int row_of(const int* start, int n, int p) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= p) lo = mid; else hi = mid - 1;
  }
  return lo;
}

struct CsrSmem {
  int64_t bbeg[kCsrThreads];
  int bstart[kCsrThreads + 1];
  int blen[kCsrThreads];
  int bneg[kCsrThreads];
  int longs[kCsrThreads];
  int scratch[32];
  uint16_t rowid[kRowIdCap];
};

template <typename T, bool SMEM>
__global__ void __launch_bounds__(kCsrThreads) cs_csr_kernel(const int64_t* __restrict__ rowptr,
                                                              const int32_t* __restrict__ colidx,
                                                              const T* __restrict__ vals, int64_t R, int64_t nnz,
                                                              const int8_t* __restrict__ s,
                                                              const int32_t* __restrict__ ptr,
                                                              const int32_t* __restrict__ rows, T* __restrict__ Y,
                                                              int64_t ldy, int* status, int vec_ok) {
  using V = typename CsrVec<T>::V;
  using C = typename CsrVec<T>::C;
  constexpr int W = CsrVec<T>::W;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CsrSmem& sm = *reinterpret_cast<CsrSmem*>(smem_raw);
  T* acc = (T*)(smem_raw + round_up((int64_t)sizeof(CsrSmem), 16));
  const int tid = threadIdx.x;
  const int64_t b = blockIdx.x;
  T* yrow = Y + b * ldy;
  T* out = SMEM ? acc : yrow;
  if (SMEM) {
    for (int64_t c = tid; c < R; c += blockDim.x) acc[c] = T(0);
  }
  __syncthreads();
  const int a0 = ptr[b], a1 = ptr[b + 1];
  for (int base = a0; base < a1; base += kCsrThreads) {
    const int n = min(kCsrThreads, a1 - base);
    int len = 0, neg = 0;
    int64_t beg = 0;
    if (tid < n) {
      const int r = rows[base + tid];
      beg = rowptr[r];
      const int64_t end = rowptr[r + 1];
      if (beg < 0 || end < beg || end > nnz) set_status(status, IDL_EDATA);
      else len = (int)(end - beg);
      neg = s[r] < 0;
    }
    const int is_long = len >= kLongRow;
    int total, nlong;
    const int excl = block_excl_scan(is_long ? 0 : len, sm.scratch, &total);
    const int lpos = block_excl_scan(is_long, sm.scratch, &nlong);
    if (tid < n) { sm.bbeg[tid] = beg; sm.bstart[tid] = excl; sm.blen[tid] = len; sm.bneg[tid] = neg; }
    if (is_long) sm.longs[lpos] = tid;
    if (tid == 0) sm.bstart[n] = total;
    const bool expand = total <= kRowIdCap;
    if (expand && tid < n && !is_long)
      for (int j = 0; j < len; ++j) sm.rowid[excl + j] = (uint16_t)tid;
    __syncthreads();
    // short rows: flattened nonzeros, kShortUnroll independent loads per thread
    for (int p0 = tid; p0 < total; p0 += kCsrThreads * kShortUnroll) {
      int cc[kShortUnroll], ng[kShortUnroll];
      T vv[kShortUnroll];
#pragma unroll
      for (int u = 0; u < kShortUnroll; ++u) {
        const int p = p0 + u * kCsrThreads;
        cc[u] = -1;
        if (p < total) {
          const int t = expand ? (int)sm.rowid[p] : row_of(sm.bstart, n, p);
          const int64_t q = sm.bbeg[t] + (p - sm.bstart[t]);
          cc[u] = __ldcs(colidx + q);
          vv[u] = __ldcs(vals + q);
          ng[u] = sm.bneg[t];
        }
      }
#pragma unroll
      for (int u = 0; u < kShortUnroll; ++u)
        if (p0 + u * kCsrThreads < total) csr_add(out, R, cc[u], vv[u], ng[u] != 0, status);
    }
    // long rows: the whole block streams each one with 16-byte loads
    for (int li = 0; li < nlong; ++li) {
      const int t = sm.longs[li];
      const int64_t q0 = sm.bbeg[t];
      const int L = sm.blen[t];
      const bool ngt = sm.bneg[t] != 0;
      const int head = vec_ok ? min(L, (int)((W - (q0 % W)) % W)) : L;
      if (tid < head) csr_add(out, R, __ldcs(colidx + q0 + tid), __ldcs(vals + q0 + tid), ngt, status);
      const int64_t qb = q0 + head;
      const int nvec = (L - head) / W;
      const C* cv = reinterpret_cast<const C*>(colidx + qb);
      const V* vv = reinterpret_cast<const V*>(vals + qb);
      for (int vi = tid; vi < nvec; vi += 2 * kCsrThreads) {
        const bool two = vi + kCsrThreads < nvec;
        const C c0 = __ldcs(cv + vi);
        const V v0 = __ldcs(vv + vi);
        C c1;
        V v1;
        if (two) { c1 = __ldcs(cv + vi + kCsrThreads); v1 = __ldcs(vv + vi + kCsrThreads); }
        if constexpr (W == 4) {
          csr_add(out, R, c0.x, v0.x, ngt, status); csr_add(out, R, c0.y, v0.y, ngt, status);
          csr_add(out, R, c0.z, v0.z, ngt, status); csr_add(out, R, c0.w, v0.w, ngt, status);
          if (two) {
            csr_add(out, R, c1.x, v1.x, ngt, status); csr_add(out, R, c1.y, v1.y, ngt, status);
            csr_add(out, R, c1.z, v1.z, ngt, status); csr_add(out, R, c1.w, v1.w, ngt, status);
          }
        } else {
          csr_add(out, R, c0.x, v0.x, ngt, status); csr_add(out, R, c0.y, v0.y, ngt, status);
          if (two) { csr_add(out, R, c1.x, v1.x, ngt, status); csr_add(out, R, c1.y, v1.y, ngt, status); }
        }
      }
      const int rem = (L - head) - nvec * W;
      if (tid < rem) {
        const int64_t q = qb + (int64_t)nvec * W + tid;
        csr_add(out, R, __ldcs(colidx + q), __ldcs(vals + q), ngt, status);
      }
    }
    __syncthreads();
  }
  if (SMEM) {
    for (int64_t c = tid; c < R; c += blockDim.x) yrow[c] = acc[c];
  }
}

static size_t csr_smem_header() { return (size_t)round_up((int64_t)sizeof(CsrSmem), 16); }

template <typename T>
static int csr_impl(idl_ctx* ctx, const int64_t* rowptr, const int32_t* colidx, const T* vals, int64_t R, int64_t nnz,
                    const int8_t* s, const int32_t* ptr, const int32_t* rows, int64_t L, T* Y, int64_t ldy) {
  const size_t head = csr_smem_header();
  const size_t want = head + sizeof(T) * (size_t)R;
  if (L > 0x7fffffffLL) return fail(ctx, IDL_ELIMIT, "countsketch csr: too many buckets");
  // a batch of kCsrThreads rows is flattened with int offsets: bound the row width
  if (R > 4000000) return fail(ctx, IDL_ELIMIT, "countsketch csr: R > 4e6");
  const int vec_ok = ((uintptr_t)colidx % 16 == 0) && ((uintptr_t)vals % 16 == 0);
  if (want <= (size_t)ctx->smem_optin) {
    auto k = cs_csr_kernel<T, true>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)want);
    if (e != cudaSuccess) return cuda_check(ctx, e, "csr smem attribute");
    k<<<(unsigned)L, kCsrThreads, want, ctx->stream>>>(rowptr, colidx, vals, R, nnz, s, ptr, rows, Y, ldy,
                                                       ctx->d_status, vec_ok), idl::count_launch();
  } else {
    cudaError_t e = cudaMemset2DAsync(Y, ldy * sizeof(T), 0, R * sizeof(T), L, ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "csr zero");
    auto k = cs_csr_kernel<T, false>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)head);
    if (e != cudaSuccess) return cuda_check(ctx, e, "csr smem attribute");
    k<<<(unsigned)L, kCsrThreads, head, ctx->stream>>>(rowptr, colidx, vals, R, nnz, s, ptr, rows, Y, ldy,
                                                       ctx->d_status, vec_ok), idl::count_launch();
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
