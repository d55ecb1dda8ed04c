// countsketch.cu -- Y1 = S A for dense and CSR A (Sec. 1.3; the sketch step of Algorithm 2).
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
//   are taken in batches of blockDim and read as 16-byte-aligned element quads
//   (masked to the row), the quads of all rows of a batch flattened into one
//   stream (a block scan of the rows' quad counts; quad -> row by a table for
//   short rows, by a binary search over the few long ones), four quads in
//   flight per thread.  Nonzeros are added with shared-memory atomics.  Rows
//   too wide for shared memory use the same kernel with global atomics on the
//   (pre-zeroed) output row.
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
                                                       int64_t ldy, int ntiles, bool accum) {
  cs_dense_block<T, VEC>(A, lda, R, s, ptr, rows, Y, ldy, blockIdx.x / ntiles, blockIdx.x % ntiles, accum);
}

template <typename T>
static int dense_impl(idl_ctx* ctx, const T* A, int64_t R, int64_t lda, const int8_t* s, const int32_t* ptr,
                      const int32_t* rows, int64_t L, T* Y, int64_t ldy, bool accum) {
  constexpr int W = 16 / sizeof(T);
  const int threads = 256;
  const int64_t tile_cols = (int64_t)threads * W;
  const int ntiles = (int)cdiv(R, tile_cols);
  const int64_t blocks = L * ntiles;
  if (blocks > 0x7fffffffLL) return fail(ctx, IDL_ELIMIT, "countsketch: too many blocks");
  const bool vec = ((uintptr_t)A % 16 == 0) && ((uintptr_t)Y % 16 == 0) && ((lda * sizeof(T)) % 16 == 0) &&
                   ((ldy * sizeof(T)) % 16 == 0);
  if (vec)
    cs_dense_kernel<T, true><<<(unsigned)blocks, threads, 0, ctx->stream>>>(A, lda, R, s, ptr, rows, Y, ldy, ntiles, accum),
        idl::count_launch();
  else
    cs_dense_kernel<T, false><<<(unsigned)blocks, threads, 0, ctx->stream>>>(A, lda, R, s, ptr, rows, Y, ldy, ntiles, accum),
        idl::count_launch();
  return cuda_check(ctx, cudaGetLastError(), "countsketch dense");
}

int launch_countsketch_dense(idl_ctx* ctx, const void* A, int64_t I, int64_t R, int64_t lda, int dtype,
                             const int8_t* s, const int32_t* bucket_ptr, const int32_t* row_list, int64_t L,
                             void* Y1, int64_t ldy, bool accum) {
  (void)I;
  if (dtype == IDL_F32)
    return dense_impl<float>(ctx, (const float*)A, R, lda, s, bucket_ptr, row_list, L, (float*)Y1, ldy, accum);
  return dense_impl<double>(ctx, (const double*)A, R, lda, s, bucket_ptr, row_list, L, (double*)Y1, ldy, accum);
}

// ----------------------------------------------------------------------------
// CSR
// ----------------------------------------------------------------------------
// Block-wide exclusive scans of two ints per thread in one pass; returns the
// exclusive prefixes, writes the block totals to *total.  scratch: >= 64 ints
// of shared memory.
__device__ __forceinline__ int2 block_excl_scan2(int2 v, int* scratch, int2* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int2 x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y0 = __shfl_up_sync(0xffffffffu, x.x, o), y1 = __shfl_up_sync(0xffffffffu, x.y, o);
    if (lane >= o) { x.x += y0; x.y += y1; }
  }
  if (lane == 31) { scratch[wid] = x.x; scratch[32 + wid] = x.y; }
  __syncthreads();
  if (wid == 0) {
    int t0 = lane < nw ? scratch[lane] : 0, t1 = lane < nw ? scratch[32 + lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y0 = __shfl_up_sync(0xffffffffu, t0, o), y1 = __shfl_up_sync(0xffffffffu, t1, o);
      if (lane >= o) { t0 += y0; t1 += y1; }
    }
    if (lane < nw) { scratch[lane] = t0; scratch[32 + lane] = t1; }
  }
  __syncthreads();
  const int2 excl = make_int2((wid ? scratch[wid - 1] : 0) + x.x - v.x, (wid ? scratch[32 + wid - 1] : 0) + x.y - v.y);
  *total = make_int2(scratch[nw - 1], scratch[32 + nw - 1]);
  __syncthreads();
  return excl;
}

constexpr int kLongRow = 256;     // rows at least this long: quads found by a search over the long rows
constexpr int kQuadUnroll = 4;    // quads in flight per thread (FP32; FP64: 2)

template <typename T>
__device__ __forceinline__ void csr_add(T* out, int64_t R, int c, T v, bool neg, int* status) {
  if (c < 0 || (int64_t)c >= R) { set_status(status, IDL_EDATA); return; }
  atomicAdd(out + c, neg ? -v : v);
}

// largest t in [0, n) with start[t] <= p  (rows without quads share a start with the next row)
__device__ __forceinline__ int row_of(const int* start, int n, int p) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= p) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int NT>
struct CsrSmem {
  static constexpr int kRowIdCap = 8 * NT;    // short-row quads expanded to a row-id table per batch
  int64_t bbeg[NT];
  int blen[NT];
  int sqstart[NT];          // first quad of each short row (long rows: the next short row's)
  int longs[NT];            // batch row of the i-th long row
  int lqstart[NT];          // first quad of the i-th long row in the long-row part of the stream
  int scratch[64];
  uint16_t rowid[kRowIdCap];
  uint8_t bneg[NT];
};

// Elements q .. q+3 of colidx / vals into c, v (only [lo, hi) loaded when the quad
// cannot be read with 16-byte loads).
template <typename T>
__device__ __forceinline__ void load_quad(const int32_t* __restrict__ colidx, const T* __restrict__ vals, int64_t q,
                                          int lo, int hi, bool vec, int (&c)[4], T (&v)[4]) {
  if (vec) {
    const int4 ci = __ldcs(reinterpret_cast<const int4*>(colidx + q));
    c[0] = ci.x; c[1] = ci.y; c[2] = ci.z; c[3] = ci.w;
    if constexpr (sizeof(T) == 4) {
      const float4 vi = __ldcs(reinterpret_cast<const float4*>(vals + q));
      v[0] = vi.x; v[1] = vi.y; v[2] = vi.z; v[3] = vi.w;
    } else {
      const double2 v0 = __ldcs(reinterpret_cast<const double2*>(vals + q));
      const double2 v1 = __ldcs(reinterpret_cast<const double2*>(vals + q + 2));
      v[0] = v0.x; v[1] = v0.y; v[2] = v1.x; v[3] = v1.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const bool in = j >= lo && j < hi;
      c[j] = in ? __ldcs(colidx + q + j) : 0;
      v[j] = in ? __ldcs(vals + q + j) : T(0);
    }
  }
}

// One block per bucket b: Y[b, :] = sum over the bucket's rows r of s[r] * A[r, :].
// The rows are taken in batches of NT (one row per thread).  Every row is read as
// the element quads that cover it (quad k of a row starting at element beg:
// elements 4*floor(beg/4) + 4k .. + 3, masked to the row), with 16-byte loads of
// colidx and vals when both arrays are 16-byte aligned and the quad ends inside
// them.  The quads of a batch form one stream -- short rows first (quad -> row by
// a table), then long rows (by a binary search over the few long rows) -- and
// thread t takes quads t, t + NT, t + 2 NT, ..., U of them into registers at a
// time, then adds their elements with shared-memory atomics into the output row
// (SMEM), or with global atomics into the pre-zeroed output row (rows too wide
// for shared memory).
// Measured on the sparse workload (1e6 x 1e4, 1.1e8 nonzeros, 3600 buckets):
// without the atomics the loop streams colidx / vals at ~6 TB/s; the atomics
// (about 4 lanes per clock per SM) do not overlap with the loads -- a cp.async
// ring of three quads per thread, double-buffered registers and bank-rotated
// lanes were each slower, as were 256-thread blocks (four buckets per SM).
template <typename T, bool SMEM, int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) cs_csr_kernel(const int64_t* __restrict__ rowptr,
                                                                const int32_t* __restrict__ colidx,
                                                                const T* __restrict__ vals, int64_t R, int64_t nnz,
                                                                const int8_t* __restrict__ s,
                                                                const int32_t* __restrict__ ptr,
                                                                const int32_t* __restrict__ rows, T* __restrict__ Y,
                                                                int64_t ldy, int* status, int vec_ok, int accum) {
  using Sm = CsrSmem<NT>;
  constexpr int U = sizeof(T) == 4 ? kQuadUnroll : 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Sm& sm = *reinterpret_cast<Sm*>(smem_raw);
  T* acc = (T*)(smem_raw + round_up((int64_t)sizeof(Sm), 16));
  const int tid = threadIdx.x;
  const int64_t b = blockIdx.x;
  T* yrow = Y + b * ldy;
  T* out = SMEM ? acc : yrow;
  const int a0 = ptr[b], a1 = ptr[b + 1];
  if (SMEM) {
    for (int64_t c = tid; c < R; c += NT) acc[c] = T(0);
  }
  for (int base = a0; base < a1; base += NT) {
    const int n = min(NT, a1 - base);
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
    const int nq = len > 0 ? (int)(((beg + len + 3) >> 2) - (beg >> 2)) : 0;
    int2 tot;
    const int2 ex = block_excl_scan2(make_int2(is_long ? 0 : nq, is_long ? nq : 0), sm.scratch, &tot);
    const int squads = tot.x, nquads = tot.x + tot.y;
    // rank of each long row among the batch's long rows
    const unsigned bal = __ballot_sync(0xffffffffu, is_long);
    if ((tid & 31) == 0) sm.scratch[tid >> 5] = __popc(bal);
    if (tid < n) { sm.bbeg[tid] = beg; sm.blen[tid] = len; sm.bneg[tid] = neg; }
    sm.sqstart[tid] = ex.x;
    __syncthreads();
    int nlong = 0, lpos = __popc(bal & ((1u << (tid & 31)) - 1));
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) {
      const int c = sm.scratch[w];
      if (w < (tid >> 5)) lpos += c;
      nlong += c;
    }
    if (is_long) { sm.longs[lpos] = tid; sm.lqstart[lpos] = squads + ex.y; }
    const bool expand = squads <= Sm::kRowIdCap;
    if (expand && !is_long)
      for (int j = 0; j < nq; ++j) sm.rowid[ex.x + j] = (uint16_t)tid;
    __syncthreads();
    // quad p of the stream: first element q, valid elements [lo, hi), row sign
    auto locate = [&](int p, int64_t& q, int& lo, int& hi, bool& ng) {
      int t, k;
      if (p < squads) {
        t = expand ? (int)sm.rowid[p] : row_of(sm.sqstart, n, p);
        k = p - sm.sqstart[t];
      } else {
        const int li = row_of(sm.lqstart, nlong, p);
        t = sm.longs[li];
        k = p - sm.lqstart[li];
      }
      const int64_t b0 = sm.bbeg[t], b1 = b0 + sm.blen[t];
      q = ((b0 >> 2) + k) << 2;
      lo = b0 > q ? (int)(b0 - q) : 0;
      hi = b1 - q < 4 ? (int)(b1 - q) : 4;
      ng = sm.bneg[t] != 0;
    };
    for (int p0 = tid; p0 < nquads; p0 += NT * U) {
      int cq[U][4], lo[U], hi[U];
      T vq[U][4];
      bool ngq[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int p = p0 + u * NT;
        lo[u] = 4;
        hi[u] = 0;
        ngq[u] = false;
        if (p < nquads) {
          int64_t q;
          locate(p, q, lo[u], hi[u], ngq[u]);
          load_quad(colidx, vals, q, lo[u], hi[u], vec_ok && q + 4 <= nnz, cq[u], vq[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (j >= lo[u] && j < hi[u]) csr_add(out, R, cq[u][j], vq[u][j], ngq[u], status);
    }
    __syncthreads();
  }
  if (SMEM) {
    if (accum) for (int64_t c = tid; c < R; c += NT) yrow[c] += acc[c];
    else for (int64_t c = tid; c < R; c += NT) yrow[c] = acc[c];
  }
}

template <typename T, int NT>
static int csr_launch(idl_ctx* ctx, const int64_t* rowptr, const int32_t* colidx, const T* vals, int64_t R,
                      int64_t nnz, const int8_t* s, const int32_t* ptr, const int32_t* rows, int64_t L, T* Y,
                      int64_t ldy, int vec_ok, int accum) {
  const size_t head = (size_t)round_up((int64_t)sizeof(CsrSmem<NT>), 16);
  const size_t want = head + sizeof(T) * (size_t)R;
  if (want <= (size_t)ctx->smem_optin) {
    auto k = cs_csr_kernel<T, true, NT>;
    cudaError_t e = ensure_smem(ctx, (const void*)k, want);
    if (e != cudaSuccess) return cuda_check(ctx, e, "csr smem attribute");
    k<<<(unsigned)L, NT, want, ctx->stream>>>(rowptr, colidx, vals, R, nnz, s, ptr, rows, Y, ldy, ctx->d_status,
                                              vec_ok, accum), idl::count_launch();
  } else {
    cudaError_t e = accum ? cudaSuccess : cudaMemset2DAsync(Y, ldy * sizeof(T), 0, R * sizeof(T), L, ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "csr zero");
    auto k = cs_csr_kernel<T, false, NT>;
    e = ensure_smem(ctx, (const void*)k, head);
    if (e != cudaSuccess) return cuda_check(ctx, e, "csr smem attribute");
    k<<<(unsigned)L, NT, head, ctx->stream>>>(rowptr, colidx, vals, R, nnz, s, ptr, rows, Y, ldy, ctx->d_status,
                                              vec_ok, accum), idl::count_launch();
  }
  return cuda_check(ctx, cudaGetLastError(), "countsketch csr");
}

template <typename T>
static int csr_impl(idl_ctx* ctx, const int64_t* rowptr, const int32_t* colidx, const T* vals, int64_t R, int64_t nnz,
                    const int8_t* s, const int32_t* ptr, const int32_t* rows, int64_t L, T* Y, int64_t ldy, int accum) {
  if (L > 0x7fffffffLL) return fail(ctx, IDL_ELIMIT, "countsketch csr: too many buckets");
  // a batch's quads are counted in int: bound the row width
  if (R > 4000000) return fail(ctx, IDL_ELIMIT, "countsketch csr: R > 4e6");
  const int vec_ok = ((uintptr_t)colidx % 16 == 0) && ((uintptr_t)vals % 16 == 0);
  return csr_launch<T, 512>(ctx, rowptr, colidx, vals, R, nnz, s, ptr, rows, L, Y, ldy, vec_ok, accum);
}

int launch_countsketch_csr(idl_ctx* ctx, const int64_t* rowptr, const int32_t* colidx, const void* vals, int64_t I,
                           int64_t R, int64_t nnz, int dtype, const int8_t* s, const int32_t* bucket_ptr,
                           const int32_t* row_list, int64_t L, void* Y1, int64_t ldy, bool accum) {
  (void)I;
  if (dtype == IDL_F32)
    return csr_impl<float>(ctx, rowptr, colidx, (const float*)vals, R, nnz, s, bucket_ptr, row_list, L, (float*)Y1, ldy,
                           accum);
  return csr_impl<double>(ctx, rowptr, colidx, (const double*)vals, R, nnz, s, bucket_ptr, row_list, L, (double*)Y1,
                          ldy, accum);
}

}  // namespace idl
