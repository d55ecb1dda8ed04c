// draws_dev.cuh -- device bodies of the draws and of the bucket-offset build,
// shared by the single-problem kernels (draws.cu) and the batched ones (batch.cu).
#pragma once

#include "common.cuh"

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

// Arguments of the CountSketch draw of one problem (host-computed).
struct CsDrawArgs {
  uint64_t bucket_base, sign_base, mask;
  FeistelKeys keys;
  int half;
};

inline int feistel_width_host(int64_t I) {
  int w = 1;
  while (w < 62 && ((int64_t)1 << w) < I) ++w;
  if (w & 1) ++w;
  return w < 2 ? 2 : w;
}

inline CsDrawArgs make_cs_draw_args(uint64_t seed, int64_t I) {
  CsDrawArgs a;
  const uint64_t pb = stream_base(seed, kTagPerm);
  for (int r = 0; r < kFeistelRounds; ++r) a.keys.k[r] = stream_at(pb, (uint64_t)r);
  const int w = feistel_width_host(I);
  a.half = w / 2;
  a.mask = (1ull << a.half) - 1;
  a.bucket_base = stream_base(seed, kTagBucket);
  a.sign_base = stream_base(seed, kTagSign);
  return a;
}

// h(i), s(i) of a CountSketch (plain or modified, Remark 2) for row i of I
__device__ __forceinline__ void cs_draw_value(int64_t i, const CsDrawArgs& a, int64_t I, int64_t L, int modified,
                                              int32_t* hv_out, int8_t* s_out, int* status) {
  const uint32_t x = bounded(stream_at(a.bucket_base, (uint64_t)i), (uint64_t)L);
  uint32_t hv = x;
  if (modified) {
    uint64_t y = feistel((uint64_t)i, a.half, a.mask, a.keys);
    // Cycle walking ends: i lies on a finite cycle of the bijection on [0, 2^w)
    // and i < I.  The cap only guards against corrupted arguments.
    int walks = 0;
    while (y >= (uint64_t)I && walks < (1 << 22)) { y = feistel(y, a.half, a.mask, a.keys); ++walks; }
    if (y >= (uint64_t)I) { set_status(status, IDL_ETIMEOUT); y = 0; }
    if (y < (uint64_t)L) hv = (uint32_t)y;
  }
  *hv_out = (int32_t)hv;
  *s_out = (stream_at(a.sign_base, (uint64_t)i) >> 63) ? (int8_t)-1 : (int8_t)1;
}

// h[i], s[i] of a CountSketch (plain or modified, Remark 2)
__device__ __forceinline__ void cs_draw_elem(int64_t i, const CsDrawArgs& a, int64_t I, int64_t L, int modified,
                                             int32_t* __restrict__ h, int8_t* __restrict__ s, int* status) {
  cs_draw_value(i, a, I, L, modified, h + i, s + i, status);
}

// Box-Muller pair p (flat indices 2p, 2p+1) of Omega; cos(2 pi u2) as cospi(2 u2)
__device__ __forceinline__ void gauss_pair(int64_t p, uint64_t base, int64_t n, double* __restrict__ Om) {
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

// The same pair in FP32 arithmetic (the draw of the FP32 pipelines and batches:
// GB300's FP64 pipes made the FP64 form several milliseconds per batch).  The
// uniforms are the same 53-bit integers; ln U1 is log1pf(-(1 - U1)) when U1 > 1/2
// (1 - U1 formed exactly in integers) and logf(U1) otherwise, and the angle
// 2 pi U2 is reduced to pi t, t in [-1, 1), in integers before the conversion.
// The result differs from the FP64 draw by a few units in the last place of
// FP32 (about 4e-7 (rho + |z|)).
__device__ __forceinline__ void gauss_pair_f32(int64_t p, uint64_t base, int64_t n, double* __restrict__ Om) {
  const uint64_t ka = stream_at(base, 2 * (uint64_t)p) >> 11;       // U1 = (ka + 1) 2^-53
  const uint64_t kc = stream_at(base, 2 * (uint64_t)p + 1) >> 11;   // U2 = kc 2^-53
  float lg;
  if (ka >= (1ull << 52)) {
    const float v = __ull2float_rn((1ull << 53) - 1 - ka) * 0x1.0p-53f;   // 1 - U1
    lg = log1pf(-v);
  } else {
    lg = logf(__ull2float_rn(ka + 1) * 0x1.0p-53f);
  }
  const float rho = sqrtf(-2.f * lg);
  const int64_t kt = kc >= (1ull << 52) ? (int64_t)kc - (int64_t)(1ull << 53) : (int64_t)kc;   // 2 U2 (- 2)
  const float t = __ll2float_rn(kt) * 0x1.0p-52f;
  float sv, cv;
  sincospif(t, &sv, &cv);
  Om[2 * p] = (double)(rho * cv);
  if (2 * p + 1 < n) Om[2 * p + 1] = (double)(rho * sv);
}

// TensorSketch map of one mode entry
__device__ __forceinline__ void mode_elem(int64_t i, uint64_t hb, uint64_t sb, int64_t L, int32_t* __restrict__ h,
                                          int8_t* __restrict__ s) {
  h[i] = (int32_t)bounded(stream_at(hb, (uint64_t)i), (uint64_t)L);
  s[i] = (stream_at(sb, (uint64_t)i) >> 63) ? (int8_t)-1 : (int8_t)1;
}

// ---------------------------------------------------------------------------
// Bucket offsets: histogram, exclusive scan, atomic scatter, per-bucket rank sort
// ---------------------------------------------------------------------------
constexpr int kHistSmem = 12288;     // buckets histogrammed in shared memory first
constexpr int kWarpSortCap = 1024;   // rows per bucket sorted by one warp
constexpr int kBlockSortCap = 12288; // rows per bucket sorted by one block

// block `blk` of `nblk` (grid-stride over rows); sh: >= L ints of shared memory when L <= kHistSmem
__device__ __forceinline__ void bucket_hist_body(const int32_t* __restrict__ h, int64_t I, int64_t L,
                                                 int32_t* __restrict__ cnt, int* status, int64_t blk, int64_t nblk,
                                                 int32_t* sh) {
  const bool local = L <= kHistSmem;
  if (local) {
    for (int64_t b = threadIdx.x; b < L; b += blockDim.x) sh[b] = 0;
    __syncthreads();
  }
  for (int64_t i = blk * blockDim.x + threadIdx.x; i < I; i += nblk * blockDim.x) {
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

// one block: exclusive scan of cnt[0..L) into ptr[0..L] and the scatter cursor
// (cnt and cursor may alias: each thread reads cnt[b] before it writes cursor[b])
__device__ __forceinline__ void bucket_scan_body(const int32_t* cnt, int64_t L, int32_t* __restrict__ ptr,
                                                 int32_t* cursor) {
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

__device__ __forceinline__ void bucket_scatter_elem(int64_t i, const int32_t* __restrict__ h, int64_t L,
                                                    int32_t* __restrict__ cursor, int32_t* __restrict__ row_list) {
  const int b = h[i];
  if (b < 0 || (int64_t)b >= L) return;        // flagged by the histogram pass
  const int pos = atomicAdd(&cursor[b], 1);
  row_list[pos] = (int32_t)i;
}

// one warp, bucket b: rank sort of its rows (distinct, so rank = #smaller); buckets
// above kWarpSortCap go to the `big` list for a block.  seg: kWarpSortCap ints.
__device__ __forceinline__ void bucket_sort_warp_body(const int32_t* __restrict__ ptr, int64_t b,
                                                      int32_t* __restrict__ row_list, int32_t* __restrict__ big,
                                                      int32_t* __restrict__ nbig, int32_t* seg) {
  const int lane = threadIdx.x & 31;
  const int a0 = ptr[b], n = ptr[b + 1] - a0;
  if (n <= 1) return;
  if (n > kWarpSortCap) {
    if (lane == 0) big[atomicAdd(nbig, 1)] = (int32_t)b;
    return;
  }
  for (int j = lane; j < n; j += 32) seg[j] = row_list[a0 + j];
  __syncwarp();
  for (int j = lane; j < n; j += 32) {
    const int x = seg[j];
    int rank = 0;
    for (int t = 0; t < n; ++t) rank += seg[t] < x;
    row_list[a0 + rank] = x;
  }
}

// one block: the rows of bucket b written in increasing order by one pass over all
// of h (for buckets above kBlockSortCap rows).  Each thread takes 16 consecutive
// rows of a chunk, a block-wide prefix of the per-thread match counts places them.
// sh: >= 32 ints of shared memory.
__device__ __forceinline__ void bucket_rescan_block_body(const int32_t* __restrict__ h, int64_t I,
                                                         const int32_t* __restrict__ ptr, int32_t b,
                                                         int32_t* __restrict__ row_list, int32_t* sh) {
  constexpr int E = 16;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int32_t base = ptr[b];
  const int64_t chunk = (int64_t)blockDim.x * E;
  for (int64_t c0 = 0; c0 < I; c0 += chunk) {
    const int64_t i0 = c0 + (int64_t)threadIdx.x * E;
    int hv[E];
#pragma unroll
    for (int u = 0; u < E; ++u) hv[u] = i0 + u < I ? __ldg(h + i0 + u) : -1;
    unsigned m = 0;
#pragma unroll
    for (int u = 0; u < E; ++u) m |= (hv[u] == b ? 1u : 0u) << u;
    const int cnt = __popc(m);
    int x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
      int t = lane < nw ? sh[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      if (lane < nw) sh[lane] = t;                       // inclusive prefix over the warps
    }
    __syncthreads();
    int pos = base + (w ? sh[w - 1] : 0) + x - cnt;
    const int32_t total = sh[nw - 1];
#pragma unroll
    for (int u = 0; u < E; ++u)
      if ((m >> u) & 1u) row_list[pos++] = (int32_t)(i0 + u);
    __syncthreads();                                     // sh is reused by the next chunk
    base += total;
  }
}

// one block: rank sort of the rows of bucket b (up to kBlockSortCap; larger ones are
// rewritten in increasing order by a pass over h).  seg: kBlockSortCap ints.
__device__ __forceinline__ void bucket_sort_block_body(const int32_t* __restrict__ ptr, int32_t b,
                                                       int32_t* __restrict__ row_list, int32_t* seg,
                                                       const int32_t* __restrict__ h, int64_t I) {
  const int a0 = ptr[b], n = ptr[b + 1] - a0;
  if (n > kBlockSortCap) {
    __syncthreads();
    bucket_rescan_block_body(h, I, ptr, b, row_list, seg);
    return;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) seg[j] = row_list[a0 + j];
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const int x = seg[j];
    int rank = 0;
    for (int t = 0; t < n; ++t) rank += seg[t] < x;
    row_list[a0 + rank] = x;
  }
}

// ---------------------------------------------------------------------------
// Stable counting sort by bucket (used when L <= kStableMaxL): row i goes to
// its bucket in increasing i without any per-bucket sort.  A block of W warps
// owns a chunk of W * kStableSub rows; warp w owns the chunk's w-th
// sub-chunk of kStableSub consecutive rows.
//   1. stable_count_block: per-warp histograms in shared memory (loads of a
//      sub-chunk in flight together), then the per-bucket sum over the warps
//      goes to cnt[blk][*];
//   2. stable_prefix_bucket: per bucket b, cnt[blk][b] becomes the exclusive
//      prefix over the blocks (one warp per bucket, lanes over blocks, warp
//      scans) and the total; one block scans the totals into bucket_ptr
//      (bucket_scan_body);
//   3. stable_scatter_block: the per-warp histograms are formed again and
//      turned into exclusive prefixes over the warps; warp w then walks its
//      rows in order, 32 at a time, lanes with the same bucket found by
//      __match_any_sync: row i of bucket b goes to ptr[b] + cnt[blk][b] +
//      (rows of b in earlier warps of the block) + (earlier rows of b in the
//      warp).
// ---------------------------------------------------------------------------
constexpr int kStableSub = 1024;                 // rows per warp
constexpr int64_t kStableMaxL = 14336;          // at least three warps' counters fit
constexpr int kStableSmemInts = 51200;          // W * L <= this (200 KB of shared memory)
__host__ __device__ constexpr int stable_warps(int64_t L) {
  return L <= 0 ? 1 : (int)(kStableSmemInts / L >= 8 ? 8 : (kStableSmemInts / L < 1 ? 1 : kStableSmemInts / L));
}

// per-warp histograms of the block's rows into hw[w * L + b]
__device__ __forceinline__ void stable_warp_hist(const int32_t* __restrict__ h, int64_t I, int L, int64_t blk,
                                                 int* status, int32_t* hw) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, W = blockDim.x >> 5;
  for (int e = threadIdx.x; e < W * L; e += blockDim.x) hw[e] = 0;
  __syncthreads();
  const int64_t i0 = (blk * W + w) * (int64_t)kStableSub;
  int32_t* cw = hw + w * L;
  // all of the lane's buckets first (one memory round trip), then the counts
  int hv[kStableSub / 32];
#pragma unroll
  for (int q = 0; q < kStableSub / 32; ++q) {
    const int64_t i = i0 + q * 32 + lane;
    hv[q] = i < I ? __ldg(h + i) : 0;
  }
#pragma unroll
  for (int q = 0; q < kStableSub / 32; ++q) {
    if (i0 + q * 32 + lane >= I) break;
    const int b = hv[q];
    if (b < 0 || b >= L) set_status(status, IDL_EDATA);
    else atomicAdd(&cw[b], 1);
  }
  __syncthreads();
}

__device__ __forceinline__ void stable_count_block(const int32_t* __restrict__ h, int64_t I, int L, int64_t blk,
                                                   int32_t* __restrict__ cnt, int* status, int32_t* hw) {
  stable_warp_hist(h, I, L, blk, status, hw);
  const int W = blockDim.x >> 5;
  int32_t* out = cnt + blk * (int64_t)L;
  for (int b = threadIdx.x; b < L; b += blockDim.x) {
    int32_t t = 0;
    for (int w = 0; w < W; ++w) t += hw[w * L + b];
    out[b] = t;
  }
}

// bucket b (one warp): exclusive prefix over the nblk blocks in place, 32
// blocks per round (lane = block); returns the total (every lane)
__device__ __forceinline__ int32_t stable_prefix_bucket(int32_t* __restrict__ cnt, int64_t nblk, int L, int b) {
  const int lane = threadIdx.x & 31;
  int32_t run = 0;
  for (int64_t c0 = 0; c0 < nblk; c0 += 32) {
    const int64_t c = c0 + lane;
    const int32_t v = c < nblk ? cnt[c * L + b] : 0;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (c < nblk) cnt[c * L + b] = run + x - v;
    run += __shfl_sync(0xffffffffu, x, 31);
  }
  return run;
}

__device__ __forceinline__ void stable_scatter_block(const int32_t* __restrict__ h, int64_t I, int L, int64_t blk,
                                                     const int32_t* __restrict__ ptr, const int32_t* __restrict__ cnt,
                                                     int32_t* __restrict__ row_list, int32_t* hw) {
  int* no_status = nullptr;
  stable_warp_hist(h, I, L, blk, no_status, hw);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, W = blockDim.x >> 5;
  // hw[w][b] <- next free slot of bucket b for warp w; the bucket bases first, 8 loads
  // of each array in flight per thread, then the shared-memory prefix over the warps
  const int32_t* pre = cnt + blk * (int64_t)L;
  for (int b0 = threadIdx.x; b0 < L; b0 += 8 * blockDim.x) {
    int32_t base[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int b = b0 + u * blockDim.x;
      base[u] = b < L ? __ldg(ptr + b) + __ldg(pre + b) : 0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int b = b0 + u * blockDim.x;
      if (b >= L) break;
      int32_t run = base[u];
      for (int ww = 0; ww < W; ++ww) {
        const int32_t v = hw[ww * L + b];
        hw[ww * L + b] = run;
        run += v;
      }
    }
  }
  __syncthreads();
  int32_t* cw = hw + w * L;
  const int64_t i0 = (blk * W + w) * (int64_t)kStableSub;
  const unsigned lt = (1u << lane) - 1u;
  int hv[kStableSub / 32];                                            // the lane's buckets, loaded at once
#pragma unroll
  for (int q = 0; q < kStableSub / 32; ++q) {
    const int64_t i = i0 + q * 32 + lane;
    hv[q] = i < I ? __ldg(h + i) : -1;
  }
#pragma unroll
  for (int q = 0; q < kStableSub / 32; ++q) {
    const int64_t i = i0 + q * 32 + lane;
    int b = hv[q];
    if (b >= L) b = -1;                                               // flagged by the counting pass
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const int slot = b >= 0 ? cw[b] : 0;
    __syncwarp();
    if (b >= 0) {
      row_list[slot + __popc(peers & lt)] = (int32_t)i;
      if ((peers & lt) == 0) cw[b] = slot + __popc(peers);             // the group's lowest lane advances it
    }
    __syncwarp();
  }
}

}  // namespace idl
