// gemm_dev.cuh -- device bodies of the tcgen05 Gaussian stage, shared by the
// single-problem kernels (gaussian_tc.cu) and the batched ones (batch.cu).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace idl {

namespace tc {

constexpr int kThreads = 256;
constexpr int kBM = 128;        // rows of D (columns r of Y1) per CTA
constexpr int kBK = 64;         // K per stage (one 128-byte swizzle atom of bf16)
constexpr int kStages = 2;
constexpr uint64_t kTimeoutNs = 1000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_timer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Bounded wait: true when the phase of the given parity completed, false once
// limit_ns (default 1 s) of %globaltimer time have passed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns = kTimeoutNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_timer() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// K-major operand, 128-byte swizzle: 8-row atoms of 1024 B, rows 128 B apart.
__device__ __forceinline__ uint64_t sw128_desc(const void* base) {
  const uint32_t a = smem_u32(base);
  return (uint64_t)((a >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) |
         ((uint64_t)2 << 61);
}

// instruction descriptor: D FP32, A and B bf16, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

// byte offset of the 16-byte chunk (row, kc) in a K-major 128-byte-swizzled tile
__host__ __device__ __forceinline__ uint32_t sw128_off(int row, int kc) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((kc ^ (row & 7)) << 4));
}

// split x into NP bf16 terms.  NP <= 2: each term the round-to-nearest of what
// the previous ones left (NP = 1 is the bf16 rounding the BF16 mode defines).
// NP = 3: the top 8 mantissa bits of what is left, by truncation -- three terms
// then hold all 24 bits of x exactly, and each step is one AND and one FSUB.
template <int NP>
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16* out) {
  float r = x;
  if constexpr (NP == 3) {
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const uint32_t hb = __float_as_uint(r) & 0xFFFF0000u;
      out[p] = __ushort_as_bfloat16((unsigned short)(hb >> 16));
      r = r - __uint_as_float(hb);
    }
  } else {
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const __nv_bfloat16 b = __float2bfloat16_rn(r);
      out[p] = b;
      r = r - __bfloat162float(b);
    }
  }
}

}  // namespace tc

// Omega (m2 x m1, FP64) -> bf16 planes of Omega^T in the swizzled K-major tile layout:
// [k block][plane][NT rows][64] with rows n = 0..NT-1 (zero beyond m2 / m1).
template <int NP>
__device__ __forceinline__ void omega_planes_elem(int64_t e, const double* __restrict__ Om, int m2, int64_t m1, int NT,
                                                  __nv_bfloat16* __restrict__ out) {
  const int kc = (int)(e & 7);
  const int n = (int)((e >> 3) % NT);
  const int kb = (int)(e / (8 * NT));
  __nv_bfloat16 pl[NP][8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int64_t k = (int64_t)kb * tc::kBK + kc * 8 + q;
    const float x = (n < m2 && k < m1) ? (float)Om[(int64_t)n * m1 + k] : 0.f;
    __nv_bfloat16 t[NP];
    tc::split_bf16<NP>(x, t);
#pragma unroll
    for (int p = 0; p < NP; ++p) pl[p][q] = t[p];
  }
  unsigned char* tile = (unsigned char*)out + (size_t)kb * NP * NT * 128;
#pragma unroll
  for (int p = 0; p < NP; ++p)
    *(uint4*)(tile + (size_t)p * NT * 128 + tc::sw128_off(n, kc)) = *(const uint4*)pl[p];
}

// Products (plane of A, plane of B) per precision mode, smallest terms first.
__host__ __device__ constexpr int n_products(int np) { return np == 1 ? 1 : (np == 2 ? 3 : 6); }
__host__ __device__ constexpr int prod_a(int np, int q) {
  return np == 1 ? 0 : (np == 2 ? (q == 0 ? 1 : 0) : (q == 0 ? 2 : q == 1 ? 1 : q == 2 ? 0 : q == 3 ? 1 : 0));
}
__host__ __device__ constexpr int prod_b(int np, int q) {
  return np == 1 ? 0 : (np == 2 ? (q == 1 ? 1 : 0) : (q == 0 ? 0 : q == 1 ? 1 : q == 2 ? 2 : q == 3 ? 0 : q == 4 ? 1 : 0));
}

// Warp-specialised: warps 0-7 convert (load FP32 Y1 one K block ahead in
// registers, split into bf16 planes, store them swizzled, arrive on a_ready);
// warp 8 feeds Omega^T planes through a ring of bulk copies (BS = 2 or 3 slots) and one of
// its lanes issues the MMAs.  Stages are handed over with mbarriers only.
constexpr int kConvThreads = 256;
constexpr int kTcThreads = kConvThreads + 32;
constexpr int kBSlots = 3;     // Omega^T ring slots (at most; the launcher may pass 2)
// The single-problem launcher passes two slots for row-major Y1 (and wherever two slots
// avoid splitting N); the batch and column-major Y1 use three.

// One CTA: rows [mt*128, +128) of D, columns [z*NTc, +NTc), K blocks [kb0, kb0 + nk);
// partial result rows go to part_base[r * NT + column]; with ldo > 0 (a CTA that
// covers all of K) the result goes straight to the output instead,
// part_base[r * ldo + column] for columns < ncols.  smem_raw: the dynamic
// shared memory (1 KB alignment slack included by the launcher).
// CM = false: Y1 row-major (Y1[b * ldy1 + r]); CM = true: column-major
// (Y1[r * ldy1 + b]), each converter thread then reads 32 consecutive K values
// of its row of D (one 128-byte line when ldy1 is a multiple of 32).
template <int NP, bool CM = false>
__device__ __forceinline__ void gauss_tc_block(const float* __restrict__ Y1, int64_t ldy1, int64_t R, int64_t m1,
                                               const __nv_bfloat16* __restrict__ Bpl, int NT, int NTc, int kb0, int nk,
                                               int64_t mt, int z, float* __restrict__ part_base, int* status,
                                               unsigned char* smem_raw, int BS = kBSlots, int64_t ldo = 0,
                                               int ncols = 0) {
  using namespace tc;
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int a_plane = kBM * kBK * 2;                   // 16 KB
  const int b_plane = NTc * kBK * 2;
  const int n0 = z * NTc;
  unsigned char* A = sm;                               // [stage][plane] a_plane
  unsigned char* B = A + kStages * NP * a_plane;       // [slot][plane] b_plane
  uint64_t* bars = (uint64_t*)(B + BS * NP * b_plane);
  uint64_t* a_ready = bars;                            // [kStages] 256 converter arrivals
  uint64_t* mma_done = bars + 2;                       // [kStages] tcgen05.commit
  uint64_t* b_full = bars + 4;                         // [BS] bulk-copy bytes
  uint64_t* b_free = bars + 7;                         // [BS] tcgen05.commit
  uint32_t* tmem_slot = (uint32_t*)(bars + 10);
  __shared__ int s_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t r0 = mt * kBM;
  // two accumulators (columns [0, NTc) and [NTc, 2 NTc)) taken in turn, so consecutive
  // MMAs do not depend on each other's result
  uint32_t tcols = 32;
  while ((int)tcols < 2 * NTc) tcols <<= 1;

  if (tid == 0) {
    for (int q = 0; q < kStages; ++q) { mbar_init(&a_ready[q], kConvThreads); mbar_init(&mma_done[q], 1); }
    for (int q = 0; q < BS; ++q) { mbar_init(&b_full[q], 1); mbar_init(&b_free[q], 1); }
    fence_barrier_init();
    s_flag = 0;
  }
  if (warp == 0) tmem_alloc(tmem_slot, tcols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t b_bytes = (uint32_t)(NP * b_plane);
  // the NP planes' row chunks [n0, n0 + NTc) of K block kb into B slot sl
  auto fetch_b = [&](int kb, int sl) {
    mbar_expect_tx(&b_full[sl], b_bytes);
#pragma unroll
    for (int p = 0; p < NP; ++p)
      bulk_g2s(B + (size_t)(sl * NP + p) * b_plane, Bpl + ((size_t)kb * NP * NT + (size_t)p * NT + n0) * kBK,
               (uint32_t)b_plane, &b_full[sl]);
  };

  if (warp < 8) {
    // ---------------- converters ----------------
    const int m = tid & (kBM - 1);
    // 8-value k-chunks of this thread: kq, kq+2, kq+4, kq+6 (row-major Y1: a warp reads
    // 32 consecutive columns of one row) or 4kq .. 4kq+3 (column-major Y1)
    const int kq = tid >> 7;
    auto kchunk = [&](int c) { return CM ? kq * 4 + c : kq + 2 * c; };
    const bool col_ok = r0 + m < R;
    const float* ycol = CM && col_ok ? Y1 + (r0 + m) * ldy1 : Y1;
    const bool cm_vec = CM && (ldy1 & 3) == 0 && (((uintptr_t)Y1) & 15) == 0;
    // two register buffers: the loads of K block i+2 are in flight while block i is converted
    float va[4][8], vb[4][8];
    auto load_block = [&](float (&v)[4][8], int kb) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int kc = kchunk(c);
        const int64_t b0 = (int64_t)kb * kBK + kc * 8;
        if (CM && cm_vec && col_ok && b0 + 8 <= m1) {
          const float4 x = __ldcs((const float4*)(ycol + b0));
          const float4 y = __ldcs((const float4*)(ycol + b0 + 4));
          v[c][0] = x.x; v[c][1] = x.y; v[c][2] = x.z; v[c][3] = x.w;
          v[c][4] = y.x; v[c][5] = y.y; v[c][6] = y.z; v[c][7] = y.w;
        } else if (!CM && col_ok && b0 + 8 <= m1) {
          // whole chunk inside Y1: one row pointer, stride ldy1, no per-value predicate
          const float* q = Y1 + b0 * ldy1 + r0 + m;
#pragma unroll
          for (int e = 0; e < 8; ++e) v[c][e] = __ldcs(q + e * ldy1);
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int64_t b = b0 + e;
            v[c][e] = (col_ok && b < m1) ? __ldcs(CM ? ycol + b : Y1 + b * ldy1 + r0 + m) : 0.f;
          }
        }
      }
    };
    // convert block i from v into A stage i&1; false when the kernel is giving up
    auto convert = [&](float (&v)[4][8], int i) -> bool {
      const int s = i & 1;
      if (i >= 2 && !mbar_wait(&mma_done[s], ((i - 2) >> 1) & 1)) { s_flag = 1; return false; }   // stage s free
      if (*(volatile int*)&s_flag) return false;
      unsigned char* As = A + (size_t)s * NP * a_plane;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int kc = kchunk(c);
        if constexpr (NP == 3) {
          // truncation split (split_bf16<3>) of two values at a time: a plane's bf16 pair
          // is the top halves of the two remainders, one byte permute
          uint32_t w[NP][4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float x0 = v[c][2 * j], x1 = v[c][2 * j + 1];
#pragma unroll
            for (int p = 0; p < NP; ++p) {
              const uint32_t u0 = __float_as_uint(x0), u1 = __float_as_uint(x1);
              w[p][j] = __byte_perm(u0, u1, 0x7632);
              if (p + 1 < NP) {
                x0 -= __uint_as_float(u0 & 0xFFFF0000u);
                x1 -= __uint_as_float(u1 & 0xFFFF0000u);
              }
            }
          }
#pragma unroll
          for (int p = 0; p < NP; ++p)
            *(uint4*)(As + (size_t)p * a_plane + sw128_off(m, kc)) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
        } else {
          __nv_bfloat16 pl[NP][8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            __nv_bfloat16 t[NP];
            split_bf16<NP>(v[c][e], t);
#pragma unroll
            for (int p = 0; p < NP; ++p) pl[p][e] = t[p];
          }
#pragma unroll
          for (int p = 0; p < NP; ++p) *(uint4*)(As + (size_t)p * a_plane + sw128_off(m, kc)) = *(const uint4*)pl[p];
        }
      }
      fence_async_smem();
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&a_ready[s])) : "memory");
      return true;
    };
    if (nk > 0) load_block(va, kb0);
    if (nk > 1) load_block(vb, kb0 + 1);
    for (int i = 0; i < nk; i += 2) {
      if (!convert(va, i)) break;
      if (i + 2 < nk) load_block(va, kb0 + i + 2);
      if (i + 1 >= nk) break;
      if (!convert(vb, i + 1)) break;
      if (i + 3 < nk) load_block(vb, kb0 + i + 3);
    }
  } else if (lane == 0) {
    // ---------------- producer of Omega^T planes + MMA issue ----------------
    int last_commit = -1, b_issued = 0, b_done = 0;
    for (int q = 0; q < BS && q < nk; ++q) { fetch_b(kb0 + q, q); b_issued = q + 1; }
    const uint32_t idesc = idesc_bf16(NTc);
    for (int i = 0; i < nk && !*(volatile int*)&s_flag; ++i) {
      const int s = i & 1, sb = i % BS;
      if (!mbar_wait(&a_ready[s], (i >> 1) & 1)) { s_flag = 1; break; }
      if (!mbar_wait(&b_full[sb], (i / BS) & 1)) { s_flag = 1; break; }
      b_done = i + 1;
      tc_fence_after();
      const unsigned char* As = A + (size_t)s * NP * a_plane;
      const unsigned char* Bs = B + (size_t)sb * NP * b_plane;
#pragma unroll
      for (int ks = 0; ks < kBK / 16; ++ks) {
#pragma unroll
        for (int q = 0; q < n_products(NP); ++q) {
          const int u = (ks * n_products(NP) + q) & 1;           // accumulator of this MMA
          const uint64_t ad = sw128_desc(As + (size_t)prod_a(NP, q) * a_plane) + (uint64_t)(ks * 2);
          const uint64_t bd = sw128_desc(Bs + (size_t)prod_b(NP, q) * b_plane) + (uint64_t)(ks * 2);
          const bool first = i == 0 && ks * n_products(NP) + q < 2;
          mma_bf16(tmem + (uint32_t)(u * NTc), ad, bd, idesc, first ? 0u : 1u);
        }
      }
      mma_commit(&mma_done[s]);
      mma_commit(&b_free[sb]);
      last_commit = i;
      // refill the B slot of block i-1 with block i-1+BS once block i-1's MMAs are done
      if (i >= 1 && i - 1 + BS < nk) {
        const int so = (i - 1) % BS;
        if (!mbar_wait(&b_free[so], ((i - 1) / BS) & 1)) { s_flag = 1; break; }
        fetch_b(kb0 + i - 1 + BS, so);
        b_issued = i + BS;
      }
    }
    // the accumulator is final once the last MMAs complete (bounded wait)
    if (last_commit >= 0 && !mbar_wait(&mma_done[last_commit & 1], (last_commit >> 1) & 1)) s_flag = 2;
    if (last_commit < nk - 1 && !s_flag) s_flag = 1;
    // after an early exit, wait (bounded) for Omega^T copies still in flight
    for (int j = b_done; j < b_issued; ++j) (void)mbar_wait(&b_full[j % BS], (j / BS) & 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (s_flag == 0 && nk > 0 && warp < 8) {
    // epilogue: warp w reads TMEM lanes 32*(w%4).. (rows of D); warps 0-3 and 4-7 split the columns
    const int lane_base = (warp & 3) * 32;
    const int64_t r = r0 + lane_base + lane;
    float* prow = part_base + r * (ldo ? ldo : NT) + n0;
    const int uses = 4 * n_products(NP) * nk;        // MMAs issued; the second accumulator is used if > 1
    for (int q = warp >> 2; q < NTc / 16; q += 2) {
      float vals[16];
      tmem_ld16(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(q * 16), vals);
      if (uses > 1) {
        float v2[16];
        tmem_ld16(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(NTc + q * 16), v2);
#pragma unroll
        for (int j = 0; j < 16; ++j) vals[j] += v2[j];
      }
      if (r < R && ldo == 0) {
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *(float4*)(prow + q * 16 + j) = make_float4(vals[j], vals[j + 1], vals[j + 2], vals[j + 3]);
      } else if (r < R) {                            // straight to Y2 (row stride ldo, ncols columns)
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (n0 + q * 16 + j < ncols) prow[q * 16 + j] = vals[j];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && s_flag) set_status(status, IDL_ETIMEOUT);
  if (warp == 0) tmem_dealloc(tmem, tcols);
}

}  // namespace idl

namespace idl {

// Pre-tiled A operand: the bf16 planes of Y1^T already in the swizzled K-major tile
// layout, one 16 KB tile per (column tile mt, K block kb, plane p) at byte offset
// ((mt * nkb + kb) * NP + p) * 16384 -- written by the producer of Y1 (the L = 8192
// TensorSketch of the batch's CP items).  Row m of a tile is column mt * 128 + m;
// within a row, the 16-byte chunk of K values 8 kc .. 8 kc + 7 at sw128_off(m, kc).
constexpr int kTileBytes = tc::kBM * tc::kBK * 2;

__host__ __device__ constexpr size_t pretiled_bytes(int64_t R, int64_t m1, int NP) {
  return (size_t)((R + tc::kBM - 1) / tc::kBM) * (size_t)((m1 + tc::kBK - 1) / tc::kBK) * (size_t)NP * kTileBytes;
}

// shared memory of gauss_tc_block_pretiled with an A ring of S stages: the 1 KB
// alignment slack, the rings, 2 S + 6 barriers and the TMEM address
constexpr int kPtMaxStages = 6;
__host__ __device__ constexpr size_t pretiled_smem_bytes(int S, int NP, int NT) {
  return 1024 + (size_t)S * NP * kTileBytes + (size_t)kBSlots * NP * NT * tc::kBK * 2 + 8 * (size_t)(2 * S + 6) + 16;
}

// Pre-tiled store of the column pair (r0, r0 + 1), r0 even: thread t of a block of T
// threads holds the pair's K entries l = T q + t (q < Q) as v[q] = (column r0, column
// r0 + 1), each to be scaled by s0 / s1.  Lanes t and t ^ 1 hold one bf16 pair of
// K entries: they swap the value of the column the other one stores, so the even
// lane writes column r0's words and the odd lane column r0 + 1's, and each plane's
// word is the split (split_bf16, same bits) of both values at once -- one 4-byte
// store per plane and q.  Past the last column s1 = 0 and row r0 + 1 gets zeros.
template <int NP, int T, int Q>
__device__ __forceinline__ void pretiled_store_pair(unsigned char* __restrict__ base, int64_t nkb, int64_t r0,
                                                    const float2* v, float s0, float s1) {
  static_assert(T % tc::kBK == 0, "a thread keeps its place in the K block");
  const int t = threadIdx.x;
  const bool odd = t & 1;
  const int64_t mt = r0 / tc::kBM;
  const int row = (int)(r0 % tc::kBM) + (odd ? 1 : 0);
  const int kk = t % tc::kBK;
  unsigned char* dst = base + (size_t)((mt * nkb + t / tc::kBK) * NP) * kTileBytes + tc::sw128_off(row, kk >> 3) +
                       2 * (kk & 6);
  constexpr size_t step = (size_t)(T / tc::kBK) * NP * kTileBytes;   // q + 1: T / 64 K blocks on
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const float x0 = v[q].x * s0, x1 = v[q].y * s1;
    const float other = __shfl_xor_sync(0xffffffffu, odd ? x0 : x1, 1);
    float lo = odd ? other : x0;          // the stored column's values at K entries 2j and 2j + 1
    float hi = odd ? x1 : other;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      uint32_t w;
      if constexpr (NP == 3) {
        // truncation split: the top halves of both remainders
        const uint32_t ul = __float_as_uint(lo), uh = __float_as_uint(hi);
        w = __byte_perm(ul, uh, 0x7632);
        lo -= __uint_as_float(ul & 0xFFFF0000u);
        hi -= __uint_as_float(uh & 0xFFFF0000u);
      } else {
        const __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);   // .x (low half) = rn(lo)
        w = *reinterpret_cast<const uint32_t*>(&b);
        if (p + 1 < NP) {
          lo -= __low2float(b);
          hi -= __high2float(b);
        }
      }
      *reinterpret_cast<uint32_t*>(dst + q * step + (size_t)p * kTileBytes) = w;
    }
  }
}

// The Gaussian-stage CTA of gauss_tc_block with the A planes fetched by bulk copies from
// the pre-tiled layout into a ring of S stages (no converter work): the elected lane of
// warp 8 feeds both rings and issues the MMAs; the other warps only join the epilogue.
template <int NP>
__device__ __forceinline__ void gauss_tc_block_pretiled(const unsigned char* __restrict__ Apl, int64_t nkb_all,
                                                        int64_t R, const __nv_bfloat16* __restrict__ Bpl, int NT,
                                                        int NTc, int kb0, int nk, int64_t mt, int z, int S,
                                                        float* __restrict__ part_base, int* status,
                                                        unsigned char* smem_raw, int64_t ldo = 0, int ncols = 0) {
  using namespace tc;
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int b_plane = NTc * kBK * 2;
  const int n0 = z * NTc;
  unsigned char* A = sm;                               // [stage][plane] 16 KB
  unsigned char* B = A + (size_t)S * NP * kTileBytes;  // [slot][plane] b_plane
  uint64_t* bars = (uint64_t*)(B + (size_t)kBSlots * NP * b_plane);
  uint64_t* a_full = bars;                             // [S] bulk-copy bytes
  uint64_t* mma_done = bars + S;                       // [S] tcgen05.commit
  uint64_t* b_full = bars + 2 * S;                     // [3]
  uint64_t* b_free = bars + 2 * S + 3;                 // [3]
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * S + 6);
  __shared__ int s_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t r0 = mt * kBM;
  uint32_t tcols = 32;
  while ((int)tcols < 2 * NTc) tcols <<= 1;
  if (tid == 0) {
    for (int q = 0; q < S; ++q) { mbar_init(&a_full[q], 1); mbar_init(&mma_done[q], 1); }
    for (int q = 0; q < kBSlots; ++q) { mbar_init(&b_full[q], 1); mbar_init(&b_free[q], 1); }
    fence_barrier_init();
    s_flag = 0;
  }
  if (warp == 0) tmem_alloc(tmem_slot, tcols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  if (warp == 8 && lane == 0) {
    const unsigned char* atile = Apl + (size_t)(mt * nkb_all) * NP * kTileBytes;
    auto fetch_a = [&](int kb, int st) {
      mbar_expect_tx(&a_full[st], (uint32_t)(NP * kTileBytes));
#pragma unroll
      for (int p = 0; p < NP; ++p)
        bulk_g2s(A + (size_t)(st * NP + p) * kTileBytes, atile + ((size_t)kb * NP + p) * kTileBytes,
                 (uint32_t)kTileBytes, &a_full[st]);
    };
    auto fetch_b = [&](int kb, int sl) {
      mbar_expect_tx(&b_full[sl], (uint32_t)(NP * b_plane));
#pragma unroll
      for (int p = 0; p < NP; ++p)
        bulk_g2s(B + (size_t)(sl * NP + p) * b_plane, Bpl + ((size_t)kb * NP * NT + (size_t)p * NT + n0) * kBK,
                 (uint32_t)b_plane, &b_full[sl]);
    };
    int last_commit = -1, a_issued = 0, b_issued = 0, done = 0;
    for (int q = 0; q < S && q < nk; ++q) { fetch_a(kb0 + q, q); a_issued = q + 1; }
    for (int q = 0; q < kBSlots && q < nk; ++q) { fetch_b(kb0 + q, q); b_issued = q + 1; }
    const uint32_t idesc = idesc_bf16(NTc);
    for (int i = 0; i < nk; ++i) {
      const int s = i % S, sb = i % kBSlots;
      if (!mbar_wait(&a_full[s], (uint32_t)((i / S) & 1))) { s_flag = 1; break; }
      if (!mbar_wait(&b_full[sb], (uint32_t)((i / kBSlots) & 1))) { s_flag = 1; break; }
      done = i + 1;
      tc_fence_after();
      const unsigned char* As = A + (size_t)s * NP * kTileBytes;
      const unsigned char* Bs = B + (size_t)sb * NP * b_plane;
#pragma unroll
      for (int ks = 0; ks < kBK / 16; ++ks) {
#pragma unroll
        for (int q = 0; q < n_products(NP); ++q) {
          const int u = (ks * n_products(NP) + q) & 1;
          const uint64_t ad = sw128_desc(As + (size_t)prod_a(NP, q) * kTileBytes) + (uint64_t)(ks * 2);
          const uint64_t bd = sw128_desc(Bs + (size_t)prod_b(NP, q) * b_plane) + (uint64_t)(ks * 2);
          const bool first = i == 0 && ks * n_products(NP) + q < 2;
          mma_bf16(tmem + (uint32_t)(u * NTc), ad, bd, idesc, first ? 0u : 1u);
        }
      }
      mma_commit(&mma_done[s]);
      mma_commit(&b_free[sb]);
      last_commit = i;
      // refill block i-1's A stage and B slot once its MMAs are done
      if (i >= 1) {
        const int so = (i - 1) % S, sbo = (i - 1) % kBSlots;
        const bool need_a = i - 1 + S < nk, need_b = i - 1 + kBSlots < nk;
        if (need_a) {
          if (!mbar_wait(&mma_done[so], (uint32_t)(((i - 1) / S) & 1))) { s_flag = 1; break; }
          fetch_a(kb0 + i - 1 + S, so);
          a_issued = i + S;
        }
        if (need_b) {
          if (!mbar_wait(&b_free[sbo], (uint32_t)(((i - 1) / kBSlots) & 1))) { s_flag = 1; break; }
          fetch_b(kb0 + i - 1 + kBSlots, sbo);
          b_issued = i + kBSlots;
        }
      }
    }
    if (last_commit >= 0 && !mbar_wait(&mma_done[last_commit % S], (uint32_t)((last_commit / S) & 1))) s_flag = 2;
    if (last_commit < nk - 1 && !s_flag) s_flag = 1;
    // after an early exit, wait (bounded) for the copies still in flight
    for (int j = done; j < a_issued; ++j) (void)mbar_wait(&a_full[j % S], (uint32_t)((j / S) & 1));
    for (int j = done; j < b_issued; ++j) (void)mbar_wait(&b_full[j % kBSlots], (uint32_t)((j / kBSlots) & 1));
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (s_flag == 0 && nk > 0 && warp < 8) {
    const int lane_base = (warp & 3) * 32;
    const int64_t r = r0 + lane_base + lane;
    float* prow = part_base + r * (ldo ? ldo : NT) + n0;
    const int uses = 4 * n_products(NP) * nk;
    for (int q = warp >> 2; q < NTc / 16; q += 2) {
      float vals[16];
      tmem_ld16(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(q * 16), vals);
      if (uses > 1) {
        float v2[16];
        tmem_ld16(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(NTc + q * 16), v2);
#pragma unroll
        for (int j = 0; j < 16; ++j) vals[j] += v2[j];
      }
      if (r < R && ldo == 0) {
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *(float4*)(prow + q * 16 + j) = make_float4(vals[j], vals[j + 1], vals[j + 2], vals[j + 3]);
      } else if (r < R) {                            // straight to Y2 (row stride ldo, ncols columns)
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (n0 + q * 16 + j < ncols) prow[q * 16 + j] = vals[j];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && s_flag) set_status(status, IDL_ETIMEOUT);
  if (warp == 0) tmem_dealloc(tmem, tcols);
}

}  // namespace idl
