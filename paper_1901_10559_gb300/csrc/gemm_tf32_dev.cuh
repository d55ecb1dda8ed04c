// gemm_tf32_dev.cuh -- the Gaussian stage Y2 = Omega Y1 (Sec. 1.2.1) in the
// TF32X3 precision mode: tcgen05.mma kind::tf32 with each FP32 operand split
// into two TF32 terms,
//   x = hi + lo,  hi = x with the low 13 mantissa bits cleared,
//                 lo = (x - hi) with the low 13 mantissa bits cleared,
// and three products hi*hi + hi*lo + lo*hi (the 3xTF32 scheme, Ootomo & Yokota
// 2022).  Both terms are exact TF32 values, so what the tensor core does with
// the low bits of a 32-bit container never matters; hi + lo keeps 22 of x's 24
// significand bits and the dropped lo*lo term is below 2^-22 |x y|.
//
// Layout as in the bf16 body (gemm_dev.cuh): D = Y1^T Omega^T, M = 128 columns r
// of Y1 per CTA, N = NTc rows of Omega, K split over CTAs.  A K block is 32 FP32
// values (one 128-byte swizzle row), both operands K-major with the 128-byte
// swizzle.  A (Y1^T):
//   * column-major Y1 (column r at Y1 + r ldy1, 16-byte aligned): each thread
//     copies 64 contiguous bytes of its column with four 16-byte cp.async
//     straight into the swizzled stage (zero fill past R and m1), S - 2 blocks
//     ahead, then splits its own values in place (hi) and beside them (lo):
//     two AND, one FSUB per value;
//   * row-major Y1 (or an unaligned column-major one): register loads two
//     blocks ahead (a warp reads 32 consecutive columns of a row), split and
//     stored transposed into the same layout.
// B (Omega^T): both TF32 planes built once per call in global memory in the
// shared-memory layout, fetched per K block by one cp.async.bulk into a
// kBSlots-slot ring.  Warp 8's lane 0 issues the MMAs; handovers use mbarriers only,
// every wait bounded as in the bf16 body.
#pragma once

#include "gemm_dev.cuh"

namespace idl {
namespace tc {

constexpr int kBKt = 32;                    // K per block: 32 FP32 = one 128-byte swizzle row
constexpr int kTf32MaxStages = 6;
constexpr uint32_t kTf32Mask = 0xFFFFE000u;

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}

// instruction descriptor: D FP32, A and B TF32 (format 2), both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
  const uint32_t h = __float_as_uint(x) & kTf32Mask;
  hi = __uint_as_float(h);
  lo = __uint_as_float(__float_as_uint(x - hi) & kTf32Mask);
}

// 16-byte cp.async with zero fill beyond src_bytes (0..16)
__device__ __forceinline__ void cp_async16(void* dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

}  // namespace tc

// Omega (m2 x m1, FP64) -> the two TF32 planes of Omega^T in the swizzled K-major
// layout [k block][plane][NT rows][32]; element e = (kb, n, kc) writes one
// 16-byte chunk (4 values) of each plane; zero beyond m2 / m1.
__device__ __forceinline__ void omega_tf32_elem(int64_t e, const double* __restrict__ Om, int m2, int64_t m1, int NT,
                                                float* __restrict__ out) {
  const int kc = (int)(e & 7);
  const int n = (int)((e >> 3) % NT);
  const int64_t kb = e / (8 * NT);
  float hi[4], lo[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t k = kb * tc::kBKt + kc * 4 + q;
    const float x = (n < m2 && k < m1) ? (float)Om[(int64_t)n * m1 + k] : 0.f;
    tc::tf32_split(x, hi[q], lo[q]);
  }
  unsigned char* tile = (unsigned char*)out + (size_t)kb * 2 * NT * 128;
  *(float4*)(tile + tc::sw128_off(n, kc)) = make_float4(hi[0], hi[1], hi[2], hi[3]);
  *(float4*)(tile + (size_t)NT * 128 + tc::sw128_off(n, kc)) = make_float4(lo[0], lo[1], lo[2], lo[3]);
}

// Shared memory of one CTA (the launcher adds 1 KB of alignment slack)
__host__ __device__ constexpr size_t tf32_smem_bytes(int stages, int ntc) {
  return 1024 + (size_t)stages * 2 * tc::kBM * 128 + (size_t)kBSlots * 2 * ntc * 128 + 8 * (2 * stages + 6) + 16;
}

// One CTA: rows [mt*128, +128) of D, columns [z*NTc, +NTc), K blocks [kb0, kb0 + nk);
// partial result rows go to part_base[r * NT + column].  S: A stages (3..6).
template <bool CM>
__device__ __forceinline__ void gauss_tf32_block(const float* __restrict__ Y1, int64_t ldy1, int64_t R, int64_t m1,
                                                 const float* __restrict__ Bpl, int NT, int NTc, int kb0, int nk,
                                                 int64_t mt, int z, int S, float* __restrict__ part_base, int* status,
                                                 unsigned char* smem_raw) {
  using namespace tc;
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int a_plane = kBM * 128;                   // 16 KB: 128 rows x 32 FP32
  const int b_plane = NTc * 128;
  const int n0 = z * NTc;
  unsigned char* A = sm;                               // [stage][plane: hi, lo]
  unsigned char* B = A + (size_t)S * 2 * a_plane;      // [slot][plane: hi, lo]
  uint64_t* bars = (uint64_t*)(B + (size_t)kBSlots * 2 * b_plane);
  uint64_t* a_ready = bars;                            // [S] 256 converter arrivals
  uint64_t* mma_done = bars + S;                       // [S] tcgen05.commit
  uint64_t* b_full = bars + 2 * S;                     // [3] bulk-copy bytes
  uint64_t* b_free = bars + 2 * S + 3;                 // [3] tcgen05.commit
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * S + 6);
  __shared__ int s_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t r0 = mt * kBM;
  uint32_t tcols = 32;
  while ((int)tcols < 2 * NTc) tcols <<= 1;

  if (tid == 0) {
    for (int q = 0; q < S; ++q) { mbar_init(&a_ready[q], kConvThreads); mbar_init(&mma_done[q], 1); }
    for (int q = 0; q < kBSlots; ++q) { mbar_init(&b_full[q], 1); mbar_init(&b_free[q], 1); }
    fence_barrier_init();
    s_flag = 0;
  }
  if (warp == 0) tmem_alloc(tmem_slot, tcols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t b_bytes = (uint32_t)(2 * b_plane);
  auto fetch_b = [&](int kb, int sl) {
    mbar_expect_tx(&b_full[sl], b_bytes);
#pragma unroll
    for (int p = 0; p < 2; ++p)
      bulk_g2s(B + (size_t)(sl * 2 + p) * b_plane, Bpl + ((size_t)kb * 2 * NT + (size_t)p * NT + n0) * kBKt,
               (uint32_t)b_plane, &b_full[sl]);
  };

  if (warp < 8) {
    // ---------------- converters: row m of D, 16-byte chunks 4h .. 4h+3 of each K block ----------------
    const int m = tid & (kBM - 1);
    const int h = tid >> 7;
    const int64_t r = r0 + m;
    const bool col_ok = r < R;
    // stage s free for block i (its block i - S done by the MMAs); false once giving up
    auto stage_free = [&](int i) -> bool {
      if (i < S) return true;
      const int s = i % S;
      if (!mbar_wait(&mma_done[s], (uint32_t)(((i - S) / S) & 1))) { s_flag = 1; return false; }
      return true;
    };
    auto publish = [&](int i) {
      fence_async_smem();
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&a_ready[i % S])) : "memory");
    };
    const bool cm_async = CM && (ldy1 & 3) == 0 && (((uintptr_t)Y1) & 15) == 0;
    if (cm_async) {
      const float* ycol = Y1 + (col_ok ? r : 0) * ldy1;
      const int P = S - 2;                             // blocks in flight ahead of the one converted
      auto issue = [&](int i) -> bool {
        if (!stage_free(i)) return false;
        unsigned char* Ah = A + (size_t)(i % S) * 2 * a_plane;
        const int64_t kbase = (int64_t)(kb0 + i) * kBKt;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int kc = 4 * h + c;
          const int64_t k = kbase + kc * 4;
          const int64_t left = col_ok ? m1 - k : 0;
          const uint32_t bytes = left >= 4 ? 16u : (left > 0 ? (uint32_t)left * 4u : 0u);
          cp_async16(Ah + sw128_off(m, kc), bytes ? (const void*)(ycol + k) : (const void*)Y1, bytes);
        }
        return true;
      };
      bool ok = true;
      for (int i = 0; i < P; ++i) {
        if (i < nk && ok) ok = issue(i);
        cp_async_commit();
      }
      for (int i = 0; i < nk && ok; ++i) {
        if (i + P < nk) ok = issue(i + P);
        cp_async_commit();
        if (!ok) break;
        // block i's group done: at most P younger groups pending
        if (P == 1) cp_async_wait<1>();
        else if (P == 2) cp_async_wait<2>();
        else if (P == 3) cp_async_wait<3>();
        else cp_async_wait<4>();
        if (*(volatile int*)&s_flag) break;
        unsigned char* Ah = A + (size_t)(i % S) * 2 * a_plane;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const uint32_t off = sw128_off(m, 4 * h + c);
          const float4 x = *(const float4*)(Ah + off);
          float4 hi, lo;
          tf32_split(x.x, hi.x, lo.x);
          tf32_split(x.y, hi.y, lo.y);
          tf32_split(x.z, hi.z, lo.z);
          tf32_split(x.w, hi.w, lo.w);
          *(float4*)(Ah + off) = hi;
          *(float4*)(Ah + a_plane + off) = lo;
        }
        publish(i);
      }
      cp_async_wait_all();                             // nothing of this thread in flight at exit
    } else {
      // register path: 16 values per K block, two blocks ahead
      auto load_block = [&](float (&v)[16], int kb) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int64_t k = (int64_t)kb * kBKt + (4 * h + c) * 4 + e;
            v[c * 4 + e] = (col_ok && k < m1) ? __ldcs(CM ? Y1 + r * ldy1 + k : Y1 + k * ldy1 + r) : 0.f;
          }
        }
      };
      auto convert = [&](float (&v)[16], int i) -> bool {
        if (!stage_free(i)) return false;
        if (*(volatile int*)&s_flag) return false;
        unsigned char* Ah = A + (size_t)(i % S) * 2 * a_plane;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const uint32_t off = sw128_off(m, 4 * h + c);
          float4 hi, lo;
          tf32_split(v[c * 4 + 0], hi.x, lo.x);
          tf32_split(v[c * 4 + 1], hi.y, lo.y);
          tf32_split(v[c * 4 + 2], hi.z, lo.z);
          tf32_split(v[c * 4 + 3], hi.w, lo.w);
          *(float4*)(Ah + off) = hi;
          *(float4*)(Ah + a_plane + off) = lo;
        }
        publish(i);
        return true;
      };
      float va[16], vb[16];
      if (nk > 0) load_block(va, kb0);
      if (nk > 1) load_block(vb, kb0 + 1);
      for (int i = 0; i < nk; i += 2) {
        if (!convert(va, i)) break;
        if (i + 2 < nk) load_block(va, kb0 + i + 2);
        if (i + 1 >= nk) break;
        if (!convert(vb, i + 1)) break;
        if (i + 3 < nk) load_block(vb, kb0 + i + 3);
      }
    }
  } else if (lane == 0) {
    // ---------------- producer of Omega^T planes + MMA issue ----------------
    int last_commit = -1, b_issued = 0, b_done = 0;
    for (int q = 0; q < kBSlots && q < nk; ++q) { fetch_b(kb0 + q, q); b_issued = q + 1; }
    const uint32_t idesc = idesc_tf32(NTc);
    for (int i = 0; i < nk && !*(volatile int*)&s_flag; ++i) {
      const int s = i % S, sb = i % kBSlots;
      if (!mbar_wait(&a_ready[s], (uint32_t)((i / S) & 1))) { s_flag = 1; break; }
      if (!mbar_wait(&b_full[sb], (uint32_t)((i / kBSlots) & 1))) { s_flag = 1; break; }
      b_done = i + 1;
      tc_fence_after();
      const unsigned char* As = A + (size_t)s * 2 * a_plane;
      const unsigned char* Bs = B + (size_t)sb * 2 * b_plane;
#pragma unroll
      for (int ks = 0; ks < kBKt / 8; ++ks) {
        // smallest terms first: lo*hi, hi*lo, hi*hi (planes: 0 = hi, 1 = lo)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int pa = q == 0 ? 1 : 0, pb = q == 1 ? 1 : 0;
          const int u = (ks * 3 + q) & 1;
          const uint64_t ad = sw128_desc(As + (size_t)pa * a_plane) + (uint64_t)(ks * 2);
          const uint64_t bd = sw128_desc(Bs + (size_t)pb * b_plane) + (uint64_t)(ks * 2);
          const bool first = i == 0 && ks * 3 + q < 2;
          mma_tf32(tmem + (uint32_t)(u * NTc), ad, bd, idesc, first ? 0u : 1u);
        }
      }
      mma_commit(&mma_done[s]);
      mma_commit(&b_free[sb]);
      last_commit = i;
      if (i >= 1 && i - 1 + kBSlots < nk) {
        const int so = (i - 1) % kBSlots;
        if (!mbar_wait(&b_free[so], (uint32_t)(((i - 1) / kBSlots) & 1))) { s_flag = 1; break; }
        fetch_b(kb0 + i - 1 + kBSlots, so);
        b_issued = i + kBSlots;
      }
    }
    if (last_commit >= 0 && !mbar_wait(&mma_done[last_commit % S], (uint32_t)((last_commit / S) & 1))) s_flag = 2;
    if (last_commit < nk - 1 && !s_flag) s_flag = 1;
    for (int j = b_done; j < b_issued; ++j) (void)mbar_wait(&b_full[j % kBSlots], (uint32_t)((j / kBSlots) & 1));
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (s_flag == 0 && nk > 0 && warp < 8) {
    const int lane_base = (warp & 3) * 32;
    const int64_t r = r0 + lane_base + lane;
    float* prow = part_base + r * NT + n0;
    for (int q = warp >> 2; q < NTc / 16; q += 2) {
      float vals[16], v2[16];
      tmem_ld16(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(q * 16), vals);
      tmem_ld16(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(NTc + q * 16), v2);   // 12 nk >= 2 MMAs
#pragma unroll
      for (int j = 0; j < 16; ++j) vals[j] += v2[j];
      if (r < R) {
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *(float4*)(prow + q * 16 + j) = make_float4(vals[j], vals[j + 1], vals[j + 2], vals[j + 3]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && s_flag) set_status(status, IDL_ETIMEOUT);
  if (warp == 0) tmem_dealloc(tmem, tcols);
}

}  // namespace idl
