// gaussian_tc.cu -- the Gaussian stage Y2 = Omega Y1 (Sec. 1.2.1) on the
// 5th-generation tensor cores (tcgen05, TMEM accumulators).
//
// Computed as D = Y1^T Omega^T: M = 128 columns r of Y1 per CTA, N = m2
// rounded up to 16, K = m1 (split over CTAs, partial sums reduced in a fixed
// order by gauss_reduce_kernel).  Both operands are K-major bf16 in shared
// memory with the 128-byte swizzle:
//   * A (Y1^T): every thread loads FP32 Y1 (row-major Y1: coalesced along r;
//     column-major Y1: 32 consecutive K values per thread), splits each
//     value into bf16 planes x = hi + mid + lo (each the bf16 rounding of the
//     remainder) and stores the planes already transposed into the K-major
//     swizzled layout -- the conversion and the transpose cost no extra HBM
//     traffic;
//   * B (Omega^T): the planes of Omega are built once per call in global
//     memory in exactly the shared-memory layout and fetched per K block with
//     one cp.async.bulk (TMA engine) completing on an mbarrier.
// One thread issues tcgen05.mma (kind::f16, FP32 accumulate) for every pair of
// planes the precision mode keeps:
//   BF16   : hi*hi                                (1 product,  8-bit operands)
//   BF16X3 : hi*hi + hi*lo + lo*hi   (2 planes)   (3 products, ~16-bit operands)
//   FP32   : hh + hm + mh + hl + mm + lh  (3 planes: the terms above 2^-24)
// Warp-specialised pipeline (measured: with one block-wide barrier per K block
// and the MMA issue on a converter thread, ncu showed ~25% barrier stalls and
// the tensor pipe active 16% of the time): eight converter warps and one
// MMA/producer warp hand over two stages of A planes and a 2- or 3-slot ring of
// Omega^T planes through mbarriers only.  Every mbarrier wait is bounded (1 s); on a timeout the kernel
// records IDL_ETIMEOUT, waits (bounded) for the MMAs it issued, frees TMEM
// and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "gemm_dev.cuh"
#include "gemm_tf32_dev.cuh"
#include "internal.h"

namespace idl {

template <int NP>
__global__ void omega_planes_kernel(const double* __restrict__ Om, int m2, int64_t m1, int NT, int nkb,
                                    __nv_bfloat16* __restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;     // (kb, n, kc)
  if (e < (int64_t)nkb * NT * 8) omega_planes_elem<NP>(e, Om, m2, m1, NT, out);
}

template <int NP, bool CM>
__global__ void __launch_bounds__(kTcThreads, CM ? 1 : 2)
gauss_tc_kernel(const float* __restrict__ Y1, int64_t ldy1, int64_t R, int64_t m1, const __nv_bfloat16* __restrict__ Bpl,
                int NT, int NTc, int kb_per_cta, int nkb, float* __restrict__ part, int* status, int bslots) {
  extern __shared__ unsigned char smem_raw[];
  const int kb0 = blockIdx.y * kb_per_cta;
  const int nk = min(nkb, kb0 + kb_per_cta) - kb0;
  gauss_tc_block<NP, CM>(Y1, ldy1, R, m1, Bpl, NT, NTc, kb0, nk, blockIdx.x, blockIdx.z,
                         part + (int64_t)blockIdx.y * R * NT, status, smem_raw, bslots);
}

__global__ void omega_tf32_kernel(const double* __restrict__ Om, int m2, int64_t m1, int NT, int nkb,
                                  float* __restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;     // (kb, n, kc)
  if (e < (int64_t)nkb * NT * 8) omega_tf32_elem(e, Om, m2, m1, NT, out);
}

template <bool CM>
__global__ void __launch_bounds__(kTcThreads, 1)
gauss_tf32_kernel(const float* __restrict__ Y1, int64_t ldy1, int64_t R, int64_t m1, const float* __restrict__ Bpl,
                  int NT, int NTc, int kb_per_cta, int nkb, int S, float* __restrict__ part, int* status) {
  extern __shared__ unsigned char smem_raw[];
  const int kb0 = blockIdx.y * kb_per_cta;
  const int nk = min(nkb, kb0 + kb_per_cta) - kb0;
  gauss_tf32_block<CM>(Y1, ldy1, R, m1, Bpl, NT, NTc, kb0, nk, blockIdx.x, blockIdx.z, S,
                       part + (int64_t)blockIdx.y * R * NT, status, smem_raw);
}

using namespace tc;

// Split K over CTAs so that (waves of CTAs) x (K blocks per CTA) is smallest: a CTA's
// time is proportional to its K blocks and a partly filled last wave costs a whole one;
// each split adds a partial result to write and reduce (about half a K block).
static void choose_splits(int64_t ctas_per_split, int nkb, int64_t slots, int* splits, int* kbpc) {
  *splits = 1;
  *kbpc = nkb;
  double best = 1e300;
  for (int sp = 1; sp <= std::min(nkb, 32); ++sp) {
    const int kb = (int)cdiv(nkb, sp);
    const int se = (int)cdiv(nkb, kb);
    const double cost = (double)cdiv(ctas_per_split * se, slots) * kb + 0.5 * se;
    if (cost < best - 1e-9) { best = cost; *splits = se; *kbpc = kb; }
  }
}

// TF32X3: K blocks of 32, stages as many as fit (3..6) after the Omega^T ring
static int tf32_impl(idl_ctx* ctx, const double* Omega, int64_t m2, int64_t m1, const float* Y1, int64_t R,
                     int64_t ldy1, bool y1_cm, float* Y2, int64_t ldy2) {
  const int nkb = (int)cdiv(m1, kBKt);
  const int mtiles = (int)cdiv(R, kBM);
  const int NT0 = (int)round_up(m2, 16);
  int nz = 1, NTc = NT0;
  while ((tf32_smem_bytes(3, NTc) > (size_t)ctx->smem_optin || 2 * NTc > 512) && NTc > 16) {
    ++nz;
    NTc = (int)round_up(cdiv(NT0, nz), 16);
  }
  int S = 3;
  while (S < kTf32MaxStages && tf32_smem_bytes(S + 1, NTc) <= (size_t)ctx->smem_optin) ++S;
  const size_t smem = tf32_smem_bytes(S, NTc);
  if (smem > (size_t)ctx->smem_optin) return fail(ctx, IDL_ELIMIT, "gaussian tf32: shared memory");
  const int NT = nz * NTc;
  const int per_sm = std::max(1, (int)(ctx->smem_optin / smem));
  int splits, kbpc;
  choose_splits((int64_t)mtiles * nz, nkb, (int64_t)ctx->num_sms * per_sm, &splits, &kbpc);
  float* Bpl = (float*)ws_get(ctx, kWsOmegaConv, (size_t)nkb * 2 * NT * 128);
  float* part = (float*)ws_get(ctx, kWsPart, sizeof(float) * (size_t)splits * R * NT);
  if (!Bpl || !part) return IDL_ENOMEM;
  {
    const int64_t n = (int64_t)nkb * NT * 8;
    omega_tf32_kernel<<<(unsigned)cdiv(n, 256), 256, 0, ctx->stream>>>(Omega, (int)m2, m1, NT, nkb, Bpl),
        count_launch();
  }
  auto k = y1_cm ? gauss_tf32_kernel<true> : gauss_tf32_kernel<false>;
  cudaError_t e = ensure_smem(ctx, (const void*)k, smem);
  if (e != cudaSuccess) return cuda_check(ctx, e, "gaussian tf32 attribute");
  dim3 grid((unsigned)mtiles, (unsigned)splits, (unsigned)nz);
  k<<<grid, kTcThreads, smem, ctx->stream>>>(Y1, ldy1, R, m1, Bpl, NT, NTc, kbpc, nkb, S, part, ctx->d_status),
      count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(ctx, e, "gaussian tf32");
  return launch_gaussian_reduce(ctx, part, splits, R, NT, m2, Y2, ldy2);
}

template <int NP>
static int tc_impl(idl_ctx* ctx, const double* Omega, int64_t m2, int64_t m1, const float* Y1, int64_t R, int64_t ldy1,
                   bool y1_cm, float* Y2, int64_t ldy2) {
  using namespace tc;
  const int nkb = (int)cdiv(m1, kBK);
  const int mtiles = (int)cdiv(R, kBM);
  const size_t a_plane = (size_t)kBM * kBK * 2;
  // N chunks: the widest chunk (multiple of 16, <= 256) whose stages fit in shared memory,
  // for an Omega^T ring of bs slots; two accumulators of NTc columns fit in TMEM (2 NTc <= 512)
  const int NT0 = (int)round_up(m2, 16);
  auto smem_for = [&](int bs, int ntc) {
    return 1024 + (size_t)kStages * NP * a_plane + (size_t)bs * NP * ntc * kBK * 2 + 128;
  };
  struct Plan { int bs, nz, NTc, per_sm; };
  auto plan = [&](int bs) {
    Plan q{bs, 1, NT0, 1};
    while ((smem_for(bs, q.NTc) > (size_t)ctx->smem_optin || 2 * q.NTc > 512) && q.NTc > 16) {
      ++q.nz;
      q.NTc = (int)round_up(cdiv(NT0, q.nz), 16);
    }
    q.per_sm = std::max(1, (int)(ctx->smem_optin / smem_for(bs, q.NTc)));
    return q;
  };
  // Fewer N chunks first (each chunk re-reads and re-splits Y1); then two slots for
  // row-major Y1 and three for column-major.  Measured: a two-slot ring that avoids N
  // chunks took the dense 14400 x 4096 FP32 shape 162 -> 107 us; on the sparse
  // 3600 x 10000 shape two slots beat three (BF16X3 62 vs 72 us, FP32 78 vs 82 us);
  // column-major Y1 was slower with two slots and two CTAs per SM (CP-item shape 75 -> 88 us).
  const Plan p3 = plan(kBSlots), p2 = plan(2);
  Plan pl = p3;
  if (p2.nz < p3.nz || (!y1_cm && p2.nz == p3.nz)) pl = p2;
  const int bslots = pl.bs, nz = pl.nz, NTc = pl.NTc;
  const size_t smem = smem_for(bslots, NTc);
  if (smem > (size_t)ctx->smem_optin) return fail(ctx, IDL_ELIMIT, "gaussian tc: shared memory");
  const int NT = nz * NTc;                            // plane rows (zero beyond m2)
  const size_t b_plane_full = (size_t)NT * kBK * 2;
  // split K so that (waves of CTAs) x (K blocks per CTA) is smallest: a CTA's time is
  // proportional to its K blocks, and a partly filled last wave costs a whole one;
  // each split adds a partial result to write and reduce (about half a K block)
  int splits, kbpc;
  choose_splits((int64_t)mtiles * nz, nkb, (int64_t)ctx->num_sms * pl.per_sm, &splits, &kbpc);
  __nv_bfloat16* Bpl = (__nv_bfloat16*)ws_get(ctx, kWsOmegaConv, (size_t)nkb * NP * b_plane_full);
  float* part = (float*)ws_get(ctx, kWsPart, sizeof(float) * (size_t)splits * R * NT);
  if (!Bpl || !part) return IDL_ENOMEM;
  {
    const int64_t n = (int64_t)nkb * NT * 8;
    omega_planes_kernel<NP><<<(unsigned)cdiv(n, 256), 256, 0, ctx->stream>>>(Omega, (int)m2, m1, NT, nkb, Bpl),
        count_launch();
  }
  auto k = y1_cm ? gauss_tc_kernel<NP, true> : gauss_tc_kernel<NP, false>;
  cudaError_t e = ensure_smem(ctx, (const void*)k, smem);
  if (e != cudaSuccess) return cuda_check(ctx, e, "gaussian tc attribute");
  dim3 grid((unsigned)mtiles, (unsigned)splits, (unsigned)nz);
  k<<<grid, kTcThreads, smem, ctx->stream>>>(Y1, ldy1, R, m1, Bpl, NT, NTc, kbpc, nkb, part, ctx->d_status, bslots),
      count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(ctx, e, "gaussian tc");
  return launch_gaussian_reduce(ctx, part, splits, R, NT, m2, Y2, ldy2);
}

int launch_gaussian_tc(idl_ctx* ctx, const double* Omega, int64_t m2, int64_t m1, const float* Y1, int64_t R,
                       int64_t ldy1, bool y1_cm, int precision, float* Y2, int64_t ldy2) {
  if (m2 > 256) return fail(ctx, IDL_ELIMIT, "gaussian tc: m2 > 256");
  switch (precision) {
    case IDL_PREC_BF16: return tc_impl<1>(ctx, Omega, m2, m1, Y1, R, ldy1, y1_cm, Y2, ldy2);
    case IDL_PREC_BF16X3: return tc_impl<2>(ctx, Omega, m2, m1, Y1, R, ldy1, y1_cm, Y2, ldy2);
    case IDL_PREC_TF32X3: return tf32_impl(ctx, Omega, m2, m1, Y1, R, ldy1, y1_cm, Y2, ldy2);
    default: return tc_impl<3>(ctx, Omega, m2, m1, Y1, R, ldy1, y1_cm, Y2, ldy2);
  }
}

}  // namespace idl

// ---------------------------------------------------------------------------
// Failure detection without a fault: one warp waits, through the same bounded
// mbarrier wait as the Gaussian stage, for a phase that completes only when the
// caller asks for the arrival (arrive != 0).  Without it the wait gives up after
// limit_ns and the kernel records IDL_ETIMEOUT in the status word and returns.
// ---------------------------------------------------------------------------
namespace idl {

__global__ void wait_probe_kernel(int arrive, uint64_t limit_ns, int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_barrier_init();
  }
  __syncwarp();
  if (threadIdx.x == 0 && arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&bar)) : "memory");
  __syncwarp();
  const bool done = tc::mbar_wait(&bar, 0, limit_ns);
  if (!done && threadIdx.x == 0) set_status(status, IDL_ETIMEOUT);
}

}  // namespace idl

// Test hook (not in the public header): runs the wait probe on the context's stream.
extern "C" int idl_debug_wait_probe(idl_ctx* ctx, int arrive, unsigned long long limit_ns) {
  using namespace idl;
  const int rc = ctx_usable(ctx);
  if (rc != IDL_OK) return rc;
  if (limit_ns < 1000ull || limit_ns > tc::kTimeoutNs) return fail(ctx, IDL_EINVAL, "wait probe: limit in [1 us, 1 s]");
  wait_probe_kernel<<<1, 32, 0, ctx->stream>>>(arrive, (uint64_t)limit_ns, ctx->d_status), count_launch();
  return cuda_check(ctx, cudaGetLastError(), "wait probe");
}
