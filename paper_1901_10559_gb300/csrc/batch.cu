// batch.cu -- many IDs of uneven sizes in one pass: every stage of the hot path
// is one launch over all items (dense matrices for Algorithm 2, CP tensors for
// Algorithm 3), and the pivoted QR runs one thread-block cluster per item in a
// single launch.
//
// Every block finds its item by a binary search over a per-stage prefix table
// of block counts, then runs the same device body as the single-problem kernel
// (sketch_dev.cuh, draws_dev.cuh, tsketch_dev.cuh, gemm_dev.cuh, cpqr_dev.cuh,
// tsolve_dev.cuh).  The item descriptors and the prefix tables live in device
// memory, so the launch sequence of a batch shape is captured once into a CUDA
// graph and replayed; descriptors are re-uploaded before each replay.
//
// Column proposal (idl_params.learned): items that ask for it get the
// proposal stages (features, MLP or norm scores, selection, one-CTA candidate
// QR, certificate) before the cluster QR launch, in which their clusters only
// run when the certificate failed (a per-item gate read at block start).
//
// Tuning: the dense sketch's block width, the Gaussian stage's split-K factor
// and the thread-block cluster sizes of the dense and the CP items' pivoted QR
// are chosen per batch shape by timing the candidates on the first call (CUDA
// events around the stage groups, one knob at a time); the choice is kept in
// the context and can be saved to / loaded from a text file (idl_tune_save /
// idl_tune_load).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <array>
#include <initializer_list>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "cpqr_dev.cuh"
#include "draws_dev.cuh"
#include "gemm_dev.cuh"
#include "gemm_tf32_dev.cuh"
#include "internal.h"
#include "proposal_dev.cuh"
#include "sketch_dev.cuh"
#include "tsketch_dev.cuh"
#include "tsketch8k_dev.cuh"
#include "tsolve_dev.cuh"

namespace idl {

using namespace tc;

constexpr int kNPTf32 = 4;      // BatchPlan::NP of the TF32X3 mode (two TF32 planes)

// ---------------------------------------------------------------------------
// device descriptor of one item
// ---------------------------------------------------------------------------
struct BItem {
  int kind, N, modified, K, vec;
  int pt;                         // CP, L = 8192: Y1 holds the pre-tiled bf16 planes (gauss_tc_block_pretiled)
  int64_t I, R, lda, m1, m2, ldy1, nkb, NT, mtiles, splits, kbpc, ntiles, mode_tot;
  const float* A;
  TsArgs ts;                      // CP: factors (column-contiguous), mode maps, dims
  uint64_t mode_hb[kTsMaxModes], mode_sb[kTsMaxModes];
  const double* lam;
  CsDrawArgs cs;
  uint64_t gauss_base;
  int32_t *h, *ptr, *rows, *cursor, *big, *nbig, *mh;
  int8_t *s, *ms;
  double* Om;
  __nv_bfloat16* Bpl;
  float *Y1, *part, *Y2;
  int32_t* rest;
  double *Rinv, *diag;
  int32_t* J;
  double* T;
  double* lam_hat;
  int nc;
  // column proposal
  int learned, C, nsplit;
  float* Yf;                       // factored sketch (== Y2 without a proposal)
  float *Gp, *nmaxp, *scal, *Linv, *G, *F, *sc, *V, *beta;
  int32_t *cand, *outl;
  double* rn;
  int* flag;                       // certificate failed
  const int* gate;                 // == flag for proposal items, nullptr otherwise
};

// stages with a flattened block list (prefix tables, one per stage)
enum BStage { kBDraw = 0, kBGauss, kBHist, kBScan, kBScatter, kBSortW, kBSortB, kBSketchD, kBSketchT, kBSketchT8,
              kBPlanes,
              kBGemm, kBReduce, kBPGram, kBPGRed, kBPChol, kBPFeat, kBPMlp, kBPNorm, kBPSel, kBPApply, kBRest, kBRinv,
              kBTgemm, kBLam, kBNumStages };

// stage groups timed by idl_debug_batch_timing
enum BTimed { kBTDrawBuckets = 0, kBTSketchCP, kBTSketchDense, kBTGauss, kBTProposal, kBTQR, kBTSolve, kBTimedStages };

__device__ __forceinline__ int find_item(const int64_t* __restrict__ pre, int n, int64_t blk) {
  int lo = 0, hi = n - 1;                          // largest p with pre[p] <= blk
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= blk) lo = mid; else hi = mid - 1;
  }
  return lo;
}

#define ITEM_OF_BLOCK(pre, n)                         \
  const int p = find_item(pre, n, (int64_t)blockIdx.x); \
  const BItem& it = items[p];                         \
  const int64_t local = (int64_t)blockIdx.x - pre[p]

__global__ void b_draw_kernel(const BItem* __restrict__ items, const int64_t* __restrict__ pre, int n, int* status) {
  ITEM_OF_BLOCK(pre, n);
  const int64_t i = local * blockDim.x + threadIdx.x;
  if (it.kind == IDL_ITEM_DENSE) {
    if (i < it.I) cs_draw_elem(i, it.cs, it.I, it.m1, it.modified, it.h, it.s, status);
  } else if (i < it.mode_tot) {
    int64_t off = 0;
    for (int q = 0; q < it.N; ++q) {
      const int64_t d = it.ts.dims[q];
      if (i < off + d) { mode_elem(i - off, it.mode_hb[q], it.mode_sb[q], it.m1, it.mh + off, it.ms + off); break; }
      off += d;
    }
  }
}

__global__ void b_gauss_draw_kernel(const BItem* __restrict__ items, const int64_t* __restrict__ pre, int n) {
  ITEM_OF_BLOCK(pre, n);
  const int64_t q = local * blockDim.x + threadIdx.x;
  const int64_t tot = it.m2 * it.m1;
  if (2 * q < tot) gauss_pair_f32(q, it.gauss_base, tot, it.Om);     // batches hold FP32 data
}

constexpr int kBHistBlocks = 64;

__global__ void b_hist_kernel(const BItem* __restrict__ items, const int64_t* __restrict__ pre, int n, int* status) {
  extern __shared__ int32_t sh[];
  ITEM_OF_BLOCK(pre, n);
  const int64_t nb = pre[p + 1] - pre[p];
  bucket_hist_body(it.h, it.I, it.m1, it.cursor, status, local, nb, sh);
}

__global__ void b_scan_kernel(const BItem* __restrict__ items, const int64_t* __restrict__ pre, int n) {
  ITEM_OF_BLOCK(pre, n);
  (void)local;
  bucket_scan_body(it.cursor, it.m1, it.ptr, it.cursor);
}

__global__ void b_scatter_kernel(const BItem* __restrict__ items, const int64_t* __restrict__ pre, int n) {
  ITEM_OF_BLOCK(pre, n);
  const int64_t i = local * blockDim.x + threadIdx.x;
  if (i < it.I) bucket_scatter_elem(i, it.h, it.m1, it.cursor, it.rows);
}

__global__ void b_sortw_kernel(const BItem* __restrict__ items, const int64_t* __restrict__ pre, int n) {
  extern __shared__ int32_t sh[];
  ITEM_OF_BLOCK(pre, n);
  const int wid = threadIdx.x >> 5;
  const int64_t b = local * (blockDim.x >> 5) + wid;
  if (b < it.m1) bucket_sort_warp_body(it.ptr, b, it.rows, it.big, it.nbig, sh + wid * kWarpSortCap);
}

constexpr int kBSortBlocks = 4;

__global__ void b_sortb_kernel(const BItem* __restrict__ items, const int64_t* __restrict__ pre, int n) {
  extern __shared__ int32_t seg[];
  ITEM_OF_BLOCK(pre, n);
  const int count = *it.nbig;
  for (int q = (int)local; q < count; q += kBSortBlocks)
    bucket_sort_block_body(it.ptr, it.big[q], it.rows, seg, it.h, it.I);
}

// blk0: first block of this launch in the stage's flattened block list (a launch may
// cover only the items whose matrices have arrived)
// At most 32 registers (2048 resident threads per SM): the kernel waits on the
// latency of its few rows per bucket, and full occupancy measured 14 % faster than
// the 40 registers it takes unbounded (small spills included).
__global__ void __launch_bounds__(512, 4) b_sketch_dense_kernel(const BItem* __restrict__ items,
                                                             const int64_t* __restrict__ pre, int n, int64_t blk0) {
  const int64_t gblk = (int64_t)blockIdx.x + blk0;
  const int p = find_item(pre, n, gblk);
  const BItem& it = items[p];
  const int64_t local = gblk - pre[p];
  const int64_t b = local / it.ntiles;
  const int tile = (int)(local % it.ntiles);
  if (it.vec)
    cs_dense_block<float, true>(it.A, it.lda, it.R, it.s, it.ptr, it.rows, it.Y1, it.ldy1, b, tile);
  else
    cs_dense_block<float, false>(it.A, it.lda, it.R, it.s, it.ptr, it.rows, it.Y1, it.ldy1, b, tile);
}

__global__ void __launch_bounds__(kTsMaxThreads, 1) b_sketch_cp_kernel(const BItem* __restrict__ items,
                                                                    const int64_t* __restrict__ pre, int n,
                                                                    const float2* __restrict__ tw) {
  extern __shared__ __align__(16) float2 sm2[];
  ITEM_OF_BLOCK(pre, n);
  int logL = 0;
  while ((1LL << logL) < it.m1) ++logL;
  // column-major: column r at Y1 + r * m1 (the Gaussian stage reads each column's K values contiguously)
  tensorsketch_block(it.ts, it.R, (int)it.m1, logL, it.lam, it.Y1, it.m1, true, local * 2, tw, sm2);
}

// CP items with L = 8192: persistent blocks (one per SM) over the column pairs of all
// such items; pre counts pairs, not blocks
// PT = 0: Y1 column-major FP32 (column r at Y1 + r m1); PT = 1..3: Y1 holds the
// Gaussian stage's PT bf16 operand planes, pre-tiled (pretiled_store_pair), so that stage
// fetches them with bulk copies and converts nothing
template <int PT>
__global__ void __launch_bounds__(ts8::kT, 1) b_sketch_cp8k_kernel(const BItem* __restrict__ items,
                                                                   const int64_t* __restrict__ pre, int n,
                                                                   const float2* __restrict__ tab) {
  extern __shared__ __align__(16) float2 sm8[];
  float2 *z, *tw1, *tw2;
  ts8::block_setup(sm8, tab, &z, &tw1, &tw2);
  const int64_t total = pre[n];
  ts8::Pre pf;
  for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
    const int p = find_item(pre, n, g);
    const BItem& it = items[p];
    const int64_t r0 = 2 * (g - pre[p]);
    const bool two = r0 + 1 < it.R;
    ts8::load_mode(it.ts, 0, r0, two, pf);
    if constexpr (PT == 0) {
      ts8::pair_body(it.ts, it.R, r0, it.lam, it.Y1, it.m1, true, pf, z, tw1, tw2);
    } else {
      float2 v[16];
      float s0, s1;
      ts8::pair_core(it.ts, it.R, r0, it.lam, pf, z, tw1, tw2, v, s0, s1);
      pretiled_store_pair<PT, ts8::kT, 16>(reinterpret_cast<unsigned char*>(it.Y1), it.nkb, r0, v, s0, s1);
      __syncthreads();              // every place of z is clear before the next pair's scatter
    }
  }
}

template <int NP>
__global__ void b_planes_kernel(const BItem* __restrict__ items, const int64_t* __restrict__ pre, int n) {
  ITEM_OF_BLOCK(pre, n);
  const int64_t e = local * blockDim.x + threadIdx.x;
  if (e < it.nkb * it.NT * 8) omega_planes_elem<NP>(e, it.Om, (int)it.m2, it.m1, (int)it.NT, it.Bpl);
}

// S: stages of the A ring of the pre-tiled items
template <int NP>
__global__ void __launch_bounds__(kTcThreads, 1) b_gemm_kernel(const BItem* __restrict__ items,
                                                               const int64_t* __restrict__ pre, int n, int* status,
                                                               int S) {
  extern __shared__ unsigned char smem_raw[];
  ITEM_OF_BLOCK(pre, n);
  const int64_t mt = local / it.splits;
  const int sp = (int)(local % it.splits);
  const int kb0 = sp * (int)it.kbpc;
  const int nk = (int)std::min<int64_t>(it.nkb, kb0 + it.kbpc) - kb0;
  // an item not split in K writes Y2 itself (no partial sums, no reduction launch)
  float* out = it.splits == 1 ? it.Y2 : it.part + (int64_t)sp * it.R * it.NT;
  const int64_t ldo = it.splits == 1 ? it.m2 : 0;
  if (it.pt)
    gauss_tc_block_pretiled<NP>(reinterpret_cast<const unsigned char*>(it.Y1), it.nkb, it.R, it.Bpl, (int)it.NT,
                                (int)it.NT, kb0, nk, mt, 0, S, out, status, smem_raw, ldo, (int)it.m2);
  else if (it.kind == IDL_ITEM_CP)
    gauss_tc_block<NP, true>(it.Y1, it.m1, it.R, it.m1, it.Bpl, (int)it.NT, (int)it.NT, kb0, nk, mt, 0, out, status,
                             smem_raw, kBSlots, ldo, (int)it.m2);
  else
    gauss_tc_block<NP, false>(it.Y1, it.ldy1, it.R, it.m1, it.Bpl, (int)it.NT, (int)it.NT, kb0, nk, mt, 0, out,
                              status, smem_raw, kBSlots, ldo, (int)it.m2);
}

__global__ void b_planes_tf32_kernel(const BItem* __restrict__ items, const int64_t* __restrict__ pre, int n) {
  ITEM_OF_BLOCK(pre, n);
  const int64_t e = local * blockDim.x + threadIdx.x;
  if (e < it.nkb * it.NT * 8) omega_tf32_elem(e, it.Om, (int)it.m2, it.m1, (int)it.NT, (float*)it.Bpl);
}

__global__ void __launch_bounds__(kTcThreads, 1) b_gemm_tf32_kernel(const BItem* __restrict__ items,
                                                                    const int64_t* __restrict__ pre, int n,
                                                                    int* status, int S) {
  extern __shared__ unsigned char smem_raw[];
  ITEM_OF_BLOCK(pre, n);
  const int64_t mt = local / it.splits;
  const int sp = (int)(local % it.splits);
  const int kb0 = sp * (int)it.kbpc;
  const int nk = (int)std::min<int64_t>(it.nkb, kb0 + it.kbpc) - kb0;
  if (it.kind == IDL_ITEM_CP)
    gauss_tf32_block<true>(it.Y1, it.m1, it.R, it.m1, (const float*)it.Bpl, (int)it.NT, (int)it.NT, kb0, nk, mt, 0, S,
                           it.part + (int64_t)sp * it.R * it.NT, status, smem_raw);
  else
    gauss_tf32_block<false>(it.Y1, it.ldy1, it.R, it.m1, (const float*)it.Bpl, (int)it.NT, (int)it.NT, kb0, nk, mt,
                            0, S, it.part + (int64_t)sp * it.R * it.NT, status, smem_raw);
}

__global__ void b_reduce_kernel(const BItem* __restrict__ items, const int64_t* __restrict__ pre, int n) {
  ITEM_OF_BLOCK(pre, n);
  const int64_t e = local * blockDim.x + threadIdx.x;
  if (e >= it.R * it.m2) return;
  const int64_t r = e / it.m2;
  const int64_t j = e - r * it.m2;
  float acc = 0.f;
  for (int q = 0; q < it.splits; ++q) acc += it.part[(int64_t)q * it.R * it.NT + r * it.NT + j];
  it.Y2[r * it.m2 + j] = acc;
}

template <int V, int TPC>
__global__ void __launch_bounds__(RegCpqr<float, V, TPC>::kMaxThreads, 1)
b_cpqr_kernel(const BItem* __restrict__ items, const int32_t* __restrict__ list, int CS, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BItem& it = items[list[blockIdx.x / CS]];
  if (proposal_certified(it.gate, it.diag)) return;     // the whole cluster belongs to this item
  cpqr_reg_body<float, V, TPC>(it.Y2, it.Yf, (int)it.m2, (int)it.R, (int)it.m2, it.K, it.nc, it.J, nullptr, it.diag,
                               status, smem_raw);
}

// ---- column proposal stages ----
__global__ void __launch_bounds__(prop::kThreads) b_pgram_kernel(const BItem* __restrict__ items,
                                                                 const int64_t* __restrict__ pre, int n) {
  extern __shared__ __align__(16) float smf[];
  ITEM_OF_BLOCK(pre, n);
  prop::gram_partial_block(it.Y2, (int)it.m2, (int)it.m2, (int)it.R, (int)local, it.Gp, it.nmaxp, smf);
}

__global__ void __launch_bounds__(prop::kThreads) b_pgred_kernel(const BItem* __restrict__ items,
                                                                 const int64_t* __restrict__ pre, int n) {
  ITEM_OF_BLOCK(pre, n);
  prop::gram_reduce_elem(it.Gp, it.nsplit, it.nmaxp, (int)it.m2, (int)(local * blockDim.x + threadIdx.x), it.G,
                         it.scal);
}

__global__ void __launch_bounds__(prop::kThreads) b_pchol_kernel(const BItem* __restrict__ items,
                                                                 const int64_t* __restrict__ pre, int n) {
  extern __shared__ __align__(16) float smf[];
  ITEM_OF_BLOCK(pre, n);
  prop::chol_inv_block(it.G, (int)it.m2, (int)local, it.Linv, it.scal, smf);
}

__global__ void __launch_bounds__(prop::kThreads) b_pfeat_kernel(const BItem* __restrict__ items,
                                                                 const int64_t* __restrict__ pre, int n) {
  extern __shared__ __align__(16) float smf[];
  ITEM_OF_BLOCK(pre, n);
  prop::features_block(it.Y2, (int)it.m2, (int)it.m2, (int)it.R, it.K, it.Linv, it.scal, (int)local, it.F, smf);
}

__global__ void __launch_bounds__(prop::kThreads, 1) b_pmlp_kernel(const BItem* __restrict__ items,
                                                                   const int64_t* __restrict__ pre, int n,
                                                                   const float* __restrict__ theta) {
  extern __shared__ __align__(16) float smf[];
  ITEM_OF_BLOCK(pre, n);
  prop::mlp_forward_tile(theta, it.F, it.R, local * prop::kTile, it.sc, smf);
}

__global__ void __launch_bounds__(prop::kThreads) b_pnorm_kernel(const BItem* __restrict__ items,
                                                                 const int64_t* __restrict__ pre, int n) {
  ITEM_OF_BLOCK(pre, n);
  const int64_t c = local * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c < it.R) prop::norm_scores_warp(it.Y2, (int)it.m2, (int)it.m2, (int)c, it.sc);
}

__global__ void __launch_bounds__(prop::kSelThreads) b_psel_kernel(const BItem* __restrict__ items,
                                                                   const int64_t* __restrict__ pre, int n) {
  ITEM_OF_BLOCK(pre, n);
  (void)local;
  prop::select_block(it.sc, (int)it.R, it.C, it.cand, it.outl);
}

__global__ void __launch_bounds__(prop::kApplyThreads) b_papply_kernel(const BItem* __restrict__ items,
                                                                       const int64_t* __restrict__ pre, int n) {
  extern __shared__ __align__(16) float smf[];
  ITEM_OF_BLOCK(pre, n);
  prop::apply_cert_block(it.Y2, it.Yf, (int)it.m2, (int)it.m2, it.K, it.outl, (int)(it.R - it.C), it.V, it.beta,
                         it.rn, it.flag, it.diag + 8, (int)local, (int)(pre[p + 1] - pre[p]), smf);
}

// candidate QR: one CTA per proposal item
template <int V, int TPC>
__global__ void __launch_bounds__(CtaCpqr<float, V, TPC>::kMaxThreads, 1)
b_cand_kernel(const BItem* __restrict__ items, const int32_t* __restrict__ list, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BItem& it = items[list[blockIdx.x]];
  cpqr_cta_body<float, V, TPC>(it.Y2, it.Yf, (int)it.m2, it.C, (int)it.m2, it.K, it.J, it.rn, it.diag + 8, status,
                               smem_raw, it.cand, it.V, it.beta);
}

__global__ void b_rest_kernel(const BItem* __restrict__ items, const int64_t* __restrict__ pre, int n) {
  extern __shared__ int32_t sJ[];
  ITEM_OF_BLOCK(pre, n);
  for (int q = threadIdx.x; q < it.K; q += blockDim.x) sJ[q] = it.J[q];
  __syncthreads();
  const int64_t r = local * blockDim.x + threadIdx.x;
  if (r < it.R) rest_elem((int)r, sJ, it.K, (int)it.R, it.rest);
}

__global__ void __launch_bounds__(32 * kRinvWarpsDf) b_rinv_kernel(const BItem* __restrict__ items, const int64_t* __restrict__ pre,
                                                     int n) {
  extern __shared__ __align__(16) double shU[];
  ITEM_OF_BLOCK(pre, n);
  rinv_block_df(it.Yf, (int)it.m2, it.K, (int)it.R, it.J, (float*)(it.Rinv + it.K * it.K), (int)local,
                (int)(pre[p + 1] - pre[p]), (float*)shU);
}

__global__ void __launch_bounds__(256) b_tgemm_kernel(const BItem* __restrict__ items, const int64_t* __restrict__ pre,
                                                      int n) {
  extern __shared__ __align__(16) float shf[];
  ITEM_OF_BLOCK(pre, n);
  tgemm_block_df(it.Yf, (int)it.m2, it.K, (int)it.R, (const float*)(it.Rinv + it.K * it.K), it.rest, (int)(it.R - it.K),
                 it.T, (int)local, shf);
}

__global__ void b_lam_kernel(const BItem* __restrict__ items, const int64_t* __restrict__ pre, int n) {
  ITEM_OF_BLOCK(pre, n);
  lambda_hat_block(it.lam, it.J, it.T, (int)(it.R - it.K), it.K, it.lam_hat, (int)local);
}

}  // namespace idl

// ===========================================================================
// host side
// ===========================================================================
using namespace idl;

namespace {

// Tuned per batch shape: the dense sketch's block width, the Gaussian stage's split-K
// factor, and the thread-block cluster size of the pivoted QR of dense and of CP items.
// split_mult >= 1: each item's K splits fill split_mult x the SMs by that item alone;
// 0: K is split only as far as the whole batch needs to give kBatchWaves waves of CTAs
// qr_cap_*: threads per QR CTA at most where an item's shape allows it (fewer lanes per
// column, more clusters on the GPU at once)
struct Tune {
  int sketch_threads = 256; int split_mult = 1; int qr_cs_dense = 16; int qr_cs_cp = 16;
  int qr_cap_dense = 1024, qr_cap_cp = 1024;
};
constexpr int kBatchWaves = 8, kMinKbPerCta = 8;

// a batch shape: the sizes that decide every launch
std::string signature(const idl_batch_item* items, int n) {
  std::string s;
  char buf[160];
  for (int i = 0; i < n; ++i) {
    const idl_batch_item& x = items[i];
    snprintf(buf, sizeof(buf), "%d:%lld:%lld:%lld:%lld:%lld:%d:%d:%d;", x.kind, (long long)x.I, (long long)x.R,
             (long long)x.K, (long long)x.params.m1, (long long)x.params.m2, x.params.precision, x.N,
             x.params.learned * 16 + x.params.cand_factor);
    s += buf;
    for (int q = 0; q < x.N && x.kind == IDL_ITEM_CP; ++q) {
      snprintf(buf, sizeof(buf), "%lld,", (long long)x.dims[q]);
      s += buf;
    }
  }
  return s;
}

uint64_t fnv1a(const std::string& s) {
  uint64_t h = 1469598103934665603ull;
  for (unsigned char c : s) { h ^= c; h *= 1099511628211ull; }
  return h;
}

struct CpqrCfg { int V = 0, TPC = 0, CS = 16, threads = 0; size_t smem = 0; };
// one QR launch: the items at [off, off + count) of the device list array, one shape
struct QrClass { CpqrCfg cfg; int off = 0, count = 0, maxK = 0; };
constexpr int kQrSide = 15;         // side streams the QR classes are spread over

}  // namespace

// context-side batch state
struct idl_batch_state {
  std::map<uint64_t, Tune> tune;
  uint64_t graph_sig = 0;
  cudaGraphExec_t graph = nullptr;
  int graph_launches = 0;
  cudaStream_t gstream = nullptr;    // private stream: capture and replay (the legacy stream cannot be captured)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  const int* d_flags = nullptr;      // certificate flags of the last batch (n ints, device)
  int nflags = 0;
  std::vector<std::pair<const int*, int>> flag_sets;   // host-array batches: one per item group
  unsigned char* pin = nullptr;      // pinned staging of the item groups' tables (host-array batches)
  size_t pin_bytes = 0;
  cudaStream_t cstream = nullptr;    // host-staged batches: the copies run here
  std::vector<cudaEvent_t> cev;      // their events (reused)
  cudaStream_t qs[kQrSide] = {};     // QR classes: side streams, forked from and joined to ctx->stream
  cudaEvent_t qfork = nullptr, qjoin[kQrSide] = {};
};

extern "C" long long idl_launch_count(void);

static idl_batch_state* bstate(idl_ctx* ctx) {
  if (!ctx->batch) ctx->batch = new idl_batch_state();
  return ctx->batch;
}

void idl_batch_state_free(idl_batch_state* b) {
  if (!b) return;
  if (b->pin) cudaFreeHost(b->pin);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->gstream) cudaStreamDestroy(b->gstream);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->cstream) { cudaStreamSynchronize(b->cstream); cudaStreamDestroy(b->cstream); }
  for (cudaEvent_t e : b->cev) cudaEventDestroy(e);
  for (int k = 0; k < kQrSide; ++k) {
    if (b->qs[k]) { cudaStreamSynchronize(b->qs[k]); cudaStreamDestroy(b->qs[k]); }
    if (b->qjoin[k]) cudaEventDestroy(b->qjoin[k]);
  }
  if (b->qfork) cudaEventDestroy(b->qfork);
  delete b;
}

#define BTRY(x)                     \
  do {                              \
    int _rc = (x);                  \
    if (_rc != IDL_OK) return _rc;  \
  } while (0)

#define TRYC(expr, where)                                   \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) return cuda_check(ctx, _e, where); \
  } while (0)

static int launch_check(idl_ctx* ctx, const char* where) { return cuda_check(ctx, cudaGetLastError(), where); }

template <int V, int TPC>
static bool cpqr_cfg_fits(const std::vector<int>& list, const std::vector<BItem>& it, int CS, CpqrCfg* cfg,
                          bool cand = false, int cap = 1 << 30) {
  int threads = 0, maxm = 0;
  for (int p : list) {
    const BItem& x = it[p];
    if (cdiv(x.m2, TPC) > V) return false;
    const int nc = cand ? x.C : (int)cdiv(x.R, CS);
    threads = std::max(threads, (int)round_up((int64_t)nc * TPC, 32));
    maxm = std::max(maxm, (int)x.m2);
  }
  const int maxt = cand ? CtaCpqr<float, V, TPC>::kMaxThreads : RegCpqr<float, V, TPC>::kMaxThreads;
  if (threads > maxt || threads > cap || threads < 32) return false;
  cfg->V = V;
  cfg->TPC = TPC;
  cfg->CS = CS;
  cfg->threads = threads;
  cfg->smem = reg_cpqr_smem<float, V, TPC>(maxm);
  return true;
}

static bool pick_cpqr(const std::vector<int>& list, const std::vector<BItem>& it, CpqrCfg* cfg, bool cand = false,
                      int cluster = 16, int cap = 1 << 30) {
  const int CS = cand ? 1 : cluster;
#define PICK(VV, TT) if (cpqr_cfg_fits<VV, TT>(list, it, CS, cfg, cand, cap)) return true;
  PICK(8, 32) PICK(8, 16) PICK(8, 8) PICK(16, 8) PICK(8, 4) PICK(16, 4) PICK(32, 4) PICK(16, 2) PICK(32, 2)
  PICK(16, 1) PICK(32, 1) PICK(64, 4) PICK(64, 2) PICK(64, 1) PICK(96, 1) PICK(128, 1)
#undef PICK
  return false;
}

// The QR launches of one list (device list array offset base): items grouped by the
// kernel shape each picks by itself (cluster size cs, at most cap threads per CTA where
// a shape fits under it) -- values per lane V, lanes per column TPC, cluster size,
// threads rounded up to a power of two -- larger CTAs first; the list is reordered
// class by class.  An item's factorization depends only on its own V and TPC, so it
// gets the same bits in every batch of the same tuning that contains it; and small
// items no longer take the CTA size of the largest, so more clusters fit at once.
static bool qr_classes(std::vector<int32_t>& list, std::vector<BItem>& it, int cs, int cap, int base,
                       std::vector<QrClass>& out) {
  std::map<std::array<int, 4>, std::pair<CpqrCfg, std::vector<int32_t>>> cls;
  for (int32_t p : list) {
    CpqrCfg c;
    const std::vector<int> one{p};
    if (!pick_cpqr(one, it, &c, false, cs, cap) && !pick_cpqr(one, it, &c, false, cs) &&
        !pick_cpqr(one, it, &c, false, 16, cap) && !pick_cpqr(one, it, &c, false, 16))
      return false;
    int tb = 32;
    while (tb < c.threads) tb *= 2;
    auto& e = cls[{-tb, c.V, c.TPC, c.CS}];
    if (e.second.empty()) {
      e.first = c;
    } else {
      e.first.threads = std::max(e.first.threads, c.threads);
      e.first.smem = std::max(e.first.smem, c.smem);
    }
    e.second.push_back(p);
  }
  list.clear();
  for (auto& kv : cls) {
    QrClass q;
    q.cfg = kv.second.first;
    q.off = base + (int)list.size();
    q.count = (int)kv.second.second.size();
    for (int32_t p : kv.second.second) {
      list.push_back(p);
      it[p].nc = (int)cdiv(it[p].R, q.cfg.CS);
      q.maxK = std::max(q.maxK, it[p].K);
    }
    out.push_back(q);
  }
  return true;
}

template <int V, int TPC>
static int launch_b_cpqr(idl_ctx* ctx, const BItem* d_items, const int32_t* d_list, int nlist, const CpqrCfg& c,
                         cudaStream_t stream) {
  auto kern = b_cpqr_kernel<V, TPC>;
  cudaError_t e = ensure_cluster_nonportable(ctx, (const void*)kern);
  if (e == cudaSuccess) e = ensure_smem(ctx, (const void*)kern, c.smem);
  if (e != cudaSuccess) return cuda_check(ctx, e, "batch cpqr attribute");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nlist * c.CS));
  cfg.blockDim = dim3((unsigned)c.threads);
  cfg.dynamicSmemBytes = c.smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = c.CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, d_items, d_list, c.CS, ctx->d_status);
  count_launch();
  return cuda_check(ctx, e, "batch cpqr");
}

template <int V, int TPC>
static int launch_b_cand(idl_ctx* ctx, const BItem* d_items, const int32_t* d_list, int nlist, const CpqrCfg& c) {
  (void)c.smem;
  b_cand_kernel<V, TPC><<<(unsigned)nlist, (unsigned)c.threads, cta_cpqr_smem<float, V, TPC>(), ctx->stream>>>(
      d_items, d_list, ctx->d_status);
  count_launch();
  return cuda_check(ctx, cudaGetLastError(), "batch candidate QR");
}

static int dispatch_b_cand(idl_ctx* ctx, const BItem* d_items, const int32_t* d_list, int nlist, const CpqrCfg& c) {
#define CASE(VV, TT) if (c.V == VV && c.TPC == TT) return launch_b_cand<VV, TT>(ctx, d_items, d_list, nlist, c);
  CASE(8, 32) CASE(8, 16) CASE(8, 8) CASE(16, 8) CASE(8, 4) CASE(16, 4) CASE(32, 4) CASE(16, 2) CASE(32, 2)
  CASE(16, 1) CASE(32, 1) CASE(64, 4) CASE(64, 2) CASE(64, 1) CASE(96, 1) CASE(128, 1)
#undef CASE
  return fail(ctx, IDL_ELIMIT, "batch candidate QR: no configuration");
}

static int dispatch_b_cpqr(idl_ctx* ctx, const BItem* d_items, const int32_t* d_list, int nlist, const CpqrCfg& c,
                           cudaStream_t stream) {
#define CASE(VV, TT) \
  if (c.V == VV && c.TPC == TT) return launch_b_cpqr<VV, TT>(ctx, d_items, d_list, nlist, c, stream);
  CASE(8, 32) CASE(8, 16) CASE(8, 8) CASE(16, 8) CASE(8, 4) CASE(16, 4) CASE(32, 4) CASE(16, 2) CASE(32, 2)
  CASE(16, 1) CASE(32, 1) CASE(64, 4) CASE(64, 2) CASE(64, 1) CASE(96, 1) CASE(128, 1)
#undef CASE
  return fail(ctx, IDL_ELIMIT, "batch cpqr: no configuration");
}

// Everything a batch needs on the host side, computed from the items.
struct BatchPlan {
  std::vector<BItem> it;
  std::vector<int64_t> pre[kBNumStages];
  std::vector<int32_t> dense_list, cp_list, prop_list;
  CpqrCfg cfg_cand;
  std::vector<QrClass> qr;         // QR launches: the dense list's classes, then the CP list's
  int NP = 3;
  bool any_pt = false;             // some item's Y1 is pre-tiled
  int64_t kbmax = 0;               // split_mult 0: K blocks per Gaussian-stage CTA at most
  int maxL_hist = 0, maxK = 0, maxNT = 0, maxL_cp = 0, maxm_prop = 0, maxKm_prop = 0;
  size_t ws_bytes = 0, zero_bytes = 0, off_flags = 0;
  size_t off_items = 0, off_pre = 0, off_lists = 0, table_bytes = 0;
};

// like (optional): a plan of a batch that contains these items; its candidate-QR shape
// and Gaussian-stage K-block cap are kept, so that every item is computed as in that batch
static int plan_batch(idl_ctx* ctx, const idl_batch_item* items, int n, const Tune& tn, BatchPlan& P,
                      const BatchPlan* like = nullptr) {
  P.it.assign(n, BItem());
  int prec = -1;
  for (int i = 0; i < n; ++i) {
    const idl_batch_item& x = items[i];
    const idl_params& pr = x.params;
    if (prec < 0) prec = pr.precision;
    if (pr.precision != prec) return fail(ctx, IDL_EINVAL, "batch: all items must use one precision");
    if (pr.learned < IDL_PROPOSAL_NONE || pr.learned > IDL_PROPOSAL_NORM)
      return fail(ctx, IDL_EINVAL, "batch: unknown proposal mode");
    if (pr.cand_factor < 0 || pr.cand_factor > 8) return fail(ctx, IDL_EINVAL, "batch: cand_factor must be in 0..8");
    if (pr.srrqr_f != 0.f) return fail(ctx, IDL_EINVAL, "batch: srrqr_f is for the single-item pipelines");
    if (pr.learned == IDL_PROPOSAL_MLP && !ctx->mlp_ready)
      return fail(ctx, IDL_EINVAL, "batch: no MLP weights (idl_mlp_init / idl_load_weights)");
    if (prec == IDL_PREC_FP64) return fail(ctx, IDL_EINVAL, "batch: FP32 data only (precision FP32, BF16X3, BF16 or TF32X3)");
    if (x.K < 1 || x.K >= x.R || pr.m2 < x.K || pr.m2 > pr.m1 || pr.m2 > 128 || x.K > 128 || !x.J || !x.T ||
        x.R > 0x7fffffffLL)
      return fail(ctx, IDL_EINVAL, "batch: need 1 <= K < R, K <= m2 <= min(m1, 128), K <= 128, outputs");
    if (x.kind == IDL_ITEM_DENSE) {
      if (!x.A || x.I < 1 || x.lda < x.R || x.I > 0x7fffffffLL) return fail(ctx, IDL_EINVAL, "batch: dense item");
      if (pr.modified && !(pr.m1 < x.I)) return fail(ctx, IDL_EINVAL, "batch: modified CountSketch needs m1 < I");
    } else if (x.kind == IDL_ITEM_CP) {
      if (x.N < 1 || x.N > 8 || !x.lambda || !x.lambda_hat || (pr.m1 & (pr.m1 - 1)) || pr.m1 < 16 || pr.m1 > 8192)
        return fail(ctx, IDL_EINVAL, "batch: CP item (1 <= N <= 8, L a power of two in [16, 8192])");
      for (int q = 0; q < x.N; ++q)
        if (!x.factors[q] || x.dims[q] < 1) return fail(ctx, IDL_EINVAL, "batch: CP factor");
    } else {
      return fail(ctx, IDL_EINVAL, "batch: item kind must be IDL_ITEM_DENSE or IDL_ITEM_CP");
    }
  }
  // operand planes of the Gaussian stage: 1..3 bf16 planes, or kNPTf32 for the two TF32 planes
  P.NP = prec == IDL_PREC_BF16 ? 1 : (prec == IDL_PREC_BF16X3 ? 2 : (prec == IDL_PREC_TF32X3 ? kNPTf32 : 3));
  const bool tf32 = P.NP == kNPTf32;
  // ---- per-item sizes and workspace layout ----
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off += (bytes + 255) & ~(size_t)255; return o; };
  std::vector<size_t> o_h(n), o_s(n), o_ptr(n), o_rows(n), o_big(n), o_Om(n), o_Bpl(n), o_Y1(n), o_part(n),
      o_Y2(n), o_rest(n), o_Rinv(n), o_mh(n), o_ms(n), o_Yf(n), o_Gp(n), o_F(n), o_V(n), o_cand(n), o_rn(n);
  // zero-initialised region first: certificate flags, cursors, nbig, diag
  P.off_flags = take(sizeof(int) * (size_t)n);
  std::vector<size_t> o_cur(n), o_nbig(n), o_diag(n);
  for (int i = 0; i < n; ++i) {
    const idl_batch_item& x = items[i];
    o_cur[i] = take(x.kind == IDL_ITEM_DENSE ? sizeof(int32_t) * (size_t)(x.params.m1 + 1) : 0);
    o_nbig[i] = take(sizeof(int32_t));
    o_diag[i] = take(sizeof(double) * 16);
  }
  P.zero_bytes = off;
  const int per_sm_gemm = 1;
  if (tn.split_mult == 0) {
    // the batch's output tiles times K blocks, in CTA-sized units; a group of a larger
    // batch (like) takes that batch's cap, so each item is split as it is there
    int64_t W = 0;
    for (int i = 0; i < n; ++i)
      W += cdiv(items[i].R, (int64_t)kBM) * cdiv(items[i].params.m1, (int64_t)(tf32 ? kBKt : kBK));
    P.kbmax = like ? like->kbmax
                   : std::max<int64_t>(kMinKbPerCta, cdiv(W, (int64_t)ctx->num_sms * kBatchWaves));
  }
  for (int i = 0; i < n; ++i) {
    const idl_batch_item& x = items[i];
    BItem& b = P.it[i];
    b.kind = x.kind;
    b.K = (int)x.K;
    b.R = x.R;
    b.m1 = x.params.m1;
    b.m2 = x.params.m2;
    b.ldy1 = round_up(x.R, 32);
    b.modified = x.params.modified;
    b.nkb = cdiv(b.m1, tf32 ? kBKt : kBK);
    b.NT = round_up(b.m2, 16);
    b.mtiles = cdiv(b.R, kBM);
    int64_t splits = tn.split_mult == 0
                         ? cdiv(b.nkb, P.kbmax)
                         : std::max<int64_t>(1, cdiv((int64_t)ctx->num_sms * per_sm_gemm * tn.split_mult, b.mtiles));
    splits = std::min<int64_t>(splits, b.nkb);
    b.kbpc = cdiv(b.nkb, splits);
    b.splits = cdiv(b.nkb, b.kbpc);
    b.gauss_base = stream_base(x.params.seed, kTagGauss);
    if (x.kind == IDL_ITEM_DENSE) {
      b.I = x.I;
      b.lda = x.lda;
      b.A = x.A;
      b.cs = make_cs_draw_args(x.params.seed, x.I);
      b.vec = ((uintptr_t)x.A % 16 == 0) && (x.lda % 4 == 0);
      b.ntiles = cdiv(x.R, (int64_t)tn.sketch_threads * 4);
      o_h[i] = take(sizeof(int32_t) * (size_t)x.I);
      o_s[i] = take((size_t)x.I);
      o_ptr[i] = take(sizeof(int32_t) * (size_t)(b.m1 + 1));
      o_rows[i] = take(sizeof(int32_t) * (size_t)x.I);
      o_big[i] = take(sizeof(int32_t) * (size_t)(b.m1 + 1));
      P.maxL_hist = std::max<int>(P.maxL_hist, (int)std::min<int64_t>(b.m1, kHistSmem));
    } else {
      b.N = x.N;
      b.lam = x.lambda;
      b.mode_tot = 0;
      for (int q = 0; q < x.N; ++q) b.mode_tot += x.dims[q];
      o_mh[i] = take(sizeof(int32_t) * (size_t)b.mode_tot);
      o_ms[i] = take((size_t)b.mode_tot);
      b.ts.N = x.N;
      for (int q = 0; q < x.N; ++q) {
        b.ts.F[q] = x.factors[q];
        b.ts.dims[q] = (int)x.dims[q];
        b.ts.ldf[q] = x.dims[q];
        b.mode_hb[q] = stream_base(x.params.seed, kTagModeBucket + q);
        b.mode_sb[q] = stream_base(x.params.seed, kTagModeSign + q);
      }
      P.maxL_cp = std::max<int>(P.maxL_cp, (int)b.m1);
    }
    o_Om[i] = take(sizeof(double) * (size_t)(b.m2 * b.m1));
    o_Bpl[i] = take(tf32 ? (size_t)b.nkb * 2 * b.NT * 128 : (size_t)b.nkb * P.NP * b.NT * kBK * 2);
    b.pt = x.kind == IDL_ITEM_CP && b.m1 == ts8::kL && !tf32;
    P.any_pt = P.any_pt || b.pt;
    o_Y1[i] = take(b.pt ? pretiled_bytes(b.R, b.m1, P.NP) : sizeof(float) * (size_t)(b.m1 * b.ldy1));
    o_part[i] = take(sizeof(float) * (size_t)(b.splits * b.R * b.NT));
    o_Y2[i] = take(sizeof(float) * (size_t)(b.R * b.m2));
    o_rest[i] = take(sizeof(int32_t) * (size_t)b.R);
    o_Rinv[i] = take(2 * sizeof(double) * (size_t)(x.K * x.K));     // FP64 inverse, then its FP32 pairs
    b.learned = x.params.learned;
    b.C = (int)std::min<int64_t>((x.params.cand_factor > 0 ? x.params.cand_factor : 2) * x.K, x.R);
    b.nsplit = (int)cdiv(x.R, prop::kGramCols);
    if (b.learned) {
      const int64_t m = b.m2;
      o_Yf[i] = take(sizeof(float) * (size_t)(b.R * m));
      o_Gp[i] = take(sizeof(float) * (size_t)(b.nsplit * m * m + b.nsplit + 4 + 4 * m * m));
      o_F[i] = take(sizeof(float) * (size_t)(b.R * prop::kNF + b.R));
      o_V[i] = take(sizeof(float) * (size_t)(x.K * m + x.K));
      o_cand[i] = take(sizeof(int32_t) * (size_t)b.R);
      o_rn[i] = take(sizeof(double) * (size_t)x.K);
      P.maxm_prop = std::max<int>(P.maxm_prop, (int)m);
      P.maxKm_prop = std::max<int>(P.maxKm_prop, (int)(x.K * m + 2 * x.K));
    }
    b.J = x.J;
    b.T = x.T;
    b.lam_hat = x.lambda_hat;
    P.maxK = std::max(P.maxK, (int)x.K);
    P.maxNT = std::max(P.maxNT, (int)b.NT);
  }
  P.ws_bytes = off;
  // tables: items, prefix arrays, cluster lists
  size_t toff = 0;
  P.off_items = toff;
  toff += sizeof(BItem) * n;
  toff = (toff + 255) & ~(size_t)255;
  P.off_pre = toff;
  toff += sizeof(int64_t) * (size_t)(n + 1) * kBNumStages;
  P.off_lists = toff;
  toff += sizeof(int32_t) * (size_t)(3 * n + 3);
  P.table_bytes = toff;
  // record workspace offsets (pointers are filled once the workspace address is known)
  for (int i = 0; i < n; ++i) {
    BItem& b = P.it[i];
    b.h = (int32_t*)o_h[i]; b.s = (int8_t*)o_s[i]; b.ptr = (int32_t*)o_ptr[i]; b.rows = (int32_t*)o_rows[i];
    b.cursor = (int32_t*)o_cur[i]; b.big = (int32_t*)o_big[i]; b.nbig = (int32_t*)o_nbig[i];
    b.mh = (int32_t*)o_mh[i]; b.ms = (int8_t*)o_ms[i]; b.Om = (double*)o_Om[i];
    b.Bpl = (__nv_bfloat16*)o_Bpl[i]; b.Y1 = (float*)o_Y1[i]; b.part = (float*)o_part[i]; b.Y2 = (float*)o_Y2[i];
    b.rest = (int32_t*)o_rest[i]; b.Rinv = (double*)o_Rinv[i]; b.diag = (double*)o_diag[i];
    b.flag = (int*)(P.off_flags + sizeof(int) * (size_t)i);
    if (b.learned) {
      const int64_t m = b.m2;
      b.Yf = (float*)o_Yf[i];
      b.Gp = (float*)o_Gp[i];
      b.nmaxp = (float*)(o_Gp[i] + sizeof(float) * (size_t)(b.nsplit * m * m));
      b.scal = (float*)((size_t)b.nmaxp + sizeof(float) * (size_t)b.nsplit);
      b.Linv = (float*)((size_t)b.scal + sizeof(float) * 4);
      b.G = (float*)((size_t)b.Linv + sizeof(float) * (size_t)(3 * m * m));
      b.F = (float*)o_F[i];
      b.sc = (float*)(o_F[i] + sizeof(float) * (size_t)(b.R * prop::kNF));
      b.V = (float*)o_V[i];
      b.beta = (float*)(o_V[i] + sizeof(float) * (size_t)(b.K * m));
      b.cand = (int32_t*)o_cand[i];
      b.outl = (int32_t*)(o_cand[i] + sizeof(int32_t) * (size_t)b.C);
      b.rn = (double*)o_rn[i];
    } else {
      b.Yf = b.Y2;
    }
  }
  // ---- prefix tables ----
  for (int st = 0; st < kBNumStages; ++st) P.pre[st].assign(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    const BItem& b = P.it[i];
    const bool d = b.kind == IDL_ITEM_DENSE, cp = !d;
    int64_t nb[kBNumStages] = {0};
    nb[kBDraw] = cdiv(d ? b.I : b.mode_tot, 256);
    nb[kBGauss] = cdiv(cdiv(b.m2 * b.m1, 2), 256);
    nb[kBHist] = d ? std::min<int64_t>(kBHistBlocks, cdiv(b.I, 4096)) : 0;
    nb[kBScan] = d ? 1 : 0;
    nb[kBScatter] = d ? cdiv(b.I, 256) : 0;
    nb[kBSortW] = d ? cdiv(b.m1, 8) : 0;
    nb[kBSortB] = d ? kBSortBlocks : 0;
    nb[kBSketchD] = d ? b.m1 * b.ntiles : 0;
    nb[kBSketchT] = cp && b.m1 != ts8::kL ? cdiv(b.R, 2) : 0;
    nb[kBSketchT8] = cp && b.m1 == ts8::kL ? cdiv(b.R, 2) : 0;    // column pairs
    nb[kBPlanes] = cdiv(b.nkb * b.NT * 8, 256);
    nb[kBGemm] = b.mtiles * b.splits;
    nb[kBReduce] = b.splits > 1 || tf32 ? cdiv(b.R * b.m2, 256) : 0;   // bf16 modes: unsplit items write Y2
    const bool mlp = b.learned == IDL_PROPOSAL_MLP, nrm = b.learned == IDL_PROPOSAL_NORM;
    nb[kBPGram] = mlp ? b.nsplit : 0;
    nb[kBPGRed] = mlp ? cdiv(b.m2 * b.m2, prop::kThreads) : 0;
    nb[kBPChol] = mlp ? 3 : 0;
    nb[kBPFeat] = mlp ? cdiv(b.R, prop::kFeatCols) : 0;
    nb[kBPMlp] = mlp ? cdiv(b.R, prop::kTile) : 0;
    nb[kBPNorm] = nrm ? cdiv(b.R, prop::kThreads / 32) : 0;
    nb[kBPSel] = b.learned ? 1 : 0;
    nb[kBPApply] = (b.learned && b.R > b.C) ? std::min<int64_t>(cdiv(b.R - b.C, prop::kApplyThreads / 32), 64) : 0;
    nb[kBRest] = cdiv(b.R, 256);
    nb[kBRinv] = cdiv(b.K, kRinvWarpsDf);                  // one warp per column
    nb[kBTgemm] = cdiv(b.R - b.K, kTNBdf);
    nb[kBLam] = cp ? b.K : 0;
    for (int st = 0; st < kBNumStages; ++st) P.pre[st][i + 1] = P.pre[st][i] + nb[st];
    if (d) P.dense_list.push_back(i); else P.cp_list.push_back(i);
    if (b.learned) P.prop_list.push_back(i);
  }
  if (!P.prop_list.empty()) {
    if (P.maxm_prop > prop::kMaxM || P.maxK > 128) return fail(ctx, IDL_ELIMIT, "batch: proposal needs m2, K <= 128");
    if (like && !like->prop_list.empty()) P.cfg_cand = like->cfg_cand;
    else if (!pick_cpqr(P.prop_list, P.it, &P.cfg_cand, true))
      return fail(ctx, IDL_ELIMIT, "batch: no candidate QR shape");
  }
  for (int i = 0; i < n; ++i) P.it[i].nc = 0;
  if (!qr_classes(P.dense_list, P.it, tn.qr_cs_dense, tn.qr_cap_dense, 0, P.qr) ||
      !qr_classes(P.cp_list, P.it, tn.qr_cs_cp, tn.qr_cap_cp, n + 1, P.qr))
    return fail(ctx, IDL_ELIMIT, "batch: no QR cluster shape");
  // launch order: the classes with the most pivot steps (the longest items) first
  std::stable_sort(P.qr.begin(), P.qr.end(), [](const QrClass& a, const QrClass& b) { return a.maxK > b.maxK; });
  return IDL_OK;
}

// one flattened launch: grid = the stage's total block count
#define BLAUNCH(kern, st, threads, smem, ...)                                                         \
  do {                                                                                                \
    const int64_t nb_ = P.pre[st][n];                                                                 \
    if (nb_ > 0) {                                                                                    \
      kern<<<(unsigned)nb_, threads, smem, ctx->stream>>>(d_items, d_pre + (size_t)(st) * (n + 1), n, \
                                                          ##__VA_ARGS__);                             \
      count_launch();                                                                                 \
      ++nlaunch;                                                                                      \
    }                                                                                                 \
  } while (0)

template <int NP>
static int run_gemm_stage(idl_ctx* ctx, const BatchPlan& P, const BItem* d_items, const int64_t* d_pre, int n,
                          int& nlaunch) {
  size_t smem = 1024 + (size_t)kStages * NP * kBM * kBK * 2 + (size_t)kBSlots * NP * P.maxNT * kBK * 2 + 128;
  // the pre-tiled items' A ring: as many stages as fit beside the B ring (2 at least)
  int S = 2;
  if (P.any_pt) {
    while (S < kPtMaxStages && pretiled_smem_bytes(S + 1, NP, P.maxNT) <= (size_t)ctx->smem_optin) ++S;
    smem = std::max(smem, pretiled_smem_bytes(S, NP, P.maxNT));
  }
  if (smem > (size_t)ctx->smem_optin) return fail(ctx, IDL_ELIMIT, "batch gemm: shared memory");
  cudaError_t e = ensure_smem(ctx, (const void*)b_gemm_kernel<NP>, smem);
  if (e != cudaSuccess) return cuda_check(ctx, e, "batch gemm attribute");
  BLAUNCH(b_planes_kernel<NP>, kBPlanes, 256, 0);
  BLAUNCH(b_gemm_kernel<NP>, kBGemm, kTcThreads, smem, ctx->d_status, S);
  return launch_check(ctx, "batch gemm");
}

static int run_gemm_stage_tf32(idl_ctx* ctx, const BatchPlan& P, const BItem* d_items, const int64_t* d_pre, int n,
                               int& nlaunch) {
  int S = 3;
  while (S < kTf32MaxStages && tf32_smem_bytes(S + 1, P.maxNT) <= (size_t)ctx->smem_optin) ++S;
  const size_t smem = tf32_smem_bytes(S, P.maxNT);
  if (smem > (size_t)ctx->smem_optin) return fail(ctx, IDL_ELIMIT, "batch gemm: shared memory");
  cudaError_t e = ensure_smem(ctx, (const void*)b_gemm_tf32_kernel, smem);
  if (e != cudaSuccess) return cuda_check(ctx, e, "batch gemm attribute");
  BLAUNCH(b_planes_tf32_kernel, kBPlanes, 256, 0);
  BLAUNCH(b_gemm_tf32_kernel, kBGemm, kTcThreads, smem, ctx->d_status, S);
  return launch_check(ctx, "batch gemm");
}

// Proposal stages: scores, selection, candidate QR, certificate (the gated
// cluster QR follows in run_stages).
static int run_proposal(idl_ctx* ctx, const BatchPlan& P, const BItem* d_items, const int64_t* d_pre,
                        const int32_t* d_plist, int n, int& nlaunch) {
  const int m = P.maxm_prop;
  const size_t sm_gram = sizeof(float) * 32 * round_up(m, 4);
  const size_t sm_chol = sizeof(float) * (2 * (size_t)m * (m + 1) + m);
  const size_t sm_feat = sizeof(float) * prop::features_smem_floats(m);
  const size_t sm_mlp = sizeof(float) * prop::mlp_fwd_smem_floats();
  const size_t sm_app = sizeof(float) * (size_t)P.maxKm_prop;
  cudaError_t e = ensure_smem(ctx, (const void*)b_pchol_kernel, sm_chol);
  if (e == cudaSuccess) e = ensure_smem(ctx, (const void*)b_pfeat_kernel, sm_feat);
  if (e == cudaSuccess) e = ensure_smem(ctx, (const void*)b_pmlp_kernel, sm_mlp);
  if (e == cudaSuccess) e = ensure_smem(ctx, (const void*)b_papply_kernel, sm_app);
  if (e != cudaSuccess) return cuda_check(ctx, e, "batch proposal attribute");
  BLAUNCH(b_pgram_kernel, kBPGram, prop::kThreads, sm_gram);
  BLAUNCH(b_pgred_kernel, kBPGRed, prop::kThreads, 0);
  BLAUNCH(b_pchol_kernel, kBPChol, prop::kThreads, sm_chol);
  BLAUNCH(b_pfeat_kernel, kBPFeat, prop::kThreads, sm_feat);
  BLAUNCH(b_pmlp_kernel, kBPMlp, prop::kThreads, sm_mlp, ctx->mlp);
  BLAUNCH(b_pnorm_kernel, kBPNorm, prop::kThreads, 0);
  BLAUNCH(b_psel_kernel, kBPSel, prop::kSelThreads, 0);
  BTRY(launch_check(ctx, "batch proposal scores"));
  BTRY(dispatch_b_cand(ctx, d_items, d_plist, (int)P.prop_list.size(), P.cfg_cand));
  ++nlaunch;
  BLAUNCH(b_papply_kernel, kBPApply, prop::kApplyThreads, sm_app);
  return launch_check(ctx, "batch proposal");
}

// The QR classes' launches: the first on ctx->stream, the others on up to kQrSide
// side streams (one per class while they last) forked from it and joined back
// (under stream capture the fork and join become graph edges), so the classes
// share the GPU.
static int run_qr(idl_ctx* ctx, const BatchPlan& P, const BItem* d_items, const int32_t* d_lists, int& nlaunch) {
  const int nq = (int)P.qr.size();
  if (nq == 0) return IDL_OK;
  idl_batch_state* bs = bstate(ctx);
  const int ns = std::min(nq - 1, kQrSide);
  if (ns > 0) {
    if (!bs->qfork) TRYC(cudaEventCreateWithFlags(&bs->qfork, cudaEventDisableTiming), "batch QR fork event");
    for (int k = 0; k < ns; ++k) {
      if (!bs->qs[k]) TRYC(cudaStreamCreateWithFlags(&bs->qs[k], cudaStreamNonBlocking), "batch QR stream");
      if (!bs->qjoin[k]) TRYC(cudaEventCreateWithFlags(&bs->qjoin[k], cudaEventDisableTiming), "batch QR join event");
    }
    TRYC(cudaEventRecord(bs->qfork, ctx->stream), "batch QR fork");
    for (int k = 0; k < ns; ++k) TRYC(cudaStreamWaitEvent(bs->qs[k], bs->qfork, 0), "batch QR fork");
  }
  for (int c = 0; c < nq; ++c) {
    const cudaStream_t st = c == 0 ? ctx->stream : bs->qs[(c - 1) % ns];
    BTRY(dispatch_b_cpqr(ctx, d_items, d_lists + P.qr[c].off, P.qr[c].count, P.qr[c].cfg, st));
    ++nlaunch;
  }
  for (int k = 0; k < ns; ++k) {
    TRYC(cudaEventRecord(bs->qjoin[k], bs->qs[k]), "batch QR join");
    TRYC(cudaStreamWaitEvent(ctx->stream, bs->qjoin[k], 0), "batch QR join");
  }
  return IDL_OK;
}

// All launches of a batch (the part that is captured into a graph).  ms (optional,
// kBTimedStages floats): CUDA-event times of the stage groups (see BTimed).
static int run_stages(idl_ctx* ctx, const BatchPlan& P, const BItem* d_items, const int64_t* d_pre,
                      const int32_t* d_lists, int n, int sketch_threads, int& nlaunch, float* ms) {
  nlaunch = 0;
  cudaEvent_t ev[kBTimedStages + 1] = {};
  const bool timed = ms != nullptr;
  if (timed)
    for (auto& x : ev) cudaEventCreate(&x);
  // stage groups as NVTX ranges (a no-op unless a profiler is attached) and, when timed, events
  static const char* const names[kBTimedStages] = {"idl:batch draws+buckets", "idl:batch sketch cp",
                                                   "idl:batch sketch dense", "idl:batch gaussian",
                                                   "idl:batch proposal", "idl:batch cpqr", "idl:batch tsolve"};
  auto mark = [&](int i) {
    if (i > 0) nvtxRangePop();
    if (i < kBTimedStages) nvtxRangePushA(names[i]);
    if (timed) cudaEventRecord(ev[i], ctx->stream);
  };
  mark(0);
  BLAUNCH(b_draw_kernel, kBDraw, 256, 0, ctx->d_status);
  BLAUNCH(b_gauss_draw_kernel, kBGauss, 256, 0);
  BLAUNCH(b_hist_kernel, kBHist, 512, sizeof(int32_t) * (size_t)P.maxL_hist, ctx->d_status);
  BLAUNCH(b_scan_kernel, kBScan, 1024, 0);
  BLAUNCH(b_scatter_kernel, kBScatter, 256, 0);
  BLAUNCH(b_sortw_kernel, kBSortW, 256, sizeof(int32_t) * 8 * kWarpSortCap);
  BLAUNCH(b_sortb_kernel, kBSortB, 512, sizeof(int32_t) * kBlockSortCap);
  BTRY(launch_check(ctx, "batch buckets"));
  mark(1);
  if (P.pre[kBSketchT][n] > 0) {
    const size_t smem = ts_smem_bytes(P.maxL_cp);
    cudaError_t e = ensure_smem(ctx, (const void*)b_sketch_cp_kernel, smem);
    if (e != cudaSuccess) return cuda_check(ctx, e, "batch tensorsketch attribute");
    BLAUNCH(b_sketch_cp_kernel, kBSketchT, ts_threads(P.maxL_cp), smem, (const float2*)ctx->ts_tw);
  }
  if (P.pre[kBSketchT8][n] > 0) {
    // pre-tiled planes for the bf16 modes (every such item is pre-tiled), FP32 otherwise
    const int pt = P.any_pt ? P.NP : 0;
    auto kern = pt == 1 ? b_sketch_cp8k_kernel<1>
                        : (pt == 2 ? b_sketch_cp8k_kernel<2> : (pt == 3 ? b_sketch_cp8k_kernel<3> : b_sketch_cp8k_kernel<0>));
    cudaError_t e = ensure_smem(ctx, (const void*)kern, ts8::kSmemBytes);
    if (e != cudaSuccess) return cuda_check(ctx, e, "batch tensorsketch attribute");
    const int64_t grid = std::min<int64_t>(P.pre[kBSketchT8][n], ctx->num_sms);
    kern<<<(unsigned)grid, ts8::kT, ts8::kSmemBytes, ctx->stream>>>(d_items, d_pre + (size_t)kBSketchT8 * (n + 1), n,
                                                                    (const float2*)ctx->ts8_tw);
    count_launch();
    ++nlaunch;
  }
  mark(2);
  {
    const int64_t nbd = P.pre[kBSketchD][n];
    const int64_t* pre_d = d_pre + (size_t)kBSketchD * (n + 1);
    if (nbd > 0) {
      b_sketch_dense_kernel<<<(unsigned)nbd, sketch_threads, 0, ctx->stream>>>(d_items, pre_d, n, 0);
      count_launch();
      ++nlaunch;
    }
  }
  BTRY(launch_check(ctx, "batch sketch"));
  mark(3);
  if (P.NP == kNPTf32) BTRY(run_gemm_stage_tf32(ctx, P, d_items, d_pre, n, nlaunch));
  else if (P.NP == 1) BTRY(run_gemm_stage<1>(ctx, P, d_items, d_pre, n, nlaunch));
  else if (P.NP == 2) BTRY(run_gemm_stage<2>(ctx, P, d_items, d_pre, n, nlaunch));
  else BTRY(run_gemm_stage<3>(ctx, P, d_items, d_pre, n, nlaunch));
  BLAUNCH(b_reduce_kernel, kBReduce, 256, 0);
  mark(4);
  if (!P.prop_list.empty()) BTRY(run_proposal(ctx, P, d_items, d_pre, d_lists + 2 * (n + 1), n, nlaunch));
  mark(5);
  BTRY(run_qr(ctx, P, d_items, d_lists, nlaunch));
  mark(6);
  BLAUNCH(b_rest_kernel, kBRest, 256, sizeof(int32_t) * (size_t)P.maxK);
  {
    const size_t smem_inv = sizeof(double) * (size_t)P.maxK * (P.maxK + 1);
    const size_t smem_t = sizeof(float) * (size_t)tgemm_df_floats(P.maxK);
    cudaError_t e = ensure_smem(ctx, (const void*)b_rinv_kernel, smem_inv);
    if (e == cudaSuccess) e = ensure_smem(ctx, (const void*)b_tgemm_kernel, smem_t);
    if (e != cudaSuccess) return cuda_check(ctx, e, "batch solve attribute");
    BLAUNCH(b_rinv_kernel, kBRinv, 32 * kRinvWarpsDf, smem_inv);
    BLAUNCH(b_tgemm_kernel, kBTgemm, 256, smem_t);
  }
  BLAUNCH(b_lam_kernel, kBLam, 256, 0);
  BTRY(launch_check(ctx, "batch solve"));
  mark(7);
  if (timed) {
    cudaEventSynchronize(ev[kBTimedStages]);
    for (int i = 0; i < kBTimedStages; ++i) cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
    for (auto& x : ev) cudaEventDestroy(x);
  }
  return IDL_OK;
}

// Uploads the tables (with workspace addresses filled in) and clears the zero region.
// pinned (optional): a pinned host region of P.table_bytes the tables pass through, so
// that the copy is queued without waiting for the stream (a pageable source may make
// the driver synchronise with the stream first)
static int upload(idl_ctx* ctx, BatchPlan& P, unsigned char* ws, unsigned char* tab, int n, bool sync = true,
                  unsigned char* pinned = nullptr) {
  std::vector<unsigned char> host(P.table_bytes, 0);
  std::vector<BItem> items = P.it;
  auto fix = [&](auto*& ptr) { ptr = (std::remove_reference_t<decltype(ptr)>)(ws + (size_t)(uintptr_t)ptr); };
  for (auto& b : items) {
    if (b.kind == IDL_ITEM_DENSE) { fix(b.h); fix(b.s); fix(b.ptr); fix(b.rows); fix(b.big); }
    else {
      fix(b.mh); fix(b.ms);
      int64_t off = 0;
      for (int q = 0; q < b.N; ++q) {
        b.ts.h[q] = b.mh + off;
        b.ts.s[q] = b.ms + off;
        off += b.ts.dims[q];
      }
    }
    fix(b.cursor); fix(b.nbig); fix(b.Om); fix(b.Bpl); fix(b.Y1); fix(b.part); fix(b.Y2); fix(b.rest); fix(b.Rinv);
    fix(b.diag); fix(b.flag); fix(b.Yf);
    if (b.learned) {
      fix(b.Gp); fix(b.nmaxp); fix(b.scal); fix(b.Linv); fix(b.G); fix(b.F); fix(b.sc); fix(b.V); fix(b.beta); fix(b.cand);
      fix(b.outl); fix(b.rn);
      b.gate = b.flag;
    } else {
      b.gate = nullptr;
    }
  }
  memcpy(host.data() + P.off_items, items.data(), sizeof(BItem) * n);
  int64_t* pre = (int64_t*)(host.data() + P.off_pre);
  for (int st = 0; st < kBNumStages; ++st) memcpy(pre + (size_t)st * (n + 1), P.pre[st].data(), sizeof(int64_t) * (n + 1));
  int32_t* lists = (int32_t*)(host.data() + P.off_lists);
  for (size_t q = 0; q < P.dense_list.size(); ++q) lists[q] = P.dense_list[q];
  for (size_t q = 0; q < P.cp_list.size(); ++q) lists[n + 1 + q] = P.cp_list[q];
  for (size_t q = 0; q < P.prop_list.size(); ++q) lists[2 * (n + 1) + q] = P.prop_list[q];
  if (pinned) memcpy(pinned, host.data(), P.table_bytes);
  cudaError_t e = cudaMemcpyAsync(tab, pinned ? pinned : host.data(), P.table_bytes, cudaMemcpyHostToDevice,
                                  ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws, 0, P.zero_bytes, ctx->stream);
  // a pageable host-to-device copy returns once its source is staged; the synchronisation
  // (sync = true) keeps the tuning runs' timing free of queued work
  if (e == cudaSuccess && sync) e = cudaStreamSynchronize(ctx->stream);
  return cuda_check(ctx, e, "batch upload");
}

// ---------------------------------------------------------------------------
// Host arrays.  The batch's inputs are copied into one device staging buffer on
// the context's copy stream -- the CP items' factors and s-values first, then the
// dense matrices in groups -- while the item groups run on the context's stream,
// each after its own inputs (run_host_groups); the outputs are copied back at the end.
// ---------------------------------------------------------------------------
struct HostStage {
  struct Copy { size_t off; const void* host; size_t bytes; };
  std::vector<Copy> in_cp, in_dense, out;
  std::vector<int> dense_item;       // item index of each in_dense entry
  size_t bytes = 0;
  unsigned char* base = nullptr;
};

static int stage_layout(idl_ctx* ctx, const idl_batch_item* items, int n, std::vector<idl_batch_item>& dv,
                        HostStage& hs) {
  dv.assign(items, items + n);
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off += (bytes + 255) & ~(size_t)255; return o; };
  for (int i = 0; i < n; ++i) {
    const idl_batch_item& x = items[i];
    if (x.K < 1 || x.K >= x.R || x.R > 0x7fffffffLL) return fail(ctx, IDL_EINVAL, "batch: need 1 <= K < R");
    if (x.kind == IDL_ITEM_DENSE) {
      if (!x.A || x.I < 1 || x.lda < x.R) return fail(ctx, IDL_EINVAL, "batch: dense item");
      const size_t b = sizeof(float) * (size_t)((x.I - 1) * x.lda + x.R);
      hs.in_dense.push_back({take(b), x.A, b});
      hs.dense_item.push_back(i);
      dv[i].A = (const float*)(uintptr_t)hs.in_dense.back().off;
    } else if (x.kind == IDL_ITEM_CP) {
      if (x.N < 1 || x.N > 8 || !x.lambda) return fail(ctx, IDL_EINVAL, "batch: CP item");
      for (int q = 0; q < x.N; ++q) {
        if (!x.factors[q] || x.dims[q] < 1) return fail(ctx, IDL_EINVAL, "batch: CP factor");
        const size_t b = sizeof(float) * (size_t)(x.dims[q] * x.R);
        hs.in_cp.push_back({take(b), x.factors[q], b});
        dv[i].factors[q] = (const float*)(uintptr_t)hs.in_cp.back().off;
      }
      const size_t b = sizeof(double) * (size_t)x.R;
      hs.in_cp.push_back({take(b), x.lambda, b});
      dv[i].lambda = (const double*)(uintptr_t)hs.in_cp.back().off;
    } else {
      return fail(ctx, IDL_EINVAL, "batch: item kind must be IDL_ITEM_DENSE or IDL_ITEM_CP");
    }
    if (!x.J || !x.T || (x.kind == IDL_ITEM_CP && !x.lambda_hat)) return fail(ctx, IDL_EINVAL, "batch: outputs");
    hs.out.push_back({take(sizeof(int32_t) * (size_t)x.K), x.J, sizeof(int32_t) * (size_t)x.K});
    dv[i].J = (int32_t*)(uintptr_t)hs.out.back().off;
    hs.out.push_back({take(sizeof(double) * (size_t)(x.K * (x.R - x.K))), x.T, sizeof(double) * (size_t)(x.K * (x.R - x.K))});
    dv[i].T = (double*)(uintptr_t)hs.out.back().off;
    if (x.kind == IDL_ITEM_CP) {
      hs.out.push_back({take(sizeof(double) * (size_t)x.K), x.lambda_hat, sizeof(double) * (size_t)x.K});
      dv[i].lambda_hat = (double*)(uintptr_t)hs.out.back().off;
    }
  }
  hs.bytes = off;
  hs.base = (unsigned char*)ws_get(ctx, kWsBatchIn, off);
  if (!hs.base) return IDL_ENOMEM;
  auto fix = [&](auto& ptr) {
    using P = std::remove_reference_t<decltype(ptr)>;
    ptr = (P)(hs.base + (size_t)(uintptr_t)ptr);
  };
  for (int i = 0; i < n; ++i) {
    if (dv[i].kind == IDL_ITEM_DENSE) fix(dv[i].A);
    else {
      for (int q = 0; q < dv[i].N; ++q) fix(dv[i].factors[q]);
      fix(dv[i].lambda);
      fix(dv[i].lambda_hat);
    }
    fix(dv[i].J);
    fix(dv[i].T);
  }
  return IDL_OK;
}

static cudaEvent_t stage_event(idl_batch_state* bs, size_t i) {
  while (bs->cev.size() <= i) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    bs->cev.push_back(e);
  }
  return bs->cev[i];
}

// All inputs of a host-array batch copied in on the copy stream; the context's stream
// waits for them (the first call's tuning runs read every input).
static int stage_all_inputs(idl_ctx* ctx, idl_batch_state* bs, const HostStage& hs) {
  if (!bs->cstream) TRYC(cudaStreamCreateWithFlags(&bs->cstream, cudaStreamNonBlocking), "batch copy stream");
  cudaEvent_t ev0 = stage_event(bs, 0), ev1 = stage_event(bs, 1);
  if (!ev0 || !ev1) return fail(ctx, IDL_ECUDA, "batch: event creation failed");
  TRYC(cudaEventRecord(ev0, ctx->stream), "batch stage order");
  TRYC(cudaStreamWaitEvent(bs->cstream, ev0, 0), "batch stage order");
  for (const auto& c : hs.in_cp)
    TRYC(cudaMemcpyAsync(hs.base + c.off, c.host, c.bytes, cudaMemcpyDefault, bs->cstream), "batch copy in");
  for (const auto& c : hs.in_dense)
    TRYC(cudaMemcpyAsync(hs.base + c.off, c.host, c.bytes, cudaMemcpyDefault, bs->cstream), "batch copy in");
  TRYC(cudaEventRecord(ev1, bs->cstream), "batch copy event");
  TRYC(cudaStreamWaitEvent(ctx->stream, ev1, 0), "batch stage wait");
  return IDL_OK;
}

static int stage_outputs(idl_ctx* ctx, const HostStage& hs) {
  for (const auto& c : hs.out)
    TRYC(cudaMemcpyAsync((void*)c.host, hs.base + c.off, c.bytes, cudaMemcpyDefault, ctx->stream), "batch copy out");
  TRYC(cudaStreamSynchronize(ctx->stream), "batch sync");
  return IDL_OK;
}

// Host arrays: the CP items, then the dense items in groups of about equal bytes (eight),
// each group copied in on the copy stream and run through every stage as soon as its
// own copies have landed, so the Gaussian stage, QR and T of all groups but the last
// overlap the later groups' copies.  Each group has its own plan, tables and workspace
// region (the regions add up to the whole batch's), so nothing is reused while queued.
// Results equal the single-plan run's: the group plans keep the whole batch's tuning and
// QR kernel shapes, and every other choice depends on the item alone.
static int run_host_groups(idl_ctx* ctx, idl_batch_state* bs, const HostStage& hs, const idl_batch_item* items,
                           int n, const Tune& tn, const BatchPlan& whole) {
  std::vector<std::vector<int>> groups;
  {
    std::vector<int> cp;
    for (int i = 0; i < n; ++i)
      if (items[i].kind == IDL_ITEM_CP) cp.push_back(i);
    if (!cp.empty()) groups.push_back(cp);
  }
  const size_t first_dense = groups.size();
  size_t tot = 0;
  for (const auto& c : hs.in_dense) tot += c.bytes;
  const size_t per = tot / 8 + 1;
  {
    std::vector<int> cur;
    size_t acc = 0;
    for (size_t q = 0; q < hs.in_dense.size(); ++q) {
      cur.push_back(hs.dense_item[q]);
      acc += hs.in_dense[q].bytes;
      if (acc >= per || q + 1 == hs.in_dense.size()) { groups.push_back(cur); cur.clear(); acc = 0; }
    }
  }
  // one plan per group, placed side by side in the workspace and the table buffer
  const size_t G = groups.size();
  std::vector<std::vector<idl_batch_item>> subs(G);
  std::vector<BatchPlan> plans(G);
  std::vector<size_t> ws_off(G), tab_off(G);
  size_t ws_tot = 0, tab_tot = 0;
  for (size_t g = 0; g < G; ++g) {
    for (int i : groups[g]) subs[g].push_back(items[i]);
    BTRY(plan_batch(ctx, subs[g].data(), (int)subs[g].size(), tn, plans[g], &whole));
    ws_off[g] = ws_tot;
    tab_off[g] = tab_tot;
    ws_tot += (plans[g].ws_bytes + 255) & ~(size_t)255;
    tab_tot += (plans[g].table_bytes + 255) & ~(size_t)255;
  }
  unsigned char* ws = (unsigned char*)ws_get(ctx, kWsBatch, ws_tot);
  unsigned char* tab = (unsigned char*)ws_get(ctx, kWsBatchTab, tab_tot);
  if (!ws || !tab) return IDL_ENOMEM;
  if (bs->pin_bytes < tab_tot) {      // reused by later calls: each call ends synchronised
    if (bs->pin) cudaFreeHost(bs->pin);
    bs->pin = nullptr;
    bs->pin_bytes = 0;
    if (cudaMallocHost((void**)&bs->pin, tab_tot) != cudaSuccess) {
      (void)cudaGetLastError();
      bs->pin = nullptr;
      return fail(ctx, IDL_ENOMEM, "batch: pinned table staging");
    }
    bs->pin_bytes = tab_tot;
  }
  // every group's tables before the input copies: host-to-device copies are served in
  // the order they are queued, so a table queued behind the inputs would wait for all
  // of them (measured: the first group then started after the last input landed)
  for (size_t g = 0; g < G; ++g)
    BTRY(upload(ctx, plans[g], ws + ws_off[g], tab + tab_off[g], (int)subs[g].size(), false, bs->pin + tab_off[g]));
  // copies: the CP group's first, then each dense group's, an event after each group
  if (!bs->cstream) TRYC(cudaStreamCreateWithFlags(&bs->cstream, cudaStreamNonBlocking), "batch copy stream");
  cudaEvent_t ev0 = stage_event(bs, 0);
  if (!ev0) return fail(ctx, IDL_ECUDA, "batch: event creation failed");
  TRYC(cudaEventRecord(ev0, ctx->stream), "batch stage order");
  TRYC(cudaStreamWaitEvent(bs->cstream, ev0, 0), "batch stage order");
  std::vector<cudaEvent_t> gev;
  size_t ne = 1;
  auto group_event = [&]() -> int {
    cudaEvent_t e = stage_event(bs, ne++);
    if (!e) return fail(ctx, IDL_ECUDA, "batch: event creation failed");
    TRYC(cudaEventRecord(e, bs->cstream), "batch copy event");
    gev.push_back(e);
    return IDL_OK;
  };
  if (first_dense == 1) {
    for (const auto& c : hs.in_cp)
      TRYC(cudaMemcpyAsync(hs.base + c.off, c.host, c.bytes, cudaMemcpyDefault, bs->cstream), "batch copy in");
    BTRY(group_event());
  }
  {
    size_t q = 0;
    for (size_t g = first_dense; g < groups.size(); ++g) {
      for (size_t k = 0; k < groups[g].size(); ++k, ++q) {
        const auto& c = hs.in_dense[q];
        TRYC(cudaMemcpyAsync(hs.base + c.off, c.host, c.bytes, cudaMemcpyDefault, bs->cstream), "batch copy in");
      }
      BTRY(group_event());
    }
  }
  bs->flag_sets.clear();
  bs->d_flags = nullptr;
  bs->nflags = 0;
  for (size_t g = 0; g < G; ++g) {
    const int ng = (int)subs[g].size();
    const BatchPlan& Q = plans[g];
    unsigned char* w = ws + ws_off[g];
    unsigned char* t = tab + tab_off[g];
    TRYC(cudaStreamWaitEvent(ctx->stream, gev[g], 0), "batch group wait");
    int nl = 0;
    BTRY(run_stages(ctx, Q, (const BItem*)(t + Q.off_items), (const int64_t*)(t + Q.off_pre),
                    (const int32_t*)(t + Q.off_lists), ng, tn.sketch_threads, nl, nullptr));
    bs->flag_sets.push_back({(const int*)(w + Q.off_flags), ng});
  }
  return IDL_OK;
}

extern "C" int idl_batch_run(idl_ctx* ctx, const idl_batch_item* items, int n) {
  BTRY(ctx_usable(ctx));
  if (n < 1 || !items) return fail(ctx, IDL_EINVAL, "batch: need n >= 1 items");
  idl_batch_state* bs = bstate(ctx);
  // host arrays: decided by the first item's input; the whole batch is then staged
  const void* first = items[0].kind == IDL_ITEM_DENSE ? (const void*)items[0].A : (const void*)items[0].factors[0];
  const bool host = first && !is_device_ptr(first);
  std::vector<idl_batch_item> staged;
  HostStage hs;
  if (host) {
    BTRY(stage_layout(ctx, items, n, staged, hs));
    items = staged.data();
  }
  const std::string sig = signature(items, n);
  const uint64_t key = fnv1a(sig);
  const bool known = bs->tune.count(key) != 0;
  Tune tn = known ? bs->tune[key] : Tune();
  BatchPlan P;
  BTRY(plan_batch(ctx, items, n, tn, P));
  if (!P.cp_list.empty() && (!ts_twiddles(ctx) || !ts8_twiddles(ctx))) return IDL_ENOMEM;   // built before any capture
  unsigned char* ws = (unsigned char*)ws_get(ctx, kWsBatch, P.ws_bytes);
  unsigned char* tab = (unsigned char*)ws_get(ctx, kWsBatchTab, P.table_bytes);
  if (!ws || !tab) return IDL_ENOMEM;
  const BItem* d_items = (const BItem*)(tab + P.off_items);
  const int64_t* d_pre = (const int64_t*)(tab + P.off_pre);
  const int32_t* d_lists = (const int32_t*)(tab + P.off_lists);
  int nlaunch = 0;
  if (!known && !ctx->batch_no_tune) {
    if (host) BTRY(stage_all_inputs(ctx, bs, hs));      // the tuning runs read the inputs
    // autotune, one knob at a time on whole-batch runs timed per stage group: the dense
    // sketch's block width, the Gaussian split-K factor, the QR cluster sizes
    auto trial = [&](const Tune& t, int stage, float* out) -> int {
      BatchPlan Q;
      BTRY(plan_batch(ctx, items, n, t, Q));
      unsigned char* ws2 = (unsigned char*)ws_get(ctx, kWsBatch, Q.ws_bytes);
      unsigned char* tab2 = (unsigned char*)ws_get(ctx, kWsBatchTab, Q.table_bytes);
      if (!ws2 || !tab2) return IDL_ENOMEM;
      BTRY(upload(ctx, Q, ws2, tab2, n));
      float ms[kBTimedStages] = {};
      BTRY(run_stages(ctx, Q, (const BItem*)(tab2 + Q.off_items), (const int64_t*)(tab2 + Q.off_pre),
                      (const int32_t*)(tab2 + Q.off_lists), n, t.sketch_threads, nlaunch, ms));
      *out = ms[stage];
      return IDL_OK;
    };
    auto tune_knob = [&](int Tune::*knob, std::initializer_list<int> values, int stage) -> int {
      float best = 1e30f;
      int pick = tn.*knob;
      for (int v : values) {
        Tune t = tn;
        t.*knob = v;
        float ms = 0.f;
        BTRY(trial(t, stage, &ms));
        if (ms < best) { best = ms; pick = v; }
      }
      tn.*knob = pick;
      return IDL_OK;
    };
    BTRY(tune_knob(&Tune::sketch_threads, {128, 256, 512}, kBTSketchDense));
    BTRY(tune_knob(&Tune::split_mult, {1, 2, 0}, kBTGauss));
    if (!P.dense_list.empty()) BTRY(tune_knob(&Tune::qr_cs_dense, {16, 8, 4}, kBTQR));
    if (!P.cp_list.empty()) BTRY(tune_knob(&Tune::qr_cs_cp, {16, 8, 4}, kBTQR));
    if (!P.dense_list.empty()) BTRY(tune_knob(&Tune::qr_cap_dense, {1024, 256, 128}, kBTQR));
    if (!P.cp_list.empty()) BTRY(tune_knob(&Tune::qr_cap_cp, {1024, 512, 320}, kBTQR));
    bs->tune[key] = tn;
    P = BatchPlan();
    BTRY(plan_batch(ctx, items, n, tn, P));
    ws = (unsigned char*)ws_get(ctx, kWsBatch, P.ws_bytes);
    tab = (unsigned char*)ws_get(ctx, kWsBatchTab, P.table_bytes);
    if (!ws || !tab) return IDL_ENOMEM;
    d_items = (const BItem*)(tab + P.off_items);
    d_pre = (const int64_t*)(tab + P.off_pre);
    d_lists = (const int32_t*)(tab + P.off_lists);
  }
  if (host) {         // item groups run as their inputs land
    BTRY(run_host_groups(ctx, bs, hs, items, n, tn, P));
    return stage_outputs(ctx, hs);
  }
  BTRY(upload(ctx, P, ws, tab, n));
  bs->d_flags = (const int*)(ws + P.off_flags);
  bs->nflags = n;
  bs->flag_sets.clear();
  if (ctx->batch_no_graph) return run_stages(ctx, P, d_items, d_pre, d_lists, n, tn.sketch_threads, nlaunch, nullptr);
  // graph: captured once per (shape, workspace address) on a private stream, replayed afterwards;
  // events order it after the caller's stream and the caller's stream after it
  if (!bs->gstream) {
    cudaError_t e = cudaStreamCreateWithFlags(&bs->gstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bs->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bs->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_check(ctx, e, "batch stream");
  }
  const uint64_t gkey = key ^ (uint64_t)(uintptr_t)ws ^ ((uint64_t)(uintptr_t)tab << 1);
  cudaStream_t user = ctx->stream;
  if (!bs->graph || bs->graph_sig != gkey) {
    if (bs->graph) { cudaGraphExecDestroy(bs->graph); bs->graph = nullptr; }
    cudaGraph_t g = nullptr;
    ctx->stream = bs->gstream;
    cudaError_t e = cudaStreamBeginCapture(bs->gstream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { ctx->stream = user; return cuda_check(ctx, e, "batch capture begin"); }
    const long long before = idl_launch_count();
    const int rc = run_stages(ctx, P, d_items, d_pre, d_lists, n, tn.sketch_threads, nlaunch, nullptr);
    e = cudaStreamEndCapture(bs->gstream, &g);
    ctx->stream = user;
    if (rc != IDL_OK) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return cuda_check(ctx, e, "batch capture end");
    e = cudaGraphInstantiate(&bs->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { bs->graph = nullptr; return cuda_check(ctx, e, "batch graph instantiate"); }
    bs->graph_sig = gkey;
    bs->graph_launches = (int)(idl_launch_count() - before);
    ctx_add_launches(-bs->graph_launches);     // counted when the graph runs
  }
  cudaError_t e = cudaEventRecord(bs->ev_in, user);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(bs->gstream, bs->ev_in, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(bs->graph, bs->gstream);
  if (e == cudaSuccess) e = cudaEventRecord(bs->ev_out, bs->gstream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(user, bs->ev_out, 0);
  ctx_add_launches(bs->graph_launches);
  return cuda_check(ctx, e, "batch graph launch");
}

extern "C" int idl_tune_save(idl_ctx* ctx, const char* path) {
  if (!ctx || !path) return IDL_EINVAL;
  FILE* f = fopen(path, "w");
  if (!f) return fail(ctx, IDL_EINVAL, "tune_save: cannot open file");
  fprintf(f, "# idl batch tuning: shape-hash sketch_threads split_mult qr_cluster_dense qr_cluster_cp "
             "qr_threads_dense qr_threads_cp\n");
  for (auto& kv : bstate(ctx)->tune)
    fprintf(f, "%016llx %d %d %d %d %d %d\n", (unsigned long long)kv.first, kv.second.sketch_threads,
            kv.second.split_mult, kv.second.qr_cs_dense, kv.second.qr_cs_cp, kv.second.qr_cap_dense,
            kv.second.qr_cap_cp);
  fclose(f);
  return IDL_OK;
}

extern "C" int idl_tune_load(idl_ctx* ctx, const char* path) {
  if (!ctx || !path) return IDL_EINVAL;
  FILE* f = fopen(path, "r");
  if (!f) return fail(ctx, IDL_EINVAL, "tune_load: cannot open file");
  char line[256];
  int loaded = 0;
  while (fgets(line, sizeof(line), f)) {
    if (line[0] == '#') continue;
    unsigned long long k;
    int a, b, c = 16, d = 16, e = 1024, g = 1024;      // the last four may be absent (older files)
    const int got = sscanf(line, "%llx %d %d %d %d %d %d", &k, &a, &b, &c, &d, &e, &g);
    auto cs_ok = [](int x) { return x == 4 || x == 8 || x == 16; };
    auto cap_ok = [](int x) { return x == 128 || x == 256 || x == 320 || x == 512 || x == 1024; };
    if (got >= 3 && (a == 128 || a == 256 || a == 512) && (b == 0 || b == 1 || b == 2) && cs_ok(c) && cs_ok(d) &&
        cap_ok(e) && cap_ok(g)) {
      Tune t;
      t.sketch_threads = a;
      t.split_mult = b;
      t.qr_cs_dense = c;
      t.qr_cs_cp = d;
      t.qr_cap_dense = e;
      t.qr_cap_cp = g;
      bstate(ctx)->tune[(uint64_t)k] = t;
      ++loaded;
    }
  }
  fclose(f);
  return loaded >= 0 ? IDL_OK : IDL_EINVAL;
}

// Runs the batch once without the graph, with CUDA events around the stage groups:
// ms[0] draws and bucket offsets, [1] CP TensorSketch, [2] dense sketch, [3] Gaussian
// stage, [4] column proposal, [5] pivoted QR, [6] T solve and lambda_hat.  Used to
// attribute time to the kernels.
extern "C" int idl_debug_batch_timing(idl_ctx* ctx, const idl_batch_item* items, int n, float* ms) {
  BTRY(ctx_usable(ctx));
  if (!items || n < 1 || !ms) return IDL_EINVAL;
  idl_batch_state* bs = bstate(ctx);
  const uint64_t key = fnv1a(signature(items, n));
  Tune tn = bs->tune.count(key) ? bs->tune[key] : Tune();
  BatchPlan P;
  BTRY(plan_batch(ctx, items, n, tn, P));
  if (!P.cp_list.empty() && (!ts_twiddles(ctx) || !ts8_twiddles(ctx))) return IDL_ENOMEM;   // built before any capture
  unsigned char* ws = (unsigned char*)ws_get(ctx, kWsBatch, P.ws_bytes);
  unsigned char* tab = (unsigned char*)ws_get(ctx, kWsBatchTab, P.table_bytes);
  if (!ws || !tab) return IDL_ENOMEM;
  BTRY(upload(ctx, P, ws, tab, n));
  int nl = 0;
  return run_stages(ctx, P, (const BItem*)(tab + P.off_items), (const int64_t*)(tab + P.off_pre),
                    (const int32_t*)(tab + P.off_lists), n, tn.sketch_threads, nl, ms);
}

extern "C" int idl_batch_fallbacks(idl_ctx* ctx) {
  if (!ctx) return -IDL_EINVAL;
  idl_batch_state* bs = bstate(ctx);
  std::vector<std::pair<const int*, int>> sets = bs->flag_sets;
  if (sets.empty() && bs->d_flags && bs->nflags > 0) sets.push_back({bs->d_flags, bs->nflags});
  int c = 0;
  for (const auto& fs : sets) {
    std::vector<int> h((size_t)fs.second);
    cudaError_t e = cudaMemcpyAsync(h.data(), fs.first, sizeof(int) * h.size(), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return -cuda_check(ctx, e, "batch fallbacks");
    for (int v : h) c += v != 0;
  }
  return c;
}

extern "C" int idl_debug_batch_mode(idl_ctx* ctx, int no_graph, int no_tune) {
  if (!ctx) return IDL_EINVAL;
  ctx->batch_no_graph = no_graph != 0;
  ctx->batch_no_tune = no_tune != 0;
  return IDL_OK;
}
