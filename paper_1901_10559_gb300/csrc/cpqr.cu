// cpqr.cu -- Algorithm 1 on the small sketch: rank-K column-pivoted Householder
// QR, T = R11^{-1} R12 in FP64, the FP64 residual check and the s-value update
// lambda_hat of Algorithm 3.
//
// QR stage design.  The sketch Y2 (m x R, m <= 256) is a few MB at most, so it
// is held entirely in the distributed shared memory of one thread-block
// cluster (up to 16 CTAs x 227 KB): CTA q owns a contiguous block of columns.
// The K pivot steps are inherently sequential; each costs one hardware cluster
// barrier:
//   1. every CTA publishes its best (largest remaining norm, smallest index)
//      column in its own shared memory;                 cluster barrier
//   2. every CTA reads the cluster's candidates and the winning column's
//      trailing part over DSMEM, and forms the same Householder reflection;
//   3. every CTA applies it to its active columns (a group of tpc lanes per
//      column, warp-shuffle reductions) and recomputes their trailing norms
//      exactly (no downdating, so no cancellation safeguard is needed).
// The pivot column itself is finalised one step later, after the next
// barrier, because other CTAs read it during the current step.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>

#include "common.cuh"
#include "cpqr_dev.cuh"
#include "internal.h"
#include "tsolve_dev.cuh"

namespace idl {

constexpr int kCpqrThreads = 1024;

template <typename T>
__global__ void __launch_bounds__(kCpqrThreads, 1)
cpqr_cluster_kernel(const T* __restrict__ Yin, T* __restrict__ Yout, int m, int R, int ld, int K, int nc, int lds,
                    int tpc, int32_t* __restrict__ J, double* __restrict__ rnorm, double* __restrict__ diag,
                    int* status, const int* gate) {
  if (proposal_certified(gate, diag)) return;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int c0 = rank * nc;
  const int ncl = max(0, min(nc, R - c0));
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int ngroups = blockDim.x / tpc, g = tid / tpc, gl = tid % tpc;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* cols = (T*)smem_raw;                           // nc * lds
  T* nrm2 = cols + (size_t)nc * lds;                // nc
  T* x = nrm2 + nc;                                 // m  (pivot column, rows t..)
  T* v = x + m;                                     // m  (Householder vector)
  Cand<T>* cand = (Cand<T>*)(v + m + 2);            // [2] published candidates (double-buffered)
  __shared__ T red_v[32];
  __shared__ int red_i[32];
  __shared__ int s_p, s_w;
  __shared__ T s_beta, s_alpha;
  __shared__ int active_bits[1];                    // unused placeholder to keep the layout obvious
  (void)active_bits;
  // active flag folded into nrm2: inactive columns get -1

  // ---- load my columns, initial norms ----
  for (int e = tid; e < ncl * m; e += blockDim.x) {
    const int c = e / m, i = e - c * m;
    cols[c * lds + i] = Yin[(int64_t)(c0 + c) * ld + i];
  }
  __syncthreads();
  double fro = 0.0;
  const int iters = (ncl + ngroups - 1) / ngroups;
  for (int it = 0; it < iters; ++it) {
    const int c = it * ngroups + g;
    T s = T(0);
    if (c < ncl)
      for (int i = gl; i < m; i += tpc) { const T y = cols[c * lds + i]; s += y * y; }
    s = group_sum(s, tpc);
    if (c < ncl && gl == 0) { nrm2[c] = s; fro += (double)s; }
  }
  if (gl == 0 && fro != 0.0) atomicAdd(&diag[1], fro);
  __syncthreads();

  int prev_pl = -1, prev_t = 0;
  T prev_alpha = T(0);
  for (int t = 0; t < K; ++t) {
    // 1. local candidate
    T bv = T(-1); int bi = -1;
    for (int c = tid; c < ncl; c += blockDim.x) {
      const T nv = nrm2[c];
      if (nv >= T(0) && better(nv, c0 + c, bv, bi)) { bv = nv; bi = c0 + c; }
    }
    for (int o = 16; o; o >>= 1) {
      const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (better(ov, oi, bv, bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { red_v[wid] = bv; red_i[wid] = bi; }
    __syncthreads();
    if (wid == 0) {
      const int nw = blockDim.x >> 5;
      bv = lane < nw ? red_v[lane] : T(-1);
      bi = lane < nw ? red_i[lane] : -1;
      for (int o = 16; o; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (better(ov, oi, bv, bi)) { bv = ov; bi = oi; }
      }
      if (lane == 0) { cand[t & 1].val = bv; cand[t & 1].idx = bi; }
    }
    cluster.sync();                                  // candidates (and pivot data) visible

    // finalise my pivot column of the previous step (nobody reads it any more)
    if (prev_pl >= 0) {
      for (int i = prev_t + tid; i < m; i += blockDim.x)
        cols[prev_pl * lds + i] = (i == prev_t) ? prev_alpha : T(0);
      prev_pl = -1;
    }
    // 2. cluster-wide winner
    if (wid == 0) {
      const int CS = (int)cluster.num_blocks();
      bv = T(-1); bi = -1; int bw = -1;
      if (lane < CS) {
        Cand<T>* rc = cluster.map_shared_rank(&cand[t & 1], (unsigned)lane);
        bv = rc->val; bi = rc->idx; bw = lane;
      }
      for (int o = 16; o; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        const int ow = __shfl_xor_sync(0xffffffffu, bw, o);
        if (better(ov, oi, bv, bi)) { bv = ov; bi = oi; bw = ow; }
      }
      if (lane == 0) { s_p = bi; s_w = bw; }
    }
    __syncthreads();
    const int p = s_p, w = s_w;
    if (p < 0) {
      // no finite remaining column (NaN/Inf input): every CTA sees the same p and
      // leaves the loop at the same step, so the cluster barriers stay matched
      if (rank == 0 && tid == 0) {
        for (int q = t; q < K; ++q) J[q] = -1;
        set_status(status, IDL_EDATA);
      }
      break;
    }
    const int pl = p - w * nc;
    {
      const T* rcol = cluster.map_shared_rank(cols, (unsigned)w) + (size_t)pl * lds;
      for (int i = t + tid; i < m; i += blockDim.x) x[i] = rcol[i];
    }
    __syncthreads();
    // 3. Householder reflection (every CTA computes the same one)
    if (wid == 0) {
      T s = T(0);
      for (int i = t + lane; i < m; i += 32) s += x[i] * x[i];
      s = warp_sum(s);
      const T nrm = sqrt(s);
      const T x0 = x[t];
      const T alpha = (x0 >= T(0)) ? -nrm : nrm;
      const T beta = (nrm > T(0)) ? T(1) / (nrm * (nrm + fabs(x0))) : T(0);
      for (int i = t + lane; i < m; i += 32) v[i] = (i == t) ? x0 - alpha : x[i];
      if (lane == 0) {
        s_alpha = alpha; s_beta = beta;
        if (rank == 0) {
          J[t] = p;
          if (rnorm) rnorm[t] = (double)fabs(alpha);
          if (t == 0) diag[3] = (double)fabs(alpha);
          if (t == K - 1) diag[4] = (double)fabs(alpha);
        }
      }
    }
    __syncthreads();
    const T beta = s_beta;
    if (w == rank && tid == 0) nrm2[pl] = T(-1);    // retire the pivot column
    if (w == rank) { prev_pl = pl; prev_t = t; prev_alpha = s_alpha; }
    __syncthreads();
    // 4. apply to active columns; recompute trailing norms exactly
    for (int it = 0; it < iters; ++it) {
      const int c = it * ngroups + g;
      const bool act = c < ncl && nrm2[c] >= T(0);
      T d = T(0);
      if (act)
        for (int i = t + gl; i < m; i += tpc) d += v[i] * cols[c * lds + i];
      d = group_sum(d, tpc) * beta;
      T s = T(0);
      if (act) {
        for (int i = t + gl; i < m; i += tpc) {
          const T y = cols[c * lds + i] - d * v[i];
          cols[c * lds + i] = y;
          if (i > t) s += y * y;
        }
      }
      s = group_sum(s, tpc);
      if (act && gl == 0) nrm2[c] = s;
    }
    __syncthreads();
  }
  cluster.sync();                                    // all DSMEM reads of the last step are done
  if (prev_pl >= 0) {
    for (int i = prev_t + tid; i < m; i += blockDim.x)
      cols[prev_pl * lds + i] = (i == prev_t) ? prev_alpha : T(0);
  }
  __syncthreads();
  // ||R22||_F^2 in FP64 over the non-pivot columns' rows K..m-1
  double r22 = 0.0;
  for (int it = 0; it < iters; ++it) {
    const int c = it * ngroups + g;
    double s = 0.0;
    if (c < ncl && nrm2[c] >= T(0))
      for (int i = K + gl; i < m; i += tpc) { const double y = (double)cols[c * lds + i]; s += y * y; }
    s = group_sum(s, tpc);
    if (gl == 0) r22 += s;
  }
  if (gl == 0 && r22 != 0.0) atomicAdd(&diag[0], r22);
  for (int e = tid; e < ncl * m; e += blockDim.x) {
    const int c = e / m, i = e - c * m;
    Yout[(int64_t)(c0 + c) * ld + i] = cols[c * lds + i];
  }
}

template <typename T, int V, int TPC>
__global__ void __launch_bounds__(RegCpqr<T, V, TPC>::kMaxThreads, 1)
cpqr_reg_kernel(const T* __restrict__ Yin, T* __restrict__ Yout, int m, int R, int ld, int K, int nc,
                int32_t* __restrict__ J, double* __restrict__ rnorm, double* __restrict__ diag, int* status,
                const int* gate, const int32_t* __restrict__ colmap, T* __restrict__ Vout, T* __restrict__ Bout,
                const int32_t* force) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (proposal_certified(gate, diag)) return;
  cpqr_reg_body<T, V, TPC>(Yin, Yout, m, R, ld, K, nc, J, rnorm, diag, status, smem_raw, colmap, Vout, Bout, force);
}

template <typename T, int V, int TPC>
static int try_reg_cpqr(idl_ctx* ctx, const T* Yin, T* Yout, int64_t m, int64_t R, int64_t ld, int64_t K, int32_t* J,
                        double* rnorm, int CS, int nc, const QrExtra& x, bool* launched) {
  constexpr int tpc = TPC;
  *launched = false;
  const int threads = (int)round_up((int64_t)nc * tpc, 32);
  if (threads > RegCpqr<T, V, TPC>::kMaxThreads || threads < 32) return IDL_OK;
  const size_t smem = reg_cpqr_smem<T, V, TPC>((int)m);
  if (smem > (size_t)ctx->smem_optin) return IDL_OK;
  auto kern = cpqr_reg_kernel<T, V, TPC>;
  cudaError_t e = ensure_cluster_nonportable(ctx, (const void*)kern);
  if (e == cudaSuccess) e = ensure_smem(ctx, (const void*)kern, smem);
  if (e != cudaSuccess) return cuda_check(ctx, e, "cpqr reg attribute");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CS);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  e = cluster_occupancy(ctx, (const void*)kern, cfg, &nclusters);
  if (e != cudaSuccess || nclusters < 1) { (void)cudaGetLastError(); return IDL_OK; }
  if (!x.colmap) ctx->last_cluster = CS;
  e = cudaLaunchKernelEx(&cfg, kern, Yin, Yout, (int)m, (int)R, (int)ld, (int)K, nc, J, rnorm,
                         x.diag ? x.diag : ctx->d_diag, ctx->d_status, x.gate, x.colmap, (T*)x.Vout, (T*)x.Bout,
                         x.force);
  idl::count_launch();
  *launched = true;
  return cuda_check(ctx, e, "cpqr reg launch");
}

// Largest cluster, then the first lane layout (reg_cpqr's order) whose register budget fits.
template <typename T, int V, int TPC>
static bool reg_try(idl_ctx* ctx, const T* Yin, T* Yout, int64_t m, int64_t R, int64_t ld, int64_t K, int32_t* J,
                    double* rnorm, int CS, int nc, const QrExtra& x, int* rc) {
  bool launched = false;
  if (cdiv(m, TPC) > V) return false;
  *rc = try_reg_cpqr<T, V, TPC>(ctx, Yin, Yout, m, R, ld, K, J, rnorm, CS, nc, x, &launched);
  return launched || *rc != IDL_OK;
}

template <typename T>
static int reg_cpqr(idl_ctx* ctx, const T* Yin, T* Yout, int64_t m, int64_t R, int64_t ld, int64_t K, int32_t* J,
                    double* rnorm, const QrExtra& x, bool* launched) {
  *launched = false;
  if (ctx->cpqr_smem_only && !x.colmap) return IDL_OK;
  int rc = IDL_OK;
  for (int CS = x.max_cs; CS >= 1; CS >>= 1) {
    const int nc = (int)cdiv(R, CS);
#define TRY_CFG(V, TPC) if (reg_try<T, V, TPC>(ctx, Yin, Yout, m, R, ld, K, J, rnorm, CS, nc, x, &rc)) { *launched = rc == IDL_OK; return rc; }
    // FP64: fewest lanes per column first.  GB300's FP64 pipe retires about two
    // lanes per clock per SM, so the per-step group reductions (log2 TPC adds on
    // all TPC lanes of a column) dominate when a column is spread over many lanes
    // (measured, 30 x 2000 sketch, 20 pivots: 431 us with 8 lanes per column,
    // 180 us with one lane and 32 values (some spilled), 156 us with two lanes).
    if constexpr (sizeof(T) == 8) { TRY_CFG(16, 1) TRY_CFG(16, 2) TRY_CFG(32, 1) TRY_CFG(32, 2) TRY_CFG(32, 4) }
    // FP32: one lane per column first as well -- fewer threads per CTA make the two
    // block barriers and candidate reductions of every step cheaper than the longer
    // per-column chain costs (measured: 60 x 1000 sketch, K = 50: 173 -> 148 us with
    // one lane and 64 values instead of 16 lanes and 8; 120 x 4096, K = 100:
    // 422 -> 388 us); then the most lanes per column
    if constexpr (sizeof(T) == 4) { TRY_CFG(16, 1) TRY_CFG(32, 1) TRY_CFG(64, 1) TRY_CFG(96, 1) TRY_CFG(128, 1) }
    TRY_CFG(8, 32) TRY_CFG(8, 16) TRY_CFG(8, 8) TRY_CFG(16, 8) TRY_CFG(8, 4) TRY_CFG(16, 4) TRY_CFG(32, 4)
    TRY_CFG(16, 2) TRY_CFG(32, 2) TRY_CFG(16, 1) TRY_CFG(32, 1)
    if constexpr (sizeof(T) == 4) { TRY_CFG(64, 4) TRY_CFG(64, 2) TRY_CFG(64, 1) TRY_CFG(96, 1) TRY_CFG(128, 1) }
#undef TRY_CFG
  }
  return IDL_OK;
}

template <typename T>
static int cpqr_impl(idl_ctx* ctx, const T* Yin, T* Yout, int64_t m, int64_t R, int64_t ld, int64_t K, int32_t* J,
                     double* rnorm, const QrExtra& x) {
  if (m > 256 || m < 1) return fail(ctx, IDL_ELIMIT, "cpqr: m must be in [1, 256]");
  {
    bool launched = false;
    const int rc = reg_cpqr<T>(ctx, Yin, Yout, m, R, ld, K, J, rnorm, x, &launched);
    if (rc != IDL_OK || launched) return rc;
  }
  if (x.colmap) return fail(ctx, IDL_ELIMIT, "cpqr: candidate set exceeds one CTA");
  if (x.force) return fail(ctx, IDL_ELIMIT, "cpqr: given pivots need the register-resident QR");
  auto kern = cpqr_cluster_kernel<T>;
  cudaError_t e = ensure_cluster_nonportable(ctx, (const void*)kern);
  if (e != cudaSuccess) return cuda_check(ctx, e, "cpqr cluster attribute");
  for (int CS = 16; CS >= 1; CS >>= 1) {
    const int nc = (int)cdiv(R, CS);
    const int threads = kCpqrThreads;
    int tpc = 1;
    while (tpc < 32 && (int64_t)nc * tpc * 2 <= threads && tpc * 2 <= m) tpc *= 2;
    int lds = (int)round_up(m, tpc);
    if (((lds / tpc) & 1) == 0) lds += tpc;
    const size_t smem = sizeof(T) * ((size_t)nc * lds + nc + 2 * m + 2) + sizeof(Cand<T>) * 2 + 16;
    if (smem > (size_t)ctx->smem_optin) {
      if (CS == 16) return fail(ctx, IDL_ELIMIT, "cpqr: sketch exceeds the cluster's shared memory");
      continue;
    }
    e = ensure_smem(ctx, (const void*)kern, smem);
    if (e != cudaSuccess) return cuda_check(ctx, e, "cpqr smem attribute");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CS);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    e = cluster_occupancy(ctx, (const void*)kern, cfg, &nclusters);
    if (e != cudaSuccess || nclusters < 1) { (void)cudaGetLastError(); continue; }
    ctx->last_cluster = CS;
    e = cudaLaunchKernelEx(&cfg, kern, Yin, Yout, (int)m, (int)R, (int)ld, (int)K, nc, lds, tpc, J, rnorm,
                           x.diag ? x.diag : ctx->d_diag, ctx->d_status, x.gate);
    idl::count_launch();
    return cuda_check(ctx, e, "cpqr launch");
  }
  return fail(ctx, IDL_ELIMIT, "cpqr: no cluster shape fits this device");
}

int launch_cpqr(idl_ctx* ctx, void* Y2, int64_t m, int64_t R, int64_t ld, int dtype, int64_t K, int32_t* J,
                double* rnorm) {
  const QrExtra x;
  if (dtype == IDL_F32) return cpqr_impl<float>(ctx, (const float*)Y2, (float*)Y2, m, R, ld, K, J, rnorm, x);
  return cpqr_impl<double>(ctx, (const double*)Y2, (double*)Y2, m, R, ld, K, J, rnorm, x);
}

int launch_cpqr_ex(idl_ctx* ctx, const float* Yin, float* Yout, int64_t m, int64_t R, int64_t ld, int64_t K,
                   int32_t* J, double* rnorm, const QrExtra& x) {
  return cpqr_impl<float>(ctx, Yin, Yout, m, R, ld, K, J, rnorm, x);
}

// ----------------------------------------------------------------------------
// Non-skeleton columns in ascending order, and T = R11^{-1} R12 (FP64).
// ----------------------------------------------------------------------------
__global__ void rest_kernel(const int32_t* __restrict__ J, int K, int R, int32_t* __restrict__ rest) {
  extern __shared__ int32_t sJ[];
  for (int q = threadIdx.x; q < K; q += blockDim.x) sJ[q] = J[q];
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < R) rest_elem(r, sJ, K, R, rest);
}

template <typename T>
__global__ void __launch_bounds__(256) rinv_kernel(const T* __restrict__ Y, int ld, int K, int R,
                                                   const int32_t* __restrict__ J, double* __restrict__ Rinv,
                                                   float* __restrict__ Rsplit) {
  extern __shared__ __align__(16) double U[];
  if constexpr (sizeof(T) == 4) rinv_block_df(Y, ld, K, R, J, Rsplit, blockIdx.x, gridDim.x, (float*)U);
  else rinv_block<T>(Y, ld, K, R, J, Rinv, blockIdx.x, gridDim.x, U, Rsplit);
}

__global__ void __launch_bounds__(256) tgemm_df_kernel(const float* __restrict__ Y, int ld, int K, int R,
                                                      const float* __restrict__ Rsplit, const int32_t* __restrict__ rest,
                                                      int nrest, double* __restrict__ Tout) {
  extern __shared__ __align__(16) float shf[];
  tgemm_block_df(Y, ld, K, R, Rsplit, rest, nrest, Tout, blockIdx.x, shf);
}

template <typename T>
__global__ void __launch_bounds__(256) tgemm_kernel(const T* __restrict__ Y, int ld, int K, int R,
                                                    const double* __restrict__ Rinv, const int32_t* __restrict__ rest,
                                                    int nrest, double* __restrict__ Tout) {
  extern __shared__ __align__(16) double sh[];
  tgemm_block<T>(Y, ld, K, R, Rinv, rest, nrest, Tout, blockIdx.x, sh);
}

int launch_t_solve(idl_ctx* ctx, const void* Y2, int64_t m, int64_t R, int64_t ld, int dtype, int64_t K,
                   const int32_t* J, double* T, int32_t* rest) {
  (void)m;
  if (K > kSolveMaxK) return fail(ctx, IDL_ELIMIT, "t_solve: K > 128");
  const int64_t nrest = R - K;
  if (!rest) {
    rest = (int32_t*)ws_get(ctx, kWsRest, sizeof(int32_t) * (size_t)(R > 0 ? R : 1));
    if (!rest) return IDL_ENOMEM;
  }
  // inv(R11): FP64 (FP64 data) or FP32 pairs (FP32 data)
  double* Rinv = (double*)ws_get(ctx, kWsRinv, 2 * sizeof(double) * (size_t)(K * K));
  if (!Rinv) return IDL_ENOMEM;
  float* Rsplit = (float*)(Rinv + K * K);
  rest_kernel<<<(unsigned)cdiv(R, 256), 256, sizeof(int32_t) * (size_t)K, ctx->stream>>>(J, (int)K, (int)R, rest),
      idl::count_launch();
  const size_t smem_inv = sizeof(double) * (size_t)K * (K + 1);
  const size_t smem_t = sizeof(double) * ((size_t)K * K + (size_t)K * (kTNB + 1)) + sizeof(int) * kTNB;
  const size_t smem_df = sizeof(float) * (size_t)tgemm_df_floats((int)K);
  const unsigned inv_blocks = (unsigned)cdiv(K, kRinvWarps);   // one warp per column
  const unsigned inv_blocks_df = (unsigned)cdiv(K, kRinvWarpsDf);
  cudaError_t e;
  if (dtype == IDL_F32) {
    e = ensure_smem(ctx, (const void*)rinv_kernel<float>, smem_inv);
    if (e == cudaSuccess) e = ensure_smem(ctx, (const void*)tgemm_df_kernel, smem_df);
    if (e == cudaSuccess) {
      rinv_kernel<float><<<inv_blocks_df, 32 * kRinvWarpsDf, smem_inv, ctx->stream>>>((const float*)Y2, (int)ld, (int)K,
                                                                                (int)R, J, Rinv, Rsplit),
          idl::count_launch();
      if (nrest > 0)
        tgemm_df_kernel<<<(unsigned)cdiv(nrest, kTNBdf), 256, smem_df, ctx->stream>>>(
            (const float*)Y2, (int)ld, (int)K, (int)R, Rsplit, rest, (int)nrest, T), idl::count_launch();
    }
  } else {
    e = ensure_smem(ctx, (const void*)rinv_kernel<double>, smem_inv);
    if (e == cudaSuccess) e = ensure_smem(ctx, (const void*)tgemm_kernel<double>, smem_t);
    if (e == cudaSuccess) {
      rinv_kernel<double><<<inv_blocks, 32 * kRinvWarps, smem_inv, ctx->stream>>>((const double*)Y2, (int)ld, (int)K,
                                                                                 (int)R, J, Rinv, nullptr),
          idl::count_launch();
      if (nrest > 0)
        tgemm_kernel<double><<<(unsigned)cdiv(nrest, kTNB), 256, smem_t, ctx->stream>>>(
            (const double*)Y2, (int)ld, (int)K, (int)R, Rinv, rest, (int)nrest, T), idl::count_launch();
    }
  }
  if (e != cudaSuccess) return cuda_check(ctx, e, "t_solve attribute");
  return cuda_check(ctx, cudaGetLastError(), "t_solve");
}

// ----------------------------------------------------------------------------
// Explicit FP64 residual  sum_c ||Y2[:, rest_c] - Y2[:, J] T[:, c]||^2  (from the
// unfactored sketch), accumulated into diag[2].
// ----------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) residual_kernel(const T* __restrict__ Y, int m, int ld, int K, int R,
                                                       const int32_t* __restrict__ J, const double* __restrict__ Tm,
                                                       const int32_t* __restrict__ rest, int nrest,
                                                       double* __restrict__ diag) {
  extern __shared__ __align__(16) double yj[];      // m x K  (Y2[:, J])
  for (int e = threadIdx.x; e < m * K; e += blockDim.x) {
    const int k = e / m, i = e - k * m;
    const int jj = J[k];
    yj[i * K + k] = (jj >= 0 && jj < R) ? (double)Y[(int64_t)jj * ld + i] : 0.0;
  }
  __syncthreads();
  double acc = 0.0;
  // one warp per column, lanes over rows
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = blockIdx.x * nw + wid; c < nrest; c += gridDim.x * nw) {
    const int r = rest[c];
    if (r < 0 || r >= R) continue;
    for (int i = lane; i < m; i += 32) {
      double y = (double)Y[(int64_t)r * ld + i];
      for (int k = 0; k < K; ++k) y -= yj[i * K + k] * Tm[(int64_t)k * nrest + c];
      acc += y * y;
    }
  }
  acc = warp_sum(acc);
  if (lane == 0 && acc != 0.0) atomicAdd(&diag[2], acc);
}

int launch_residual(idl_ctx* ctx, const void* Y2orig, const void* Y2fact, int64_t m, int64_t R, int64_t ld,
                    int dtype, int64_t K, const int32_t* J, const double* T, const int32_t* rest) {
  (void)Y2fact;
  const int64_t nrest = R - K;
  if (nrest <= 0) return IDL_OK;
  const size_t smem = sizeof(double) * (size_t)m * K;
  if (smem > (size_t)ctx->smem_optin) return fail(ctx, IDL_ELIMIT, "residual: m*K too large");
  const int blocks = (int)std::min<int64_t>(cdiv(nrest, 8), 4 * ctx->num_sms);
  cudaError_t e;
  if (dtype == IDL_F32) {
    e = ensure_smem(ctx, (const void*)residual_kernel<float>, smem);
    if (e == cudaSuccess)
      residual_kernel<float><<<blocks, 256, smem, ctx->stream>>>((const float*)Y2orig, (int)m, (int)ld, (int)K, (int)R, J, T,
                                                                 rest, (int)nrest, ctx->d_diag), idl::count_launch();
  } else {
    e = ensure_smem(ctx, (const void*)residual_kernel<double>, smem);
    if (e == cudaSuccess)
      residual_kernel<double><<<blocks, 256, smem, ctx->stream>>>((const double*)Y2orig, (int)m, (int)ld, (int)K, (int)R, J,
                                                                  T, rest, (int)nrest, ctx->d_diag), idl::count_launch();
  }
  if (e != cudaSuccess) return cuda_check(ctx, e, "residual attribute");
  return cuda_check(ctx, cudaGetLastError(), "residual");
}

// ----------------------------------------------------------------------------
// lambda_hat_k = lambda_{J_k} (1 + sum_c T_kc)  (Algorithm 3)
// ----------------------------------------------------------------------------
__global__ void lambda_hat_kernel(const double* __restrict__ lam, const int32_t* __restrict__ J,
                                  const double* __restrict__ Tm, int nrest, double* __restrict__ out) {
  lambda_hat_block(lam, J, Tm, nrest, (int)gridDim.x, out, blockIdx.x);
}

int launch_lambda_hat(idl_ctx* ctx, const double* lambda, const int32_t* J, const double* T, int64_t K, int64_t R,
                      double* lambda_hat) {
  if (K <= 0) return IDL_OK;
  lambda_hat_kernel<<<(unsigned)K, 256, 0, ctx->stream>>>(lambda, J, T, (int)(R - K), lambda_hat), idl::count_launch();
  return cuda_check(ctx, cudaGetLastError(), "lambda_hat");
}

// ----------------------------------------------------------------------------
// Row-major m x R  ->  column-major (R columns of ldy2), for m2 = 0.
// ----------------------------------------------------------------------------
template <typename T>
__global__ void transpose_kernel(const T* __restrict__ A, int64_t m, int64_t R, int64_t lda, T* __restrict__ B,
                                 int64_t ldb) {
  __shared__ T tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32, i0 = (int64_t)blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t i = i0 + y, r = r0 + threadIdx.x;
    if (i < m && r < R) tile[y][threadIdx.x] = A[i * lda + r];
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t r = r0 + y, i = i0 + threadIdx.x;
    if (i < m && r < R) B[r * ldb + i] = tile[threadIdx.x][y];
  }
}

int launch_transpose_to_colmajor(idl_ctx* ctx, const void* Y1, int64_t m, int64_t R, int64_t ldy1, int dtype,
                                 void* Y2, int64_t ldy2) {
  dim3 grid((unsigned)cdiv(R, 32), (unsigned)cdiv(m, 32));
  dim3 block(32, 8);
  if (dtype == IDL_F32)
    transpose_kernel<float><<<grid, block, 0, ctx->stream>>>((const float*)Y1, m, R, ldy1, (float*)Y2, ldy2), idl::count_launch();
  else
    transpose_kernel<double><<<grid, block, 0, ctx->stream>>>((const double*)Y1, m, R, ldy1, (double*)Y2, ldy2), idl::count_launch();
  return cuda_check(ctx, cudaGetLastError(), "transpose");
}

}  // namespace idl

// ----------------------------------------------------------------------------
// Strong rank-revealing refinement (Fact 1; Gu & Eisenstat 1996): with the
// factored sketch of the current selection J (R11 on J's columns, R12 and R22 on
// the rest) and W = T = R11^{-1} R12 from the T solve, rho_ij = W_ij^2 +
// gamma_j^2 ||e_i^T R11^{-1}||^2 (gamma_j = ||R22 e_j||); while the largest rho
// exceeds f^2, J[i] is exchanged for rest[j] (ties: smallest i, then j) and the
// sketch is factored again with J as given pivots.  Each exchange multiplies
// |det R11| by sqrt(rho) > f.
// ----------------------------------------------------------------------------
namespace idl {

constexpr int kSrrqrMaxSwaps = 256;

// winv2[i] = ||e_i^T R11^{-1}||^2: row i of the inverse by forward substitution
// (r R11 = e_i), one warp per row, FP64
template <typename T>
__global__ void srrqr_rinv_rows_kernel(const T* __restrict__ Yf, int64_t ld, int K, const int32_t* __restrict__ J,
                                       double* __restrict__ rowbuf, double* __restrict__ winv2) {
  const int i = blockIdx.x, lane = threadIdx.x;
  double* r = rowbuf + (int64_t)i * K;                   // r[l], l >= i
  double s2 = 0.0;
  for (int j = i; j < K; ++j) {
    const T* col = Yf + (int64_t)J[j] * ld;              // column j of R11: rows 0..j
    double acc = 0.0;
    for (int l = i + lane; l < j; l += 32) acc += r[l] * (double)col[l];
    acc = warp_sum(acc);
    const double v = ((j == i ? 1.0 : 0.0) - acc) / (double)col[j];
    if (lane == 0) r[j] = v;
    __syncwarp();
    s2 += v * v;
  }
  if (lane == 0) winv2[i] = s2;
}

// gam2[c] = ||R22 e_c||^2 over rows K..m-1 of the non-skeleton column rest[c]
template <typename T>
__global__ void srrqr_gamma_kernel(const T* __restrict__ Yf, int64_t ld, int m, int K,
                                   const int32_t* __restrict__ rest, int nr, double* __restrict__ gam2) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nr) return;
  const T* col = Yf + (int64_t)rest[c] * ld;
  double s = 0.0;
  for (int l = K; l < m; ++l) { const double y = (double)col[l]; s += y * y; }
  gam2[c] = s;
}

// key = max over (i, c) of (FP32 bits of rho_ic) << 32 | (~(i nr + c)): the largest rho,
// then the smallest flat index
__global__ void srrqr_argmax_kernel(const double* __restrict__ T, const double* __restrict__ winv2,
                                    const double* __restrict__ gam2, int K, int nr,
                                    unsigned long long* __restrict__ key) {
  unsigned long long best = 0ull;
  const int64_t tot = (int64_t)K * nr;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / nr), c = (int)(e - (int64_t)i * nr);
    const double w = T[e];
    const float rho = (float)(w * w + gam2[c] * winv2[i]);
    const unsigned long long k = ((unsigned long long)__float_as_uint(rho) << 32) | (0xffffffffu - (unsigned)e);
    best = k > best ? k : best;
  }
  for (int o = 16; o; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
    best = v > best ? v : best;
  }
  if ((threadIdx.x & 31) == 0 && best) atomicMax(key, best);
}

// the exchange (flag = 1) or the end (flag = 0)
__global__ void srrqr_swap_kernel(const unsigned long long* __restrict__ key, const int32_t* __restrict__ rest, int nr,
                                  float f2, int32_t* __restrict__ J, int* __restrict__ flag) {
  const unsigned long long k = *key;
  const float rho = __uint_as_float((unsigned)(k >> 32));
  const unsigned e = 0xffffffffu - (unsigned)(k & 0xffffffffull);
  if (!(rho > f2) || k == 0ull) { *flag = 0; return; }
  const unsigned i = e / (unsigned)nr, c = e - i * (unsigned)nr;
  J[i] = rest[c];
  *flag = 1;
}

int launch_srrqr(idl_ctx* ctx, const void* Yorig, void* Yf, int64_t m, int64_t R, int64_t ld, int dtype, int64_t K,
                 int32_t* J, double* T, int32_t* rest, float f) {
  const int nr = (int)(R - K);
  unsigned char* ws = (unsigned char*)ws_get(ctx, kWsSrrqr,
                                             sizeof(double) * (size_t)(K * K + K + nr) + 2 * sizeof(unsigned long long));
  if (!ws) return IDL_ENOMEM;
  double* rowbuf = (double*)ws;
  double* winv2 = rowbuf + K * K;
  double* gam2 = winv2 + K;
  unsigned long long* key = (unsigned long long*)(gam2 + nr);
  int* flag = (int*)(key + 1);
  QrExtra x;
  x.force = J;
  for (int s = 0; s <= kSrrqrMaxSwaps; ++s) {
    int rc = launch_t_solve(ctx, Yf, m, R, ld, dtype, K, J, T, rest);
    if (rc != IDL_OK) return rc;
    if (s == kSrrqrMaxSwaps) break;
    cudaStream_t st = ctx->stream;
    if (dtype == IDL_F32) {
      srrqr_rinv_rows_kernel<float><<<(unsigned)K, 32, 0, st>>>((const float*)Yf, ld, (int)K, J, rowbuf, winv2);
      srrqr_gamma_kernel<float><<<(unsigned)cdiv(nr, 256), 256, 0, st>>>((const float*)Yf, ld, (int)m, (int)K, rest,
                                                                         nr, gam2);
    } else {
      srrqr_rinv_rows_kernel<double><<<(unsigned)K, 32, 0, st>>>((const double*)Yf, ld, (int)K, J, rowbuf, winv2);
      srrqr_gamma_kernel<double><<<(unsigned)cdiv(nr, 256), 256, 0, st>>>((const double*)Yf, ld, (int)m, (int)K, rest,
                                                                          nr, gam2);
    }
    idl::count_launch();
    idl::count_launch();
    cudaMemsetAsync(key, 0, sizeof(unsigned long long), st);
    srrqr_argmax_kernel<<<(unsigned)std::min<int64_t>(cdiv((int64_t)K * nr, 256), 4LL * ctx->num_sms), 256, 0, st>>>(
        T, winv2, gam2, (int)K, nr, key), idl::count_launch();
    srrqr_swap_kernel<<<1, 1, 0, st>>>(key, rest, nr, f * f, J, flag), idl::count_launch();
    int hflag = 0;
    cudaError_t e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_check(ctx, e, "srrqr");
    if (!hflag) return IDL_OK;
    // factor the sketch again with the exchanged selection as given pivots
    e = cudaMemsetAsync(ctx->d_diag, 0, sizeof(double) * 16, st);
    if (e != cudaSuccess) return cuda_check(ctx, e, "srrqr");
    rc = dtype == IDL_F32 ? cpqr_impl<float>(ctx, (const float*)Yorig, (float*)Yf, m, R, ld, K, J, nullptr, x)
                          : cpqr_impl<double>(ctx, (const double*)Yorig, (double*)Yf, m, R, ld, K, J, nullptr, x);
    if (rc != IDL_OK) return rc;
  }
  return IDL_OK;
}

}  // namespace idl
