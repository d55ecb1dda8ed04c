// proposal_dev.cuh -- device bodies of the learned column proposal for the
// pivoted QR stage, shared by proposal.cu (one problem) and batch.cu.
//
// The QR stage of Algorithm 1 takes K pivots greedily by remaining column norm
// over all R columns of the small sketch Y (m x R): K dependent steps, each a
// cluster-wide argmax.  The proposal path instead
//   1. scores every column: features (norms and ridge leverage scores of the
//      sketch) through a 3-layer MLP of width 128 with bfloat16 operands;
//   2. keeps the C = min(2K, R) best columns (ties: smaller index);
//   3. runs the same pivoted QR on those C columns in one CTA, recording its
//      Householder reflectors;
//   4. applies the reflectors to every other column in parallel and checks the
//      certificate: each outside column's remaining norm before step t stays
//      below that step's pivot norm |r_tt|, for all t < K.  Then the QR of all
//      R columns would take the same pivots in the same order, and its factor
//      rows 0..K-1 equal the ones computed here;
//   5. otherwise the plain QR runs (a gated launch that exits at once when the
//      certificate holds).
// Features of column c (n_c = ||y_c||^2, G = Y Y^T, lambda_q = rho_q tr(G)/m):
//   f0 = max(log(n_c / max n), -64)/16, f1 = sqrt(n_c / max n),
//   f2..f4 = y_c^T (G + lambda_q I)^{-1} y_c for rho = 1e-1, 1e-2, 1e-3,
//   f5 = max_i |y_ic| / sqrt(n_c), f6 = K/R, f7 = m/R.
// The ridge leverage scores use the Cholesky factor L of G + lambda I and its
// explicit inverse: y^T (L L^T)^{-1} y = ||L^{-1} y||^2, a matrix-vector
// product per column with no sequential dependence between columns.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace idl {
namespace prop {

constexpr int kNF = 8, kHid = 128;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kHid * kNF;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid;
constexpr int kOffB3 = kOffW3 + kHid;
constexpr int kNParam = kOffB3 + 1;
static_assert(kNParam == IDL_MLP_NPARAM, "parameter layout");

constexpr int kMaxM = 128;         // sketch rows the proposal path handles
constexpr int kThreads = 256;      // block size of every proposal kernel but the selection
constexpr int kGramCols = 64;      // columns per Gram partial
constexpr int kFeatCols = 32;      // columns per feature block
constexpr int kTile = 128;         // examples per MLP block
constexpr int kLD = kTile + 1;     // odd leading dimension of the MLP's shared tiles
constexpr int kSelThreads = 1024;
constexpr int kApplyThreads = 256;
// The certificate compares squared norms computed in FP32 on both sides; a
// relative margin keeps a near tie (which the plain QR might resolve either
// way after rounding) on the fallback side.
constexpr float kCertMargin = 0.9999f;

__device__ __forceinline__ float ridge(int q) { return q == 0 ? 1e-1f : (q == 1 ? 1e-2f : 1e-3f); }
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// ---------------------------------------------------------------------------
// Gram partial: Gp[blk] = sum over this block's columns of y y^T (full m x m,
// both triangles of the diagonal tiles; the consumer reads i <= j), and the
// block's largest column norm^2.  4x4 register tiles of the upper triangle.
// smem: 32 * round_up(m, 4) floats.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void gram_partial_block(const float* __restrict__ Y, int ld, int m, int R, int blk,
                                                   float* __restrict__ Gp, float* __restrict__ nmaxp, float* smem) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int TB = (m + 3) >> 2, MP = TB * 4;
  const int ntile = TB * (TB + 1) / 2;
  const int c0 = blk * kGramCols, c1 = min(R, c0 + kGramCols);
  float* Ys = smem;                                         // [32][MP]
  __shared__ float red[32];
  constexpr int kMaxTiles = 3;                              // ceil(528 / 256) for m <= 128
  int ta[kMaxTiles], tb[kMaxTiles];
#pragma unroll
  for (int q = 0; q < kMaxTiles; ++q) {
    int e = tid + q * blockDim.x, a = 0;
    if (e < ntile) {
      while (e >= TB - a) { e -= TB - a; ++a; }
      ta[q] = a;
      tb[q] = a + e;
    } else {
      ta[q] = tb[q] = -1;
    }
  }
  float acc[kMaxTiles][16];
#pragma unroll
  for (int q = 0; q < kMaxTiles; ++q)
#pragma unroll
    for (int r = 0; r < 16; ++r) acc[q][r] = 0.f;
  float nmax = 0.f;
  for (int cc = c0; cc < c1; cc += 32) {
    const int nc = min(32, c1 - cc);
    for (int e = tid; e < 32 * MP; e += blockDim.x) {
      const int c = e / MP, i = e - c * MP;
      Ys[e] = (c < nc && i < m) ? Y[(int64_t)(cc + c) * ld + i] : 0.f;
    }
    __syncthreads();
    for (int c = wid; c < nc; c += nw) {
      float s = 0.f;
      for (int i = lane; i < m; i += 32) s = fmaf(Ys[c * MP + i], Ys[c * MP + i], s);
      s = warp_sum(s);
      nmax = fmaxf(nmax, s);
    }
#pragma unroll
    for (int q = 0; q < kMaxTiles; ++q) {
      if (ta[q] < 0) continue;
      for (int c = 0; c < nc; ++c) {
        const float4 x = *reinterpret_cast<const float4*>(Ys + c * MP + 4 * ta[q]);
        const float4 y = *reinterpret_cast<const float4*>(Ys + c * MP + 4 * tb[q]);
        const float xv[4] = {x.x, x.y, x.z, x.w}, yv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int s = 0; s < 4; ++s) acc[q][r * 4 + s] = fmaf(xv[r], yv[s], acc[q][r * 4 + s]);
      }
    }
    __syncthreads();
  }
  float* G = Gp + (int64_t)blk * m * m;
#pragma unroll
  for (int q = 0; q < kMaxTiles; ++q) {
    if (ta[q] < 0) continue;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int i = 4 * ta[q] + r, j = 4 * tb[q] + s;
        if (i < m && j < m) G[i * m + j] = acc[q][r * 4 + s];
      }
  }
  if (lane == 0) red[wid] = nmax;
  __syncthreads();
  if (tid == 0) {
    float v = 0.f;
    for (int w = 0; w < nw; ++w) v = fmaxf(v, red[w]);
    nmaxp[blk] = v;
  }
}

// ---------------------------------------------------------------------------
// G = the sum of the nsplit Gram partials in a fixed order (deterministic), one
// thread per entry; entry 0 also reduces the largest column norm into scal[0].
// ---------------------------------------------------------------------------
__device__ __forceinline__ void gram_reduce_elem(const float* __restrict__ Gp, int nsplit,
                                                 const float* __restrict__ nmaxp, int m, int e, float* __restrict__ G,
                                                 float* __restrict__ scal) {
  if (e >= m * m) return;
  float s = 0.f;
  for (int p = 0; p < nsplit; ++p) s += Gp[(int64_t)p * m * m + e];
  G[e] = s;
  if (e == 0) {
    float nm = 0.f;
    for (int p = 0; p < nsplit; ++p) nm = fmaxf(nm, nmaxp[p]);
    scal[0] = nm;
  }
}

// ---------------------------------------------------------------------------
// Cholesky factor of G + lambda_q I and its inverse (block q of three, 256
// threads).  Reads the upper triangle of G (m x m row-major).  Writes Linv[q]
// (m x m row-major, lower triangular); block 0 also writes scal[1] = tr(G).
// A zero (or non-finite) trace gives a zero Linv, i.e. zero leverage features.
// smem: 2 * m * (m + 1) + m floats.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void chol_inv_block(const float* __restrict__ G, int m, int q, float* __restrict__ Linv,
                                               float* __restrict__ scal, float* smem) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ld = m + 1;
  float* M = smem;
  float* X = M + m * ld;
  float* D = X + m * ld;
  __shared__ float s_tr;
  for (int e = tid; e < m * m; e += nt) {
    const int i = e / m, j = e - i * m;
    if (i <= j) {
      const float v = G[e];
      M[i * ld + j] = v;
      M[j * ld + i] = v;
    }
  }
  __syncthreads();
  if (tid == 0) {
    float tr = 0.f;
    for (int i = 0; i < m; ++i) tr += M[i * ld + i];
    s_tr = tr;
    if (q == 0) scal[1] = tr;
  }
  __syncthreads();
  const float tr = s_tr;
  float* Lq = Linv + (int64_t)q * m * m;
  if (!(tr > 0.f) || !isfinite(tr)) {
    for (int e = tid; e < m * m; e += nt) Lq[e] = 0.f;
    return;
  }
  const float lam = ridge(q) * tr / (float)m;
  for (int i = tid; i < m; i += nt) M[i * ld + i] += lam;
  __syncthreads();
  // right-looking elimination on the lower triangle with the unscaled pivot
  // column, M_ik -= M_ij M_kj / M_jj (j < k <= i), threads on a 16 x 16 grid of
  // (i, k) residues; column j is not written in step j: one barrier per step
  const int r0 = tid >> 4, c0 = tid & 15;
  for (int j = 0; j < m - 1; ++j) {
    const float rinv = 1.f / fmaxf(M[j * ld + j], lam * 1e-6f);
    for (int i = j + 1 + r0; i < m; i += 16) {
      const float a = M[i * ld + j] * rinv;
      for (int k = j + 1 + c0; k <= i; k += 16) M[i * ld + k] = fmaf(-a, M[k * ld + j], M[i * ld + k]);
    }
    __syncthreads();
  }
  for (int j = tid; j < m; j += nt) D[j] = sqrtf(fmaxf(M[j * ld + j], lam * 1e-6f));
  __syncthreads();
  for (int e = tid; e < m * m; e += nt) {
    const int i = e / m, j = e - i * m;
    if (j < i) M[i * ld + j] /= D[j];
  }
  for (int j = tid; j < m; j += nt) M[j * ld + j] = D[j];
  __syncthreads();
  // X = L^{-1}: thread j forms column j by forward substitution (four partial sums)
  for (int j = tid; j < m; j += nt) {
    for (int i = 0; i < j; ++i) X[i * ld + j] = 0.f;
    for (int i = j; i < m; ++i) {
      float a0 = (i == j) ? 1.f : 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
      int k = j;
      for (; k + 3 < i; k += 4) {
        a0 = fmaf(-M[i * ld + k], X[k * ld + j], a0);
        a1 = fmaf(-M[i * ld + k + 1], X[(k + 1) * ld + j], a1);
        a2 = fmaf(-M[i * ld + k + 2], X[(k + 2) * ld + j], a2);
        a3 = fmaf(-M[i * ld + k + 3], X[(k + 3) * ld + j], a3);
      }
      for (; k < i; ++k) a0 = fmaf(-M[i * ld + k], X[k * ld + j], a0);
      X[i * ld + j] = ((a0 + a1) + (a2 + a3)) / M[i * ld + i];
    }
  }
  __syncthreads();
  for (int e = tid; e < m * m; e += nt) {
    const int i = e / m, j = e - i * m;
    Lq[e] = X[i * ld + j];
  }
}

// ---------------------------------------------------------------------------
// Features of columns [blk*32, blk*32 + 32): F row-major R x 8 (FP32).
// The leverage scores ||L_q^{-1} y_c||^2 come from W = L_q^{-1} Y_blk, a
// register-tiled product: thread (ti, tc) of a 32 x 8 grid owns rows ti + 32 u
// and columns tc + 8 v; partial column sums of W^2 meet in shared memory.
// Small column blocks keep many blocks in flight (the kernel is latency-bound
// for the sketch sizes of the QR stage).  smem: features_smem_floats(m).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr size_t features_smem_floats(int m) {
  return (size_t)m * (m + 1) + (size_t)kFeatCols * (m + 1) + 32 * (size_t)kFeatCols + 3 * (size_t)kFeatCols;
}

__device__ __forceinline__ void features_block(const float* __restrict__ Y, int ld, int m, int R, int K,
                                               const float* __restrict__ Linv, const float* __restrict__ scal, int blk,
                                               float* __restrict__ F, float* smem) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int lds = m + 1;
  float* Ls = smem;                                    // m x (m+1)
  float* Yc = Ls + m * lds;                            // kFeatCols x (m+1)
  float* part = Yc + kFeatCols * lds;                  // 32 x kFeatCols
  float* Lev = part + 32 * kFeatCols;                  // kFeatCols x 3
  const int c0 = blk * kFeatCols;
  const int nc = min(kFeatCols, R - c0);
  for (int e = tid; e < kFeatCols * m; e += blockDim.x) {
    const int c = e / m, i = e - c * m;
    Yc[c * lds + i] = c < nc ? Y[(int64_t)(c0 + c) * ld + i] : 0.f;
  }
  const int ti = tid >> 3, tc = tid & 7;
  for (int q = 0; q < 3; ++q) {
    __syncthreads();
    for (int e = tid; e < m * m; e += blockDim.x) {
      const int i = e / m, j = e - i * m;
      Ls[i * lds + j] = Linv[(int64_t)q * m * m + e];
    }
    __syncthreads();
    float acc[kMaxM / 32][4];
#pragma unroll
    for (int u = 0; u < kMaxM / 32; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
    for (int k = 0; k < m; ++k) {
      float b[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) b[v] = Yc[(tc + 8 * v) * lds + k];
#pragma unroll
      for (int u = 0; u < kMaxM / 32; ++u) {
        const int i = ti + 32 * u;
        if (i < m) {
          const float a = Ls[i * lds + k];
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a, b[v], acc[u][v]);
        }
      }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      float sq = 0.f;
#pragma unroll
      for (int u = 0; u < kMaxM / 32; ++u) sq = fmaf(acc[u][v], acc[u][v], sq);
      part[ti * kFeatCols + tc + 8 * v] = sq;
    }
    __syncthreads();
    for (int c = tid; c < kFeatCols; c += blockDim.x) {
      float sq = 0.f;
      for (int r = 0; r < 32; ++r) sq += part[r * kFeatCols + c];
      Lev[c * 3 + q] = sq;
    }
  }
  __syncthreads();
  const float nmax = scal[0];
  for (int c = wid; c < nc; c += nw) {
    const float* y = Yc + c * lds;
    float n2 = 0.f, am = 0.f;
    for (int i = lane; i < m; i += 32) {
      n2 = fmaf(y[i], y[i], n2);
      am = fmaxf(am, fabsf(y[i]));
    }
    n2 = warp_sum(n2);
#pragma unroll
    for (int o = 16; o; o >>= 1) am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
    if (lane == 0) {
      float* f = F + (int64_t)(c0 + c) * kNF;
      const bool pos = nmax > 0.f && n2 > 0.f;
      f[0] = pos ? fmaxf(logf(n2 / nmax), -64.f) * (1.f / 16.f) : -4.f;
      f[1] = nmax > 0.f ? sqrtf(n2 / nmax) : 0.f;
      f[2] = Lev[c * 3 + 0];
      f[3] = Lev[c * 3 + 1];
      f[4] = Lev[c * 3 + 2];
      f[5] = n2 > 0.f ? am / sqrtf(n2) : 0.f;
      f[6] = (float)K / (float)R;
      f[7] = (float)m / (float)R;
    }
  }
}

// Norm-heuristic ablation: score = ||y_c||^2 (one warp per column).
__device__ __forceinline__ void norm_scores_warp(const float* __restrict__ Y, int ld, int m, int c, float* __restrict__ s) {
  const int lane = threadIdx.x & 31;
  float v = 0.f;
  for (int i = lane; i < m; i += 32) {
    const float y = Y[(int64_t)c * ld + i];
    v = fmaf(y, y, v);
  }
  v = warp_sum(v);
  if (lane == 0) s[c] = v;
}

// ---------------------------------------------------------------------------
// MLP.  Shared tiles (floats): W2 [h][k] and Z1 [e][k] with leading dimension
// 129, so that a thread owning rows {ti + 16 r} and columns {tj + 16 c} reads
// conflict-free.  Operands are rounded to bfloat16 (round to nearest even) as
// they are staged; products are exact in FP32 and accumulate in FP32.
// ---------------------------------------------------------------------------
struct MlpSmem {
  float* W2; float* Z1; float* DA; float* W1; float* Fs; float* b1; float* b2; float* w3; float* red;
};
constexpr size_t mlp_fwd_smem_floats() { return 2 * (size_t)kHid * kLD + 2 * kHid * kNF + 3 * kHid; }
constexpr size_t mlp_bwd_smem_floats() { return 3 * (size_t)kHid * kLD + 2 * kHid * kNF + 3 * kHid + 16 * kHid + 2 * kTile; }

__device__ __forceinline__ MlpSmem mlp_carve(float* smem, bool bwd) {
  MlpSmem s;
  s.W2 = smem;
  s.Z1 = s.W2 + kHid * kLD;
  s.DA = bwd ? s.Z1 + kTile * kLD : nullptr;
  s.W1 = (bwd ? s.DA + kTile * kLD : s.Z1 + kTile * kLD);
  s.Fs = s.W1 + kHid * kNF;
  s.b1 = s.Fs + kTile * kNF;
  s.b2 = s.b1 + kHid;
  s.w3 = s.b2 + kHid;
  s.red = s.w3 + kHid;             // bwd: 16 x kHid partial sums, then ds[kTile], y[kTile]
  return s;
}

// Stages weights and the tile's features, then layer 1 into Z1 (bf16-rounded).
__device__ __forceinline__ void mlp_stage_and_layer1(const float* __restrict__ theta, const float* __restrict__ F,
                                                     int64_t n, int64_t e0, const MlpSmem& s) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < kHid * kHid; e += nt) {
    const int h = e >> 7, k = e & 127;
    s.W2[h * kLD + k] = bf16r(theta[kOffW2 + e]);
  }
  for (int e = tid; e < kHid * kNF; e += nt) {
    s.W1[e] = bf16r(theta[kOffW1 + e]);
    const int ex = e / kNF;
    s.Fs[e] = (e0 + ex < n) ? bf16r(F[(e0 + ex) * kNF + (e - ex * kNF)]) : 0.f;
  }
  for (int h = tid; h < kHid; h += nt) {
    s.b1[h] = theta[kOffB1 + h];
    s.b2[h] = theta[kOffB2 + h];
    s.w3[h] = bf16r(theta[kOffW3 + h]);
  }
  __syncthreads();
  for (int e = tid; e < kTile * kHid; e += nt) {
    const int ex = e >> 7, h = e & 127;
    float a = 0.f;
#pragma unroll
    for (int f = 0; f < kNF; ++f) a = fmaf(s.W1[h * kNF + f], s.Fs[ex * kNF + f], a);
    a += s.b1[h];
    s.Z1[ex * kLD + h] = bf16r(fmaxf(a, 0.f));
  }
  __syncthreads();
}

// acc[r][c] = sum_k A(ti + 16 r, k) B(k, tj + 16 c) over k < 128, with
// A(i, k) = A[i * sAi + k * sAk] and B(k, j) = B[k * sBk + j * sBj].
__device__ __forceinline__ void tile_gemm(const float* A, int sAi, int sAk, const float* B, int sBk, int sBj,
                                          float acc[8][8]) {
  const int ti = threadIdx.x >> 4, tj = threadIdx.x & 15;
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
#pragma unroll 2
  for (int k = 0; k < 128; ++k) {
    float a[8], b[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) a[r] = A[(ti + 16 * r) * sAi + k * sAk];
#pragma unroll
    for (int c = 0; c < 8; ++c) b[c] = B[k * sBk + (tj + 16 * c) * sBj];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
  }
}

// Scores of examples [e0, e0 + 128) (kThreads = 256 threads).
__device__ __forceinline__ void mlp_forward_tile(const float* __restrict__ theta, const float* __restrict__ F, int64_t n,
                                                 int64_t e0, float* __restrict__ scores, float* smem) {
  const MlpSmem s = mlp_carve(smem, false);
  mlp_stage_and_layer1(theta, F, n, e0, s);
  float acc[8][8];
  tile_gemm(s.Z1, kLD, 1, s.W2, 1, kLD, acc);       // a2[e][h] - b2[h]
  const int ti = threadIdx.x >> 4, tj = threadIdx.x & 15;
  const float b3 = theta[kOffB3];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    float p = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int h = tj + 16 * c;
      p = fmaf(s.w3[h], fmaxf(acc[r][c] + s.b2[h], 0.f), p);
    }
#pragma unroll
    for (int o = 8; o; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
    const int64_t e = e0 + ti + 16 * r;
    if (tj == 0 && e < n) scores[e] = p + b3;
  }
}

__device__ __forceinline__ float softplusf(float x) { return fmaxf(x, 0.f) + log1pf(expf(-fabsf(x))); }

// Forward + backward of examples [e0, e0 + 128): the tile's contribution to the
// gradient of the mean loss over a minibatch of nb examples (inv_nb = 1/nb)
// goes to gout[0 .. kNParam) (this block's partial), its loss sum to *lout.
// Gradients take the bfloat16 rounding of the operands as the identity.
__device__ __forceinline__ void mlp_backward_tile(const float* __restrict__ theta, const float* __restrict__ F,
                                                  const float* __restrict__ yl, int64_t n, int64_t e0, float pos_weight,
                                                  float inv_nb, float* __restrict__ gout, float* __restrict__ lout,
                                                  float* smem) {
  const MlpSmem s = mlp_carve(smem, true);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ti = tid >> 4, tj = tid & 15;
  float* part = s.red;                      // 16 x kHid
  float* dsv = part + 16 * kHid;            // kTile
  float* lsum = dsv + kTile;                // kTile (per-example loss)
  mlp_stage_and_layer1(theta, F, n, e0, s);
  float acc[8][8];
  tile_gemm(s.Z1, kLD, 1, s.W2, 1, kLD, acc);
  const float b3 = theta[kOffB3];
  // scores, dL/ds
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    float p = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int h = tj + 16 * c;
      p = fmaf(s.w3[h], fmaxf(acc[r][c] + s.b2[h], 0.f), p);
    }
#pragma unroll
    for (int o = 8; o; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
    const int ex = ti + 16 * r;
    const int64_t e = e0 + ex;
    if (tj == 0) {
      float ds = 0.f, l = 0.f;
      if (e < n) {
        const float sc = p + b3;
        const float y = yl[e];
        const float sig = 1.f / (1.f + expf(-sc));
        ds = (pos_weight * y * (sig - 1.f) + (1.f - y) * sig) * inv_nb;
        l = (pos_weight * y * softplusf(-sc) + (1.f - y) * softplusf(sc)) * inv_nb;
      }
      dsv[ex] = ds;
      lsum[ex] = l;
    }
  }
  __syncthreads();
  // dw3, db2 (per-thread partials over its 8 examples, then a fixed-order sum over ti)
  float pw3[8], pb2[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) { pw3[c] = 0.f; pb2[c] = 0.f; }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int ex = ti + 16 * r;
    const float ds = dsv[ex];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int h = tj + 16 * c;
      const float a2 = acc[r][c] + s.b2[h];
      const float z2 = fmaxf(a2, 0.f);
      pw3[c] = fmaf(ds, z2, pw3[c]);
      const float da2 = a2 > 0.f ? ds * s.w3[h] : 0.f;
      s.DA[ex * kLD + h] = da2;
      pb2[c] += da2;
    }
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) part[ti * kHid + tj + 16 * c] = pw3[c];
  __syncthreads();
  for (int h = tid; h < kHid; h += nt) {
    float v = 0.f;
    for (int q = 0; q < 16; ++q) v += part[q * kHid + h];
    gout[kOffW3 + h] = v;
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 8; ++c) part[ti * kHid + tj + 16 * c] = pb2[c];
  __syncthreads();
  for (int h = tid; h < kHid; h += nt) {
    float v = 0.f;
    for (int q = 0; q < 16; ++q) v += part[q * kHid + h];
    gout[kOffB2 + h] = v;
  }
  if (tid == 0) {
    float v = 0.f, l = 0.f;
    for (int ex = 0; ex < kTile; ++ex) { v += dsv[ex]; l += lsum[ex]; }
    gout[kOffB3] = v;
    *lout = l;
  }
  // dW2[h][k] = sum_e DA[e][h] Z1[e][k]
  tile_gemm(s.DA, 1, kLD, s.Z1, kLD, 1, acc);
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) gout[kOffW2 + (ti + 16 * r) * kHid + tj + 16 * c] = acc[r][c];
  // dZ1[e][k] = sum_h DA[e][h] W2[h][k]; DA1 = dZ1 where z1 > 0
  tile_gemm(s.DA, kLD, 1, s.W2, kLD, 1, acc);
  __syncthreads();                          // every read of DA is done
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int ex = ti + 16 * r, k = tj + 16 * c;
      s.DA[ex * kLD + k] = s.Z1[ex * kLD + k] > 0.f ? acc[r][c] : 0.f;
    }
  __syncthreads();
  // dW1[h][f] = sum_e DA1[e][h] F[e][f]; db1[h] = sum_e DA1[e][h]
  for (int o = tid; o < kHid * kNF; o += nt) {
    const int h = o & 127, f = o >> 7;
    float v = 0.f;
    for (int ex = 0; ex < kTile; ++ex) v = fmaf(s.DA[ex * kLD + h], s.Fs[ex * kNF + f], v);
    gout[kOffW1 + h * kNF + f] = v;
  }
  for (int h = tid; h < kHid; h += nt) {
    float v = 0.f;
    for (int ex = 0; ex < kTile; ++ex) v += s.DA[ex * kLD + h];
    gout[kOffB1 + h] = v;
  }
}

// ---------------------------------------------------------------------------
// Candidate selection (one block of kSelThreads): the C highest scores, ties
// to the smaller index (NaN ranks lowest).  cand[0..C) ascending; outl: the
// other R - C columns ascending.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t order_key(float s) {
  const uint32_t b = __float_as_uint(s);
  if (s != s) return 0u;
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// exclusive block scan of one int per thread (blockDim.x <= 1024); returns the total in *total
__device__ __forceinline__ int block_exclusive_scan(int v, int* total, int* sh32) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) sh32[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = lane < nw ? sh32[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) sh32[lane] = w;           // inclusive prefix of warp totals
  }
  __syncthreads();
  const int before = (wid > 0 ? sh32[wid - 1] : 0) + x - v;
  *total = sh32[nw - 1];
  return before;
}

__device__ __forceinline__ void select_block(const float* __restrict__ scores, int R, int C, int32_t* __restrict__ cand,
                                             int32_t* __restrict__ outl) {
  __shared__ int hist[256];
  __shared__ int sh32[32];
  __shared__ uint32_t s_prefix;
  __shared__ int s_need;
  const int tid = threadIdx.x, nt = blockDim.x;
  uint32_t prefix = 0, mask = 0;
  int need = C;
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    for (int b = tid; b < 256; b += nt) hist[b] = 0;
    __syncthreads();
    for (int c = tid; c < R; c += nt) {
      const uint32_t k = order_key(scores[c]);
      if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & 255], 1);
    }
    __syncthreads();
    if (tid < 32) {
      // lane l holds bins 255 - 8 l - q (q < 8), i.e. the bins in descending order
      int cnt[8], sum = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) { cnt[q] = hist[255 - (tid * 8 + q)]; sum += cnt[q]; }
      int incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (tid >= o) incl += y;
      }
      const int excl = incl - sum;
      const unsigned hit = __ballot_sync(0xffffffffu, excl < need && incl >= need);
      if (tid == __ffs(hit) - 1) {
        int cum = excl, sel = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (cum + cnt[q] >= need) { sel = 255 - (tid * 8 + q); break; }
          cum += cnt[q];
        }
        s_prefix = prefix | ((uint32_t)sel << shift);
        s_need = need - cum;
      }
    }
    __syncthreads();
    prefix = s_prefix;
    need = s_need;
    mask |= 255u << shift;
    __syncthreads();
  }
  const uint32_t tau = prefix;
  // contiguous index range per thread
  const int per = (R + nt - 1) / nt;
  const int lo = min(R, tid * per), hi = min(R, lo + per);
  int eq = 0;
  for (int c = lo; c < hi; ++c) eq += order_key(scores[c]) == tau;
  int tot;
  int eq_before = block_exclusive_scan(eq, &tot, sh32);
  int take = 0;
  {
    int r = eq_before;
    for (int c = lo; c < hi; ++c) {
      const uint32_t k = order_key(scores[c]);
      if (k > tau || (k == tau && r < need)) ++take;
      if (k == tau) ++r;
    }
  }
  int pos = block_exclusive_scan(take, &tot, sh32);
  int r = eq_before;
  for (int c = lo; c < hi; ++c) {
    const uint32_t k = order_key(scores[c]);
    const bool t = k > tau || (k == tau && r < need);
    if (k == tau) ++r;
    if (t) cand[pos++] = c;
    else outl[c - pos] = c;
  }
}

// ---------------------------------------------------------------------------
// Outside columns: apply the K reflectors of the candidate QR, check the
// certificate, write the transformed column into Yf.  One warp per column,
// rows lane + 32 r in registers.  V: K x m (reflector t at V + t*m, zero
// above row t), beta: K, rn: K pivot norms |r_tt|.  cert_fail is set to 1 on
// the first violation.  diag[0] += ||R22 part||^2, diag[1] += ||y||^2 (FP64).
// smem: K * m + 2 * K floats.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void apply_cert_block(const float* __restrict__ Y2, float* __restrict__ Yf, int ld, int m,
                                                 int K, const int32_t* __restrict__ outl, int nout,
                                                 const float* __restrict__ V, const float* __restrict__ beta,
                                                 const double* __restrict__ rn, int* cert_fail, double* diag, int blk,
                                                 int nblk, float* smem) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  float* Vs = smem;
  float* Bs = Vs + K * m;
  float* Th = Bs + K;
  for (int e = tid; e < K * m; e += blockDim.x) Vs[e] = V[e];
  for (int t = tid; t < K; t += blockDim.x) {
    Bs[t] = beta[t];
    const float r = (float)rn[t];
    Th[t] = kCertMargin * r * r;
  }
  __syncthreads();
  double r22 = 0.0, ynorm = 0.0;
  for (int q = blk * nw + wid; q < nout; q += nblk * nw) {
    if (*(volatile int*)cert_fail) break;
    const int o = outl[q];
    float y[kMaxM / 32];
    float n0 = 0.f;
#pragma unroll
    for (int r = 0; r < kMaxM / 32; ++r) {
      const int i = lane + 32 * r;
      y[r] = i < m ? Y2[(int64_t)o * ld + i] : 0.f;
      n0 = fmaf(y[r], y[r], n0);
    }
    bool ok = true;
    for (int t = 0; t < K; ++t) {
      const float* v = Vs + t * m;
      float rho = 0.f, d = 0.f;
#pragma unroll
      for (int r = 0; r < kMaxM / 32; ++r) {
        const int i = lane + 32 * r;
        if (i >= t && i < m) {
          rho = fmaf(y[r], y[r], rho);
          d = fmaf(v[i], y[r], d);
        }
      }
#pragma unroll
      for (int o2 = 16; o2; o2 >>= 1) {
        rho += __shfl_xor_sync(0xffffffffu, rho, o2);
        d += __shfl_xor_sync(0xffffffffu, d, o2);
      }
      if (!(rho < Th[t])) { ok = false; break; }
      d *= Bs[t];
#pragma unroll
      for (int r = 0; r < kMaxM / 32; ++r) {
        const int i = lane + 32 * r;
        if (i >= t && i < m) y[r] = fmaf(-d, v[i], y[r]);
      }
    }
    if (!ok) {
      if (lane == 0) atomicExch(cert_fail, 1);
      break;
    }
    float tail = 0.f;
#pragma unroll
    for (int r = 0; r < kMaxM / 32; ++r) {
      const int i = lane + 32 * r;
      if (i < m) {
        Yf[(int64_t)o * ld + i] = y[r];
        if (i >= K) tail = fmaf(y[r], y[r], tail);
      }
    }
    tail = warp_sum(tail);
    n0 = warp_sum(n0);
    r22 += (double)tail;
    ynorm += (double)n0;
  }
  if (lane == 0) {
    if (r22 != 0.0) atomicAdd(&diag[0], r22);
    if (ynorm != 0.0) atomicAdd(&diag[1], ynorm);
  }
}

}  // namespace prop
}  // namespace idl
