// cpqr_dev.cuh -- device bodies of the pivoted QR stage, shared by the
// single-problem kernels (cpqr.cu) and the batched ones (batch.cu).
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"

namespace idl {

namespace cg = cooperative_groups;

template <typename T> struct Cand { T val; int idx; int pad; };

template <typename T>
__device__ __forceinline__ bool better(T va, int ia, T vb, int ib) {
  return va > vb || (va == vb && ia < ib && ia >= 0) || (ib < 0 && ia >= 0);
}

// Pivot search key of a remaining squared norm.  FP32: the value itself.  FP64:
// the bit pattern as a signed integer (non-negative doubles order like their
// bits), so the block / cluster argmax runs on the integer pipes -- GB300's
// FP64 pipe retires about two lanes per clock per SM.  Retired columns and NaN
// norms get -1 (never chosen).
template <typename T> struct PivKey;
template <> struct PivKey<float> {
  using K = float;
  static __device__ __forceinline__ K of(float v, bool ok) { return ok && v >= 0.f ? v : -1.f; }
  static __device__ __forceinline__ float store(K k) { return k; }
  static __device__ __forceinline__ K load(float v) { return v; }
};
template <> struct PivKey<double> {
  using K = long long;
  static __device__ __forceinline__ K of(double v, bool ok) {
    const long long b = __double_as_longlong(v);
    return ok && b >= 0 && (b & 0x7fffffffffffffffLL) <= 0x7ff0000000000000LL ? b : -1LL;
  }
  static __device__ __forceinline__ double store(K k) { return __longlong_as_double(k); }
  static __device__ __forceinline__ K load(double v) { return __double_as_longlong(v); }
};

__device__ __forceinline__ float group_sum(float v, int tpc) {
  for (int o = tpc >> 1; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double group_sum(double v, int tpc) {
  for (int o = tpc >> 1; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The Householder vector in shared memory is stored by thread slot: row
// i = gl + TPC j (gl: lane within the column's group) at vslot(i) = gl V + j,
// so that each thread's V values are contiguous and read as 16-byte vectors
// (V is a multiple of 4 in every compiled variant).
template <int V, int TPC>
__device__ __forceinline__ int vslot(int i) { return (i % TPC) * V + i / TPC; }

// sum_j v_j y_j over a thread's rows (four partial sums).  Slots j < jskip
// (a multiple of 4, the same for every lane) hold rows above the current
// step, where v is zero, and slots j >= jend (a multiple of 4) rows past m for
// every lane: those chunks are skipped (warp-uniform branches).
template <typename T, int V>
__device__ __forceinline__ T house_dot(const T* __restrict__ vrow, const T (&y)[V], int jskip, int jend) {
  static_assert(V % 4 == 0, "V must be a multiple of 4");
  T d0 = T(0), d1 = T(0), d2 = T(0), d3 = T(0);
#pragma unroll
  for (int j = 0; j < V; j += 4) {
    if (j < jskip || j >= jend) continue;
    if constexpr (sizeof(T) == 4) {
      const float4 w = *reinterpret_cast<const float4*>(vrow + j);
      d0 = fma(w.x, y[j], d0); d1 = fma(w.y, y[j + 1], d1); d2 = fma(w.z, y[j + 2], d2); d3 = fma(w.w, y[j + 3], d3);
    } else {
      const double2 a = *reinterpret_cast<const double2*>(vrow + j);
      const double2 b = *reinterpret_cast<const double2*>(vrow + j + 2);
      d0 = fma(a.x, y[j], d0); d1 = fma(a.y, y[j + 1], d1); d2 = fma(b.x, y[j + 2], d2); d3 = fma(b.y, y[j + 3], d3);
    }
  }
  return (d0 + d1) + (d2 + d3);
}

// y -= d v over a thread's rows; returns the thread's part of the trailing
// norm^2 over rows with slot index j >= jt (four partial sums); chunks below
// jskip or from jend on are left alone (v is zero there, jt > jskip, and the
// rows past m stay zero)
template <typename T, int V>
__device__ __forceinline__ T house_update(const T* __restrict__ vrow, T (&y)[V], T d, int jt, int jskip, int jend) {
  T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
#pragma unroll
  for (int j = 0; j < V; j += 4) {
    if (j < jskip || j >= jend) continue;
    T w0, w1, w2, w3;
    if constexpr (sizeof(T) == 4) {
      const float4 w = *reinterpret_cast<const float4*>(vrow + j);
      w0 = w.x; w1 = w.y; w2 = w.z; w3 = w.w;
    } else {
      const double2 a = *reinterpret_cast<const double2*>(vrow + j);
      const double2 b = *reinterpret_cast<const double2*>(vrow + j + 2);
      w0 = a.x; w1 = a.y; w2 = b.x; w3 = b.y;
    }
    y[j] = fma(-d, w0, y[j]);
    y[j + 1] = fma(-d, w1, y[j + 1]);
    y[j + 2] = fma(-d, w2, y[j + 2]);
    y[j + 3] = fma(-d, w3, y[j + 3]);
    if (j >= jt) {                     // the whole chunk is trailing: one FMA per row
      s0 = fma(y[j], y[j], s0);
      s1 = fma(y[j + 1], y[j + 1], s1);
      s2 = fma(y[j + 2], y[j + 2], s2);
      s3 = fma(y[j + 3], y[j + 3], s3);
    } else {                           // the chunk holding row t (or above it): masked
      s0 += (j >= jt) ? y[j] * y[j] : T(0);
      s1 += (j + 1 >= jt) ? y[j + 1] * y[j + 1] : T(0);
      s2 += (j + 2 >= jt) ? y[j + 2] * y[j + 2] : T(0);
      s3 += (j + 3 >= jt) ? y[j + 3] * y[j + 3] : T(0);
    }
  }
  return (s0 + s1) + (s2 + s3);
}

// first slot chunk (multiple of 4) that can hold rows >= t for some lane of a
// TPC-lane group: rows gl + TPC j < t for all gl when TPC (j + 4) <= t
__device__ __forceinline__ int skip_slots(int t, int tpc) { return (t / tpc) & ~3; }
// end of the slot chunks that hold some row < m for some lane
__device__ __forceinline__ int end_slots(int m, int tpc) { return ((m + tpc - 1) / tpc + 3) & ~3; }

// ----------------------------------------------------------------------------
// Register-resident variant (used whenever a cluster shape fits).  Each group
// of TPC lanes keeps one column in registers (rows gl, gl + TPC, ...).  Per
// pivot step:
//   1. block argmax of the remaining norms (warp shuffles, one block barrier);
//      warp 0 publishes the CTA's candidate in its own shared memory and,
//      after a second block barrier, the owning group copies that column's
//      trailing part into a double-buffered staging slot;
//   2. one hardware cluster barrier;
//   3. warp 0 of every CTA pulls the CS candidates (one DSMEM load per lane),
//      reduces them (same result everywhere), pulls the winner's staged
//      column and forms the Householder reflection (v in shared memory);
//   4. one block barrier; every group applies the reflection to its column in
//      registers and recomputes the trailing norm exactly.
// Measured on GB300: cluster barrier ~580 cycles, DSMEM pull of a column
// ~450, block barrier ~130; remote stores before the barrier (a push model)
// made its release wait ~2000 cycles, so candidates are pulled instead.
// ----------------------------------------------------------------------------
// Threads per CTA each (type, values per lane, lanes per column) variant is
// compiled for: sized so the column registers fit without spilling.
template <typename T, int V, int TPC> struct RegCpqr {
  static constexpr int kWords = V * (int)(sizeof(T) / 4);
  static constexpr int kMaxThreads = kWords <= 16 ? 1024 : kWords <= 32 ? (TPC == 1 ? 896 : 768)
                                   : kWords <= 64 ? (TPC == 1 ? 640 : 512) : kWords <= 96 ? 448 : 384;
};

// Body of one cluster working on one problem (Yin/Yout m x R column-major, ld);
// smem_raw: the dynamic shared memory (reg_cpqr_smem bytes).
// colmap (optional): the problem's column c is column colmap[c] of Yin/Yout
// (ascending, so ties still go to the smaller original index); J reports
// original indices.  Vout/Bout (optional): reflector t (zero above row t) at
// Vout + t*m and its beta at Bout[t] -- the learned proposal's candidate QR.
// force (optional, no colmap): the pivot of step t is column force[t] (the QR
// of a given column selection in a given order; force may alias J).
// Per pivot step: every warp publishes its best column, one block barrier;
// every warp reduces those (the same winner everywhere), the winner's group
// stages its column and thread 0 publishes the CTA's candidate; one cluster
// barrier; warp 0 pulls every CTA's candidate, picks the winner, pulls its
// staged column and forms the reflection; one block barrier; every group
// updates its column.
template <typename T, int V, int TPC>
__device__ __forceinline__ void cpqr_reg_body(const T* __restrict__ Yin, T* __restrict__ Yout, int m, int R, int ld,
                                              int K, int nc, int32_t* __restrict__ J, double* __restrict__ rnorm,
                                              double* __restrict__ diag, int* status, unsigned char* smem_raw,
                                              const int32_t* __restrict__ colmap = nullptr, T* __restrict__ Vout = nullptr,
                                              T* __restrict__ Bout = nullptr, const int32_t* __restrict__ force = nullptr) {
  constexpr int tpc = TPC;
  cg::cluster_group cluster = cg::this_cluster();
  const int CS = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, NW = blockDim.x >> 5;
  const int g = tid / tpc, gl = tid - g * tpc;
  const int c0 = rank * nc;
  const int ncl = max(0, min(nc, R - c0));
  const bool own = g < ncl;
  const int col = c0 + g;
  const int64_t scol = own ? (colmap ? (int64_t)colmap[col] : (int64_t)col) : 0;   // column of Yin / Yout
  const int mp = (m + 3) & ~3;
  const int jend = end_slots(m, tpc);

  T* vs = (T*)smem_raw;                                             // V*TPC: v by thread slot, zero outside rows [t, m)
  T* stage = vs + V * TPC;                                          // [2][mp] this CTA's staged candidate column
  Cand<T>* cand = (Cand<T>*)(smem_raw + round_up((int64_t)sizeof(T) * (V * TPC + 2 * mp), 16));   // [2]
  using PK = PivKey<T>;
  using KT = typename PK::K;
  __shared__ KT red_v[32];
  __shared__ int red_i[32];
  __shared__ T s_beta, s_alpha;
  __shared__ int s_p, s_stop;
  if (tid == 0) s_stop = 0;
  for (int i = tid; i < V * TPC; i += blockDim.x) vs[i] = T(0);

  // one thread per whole column with 16-byte aligned columns: vector loads and stores
  bool vecio = false;
  if constexpr (TPC == 1 && sizeof(T) == 4)
    vecio = ((ld & 3) == 0) && ((((uintptr_t)Yin) & 15) == 0) && ((((uintptr_t)Yout) & 15) == 0);
  T y[V];
  if (vecio) {
#pragma unroll
    for (int j = 0; j < V; j += 4) {
      if (own && j + 4 <= m) {
        const float4 q = *reinterpret_cast<const float4*>(Yin + scol * ld + j);
        y[j] = q.x; y[j + 1] = q.y; y[j + 2] = q.z; y[j + 3] = q.w;
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) y[j + u] = (own && j + u < m) ? Yin[scol * ld + j + u] : T(0);
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < V; ++j) {
      const int i = gl + tpc * j;
      y[j] = (own && i < m) ? Yin[scol * ld + i] : T(0);
    }
  }
  T nn = T(0);
#pragma unroll
  for (int j = 0; j < V; ++j) nn += y[j] * y[j];
  nn = group_sum(nn, tpc);
  {
    double f = (own && gl == 0) ? (double)nn : 0.0;
    f = warp_sum(f);
    if (lane == 0 && f != 0.0) atomicAdd(&diag[1], f);
  }
  T nrm2 = own ? nn : T(-1);          // < 0: retired or no column
  bool alive = own;                   // the column is still a pivot candidate
  int tp = -1;
  T alpha_p = T(0);
  for (int t = 0; t < K; ++t) {
    // A. warp candidates (with forced pivots, step t's only candidate is column force[t])
    KT bv = PK::of(nrm2, gl == 0 && alive && (!force || col == force[t]));
    int bi = bv >= KT(0) ? col : -1;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const KT ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (better(ov, oi, bv, bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { red_v[wid] = bv; red_i[wid] = bi; }
    __syncthreads();
    // B. the CTA's candidate, reduced by every warp (same result everywhere)
    bv = lane < NW ? red_v[lane] : KT(-1);
    bi = lane < NW ? red_i[lane] : -1;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const KT ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (better(ov, oi, bv, bi)) { bv = ov; bi = oi; }
    }
    if (own && col == bi) {
      T* st = stage + (t & 1) * mp;
      if (vecio) {
#pragma unroll
        for (int j = 0; j < V; j += 4)
          if (j + 4 > t && j < mp) *reinterpret_cast<float4*>(st + j) = make_float4(y[j], y[j + 1], y[j + 2], y[j + 3]);
      } else {
#pragma unroll
        for (int j = 0; j < V; ++j) {
          const int i = gl + tpc * j;
          if (i >= t && i < m) st[i] = y[j];
        }
      }
    }
    if (tid == 0) {
      cand[t & 1].val = PK::store(bv);   // published locally; the other CTAs pull it after the barrier
      cand[t & 1].idx = bi;
    }
    cluster.sync();
    // C. winner, pivot column, reflection (warp 0)
    if (wid == 0) {
      KT v = KT(-1);
      int ix = -1;
      if (lane < CS) {
        const Cand<T>* rc = cluster.map_shared_rank(cand + (t & 1), (unsigned)lane);
        v = PK::load(rc->val);
        ix = rc->idx;
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        const KT ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, ix, o);
        if (better(ov, oi, v, ix)) { v = ov; ix = oi; }
      }
      if (ix < 0) {
        if (lane == 0) {
          s_stop = 1;
          if (rank == 0) {
            for (int q = t; q < K; ++q) J[q] = -1;
            set_status(status, IDL_EDATA);
          }
        }
      } else {
        const int w = ix / nc;
        if (lane == 0 && t > 0) vs[vslot<V, TPC>(t - 1)] = T(0);     // rows above t stay zero
        const T* rm = cluster.map_shared_rank(stage + (t & 1) * mp, (unsigned)w);
        T xs = T(0), x0 = T(0);
        T xv[8];                                                     // m <= 256: every remote load issued first
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = t + lane + 32 * q;
          xv[q] = i < m ? rm[i] : T(0);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = t + lane + 32 * q;
          if (i < m) {
            const T x = xv[q];
            vs[vslot<V, TPC>(i)] = x;
            xs += x * x;
            if (i == t) x0 = x;
            if (Vout && rank == 0) Vout[(int64_t)t * m + i] = x;
          }
        }
        if (Vout && rank == 0)
          for (int i = lane; i < t; i += 32) Vout[(int64_t)t * m + i] = T(0);
        xs = warp_sum(xs);
        x0 = __shfl_sync(0xffffffffu, x0, 0);
        const T nrm = sqrt(xs);
        const T alpha = (x0 >= T(0)) ? -nrm : nrm;
        const T beta = (nrm > T(0)) ? T(1) / (nrm * (nrm + fabs(x0))) : T(0);
        if (lane == 0) {
          vs[vslot<V, TPC>(t)] = x0 - alpha;
          s_alpha = alpha;
          s_beta = beta;
          s_p = ix;
          if (rank == 0) {
            J[t] = colmap ? colmap[ix] : ix;
            if (Vout) { Vout[(int64_t)t * m + t] = x0 - alpha; Bout[t] = beta; }
            if (rnorm) rnorm[t] = (double)fabs(alpha);
            if (t == 0) diag[3] = (double)fabs(alpha);
            if (t == K - 1) diag[4] = (double)fabs(alpha);
          }
        }
      }
    }
    __syncthreads();
    if (s_stop) break;
    // D. update
    const int p = s_p;
    const T beta = s_beta;
    const bool act = alive;
    const bool piv = act && col == p;
    const bool upd = act && !piv;
    if (piv) { nrm2 = T(-1); alive = false; tp = t; alpha_p = s_alpha; }
    // vs is zero outside rows [t, m): no per-row predicates in the dot product and the update
    const T* vrow = vs + gl * V;
    const int jskip = skip_slots(t, tpc);
    T d = group_sum(house_dot<T, V>(vrow, y, jskip, jend), tpc) * beta;
    if (!upd) d = T(0);
    __syncwarp();   // re-read v below instead of keeping all of it in registers
    // trailing norm over rows > t: rows gl + tpc*j with j >= jt
    const int jt = (t - gl) >= 0 ? (t - gl) / tpc + 1 : 0;
    const T s2 = group_sum(house_update<T, V>(vrow, y, d, jt, jskip, jend), tpc);
    if (upd) nrm2 = s2;
  }
  cluster.sync();                 // no CTA reads another's staging slot after this point
  T r22t = T(0);                  // per-thread part in the working precision (FP64 pipes are scarce)
#pragma unroll
  for (int j = 0; j < V; ++j) {
    const int i = gl + tpc * j;
    if (tp >= 0) y[j] = (i < tp) ? y[j] : (i == tp ? alpha_p : T(0));
    else if (own && i >= K && i < m) r22t = fma(y[j], y[j], r22t);
  }
  if (vecio) {
#pragma unroll
    for (int j = 0; j < V; j += 4) {
      if (own && j + 4 <= m) {
        *reinterpret_cast<float4*>(Yout + scol * ld + j) = make_float4(y[j], y[j + 1], y[j + 2], y[j + 3]);
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (own && j + u < m) Yout[scol * ld + j + u] = y[j + u];
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < V; ++j) {
      const int i = gl + tpc * j;
      if (own && i < m) Yout[scol * ld + i] = y[j];
    }
  }
  double r22 = warp_sum((double)r22t);
  if (lane == 0 && r22 != 0.0) atomicAdd(&diag[0], r22);
}

// ----------------------------------------------------------------------------
// One-CTA variant for a column subset that fits one block (the learned
// proposal's candidate QR).  Two block barriers per pivot step:
//   A. every warp reduces its groups' remaining norms and publishes its best;
//      barrier;
//   B. every warp reduces the published candidates (same winner everywhere);
//      the winner's own group forms the Householder reflection from its
//      registers (group reductions, no staging) and writes v and beta to
//      shared memory; barrier;
//   C. every group applies the reflection to its column in registers and
//      recomputes the trailing norm exactly.
// Same arguments and outputs as cpqr_reg_body; colmap is required (column c
// of the subset is column colmap[c] of Yin / Yout).
// ----------------------------------------------------------------------------
template <typename T, int V, int TPC>
__device__ __forceinline__ void cpqr_cta_body(const T* __restrict__ Yin, T* __restrict__ Yout, int m, int C, int ld,
                                              int K, int32_t* __restrict__ J, double* __restrict__ rnorm,
                                              double* __restrict__ diag, int* status, unsigned char* smem_raw,
                                              const int32_t* __restrict__ colmap, T* __restrict__ Vout,
                                              T* __restrict__ Bout) {
  static_assert(sizeof(T) == 4, "the one-CTA variant orders FP32 norms by their bit patterns");
  constexpr int tpc = TPC;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, NW = blockDim.x >> 5;
  const int g = tid / tpc, gl = tid - g * tpc;
  const bool own = g < C;
  const int64_t scol = own ? (int64_t)colmap[g] : 0;
  T* vs = (T*)smem_raw;                                             // V*TPC: v by thread slot, zero outside rows [t, m)
  __shared__ unsigned red_k[32], red_i[32];
  __shared__ int s_piv[128];                                        // pivots (subset indices), K <= 128
  __shared__ T s_beta;
  for (int q = tid; q < K; q += blockDim.x) s_piv[q] = -1;
  T y[V];
#pragma unroll
  for (int j = 0; j < V; ++j) {
    const int i = gl + tpc * j;
    y[j] = (own && i < m) ? Yin[scol * ld + i] : T(0);
  }
  T nn = T(0);
#pragma unroll
  for (int j = 0; j < V; ++j) nn += y[j] * y[j];
  nn = group_sum(nn, tpc);
  {
    double f = (own && gl == 0) ? (double)nn : 0.0;
    f = warp_sum(f);
    if (lane == 0 && f != 0.0) atomicAdd(&diag[1], f);
  }
  T nrm2 = own ? nn : T(-1);
  int tp = -1;
  T alpha_p = T(0);
  for (int t = 0; t < K; ++t) {
    // A. warp candidates: the largest remaining norm (its FP32 bit pattern + 1;
    // 0 marks a retired column or none), then the smallest index -- the same
    // order as the cluster variant's comparison, by two warp reductions
    const unsigned key = (gl == 0 && nrm2 >= T(0)) ? __float_as_uint((float)nrm2) + 1u : 0u;
    const unsigned wk = __reduce_max_sync(0xffffffffu, key);
    const unsigned wi = __reduce_min_sync(0xffffffffu, (key == wk && wk != 0u) ? (unsigned)g : 0xffffffffu);
    if (lane == 0) { red_k[wid] = wk; red_i[wid] = wi; }
    __syncthreads();
    // B. block winner (every warp), reflection by the winner's group
    const unsigned k2 = lane < NW ? red_k[lane] : 0u;
    const unsigned bk = __reduce_max_sync(0xffffffffu, k2);
    const unsigned i2 = (lane < NW && k2 == bk && bk != 0u) ? red_i[lane] : 0xffffffffu;
    const unsigned bi = __reduce_min_sync(0xffffffffu, i2);
    const int p = bk == 0u ? -1 : (int)bi;
    if (p < 0) {                                                     // no finite remaining column
      if (tid == 0) set_status(status, IDL_EDATA);
      break;                                                         // uniform: every thread saw p < 0
    }
    const bool piv = own && g == p;
    if ((p * tpc) >> 5 == wid) {
      // the pivot's warp: trailing norm and x_t per group (all lanes shuffle;
      // only the pivot's group uses the result)
      T xs = T(0), x0 = T(0);
#pragma unroll
      for (int j = 0; j < V; ++j) {
        const int i = gl + tpc * j;
        if (i >= t) xs += y[j] * y[j];
        if (i == t) x0 = y[j];
      }
      xs = group_sum(xs, tpc);
      x0 = group_sum(x0, tpc);                                       // one lane of a group holds row t
      if (piv) {
      const T nrm = sqrt(xs);
      const T alpha = (x0 >= T(0)) ? -nrm : nrm;
      const T beta = (nrm > T(0)) ? T(1) / (nrm * (nrm + fabs(x0))) : T(0);
#pragma unroll
      for (int j = 0; j < V; ++j) {
        const int i = gl + tpc * j;
        const T v = (i < t || i >= m) ? T(0) : (i == t ? x0 - alpha : y[j]);
        vs[gl * V + j] = v;
        if (i < m) Vout[(int64_t)t * m + i] = v;
      }
      if (gl == 0) {
        s_beta = beta;
        s_piv[t] = p;
        Bout[t] = beta;
        if (rnorm) rnorm[t] = (double)fabs(alpha);
        if (t == 0) diag[3] = (double)fabs(alpha);
        if (t == K - 1) diag[4] = (double)fabs(alpha);
      }
      nrm2 = T(-1);
      tp = t;
      alpha_p = alpha;
      }
    }
    __syncthreads();
    // C. apply to the remaining columns
    const T beta = s_beta;
    const bool upd = own && nrm2 >= T(0);
    const T* vrow = vs + gl * V;
    const int jskip = skip_slots(t, tpc);
    T d = group_sum(house_dot<T, V>(vrow, y, jskip, V), tpc) * beta;
    if (!upd) d = T(0);
    const int jt = (t - gl) >= 0 ? (t - gl) / tpc + 1 : 0;
    const T s2 = group_sum(house_update<T, V>(vrow, y, d, jt, jskip, V), tpc);
    if (upd) nrm2 = s2;
  }
  T r22t = T(0);
#pragma unroll
  for (int j = 0; j < V; ++j) {
    const int i = gl + tpc * j;
    if (own && i < m) {
      T out = y[j];
      if (tp >= 0) out = (i < tp) ? y[j] : (i == tp ? alpha_p : T(0));
      Yout[scol * ld + i] = out;
      if (tp < 0 && i >= K) r22t = fma(y[j], y[j], r22t);
    }
  }
  double r22 = warp_sum((double)r22t);
  if (lane == 0 && r22 != 0.0) atomicAdd(&diag[0], r22);
  __syncthreads();
  for (int q = tid; q < K; q += blockDim.x) J[q] = s_piv[q] >= 0 ? colmap[s_piv[q]] : -1;
}

template <typename T, int V, int TPC>
__host__ __device__ constexpr size_t cta_cpqr_smem() { return sizeof(T) * (size_t)V * TPC; }

// Threads per CTA of the one-CTA variant (no staging buffer, more registers
// per thread than the cluster variant needs).
template <typename T, int V, int TPC> struct CtaCpqr {
  static constexpr int kWords = V * (int)(sizeof(T) / 4);
  static constexpr int kMaxThreads = kWords <= 16 ? 1024 : kWords <= 32 ? 640 : kWords <= 64 ? 448 : 320;
};

// Fallback gate of the learned proposal.  With a gate, a QR launch is the
// proposal's fallback and only runs when the certificate failed (*gate != 0);
// otherwise block 0 moves the proposal's diagnostics (diag[8..12]) into
// place and every block returns before any barrier.
__device__ __forceinline__ bool proposal_certified(const int* gate, double* diag) {
  if (!gate) return false;
  if (*(volatile const int*)gate != 0) return false;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    diag[0] = diag[8];
    diag[1] = diag[9];
    diag[3] = diag[11];
    diag[4] = diag[12];
  }
  return true;
}

template <typename T, int V, int TPC>
__host__ __device__ constexpr size_t reg_cpqr_smem(int m) {
  return (size_t)(((int64_t)sizeof(T) * (V * TPC + 2 * ((m + 3) & ~3)) + 15) / 16 * 16) + sizeof(Cand<T>) * 2;
}

}  // namespace idl
