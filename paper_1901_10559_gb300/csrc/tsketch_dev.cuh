// tsketch_dev.cuh -- device body of the TensorSketch kernel, shared by the
// single-problem kernel (tensorsketch.cu) and the batched one (batch.cu).
//
// One block per pair of columns (r, r+1), L/16 threads (at least 32), 16
// complex values per thread:
//   * per mode n the two columns' CountSketches are packed as the real and
//     imaginary parts of one complex length-L vector z (shared-memory atomics
//     at natural-order positions) and transformed by a Stockham autosort FFT
//     (radix-16 passes, one radix-2/4/8 pass for the remaining bits): every
//     pass reads 16 values per thread, applies the pass's twiddles (read from
//     a precomputed table, laid out so that a warp's reads are contiguous),
//     runs the small DFT in registers and writes the values to their output
//     positions (one barrier between the reads and the writes, one after);
//   * the spectra of the two columns are separated by Hermitian symmetry,
//        C_r[f] = (Z[f] + conj Z[-f]) / 2,   C_{r+1}[f] = (Z[f] - conj Z[-f]) / 2i,
//     and multiplied into the running products P_r, P_{r+1} (f = 0..L/2,
//     shared memory; registers stay with the FFT);
//   * the inverse FFT of P_r + i P_{r+1} is the forward FFT of the conjugate,
//     conjugated: both real columns at once.
// Shared memory: the length-L vector with one pad entry per 16 (bank spread),
// then P_r and P_{r+1}.
#pragma once

#include <utility>

#include "common.cuh"

namespace idl {

constexpr int kTsMaxModes = 8;
constexpr int kTsVals = 16;          // complex values per thread
constexpr int kTsMaxThreads = 512;   // L = 8192

struct TsArgs {
  const float* F[kTsMaxModes];
  const int32_t* h[kTsMaxModes];
  const int8_t* s[kTsMaxModes];
  int64_t ldf[kTsMaxModes];
  int dims[kTsMaxModes];
  int N;
};

__host__ __device__ constexpr int ts_threads(int L) { return L / kTsVals < 32 ? 32 : L / kTsVals; }

// Twiddle table: for each (radix R, span Ns) a pass of an L <= 8192 transform
// uses, entries exp(-2 pi i k r / (Ns R)) at [(r - 1) Ns + k], r = 1..R-1,
// k < Ns.  Pairs: (16, 16), (16, 256), (2|4|8, 16), (2|4|8, 256), (2, 4096).
__host__ __device__ constexpr int ts_tw_offset(int R, int Ns) {
  return R == 16 ? (Ns == 16 ? 0 : 240)
       : Ns == 16 ? 4080 + (R == 2 ? 0 : R == 4 ? 16 : 64)
       : Ns == 256 ? 4256 + (R == 2 ? 0 : R == 4 ? 256 : 1024)
       : 7072;                                                       // (2, 4096)
}
constexpr int kTsTwEntries = 7072 + 4096;
__host__ __device__ constexpr size_t ts_smem_bytes(int L) {
  return sizeof(float2) * (size_t)(L + L / 16 + 1 + 2 * (L / 2 + 1));
}

namespace ts {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }

// Twiddle read that stays where it is written (a volatile load is not
// hoisted across the passes' barriers, which would keep every pass's
// twiddles live in registers at once).
__device__ __forceinline__ float2 ld_tw(const float2* p) {
  float2 v;
  asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}

// An opaque copy of x: values derived from it are recomputed where they are
// used instead of being hoisted out of the mode loop (register pressure).
__device__ __forceinline__ int opaque(int x) {
  asm volatile("" : "+r"(x));
  return x;
}

// d * exp(-2 pi i k / 16), k < 8 (mathematical constants cos, sin of k pi / 8)
template <int K>
__device__ __forceinline__ float2 w16(float2 d) {
  constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508977f, h = 0.70710678118654752f;
  if constexpr (K == 0) return d;
  else if constexpr (K == 4) return make_float2(d.y, -d.x);
  else {
    constexpr float wr = K == 1 ? c1 : K == 2 ? h : K == 3 ? s1 : K == 5 ? -s1 : K == 6 ? -h : -c1;
    constexpr float wi = K == 1 ? -s1 : K == 2 ? -h : K == 3 ? -c1 : K == 5 ? -c1 : K == 6 ? -h : -s1;
    return make_float2(d.x * wr - d.y * wi, d.x * wi + d.y * wr);
  }
}

template <int R, int S, int A>
__device__ __forceinline__ void dif_pair(float2* v) {
  if constexpr ((A & S) == 0) {
    const float2 x = v[A], y = v[A + S];
    v[A] = make_float2(x.x + y.x, x.y + y.y);
    v[A + S] = w16<(A & (S - 1)) * (8 / S)>(make_float2(x.x - y.x, x.y - y.y));
  }
}

template <int R, int S, int... A>
__device__ __forceinline__ void dif_stage(float2* v, std::integer_sequence<int, A...>) {
  (dif_pair<R, S, A>(v), ...);
}

template <int R, int S>
__device__ __forceinline__ void dif_stages(float2* v) {
  if constexpr (S >= 1) {
    dif_stage<R, S>(v, std::make_integer_sequence<int, R>{});
    dif_stages<R, S / 2>(v);
  }
}

template <int B, int X>
constexpr int bitrev() {
  int r = 0;
  for (int i = 0; i < B; ++i) r |= ((X >> i) & 1) << (B - 1 - i);
  return r;
}

template <int R, int B, int... A>
__device__ __forceinline__ void bitrev_perm(float2* v, std::integer_sequence<int, A...>) {
  float2 t[R];
  ((t[A] = v[bitrev<B, A>()]), ...);
  ((v[A] = t[A]), ...);
}

// Natural-order R-point DFT in registers: v[k] <- sum_r v[r] exp(-2 pi i r k / R), R <= 16
// (radix-2 decimation in frequency, then a compile-time bit-reversal permutation).
template <int R>
__device__ __forceinline__ void dft(float2* v) {
  dif_stages<R, R / 2>(v);
  constexpr int B = R == 16 ? 4 : R == 8 ? 3 : R == 4 ? 2 : 1;
  bitrev_perm<R, B>(v, std::make_integer_sequence<int, R>{});
}

// One Stockham pass of radix R over span Ns (product of the earlier radices):
// butterfly j reads z[j + r L/R], multiplies by exp(-2 pi i (j mod Ns) r / (Ns R)),
// transforms, and writes z[(j / Ns) Ns R + (j mod Ns) + r Ns].  Thread t owns
// butterflies t + T b (b < 16/R), T = L / 16.
template <int R>
__device__ __forceinline__ void pass(float2* z, const float2* __restrict__ tw, int L, int Ns, int t, int T) {
  constexpr int NB = kTsVals / R;
  const int stride = L / R;
  // padded positions advance by a constant when the stride is a multiple of 16
  const int sin_ = (stride & 15) == 0 ? stride + (stride >> 4) : 0;
  const int sout = Ns == 1 ? 1 : Ns + (Ns >> 4);                    // Ns is 1 or a multiple of 16
  float2 v[NB][R];
  const bool act = t < T;
  if (act) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = t + T * b;
      const int p0 = pad(j);
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = z[sin_ ? p0 + r * sin_ : pad(j + r * stride)];
    }
  }
  __syncthreads();
  if (act) {
    const float2* twp = Ns > 1 ? tw + ts_tw_offset(R, Ns) : nullptr;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = t + T * b;
      const int k = j & (Ns - 1);
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], ld_tw(twp + (r - 1) * Ns + k));
      }
      dft<R>(v[b]);
      const int q0 = pad((j - k) * R + k);
#pragma unroll
      for (int r = 0; r < R; ++r) z[q0 + r * sout] = v[b][r];
    }
  }
  __syncthreads();
}

// Forward FFT of z (natural order in and out), L = 2^logL, 16 <= L <= 8192.
__device__ __forceinline__ void fft(float2* z, const float2* __restrict__ tw, int L, int logL, int t, int T) {
  int Ns = 1, bits = logL;
  while (bits >= 4) {
    pass<16>(z, tw, L, Ns, t, T);
    Ns <<= 4;
    bits -= 4;
  }
  if (bits == 3) pass<8>(z, tw, L, Ns, t, T);
  else if (bits == 2) pass<4>(z, tw, L, Ns, t, T);
  else if (bits == 1) pass<2>(z, tw, L, Ns, t, T);
}

// Builds the twiddle table (one thread per entry, kTsTwEntries entries).
__device__ __forceinline__ void twiddle_entry(int e, float2* tw) {
  int R, Ns, off;
  if (e < 240) { R = 16; Ns = 16; off = 0; }
  else if (e < 4080) { R = 16; Ns = 256; off = 240; }
  else if (e < 4096) { R = 2; Ns = 16; off = 4080; }
  else if (e < 4144) { R = 4; Ns = 16; off = 4096; }
  else if (e < 4256) { R = 8; Ns = 16; off = 4144; }
  else if (e < 4512) { R = 2; Ns = 256; off = 4256; }
  else if (e < 5280) { R = 4; Ns = 256; off = 4512; }
  else if (e < 7072) { R = 8; Ns = 256; off = 5280; }
  else { R = 2; Ns = 4096; off = 7072; }
  const int q = e - off, r = q / Ns + 1, k = q - (r - 1) * Ns;
  float sv, cv;
  sincospif(-2.f * (float)((k * r) % (Ns * R)) / (float)(Ns * R), &sv, &cv);
  tw[e] = make_float2(cv, sv);
}

}  // namespace ts

// One block: columns r0 and r0 + 1.  sm: ts_smem_bytes(L) of shared memory.
// cm = false: Y row-major (Y[l * ldy + r]); cm = true: column-major (Y[r * ldy + l]).
__device__ __forceinline__ void tensorsketch_block(const TsArgs& a, int64_t R, int L, int logL,
                                                   const double* __restrict__ lambda, float* __restrict__ Y,
                                                   int64_t ldy, bool cm, int64_t r0, const float2* __restrict__ tw,
                                                   float2* z) {
  using ts::pad;
  const int t = threadIdx.x, nt = blockDim.x;
  const int T = L / kTsVals;
  const bool two = r0 + 1 < R;
  const int half = L / 2;
  const int zlen = L + L / 16;
  float2* P0 = z + zlen + 1;           // L/2 + 1
  float2* P1 = P0 + half + 1;          // L/2 + 1
  for (int f = t; f <= half; f += nt) {
    P0[f] = make_float2(1.f, 0.f);
    P1[f] = make_float2(1.f, 0.f);
  }
  for (int n = 0; n < a.N; ++n) {
    for (int q = t; q < zlen; q += nt) z[q] = make_float2(0.f, 0.f);
    __syncthreads();
    const float* f0 = a.F[n] + r0 * a.ldf[n];
    const float* f1 = f0 + a.ldf[n];
    const int In = a.dims[n];
    // four entries per thread loaded together, then added (one memory round trip per four)
    for (int i0 = t; i0 < In; i0 += 4 * nt) {
      unsigned hv[4];
      float x0[4], x1[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * nt;
        const bool in = i < In;
        hv[u] = in ? (unsigned)__ldg(a.h[n] + i) : 0xffffffffu;
        const float sg = in && __ldg(a.s[n] + i) < 0 ? -1.f : 1.f;
        x0[u] = in ? sg * __ldg(f0 + i) : 0.f;
        x1[u] = in && two ? sg * __ldg(f1 + i) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (hv[u] >= (unsigned)L) continue;          // past the mode, or a caller-supplied map out of range
        float2* d = z + pad((int)hv[u]);
        atomicAdd(&d->x, x0[u]);
        if (two) atomicAdd(&d->y, x1[u]);
      }
    }
    __syncthreads();
    {
      const int Lo = ts::opaque(L);
      ts::fft(z, tw, Lo, ts::opaque(logL), ts::opaque(t), Lo / kTsVals);
    }
    for (int f = t; f <= half; f += nt) {
      const float2 zf = z[pad(f)];
      const float2 zc = z[pad((L - f) & (L - 1))];
      const float2 c0 = make_float2(0.5f * (zf.x + zc.x), 0.5f * (zf.y - zc.y));   // (Z + conj Zc)/2
      const float2 c1 = make_float2(0.5f * (zf.y + zc.y), -0.5f * (zf.x - zc.x));  // (Z - conj Zc)/2i
      P0[f] = ts::cmul(P0[f], c0);
      P1[f] = ts::cmul(P1[f], c1);
    }
    __syncthreads();
  }
  // conj(W) with W = P_r + i P_{r+1} over the whole spectrum (W[L-f] = conj P_r[f] + i conj P_{r+1}[f])
  for (int f = t; f <= half; f += nt) {
    const float2 p0 = P0[f], p1 = P1[f];
    z[pad(f)] = make_float2(p0.x - p1.y, -(p0.y + p1.x));
    if (f > 0 && f < half) z[pad(L - f)] = make_float2(p0.x + p1.y, p0.y - p1.x);
  }
  __syncthreads();
  ts::fft(z, tw, L, logL, t, T);
  // x = conj(FFT(conj W)) / L: column r0 = Re, column r0 + 1 = Im
  const float s0 = (float)(lambda[r0] / (double)L);
  const float s1 = two ? (float)(lambda[r0 + 1] / (double)L) : 0.f;
  if (cm) {
    // each column is contiguous: consecutive threads store consecutive l
    float* y0 = Y + r0 * ldy;
    float* y1 = y0 + ldy;
    for (int l = t; l < L; l += nt) {
      const float2 v = z[pad(l)];
      y0[l] = v.x * s0;
      if (two) y1[l] = -v.y * s1;
    }
    return;
  }
  const bool vec = two && ((ldy & 1) == 0) && ((((uintptr_t)(Y + r0)) & 7) == 0);
  for (int l = t; l < L; l += nt) {
    const float2 v = z[pad(l)];
    float* y = Y + (int64_t)l * ldy + r0;
    if (vec) {
      *reinterpret_cast<float2*>(y) = make_float2(v.x * s0, -v.y * s1);
    } else {
      y[0] = v.x * s0;
      if (two) y[1] = -v.y * s1;
    }
  }
}

}  // namespace idl
