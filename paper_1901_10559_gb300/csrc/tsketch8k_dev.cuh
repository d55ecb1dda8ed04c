// tsketch8k_dev.cuh -- TensorSketch for the sketch length L = 8192 (Sec. 1.3,
// Eq. TA-formula; the sketch step of Algorithm 3):  Y[:, r] = lambda_r * IFFT(prod_n FFT(S^(n) a^(n)_r)).
//
// Persistent blocks of 512 threads, one per SM; each block takes pairs of
// columns (r, r+1) in turn.  The two columns of a pair are packed as the real
// and imaginary parts of one complex length-8192 vector per mode.
//
// The FFT is an in-place mixed-radix decimation in frequency with
// 8192 = 16 * 16 * 32 (index digits n = 512 n1 + 32 n2 + n'', frequency
// f = k1 + 16 k2 + 256 k''):
//   pass 1: thread t (= n' = 32 n2 + n'') takes the 16 values x[512 n1 + t],
//           a 16-point DFT over n1, the twiddles exp(-2 pi i t k1 / 8192) (formed
//           from the table's powers k1 = 1, 2, 4, 8 by products), and
//           writes them back to the same 16 places (segment k1);
//   pass 2: warp w (segment k1 = w), lane n'' takes x[512 w + 32 n2 + n''],
//           a 16-point DFT over n2, the twiddles exp(-2 pi i n'' k2 / 512),
//           written back in place;
//   pass 3: the 32 values of (w, k2) are contiguous; lanes k2 and k2 + 16 of
//           warp w split the 32-point DFT into its even (k'' = 2k') and odd
//           (k'' = 2k' + 1) outputs (one radix-2 step, then 16-point DFTs).
// Every pass reads and writes one index set per thread, so no barrier sits
// between a pass's reads and writes; passes 2 and 3 of a warp touch only its
// own segment (a warp barrier between them).  The spectrum ends in
// digit-reversed order: frequency f sits at position 512 k1 + 32 k2 + k''.
// The products of the spectra are elementwise, so that order is kept, and the
// inverse transform runs the adjoint passes in reverse order (pass 3^H, 2^H,
// 1^H with conjugate twiddles), giving natural order in registers, which are
// stored straight to Y.
//
// The spectra of the two real columns are separated by Hermitian symmetry,
//   C_r[f] = (Z[f] + conj Z[-f]) / 2,   C_{r+1}[f] = (Z[f] - conj Z[-f]) / 2i,
// for one representative f of each pair {f, -f} (8 per thread, plus f = 4096
// on thread 0), and multiplied into running products kept in registers (the
// self-paired f = 4096 in shared memory).  The
// thread that reads Z[f] and Z[-f] zeroes both places, so the vector is clear
// for the next mode's scatter without another pass.
//
// Shared memory: the vector (one pad entry per 32, so every pass is free of
// bank conflicts beyond the two wavefronts of a 64-bit warp access), the
// pass-1 twiddles (4 x 512) and the pass-2 twiddles (4 x 32), built once per
// context in FP64 (GB300's FP64 pipes are narrow: a per-block build cost more
// than the transforms) and copied in by every block.
#pragma once

#include <utility>

#include "common.cuh"
#include "tsketch_dev.cuh"

namespace idl {
namespace ts8 {

constexpr int kL = 8192;
constexpr int kT = 512;                 // threads per block
constexpr int kZ = kL + kL / 32;        // padded vector
constexpr int kTw1 = 4 * kT;               // w^1, w^2, w^4, w^8 of w = exp(-2 pi i t / 8192), per thread t
constexpr int kTw2 = 4 * 32;               // the same of exp(-2 pi i l / 512), per lane l
constexpr int kSeg = 528;               // padded segment of 512 values
constexpr int kMaxPre = 2;              // factor entries per thread held in registers (I_n <= 1024)
constexpr size_t kSmemBytes = sizeof(float2) * (size_t)(kZ + kTw1 + kTw2 + 2);

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {   // a * conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// cos(pi m / 16), sin(pi m / 16) for m = 0..8 (mathematical constants)
__host__ __device__ constexpr float cos16(int m) {
  return m == 0 ? 1.0f : m == 1 ? 0.98078528040323044913f : m == 2 ? 0.92387953251128675613f
       : m == 3 ? 0.83146961230254523708f : m == 4 ? 0.70710678118654752440f : m == 5 ? 0.55557023301960222474f
       : m == 6 ? 0.38268343236508977173f : m == 7 ? 0.19509032201612826785f : 0.0f;
}
__host__ __device__ constexpr float sin16(int m) { return cos16(8 - m); }

// d * exp(-/+ 2 pi i m / 32), 0 <= m < 16  (INV: the + sign)
template <int M, bool INV>
__device__ __forceinline__ float2 rot32(float2 d) {
  constexpr float c = M <= 8 ? cos16(M) : -cos16(16 - M);
  constexpr float s0 = M <= 8 ? sin16(M) : sin16(16 - M);
  constexpr float s = INV ? s0 : -s0;                        // imaginary part of the factor
  if constexpr (M == 0) return d;
  else if constexpr (M == 8) return INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
  else return make_float2(d.x * c - d.y * s, d.x * s + d.y * c);
}

// Radix-2 decimation-in-frequency 16-point DFT in registers, natural order in
// and out: v[k] <- sum_n v[n] exp(-/+ 2 pi i n k / 16).
template <bool INV, int S, int A>
__device__ __forceinline__ void dif_pair(float2* v) {
  if constexpr ((A & S) == 0) {
    const float2 x = v[A], y = v[A + S];
    v[A] = make_float2(x.x + y.x, x.y + y.y);
    v[A + S] = rot32<2 * (A & (S - 1)) * (8 / S), INV>(make_float2(x.x - y.x, x.y - y.y));
  }
}
template <bool INV, int S, int... A>
__device__ __forceinline__ void dif_stage(float2* v, std::integer_sequence<int, A...>) {
  (dif_pair<INV, S, A>(v), ...);
}
template <bool INV, int S>
__device__ __forceinline__ void dif_stages(float2* v) {
  if constexpr (S >= 1) {
    dif_stage<INV, S>(v, std::make_integer_sequence<int, 16>{});
    dif_stages<INV, S / 2>(v);
  }
}
template <int X>
constexpr int rev4() {
  return ((X & 1) << 3) | ((X & 2) << 1) | ((X & 4) >> 1) | ((X & 8) >> 3);
}
template <int... A>
__device__ __forceinline__ void rev_perm(float2* v, std::integer_sequence<int, A...>) {
  float2 t[16];
  ((t[A] = v[rev4<A>()]), ...);
  ((v[A] = t[A]), ...);
}
template <bool INV>
__device__ __forceinline__ void dft16(float2* v) {
  dif_stages<INV, 8>(v);
  rev_perm(v, std::make_integer_sequence<int, 16>{});
}

// pass 3 helpers (the radix-2 step of the 32-point DFT and its adjoint)
template <int... M>
__device__ __forceinline__ void split32(float2* y, const float2* z, bool odd, std::integer_sequence<int, M...>) {
  // even lane: y[m] = w[m] + w[m+16]; odd lane: (w[m] - w[m+16]) * exp(-2 pi i m / 32)
  ((y[M] = [&] {
     const float2 a = z[M], c = z[M + 16];
     const float2 d = odd ? make_float2(a.x - c.x, a.y - c.y) : make_float2(a.x + c.x, a.y + c.y);
     const float2 r = rot32<M, false>(d);
     return odd ? r : d;
   }()), ...);
}
template <int... M>
__device__ __forceinline__ void rot_odd_inv(float2* v, bool odd, std::integer_sequence<int, M...>) {
  ((v[M] = odd ? rot32<M, true>(v[M]) : v[M]), ...);
}

// The pass twiddles w^1 .. w^15 from the table's w, w^2, w^4, w^8 (w^3 = w^2 w, w^5 = w^4 w,
// ..., w^15 = w^8 w^7: at most three products of rounded factors), multiplied into
// v[1..15] (conjugated for the inverse passes).  Four shared-memory loads instead of
// fifteen: the transform is bound by shared-memory bandwidth, not by the FMA pipe.
template <bool CONJ>
__device__ __forceinline__ void apply_twiddles(float2* v, const float2* w) {
  const float2 w1 = w[0], w2 = w[1], w4 = w[2], w8 = w[3];
  auto app = [&](int q, float2 w) { v[q] = CONJ ? cmulc(v[q], w) : cmul(v[q], w); };
  const float2 w3 = cmul(w2, w1);
  const float2 w5 = cmul(w4, w1), w6 = cmul(w4, w2), w7 = cmul(w4, w3);
  app(1, w1); app(2, w2); app(3, w3); app(4, w4); app(5, w5); app(6, w6); app(7, w7); app(8, w8);
  app(9, cmul(w8, w1)); app(10, cmul(w8, w2)); app(11, cmul(w8, w3)); app(12, cmul(w8, w4));
  app(13, cmul(w8, w5)); app(14, cmul(w8, w6)); app(15, cmul(w8, w7));
}

// Entry e of the twiddle table of passes 1 and 2 (kTw1 + kTw2 entries, built once
// per context in FP64 and rounded): e < kTw1: exp(-2 pi i t 2^j / 8192) at
// [j 512 + t], j = 0..3; then exp(-2 pi i l 2^j / 512) at [kTw1 + j 32 + l].
__device__ __forceinline__ float2 table_entry(int e) {
  int num, den;
  if (e < kTw1) { const int j = e / kT, t = e % kT; num = t << j; den = kL; }
  else { const int q = e - kTw1, j = q / 32, l = q % 32; num = l << j; den = 512; }
  double sv, cv;
  sincospi(-2.0 * (double)(num % den) / (double)den, &sv, &cv);
  return make_float2((float)cv, (float)sv);
}

__device__ __forceinline__ int pz(int i) { return i + (i >> 5); }

// Entries of one mode held in registers ahead of their scatter.
struct Pre {
  int h[kMaxPre];
  float x0[kMaxPre], x1[kMaxPre];
};

__device__ __forceinline__ void load_mode(const TsArgs& a, int n, int64_t r0, bool two, Pre& p) {
  const float* f0 = a.F[n] + r0 * a.ldf[n];
  const float* f1 = f0 + a.ldf[n];
  const int In = a.dims[n];
#pragma unroll
  for (int u = 0; u < kMaxPre; ++u) {
    const int i = threadIdx.x + u * kT;
    const bool in = i < In;
    p.h[u] = in ? __ldg(a.h[n] + i) : -1;
    const float sg = in && __ldg(a.s[n] + i) < 0 ? -1.f : 1.f;
    p.x0[u] = in ? sg * __ldg(f0 + i) : 0.f;
    p.x1[u] = in && two ? sg * __ldg(f1 + i) : 0.f;
  }
}

__device__ __forceinline__ void scatter_mode(const TsArgs& a, int n, int64_t r0, bool two, const Pre& p, float2* z) {
#pragma unroll
  for (int u = 0; u < kMaxPre; ++u) {
    const unsigned hv = (unsigned)p.h[u];
    if (hv < (unsigned)kL) {               // past the mode, or a caller-supplied map out of range
      float2* d = z + pz((int)hv);
      atomicAdd(&d->x, p.x0[u]);
      if (two) atomicAdd(&d->y, p.x1[u]);
    }
  }
  // entries beyond the register-held ones (I_n > 1024)
  const int In = a.dims[n];
  if (In > kMaxPre * kT) {
    const float* f0 = a.F[n] + r0 * a.ldf[n];
    const float* f1 = f0 + a.ldf[n];
    for (int i = threadIdx.x + kMaxPre * kT; i < In; i += kT) {
      const unsigned hv = (unsigned)__ldg(a.h[n] + i);
      if (hv >= (unsigned)kL) continue;
      const float sg = __ldg(a.s[n] + i) < 0 ? -1.f : 1.f;
      float2* d = z + pz((int)hv);
      atomicAdd(&d->x, sg * __ldg(f0 + i));
      if (two) atomicAdd(&d->y, sg * __ldg(f1 + i));
    }
  }
}

// forward passes; z holds the mode's vector, natural order in, digit-reversed out
__device__ __forceinline__ void fwd_pass1(float2* z, const float2* tw1) {  // tw1: this thread's 4 powers
  const int t = threadIdx.x, base = t + (t >> 5);
  float2 v[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = z[q * kSeg + base];
  dft16<false>(v);
  apply_twiddles<false>(v, tw1);
#pragma unroll
  for (int q = 0; q < 16; ++q) z[q * kSeg + base] = v[q];
}

__device__ __forceinline__ void fwd_pass23(float2* z, const float2* tw2) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  {
    const int b2 = w * kSeg + lane;
    float2 v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = z[b2 + q * 33];
    dft16<false>(v);
    apply_twiddles<false>(v, tw2);
#pragma unroll
    for (int q = 0; q < 16; ++q) z[b2 + q * 33] = v[q];
  }
  __syncwarp();
  {
    const bool odd = lane >= 16;
    const int b3 = w * kSeg + (lane & 15) * 33;
    float2 y[16];
    split32(y, z + b3, odd, std::make_integer_sequence<int, 16>{});
    dft16<false>(y);
    __syncwarp();                                   // the partner lane has read its inputs
    const int e = odd ? 1 : 0;
#pragma unroll
    for (int q = 0; q < 16; ++q) z[b3 + 2 * q + e] = y[q];
  }
}

// position of frequency f (digit-reversed, padded)
__device__ __forceinline__ int fpos(int f) {
  return (f & 15) * kSeg + ((f >> 4) & 15) * 33 + (f >> 8);
}

// Representative j (0..7) of this thread: f = c + 256 k'' with c = 16 w + 2 j + b,
// k'' = lane & 15, b = lane >> 4.
__device__ __forceinline__ int rep_f(int j) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  return (16 * w + 2 * j + (lane >> 4)) + 256 * (lane & 15);
}

// Hermitian separation of one frequency pair {f, -f} of the packed spectrum into the
// two columns' spectra, multiplied into their running products; clears both places.
__device__ __forceinline__ void sep_mul(float2* z, int f, float2& P0, float2& P1) {
  const int fc = (kL - f) & (kL - 1);
  const int p = fpos(f), pc = fpos(fc);
  const float2 zf = z[p], zc = z[pc];
  z[p] = make_float2(0.f, 0.f);
  z[pc] = make_float2(0.f, 0.f);
  const float2 c0 = make_float2(0.5f * (zf.x + zc.x), 0.5f * (zf.y - zc.y));   // (Z + conj Zc)/2
  const float2 c1 = make_float2(0.5f * (zf.y + zc.y), -0.5f * (zf.x - zc.x));  // (Z - conj Zc)/2i
  P0 = cmul(P0, c0);
  P1 = cmul(P1, c1);
}

// W = P_r + i P_{r+1} at f and -f (digit-reversed layout)
__device__ __forceinline__ void put_w(float2* z, int f, float2 p0, float2 p1) {
  const int fc = (kL - f) & (kL - 1);
  z[fpos(f)] = make_float2(p0.x - p1.y, p0.y + p1.x);
  if (fc != f) z[fpos(fc)] = make_float2(p0.x + p1.y, p1.x - p0.y);   // conj P_r + i conj P_{r+1}
}

// All representatives of the thread; the self-paired f = 4096 (thread 0) keeps its
// products in shared memory (ext[0], ext[1]).
__device__ __forceinline__ void hadamard(float2* z, float2* P0, float2* P1, float2* ext) {
#pragma unroll
  for (int j = 0; j < 8; ++j) sep_mul(z, rep_f(j), P0[j], P1[j]);
  if (threadIdx.x == 0) sep_mul(z, kL / 2, ext[0], ext[1]);
}

__device__ __forceinline__ void build_w(float2* z, const float2* P0, const float2* P1, const float2* ext) {
#pragma unroll
  for (int j = 0; j < 8; ++j) put_w(z, rep_f(j), P0[j], P1[j]);
  if (threadIdx.x == 0) put_w(z, kL / 2, ext[0], ext[1]);
}

// inverse passes 3^H and 2^H (warp-local)
__device__ __forceinline__ void inv_pass32(float2* z, const float2* tw2) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  {
    const bool odd = lane >= 16;
    const int e = odd ? 1 : 0;
    const int b3 = w * kSeg + (lane & 15) * 33;
    float2 v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = z[b3 + 2 * q + e];
    dft16<true>(v);                                  // A_e[m]
    rot_odd_inv(v, odd, std::make_integer_sequence<int, 16>{});
    float2 o[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const float2 r = make_float2(__shfl_xor_sync(0xffffffffu, v[q].x, 16), __shfl_xor_sync(0xffffffffu, v[q].y, 16));
      // even lane: A0 + B1 (own A0, partner's B1); odd lane: A0 - B1 (partner's A0, own B1)
      o[q] = odd ? make_float2(r.x - v[q].x, r.y - v[q].y) : make_float2(v[q].x + r.x, v[q].y + r.y);
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 16; ++q) z[b3 + 16 * e + q] = o[q];
  }
  __syncwarp();
  {
    const int b2 = w * kSeg + lane;
    float2 v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = z[b2 + q * 33];
    apply_twiddles<true>(v, tw2);
    dft16<true>(v);
#pragma unroll
    for (int q = 0; q < 16; ++q) z[b2 + q * 33] = v[q];
  }
}

// inverse pass 1^H: natural-order results x[512 q + t] in v; clears the thread's places
__device__ __forceinline__ void inv_pass1(float2* z, const float2* tw1, float2* v) {
  const int t = threadIdx.x, base = t + (t >> 5);
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    v[q] = z[q * kSeg + base];
    z[q * kSeg + base] = make_float2(0.f, 0.f);
  }
  apply_twiddles<true>(v, tw1);
  dft16<true>(v);
}

// The transforms of one pair of columns (r0, r0 + 1): on return v[q] holds entry
// l = 512 q + t of column r0 (.x) and r0 + 1 (.y) before the scale s0 / s1 (lambda_r / L;
// s1 = 0 past the last column).  z must be zero on entry and is zero on return, but
// the caller synchronises the block before z is used again.  pre: mode 0's entries
// (loaded by the caller).
__device__ __forceinline__ void pair_core(const TsArgs& a, int64_t R, int64_t r0, const double* __restrict__ lambda,
                                          Pre& pre, float2* z, const float2* tw1, const float2* tw2, float2* v,
                                          float& s0, float& s1) {
  const bool two = r0 + 1 < R;
  // this thread's twiddle powers, held in registers for the pair's 2N + 2 passes
  float2 w1[4], w2[4];
  {
    const int t = threadIdx.x, lane = t & 31;
#pragma unroll
    for (int j = 0; j < 4; ++j) { w1[j] = tw1[j * kT + t]; w2[j] = tw2[j * 32 + lane]; }
  }
  float2 P0[8], P1[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) { P0[j] = make_float2(1.f, 0.f); P1[j] = make_float2(1.f, 0.f); }
  float2* ext = z + kZ + kTw1 + kTw2;              // products of f = 4096 (thread 0)
  if (threadIdx.x == 0) { ext[0] = make_float2(1.f, 0.f); ext[1] = make_float2(1.f, 0.f); }
  for (int n = 0; n < a.N; ++n) {
    scatter_mode(a, n, r0, two, pre, z);
    if (n + 1 < a.N) load_mode(a, n + 1, r0, two, pre);     // in flight during this mode's transform
    __syncthreads();
    fwd_pass1(z, w1);
    __syncthreads();
    fwd_pass23(z, w2);
    __syncthreads();
    hadamard(z, P0, P1, ext);
    __syncthreads();
  }
  build_w(z, P0, P1, ext);
  __syncthreads();
  inv_pass32(z, w2);
  __syncthreads();
  inv_pass1(z, w1, v);
  s0 = (float)(lambda[r0] / (double)kL);
  s1 = two ? (float)(lambda[r0 + 1] / (double)kL) : 0.f;
}

// One pair of columns (r0, r0 + 1) written to Y: column-major (cm: column r at
// Y + r ldy) or row-major (Y[l ldy + r]).  z must be zero on entry and is zero on exit.
__device__ __forceinline__ void pair_body(const TsArgs& a, int64_t R, int64_t r0, const double* __restrict__ lambda,
                                          float* __restrict__ Y, int64_t ldy, bool cm, Pre& pre, float2* z,
                                          const float2* tw1, const float2* tw2) {
  const bool two = r0 + 1 < R;
  float2 v[16];
  float s0, s1;
  pair_core(a, R, r0, lambda, pre, z, tw1, tw2, v, s0, s1);
  const int t = threadIdx.x;
  if (cm) {
    float* y0 = Y + r0 * ldy;
    float* y1 = y0 + ldy;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      y0[q * kT + t] = v[q].x * s0;
      if (two) y1[q * kT + t] = v[q].y * s1;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      float* y = Y + (int64_t)(q * kT + t) * ldy + r0;
      y[0] = v[q].x * s0;
      if (two) y[1] = v[q].y * s1;
    }
  }
  __syncthreads();                  // every place of z is clear before the next pair's scatter
}

// Shared-memory set-up of a persistent block: the twiddle table copied in from
// global memory (tab: kTw1 + kTw2 entries), the vector cleared.
__device__ __forceinline__ void block_setup(float2* sm, const float2* __restrict__ tab, float2** z, float2** tw1,
                                            float2** tw2) {
  *z = sm;
  *tw1 = sm + kZ;
  *tw2 = *tw1 + kTw1;
  const float4* src = reinterpret_cast<const float4*>(tab);
  float4* dst = reinterpret_cast<float4*>(*tw1);
  for (int q = threadIdx.x; q < (kTw1 + kTw2) / 2; q += blockDim.x) dst[q] = __ldg(src + q);
  for (int q = threadIdx.x; q < kZ; q += blockDim.x) sm[q] = make_float2(0.f, 0.f);
  __syncthreads();
}

}  // namespace ts8
}  // namespace idl
