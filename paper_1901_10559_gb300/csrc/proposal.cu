// proposal.cu -- the learned column proposal of the QR stage for one problem
// (features -> MLP scores -> top-C candidates -> candidate QR -> certificate ->
// gated fallback), the MLP's training kernels (forward + backward per tile,
// fixed-order gradient reduction fused with the Adam step) and the weight file.
// Device bodies: proposal_dev.cuh.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "cpqr_dev.cuh"
#include "proposal_dev.cuh"

#define TRY(x)                     \
  do {                             \
    int _rc = (x);                 \
    if (_rc != IDL_OK) return _rc; \
  } while (0)

namespace idl {

using namespace prop;

// Example order of an epoch: position g -> example (a g + b) mod n with
// gcd(a, n) = 1, a permutation of [0, n).
struct Perm { int64_t a, b; };

__global__ void __launch_bounds__(kThreads) prop_gram_kernel(const float* __restrict__ Y, int ld, int m, int R,
                                                             float* __restrict__ Gp, float* __restrict__ nmaxp) {
  extern __shared__ __align__(16) float smf[];
  gram_partial_block(Y, ld, m, R, blockIdx.x, Gp, nmaxp, smf);
}

__global__ void __launch_bounds__(kThreads) prop_gram_reduce_kernel(const float* __restrict__ Gp, int nsplit,
                                                                    const float* __restrict__ nmaxp, int m,
                                                                    float* __restrict__ G, float* __restrict__ scal) {
  gram_reduce_elem(Gp, nsplit, nmaxp, m, blockIdx.x * blockDim.x + threadIdx.x, G, scal);
}

__global__ void __launch_bounds__(kThreads) prop_chol_kernel(const float* __restrict__ G, int m,
                                                             float* __restrict__ Linv, float* __restrict__ scal) {
  extern __shared__ __align__(16) float smf[];
  chol_inv_block(G, m, blockIdx.x, Linv, scal, smf);
}

__global__ void __launch_bounds__(kThreads) prop_features_kernel(const float* __restrict__ Y, int ld, int m, int R,
                                                                 int K, const float* __restrict__ Linv,
                                                                 const float* __restrict__ scal, float* __restrict__ F) {
  extern __shared__ __align__(16) float smf[];
  features_block(Y, ld, m, R, K, Linv, scal, blockIdx.x, F, smf);
}

__global__ void __launch_bounds__(kThreads) prop_norm_kernel(const float* __restrict__ Y, int ld, int m, int R,
                                                             float* __restrict__ s) {
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c < R) norm_scores_warp(Y, ld, m, c, s);
}

__global__ void __launch_bounds__(kThreads, 1) prop_mlp_fwd_kernel(const float* __restrict__ theta,
                                                                   const float* __restrict__ F, int64_t n,
                                                                   float* __restrict__ s) {
  extern __shared__ __align__(16) float smf[];
  mlp_forward_tile(theta, F, n, (int64_t)blockIdx.x * kTile, s, smf);
}

__global__ void __launch_bounds__(kSelThreads) prop_select_kernel(const float* __restrict__ s, int R, int C,
                                                                  int32_t* __restrict__ cand, int32_t* __restrict__ outl) {
  select_block(s, R, C, cand, outl);
}

__global__ void __launch_bounds__(kApplyThreads) prop_apply_kernel(const float* __restrict__ Y2, float* __restrict__ Yf,
                                                                   int ld, int m, int K, const int32_t* __restrict__ outl,
                                                                   int nout, const float* __restrict__ V,
                                                                   const float* __restrict__ beta,
                                                                   const double* __restrict__ rn, int* cert_fail,
                                                                   double* diag) {
  extern __shared__ __align__(16) float smf[];
  apply_cert_block(Y2, Yf, ld, m, K, outl, nout, V, beta, rn, cert_fail, diag, blockIdx.x, gridDim.x, smf);
}

// Candidate QR: the K-step pivoted QR of the C candidate columns in one CTA,
// recording the reflectors (cpqr_cta_body).
template <int V, int TPC>
__global__ void __launch_bounds__(CtaCpqr<float, V, TPC>::kMaxThreads, 1)
prop_cand_kernel(const float* __restrict__ Y2, float* __restrict__ Yf, int m, int C, int ld, int K,
                 int32_t* __restrict__ J, double* __restrict__ rn, double* __restrict__ diag, int* status,
                 const int32_t* __restrict__ cand, float* __restrict__ V_, float* __restrict__ beta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpqr_cta_body<float, V, TPC>(Y2, Yf, m, C, ld, K, J, rn, diag, status, smem_raw, cand, V_, beta);
}

// Gathers minibatch positions [p0, p0 + nb) of the epoch order into contiguous rows.
__global__ void prop_gather_kernel(const float* __restrict__ F, const float* __restrict__ y, int64_t n, Perm pm,
                                   int64_t p0, int nb, float* __restrict__ Fb, float* __restrict__ yb) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nb) return;
  const int64_t src = (pm.a * (p0 + e) + pm.b) % n;
#pragma unroll
  for (int f = 0; f < kNF; ++f) Fb[(int64_t)e * kNF + f] = F[src * kNF + f];
  yb[e] = y[src];
}

__global__ void __launch_bounds__(kThreads, 1) prop_mlp_bwd_kernel(const float* __restrict__ theta,
                                                                   const float* __restrict__ F,
                                                                   const float* __restrict__ y, int64_t n,
                                                                   float pos_weight, float inv_nb,
                                                                   float* __restrict__ gpart, float* __restrict__ lpart) {
  extern __shared__ __align__(16) float smf[];
  mlp_backward_tile(theta, F, y, n, (int64_t)blockIdx.x * kTile, pos_weight, inv_nb,
                    gpart + (int64_t)blockIdx.x * kNParam, lpart + blockIdx.x, smf);
}

// grad = sum of the block partials in block order; optionally one Adam step
// (Kingma & Ba 2015) on the FP32 master weights; loss = sum of the block losses.
__global__ void prop_reduce_adam_kernel(float* __restrict__ theta, float* __restrict__ mom, float* __restrict__ vel,
                                        const float* __restrict__ gpart, int nblk, const float* __restrict__ lpart,
                                        float* __restrict__ grad_out, float* __restrict__ loss_out, int update, float lr,
                                        float b1, float b2, float eps, float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0 && loss_out) {
    float l = 0.f;
    for (int b = 0; b < nblk; ++b) l += lpart[b];
    *loss_out = l;
  }
  if (p >= kNParam) return;
  float g = 0.f;
  for (int b = 0; b < nblk; ++b) g += gpart[(int64_t)b * kNParam + p];
  if (grad_out) grad_out[p] = g;
  if (!update) return;
  const float mm = b1 * mom[p] + (1.f - b1) * g;
  const float vv = b2 * vel[p] + (1.f - b2) * g * g;
  mom[p] = mm;
  vel[p] = vv;
  theta[p] -= lr * (mm * c1) / (sqrtf(vv * c2) + eps);
}

// labels[J[t]] = 1 (J from the plain QR)
__global__ void prop_labels_kernel(const int32_t* __restrict__ J, int K, int R, float* __restrict__ y) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < K) {
    const int j = J[t];
    if (j >= 0 && j < R) y[j] = 1.f;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int set_smem(idl_ctx* ctx, const void* kern, size_t bytes) {
  if (bytes > (size_t)ctx->smem_optin) return fail(ctx, IDL_ELIMIT, "proposal: shared memory");
  return cuda_check(ctx, ensure_smem(ctx, (const void*)kern, bytes),
                    "proposal smem attribute");
}

static float* mlp_state(idl_ctx* ctx) {
  if (!ctx->mlp) {
    if (cudaMalloc(&ctx->mlp, sizeof(float) * 3 * kNParam) != cudaSuccess) {
      (void)cudaGetLastError();
      ctx->mlp = nullptr;
      ctx->err = "MLP state allocation failed";
      return nullptr;
    }
    cudaMemsetAsync(ctx->mlp, 0, sizeof(float) * 3 * kNParam, ctx->stream);
  }
  return ctx->mlp;
}

int launch_features(idl_ctx* ctx, const float* Y, int64_t m, int64_t R, int64_t ld, int64_t K, float* F) {
  if (m < 1 || m > kMaxM) return fail(ctx, IDL_ELIMIT, "proposal: needs 1 <= m <= 128");
  const int nsplit = (int)cdiv(R, kGramCols);
  float* Gp = (float*)ws_get(ctx, kWsPropGram, sizeof(float) * ((size_t)nsplit * m * m + nsplit + 4 + 4 * m * m));
  if (!Gp) return IDL_ENOMEM;
  float* nmaxp = Gp + (size_t)nsplit * m * m;
  float* scal = nmaxp + nsplit;
  float* Linv = scal + 4;
  float* G = Linv + 3 * m * m;
  const size_t sm_gram = sizeof(float) * 32 * round_up(m, 4);
  const size_t sm_chol = sizeof(float) * (2 * (size_t)m * (m + 1) + m);
  const size_t sm_feat = sizeof(float) * features_smem_floats((int)m);
  TRY(set_smem(ctx, (const void*)prop_chol_kernel, sm_chol));
  TRY(set_smem(ctx, (const void*)prop_features_kernel, sm_feat));
  prop_gram_kernel<<<nsplit, kThreads, sm_gram, ctx->stream>>>(Y, (int)ld, (int)m, (int)R, Gp, nmaxp), count_launch();
  prop_gram_reduce_kernel<<<(unsigned)cdiv(m * m, kThreads), kThreads, 0, ctx->stream>>>(Gp, nsplit, nmaxp, (int)m, G,
                                                                                       scal), count_launch();
  prop_chol_kernel<<<3, kThreads, sm_chol, ctx->stream>>>(G, (int)m, Linv, scal), count_launch();
  prop_features_kernel<<<(unsigned)cdiv(R, kFeatCols), kThreads, sm_feat, ctx->stream>>>(Y, (int)ld, (int)m, (int)R,
                                                                                       (int)K, Linv, scal, F),
      count_launch();
  return cuda_check(ctx, cudaGetLastError(), "proposal features");
}

int launch_mlp_scores(idl_ctx* ctx, const float* F, int64_t n, float* s) {
  if (!ctx->mlp_ready) return fail(ctx, IDL_EINVAL, "proposal: no MLP weights (idl_mlp_init / idl_load_weights)");
  const size_t sm = sizeof(float) * mlp_fwd_smem_floats();
  TRY(set_smem(ctx, (const void*)prop_mlp_fwd_kernel, sm));
  prop_mlp_fwd_kernel<<<(unsigned)cdiv(n, kTile), kThreads, sm, ctx->stream>>>(ctx->mlp, F, n, s), count_launch();
  return cuda_check(ctx, cudaGetLastError(), "mlp scores");
}

template <int VV, int TT>
static bool cand_try(idl_ctx* ctx, const float* Y2, float* Yf, int64_t m, int64_t C, int64_t ld, int64_t K, int32_t* J,
                     double* rn, double* diag, const int32_t* cand, float* V, float* beta, int* rc) {
  if (cdiv(m, TT) > VV) return false;
  const int threads = (int)round_up(C * TT, 32);
  if (threads > CtaCpqr<float, VV, TT>::kMaxThreads) return false;
  prop_cand_kernel<VV, TT><<<1, threads, cta_cpqr_smem<float, VV, TT>(), ctx->stream>>>(
      Y2, Yf, (int)m, (int)C, (int)ld, (int)K, J, rn, diag, ctx->d_status, cand, V, beta);
  count_launch();
  *rc = cuda_check(ctx, cudaGetLastError(), "candidate QR");
  return true;
}

// Most lanes per column first (shortest serial chain per step).
static int launch_cand_qr(idl_ctx* ctx, const float* Y2, float* Yf, int64_t m, int64_t C, int64_t ld, int64_t K,
                          int32_t* J, double* rn, double* diag, const int32_t* cand, float* V, float* beta) {
  int rc = IDL_OK;
#define CAND(VV, TT) if (cand_try<VV, TT>(ctx, Y2, Yf, m, C, ld, K, J, rn, diag, cand, V, beta, &rc)) return rc;
  CAND(8, 32) CAND(8, 16) CAND(8, 8) CAND(16, 8) CAND(8, 4) CAND(16, 4) CAND(32, 4) CAND(16, 2) CAND(32, 2)
  CAND(16, 1) CAND(32, 1) CAND(64, 4) CAND(64, 2) CAND(64, 1) CAND(96, 1) CAND(128, 1)
#undef CAND
  return fail(ctx, IDL_ELIMIT, "proposal: the candidate set does not fit one CTA (lower cand_factor)");
}

// The QR stage through the proposal: Y2 (original sketch, read only) -> Yf
// (factored, the layout idl_cpqr produces), J.  The certificate flag is
// ctx->d_status[1]; the proposal's diagnostics go to d_diag[8..12] and the
// gated fallback moves or recomputes d_diag[0..4].
int launch_proposal_qr(idl_ctx* ctx, const float* Y2, float* Yf, int64_t m, int64_t R, int64_t ld, int64_t K,
                       int mode, int cand_factor, int32_t* J) {
  if (m > kMaxM) return fail(ctx, IDL_ELIMIT, "proposal: needs m <= 128");
  if (cand_factor < 0 || cand_factor > 8) return fail(ctx, IDL_EINVAL, "proposal: cand_factor must be in 0..8");
  if (K > 128) return fail(ctx, IDL_ELIMIT, "proposal: needs K <= 128");
  if (mode == IDL_PROPOSAL_MLP && !ctx->mlp_ready)
    return fail(ctx, IDL_EINVAL, "proposal: no MLP weights (idl_mlp_init / idl_load_weights)");
  const int64_t C = std::min<int64_t>((cand_factor ? cand_factor : 2) * K, R);
  const int64_t nout = R - C;
  // workspace: F (R x 8), scores (R), cand (C), outl (R - C), V (K x m), beta (K), rn (K doubles)
  const size_t bytes = sizeof(float) * (size_t)R * kNF + sizeof(float) * R + sizeof(int32_t) * (size_t)R +
                       sizeof(float) * (size_t)(K * m + K) + sizeof(double) * K + 64;
  unsigned char* w = (unsigned char*)ws_get(ctx, kWsProp, bytes);
  if (!w) return IDL_ENOMEM;
  double* rn = (double*)w;
  float* F = (float*)(rn + K);
  float* sc = F + (size_t)R * kNF;
  float* V = sc + R;
  float* beta = V + K * m;
  int32_t* cand = (int32_t*)(beta + K);
  int32_t* outl = cand + C;
  int* flag = ctx->d_status + 1;
  double* pdiag = ctx->d_diag + 8;
  TRY(cuda_check(ctx, cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream), "proposal flag"));
  if (mode == IDL_PROPOSAL_MLP) {
    TRY(launch_features(ctx, Y2, m, R, ld, K, F));
    TRY(launch_mlp_scores(ctx, F, R, sc));
  } else {
    prop_norm_kernel<<<(unsigned)cdiv(R, kThreads / 32), kThreads, 0, ctx->stream>>>(Y2, (int)ld, (int)m, (int)R, sc),
        count_launch();
  }
  prop_select_kernel<<<1, kSelThreads, 0, ctx->stream>>>(sc, (int)R, (int)C, cand, outl), count_launch();
  TRY(launch_cand_qr(ctx, Y2, Yf, m, C, ld, K, J, rn, pdiag, cand, V, beta));
  if (nout > 0) {
    const size_t sm = sizeof(float) * (size_t)(K * m + 2 * K);
    TRY(set_smem(ctx, (const void*)prop_apply_kernel, sm));
    const int nw = kApplyThreads / 32;
    const int blocks = (int)std::min<int64_t>(cdiv(nout, nw), 4 * (int64_t)ctx->num_sms);
    prop_apply_kernel<<<blocks, kApplyThreads, sm, ctx->stream>>>(Y2, Yf, (int)ld, (int)m, (int)K, outl, (int)nout, V,
                                                                  beta, rn, flag, pdiag), count_launch();
    TRY(cuda_check(ctx, cudaGetLastError(), "proposal apply"));
  }
  QrExtra xf;
  xf.gate = flag;
  return launch_cpqr_ex(ctx, Y2, Yf, m, R, ld, K, J, nullptr, xf);
}

}  // namespace idl

using namespace idl;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
static bool dev_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static int ctx_ok(idl_ctx* ctx) { return ctx_usable(ctx); }

extern "C" int idl_mlp_set_weights(idl_ctx* ctx, const float* theta) {
  TRY(ctx_ok(ctx));
  if (!theta) return fail(ctx, IDL_EINVAL, "mlp_set_weights: null");
  float* st = mlp_state(ctx);
  if (!st) return IDL_ENOMEM;
  cudaError_t e = cudaMemcpyAsync(st, theta, sizeof(float) * kNParam,
                                  dev_ptr(theta) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(st + kNParam, 0, sizeof(float) * 2 * kNParam, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  TRY(cuda_check(ctx, e, "mlp_set_weights"));
  ctx->mlp_step = 0;
  ctx->mlp_ready = true;
  return IDL_OK;
}

extern "C" int idl_mlp_get_weights(idl_ctx* ctx, float* theta) {
  TRY(ctx_ok(ctx));
  if (!theta) return fail(ctx, IDL_EINVAL, "mlp_get_weights: null");
  if (!ctx->mlp_ready) return fail(ctx, IDL_EINVAL, "mlp_get_weights: no weights");
  cudaError_t e = cudaMemcpyAsync(theta, ctx->mlp, sizeof(float) * kNParam,
                                  dev_ptr(theta) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  return cuda_check(ctx, e, "mlp_get_weights");
}

// He-style initial weights from the counter-based generator (host side, once).
extern "C" int idl_mlp_init(idl_ctx* ctx, uint64_t seed) {
  TRY(ctx_ok(ctx));
  std::vector<float> th(kNParam, 0.f);
  const uint64_t base = stream_base(seed, 64);
  auto gauss = [&](uint64_t i) {
    const uint64_t a = stream_at(base, 2 * i), b = stream_at(base, 2 * i + 1);
    const double u1 = ((a >> 11) + 1.0) * (1.0 / 9007199254740993.0);     // (0, 1]
    const double u2 = (b >> 11) * (1.0 / 9007199254740992.0);              // [0, 1)
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  };
  for (int i = 0; i < kHid * kNF; ++i) th[kOffW1 + i] = (float)(gauss(i) * std::sqrt(2.0 / kNF));
  for (int i = 0; i < kHid * kHid; ++i) th[kOffW2 + i] = (float)(gauss(100000 + i) * std::sqrt(2.0 / kHid));
  for (int i = 0; i < kHid; ++i) th[kOffW3 + i] = (float)(gauss(200000 + i) * std::sqrt(1.0 / kHid));
  return idl_mlp_set_weights(ctx, th.data());
}

// Weight file: "IDLMLP01", uint32 version 1, nf, hidden, nparam, nparam float32
// (little endian), uint64 FNV-1a hash of the parameter bytes.
static uint64_t fnv_bytes(const unsigned char* p, size_t n) {
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) { h ^= p[i]; h *= 1099511628211ull; }
  return h;
}

extern "C" int idl_save_weights(idl_ctx* ctx, const char* path) {
  TRY(ctx_ok(ctx));
  if (!path) return fail(ctx, IDL_EINVAL, "save_weights: null path");
  std::vector<float> th(kNParam);
  TRY(idl_mlp_get_weights(ctx, th.data()));
  FILE* f = fopen(path, "wb");
  if (!f) return fail(ctx, IDL_EINVAL, "save_weights: cannot open file");
  const uint32_t hdr[4] = {1u, (uint32_t)kNF, (uint32_t)kHid, (uint32_t)kNParam};
  const uint64_t h = fnv_bytes((const unsigned char*)th.data(), sizeof(float) * kNParam);
  bool ok = fwrite("IDLMLP01", 1, 8, f) == 8 && fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
            fwrite(th.data(), sizeof(float), kNParam, f) == (size_t)kNParam && fwrite(&h, sizeof(h), 1, f) == 1;
  ok = (fclose(f) == 0) && ok;
  return ok ? IDL_OK : fail(ctx, IDL_EINVAL, "save_weights: write failed");
}

extern "C" int idl_load_weights(idl_ctx* ctx, const char* path) {
  TRY(ctx_ok(ctx));
  if (!path) return fail(ctx, IDL_EINVAL, "load_weights: null path");
  FILE* f = fopen(path, "rb");
  if (!f) return fail(ctx, IDL_EINVAL, "load_weights: cannot open file");
  char magic[8];
  uint32_t hdr[4];
  std::vector<float> th(kNParam);
  uint64_t h = 0;
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "IDLMLP01", 8) == 0 && fread(hdr, sizeof(hdr), 1, f) == 1 &&
            hdr[0] == 1u && hdr[1] == (uint32_t)kNF && hdr[2] == (uint32_t)kHid && hdr[3] == (uint32_t)kNParam &&
            fread(th.data(), sizeof(float), kNParam, f) == (size_t)kNParam && fread(&h, sizeof(h), 1, f) == 1;
  fclose(f);
  if (!ok) return fail(ctx, IDL_EINVAL, "load_weights: not a weight file of this layout");
  if (fnv_bytes((const unsigned char*)th.data(), sizeof(float) * kNParam) != h)
    return fail(ctx, IDL_EINVAL, "load_weights: checksum mismatch");
  return idl_mlp_set_weights(ctx, th.data());
}

extern "C" int idl_proposal_features(idl_ctx* ctx, const float* Y, int64_t m, int64_t R, int64_t ldy, int64_t K,
                                     float* F) {
  TRY(ctx_ok(ctx));
  if (!Y || !F || R < 1 || ldy < m || K < 1) return fail(ctx, IDL_EINVAL, "proposal_features: bad arguments");
  return launch_features(ctx, Y, m, R, ldy, K, F);
}

extern "C" int idl_mlp_scores(idl_ctx* ctx, const float* F, int64_t n, float* s) {
  TRY(ctx_ok(ctx));
  if (!F || !s || n < 1) return fail(ctx, IDL_EINVAL, "mlp_scores: bad arguments");
  return launch_mlp_scores(ctx, F, n, s);
}

// Loss and gradient over n examples (one minibatch), no update.
extern "C" int idl_mlp_grad(idl_ctx* ctx, const float* F, const float* y, int64_t n, float pos_weight, float* grad,
                            float* loss) {
  TRY(ctx_ok(ctx));
  if (!F || !y || n < 1 || !grad || !loss) return fail(ctx, IDL_EINVAL, "mlp_grad: bad arguments");
  if (!ctx->mlp_ready) return fail(ctx, IDL_EINVAL, "mlp_grad: no weights");
  const int nblk = (int)cdiv(n, kTile);
  float* part = (float*)ws_get(ctx, kWsPropTrain, sizeof(float) * ((size_t)nblk * kNParam + nblk));
  if (!part) return IDL_ENOMEM;
  const size_t sm = sizeof(float) * mlp_bwd_smem_floats();
  TRY(set_smem(ctx, (const void*)prop_mlp_bwd_kernel, sm));
  prop_mlp_bwd_kernel<<<nblk, kThreads, sm, ctx->stream>>>(ctx->mlp, F, y, n, pos_weight, 1.f / (float)n, part,
                                                           part + (size_t)nblk * kNParam), count_launch();
  prop_reduce_adam_kernel<<<(unsigned)cdiv(kNParam, 256), 256, 0, ctx->stream>>>(
      ctx->mlp, ctx->mlp + kNParam, ctx->mlp + 2 * kNParam, part, nblk, part + (size_t)nblk * kNParam, grad, loss, 0,
      0.f, 0.f, 0.f, 0.f, 0.f, 0.f), count_launch();
  return cuda_check(ctx, cudaGetLastError(), "mlp_grad");
}

static int64_t gcd64(int64_t a, int64_t b) { while (b) { const int64_t t = a % b; a = b; b = t; } return a; }

extern "C" int idl_train_proposal(idl_ctx* ctx, const float* F, const float* y, int64_t n, const idl_train_params* tp,
                                  float* epoch_loss) {
  TRY(ctx_ok(ctx));
  if (!F || !y || n < 1 || !tp || tp->epochs < 1 || tp->batch < 1 || tp->batch > (1 << 20) || !(tp->lr > 0.f))
    return fail(ctx, IDL_EINVAL, "train_proposal: bad arguments");
  if (!dev_ptr(F) || !dev_ptr(y)) return fail(ctx, IDL_EINVAL, "train_proposal: F and y must be device pointers");
  if (!ctx->mlp_ready) TRY(idl_mlp_init(ctx, tp->seed));
  const int B = (int)std::min<int64_t>(tp->batch, n);
  const int nblk = (int)cdiv(B, kTile);
  const size_t part_f = (size_t)nblk * kNParam + nblk;
  float* part = (float*)ws_get(ctx, kWsPropTrain, sizeof(float) * (part_f + (size_t)B * (kNF + 1) + 64));
  if (!part) return IDL_ENOMEM;
  float* Fb = part + part_f;
  float* yb = Fb + (size_t)B * kNF;
  float* dloss = yb + B;
  const size_t sm = sizeof(float) * mlp_bwd_smem_floats();
  TRY(set_smem(ctx, (const void*)prop_mlp_bwd_kernel, sm));
  const float b1 = tp->beta1 > 0.f ? tp->beta1 : 0.9f, b2 = tp->beta2 > 0.f ? tp->beta2 : 0.999f;
  const float eps = tp->eps > 0.f ? tp->eps : 1e-8f;
  const float pw = tp->pos_weight > 0.f ? tp->pos_weight : 1.f;
  const int64_t steps_per_epoch = cdiv(n, B);
  std::vector<float> losses((size_t)steps_per_epoch);
  for (int ep = 0; ep < tp->epochs; ++ep) {
    // epoch order: a multiplicative permutation drawn from the seed
    const uint64_t u = stream_at(stream_base(tp->seed, 65), (uint64_t)ep);
    int64_t a = 1 + (int64_t)(u % (uint64_t)n);
    while (gcd64(a, n) != 1) ++a;
    const Perm pm{a, (int64_t)((u >> 32) % (uint64_t)n)};
    double ep_loss = 0.0;
    for (int64_t st = 0; st < steps_per_epoch; ++st) {
      const int64_t p0 = st * B;
      const int nb = (int)std::min<int64_t>(B, n - p0);
      const int blocks = (int)cdiv(nb, kTile);
      prop_gather_kernel<<<(unsigned)cdiv(nb, 256), 256, 0, ctx->stream>>>(F, y, n, pm, p0, nb, Fb, yb), count_launch();
      prop_mlp_bwd_kernel<<<blocks, kThreads, sm, ctx->stream>>>(ctx->mlp, Fb, yb, nb, pw, 1.f / (float)nb, part,
                                                                 part + (size_t)nblk * kNParam), count_launch();
      ++ctx->mlp_step;
      const double t = (double)ctx->mlp_step;
      const float c1 = (float)(1.0 / (1.0 - std::pow((double)b1, t)));
      const float c2 = (float)(1.0 / (1.0 - std::pow((double)b2, t)));
      prop_reduce_adam_kernel<<<(unsigned)cdiv(kNParam, 256), 256, 0, ctx->stream>>>(
          ctx->mlp, ctx->mlp + kNParam, ctx->mlp + 2 * kNParam, part, blocks, part + (size_t)nblk * kNParam, nullptr,
          dloss + (st % 32), 1, tp->lr, b1, b2, eps, c1, c2), count_launch();
      if (epoch_loss && (st % 32 == 31 || st == steps_per_epoch - 1)) {
        float h[32];
        const int cnt = (int)(st % 32) + 1;
        cudaError_t e = cudaMemcpyAsync(h, dloss, sizeof(float) * cnt, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        TRY(cuda_check(ctx, e, "train loss"));
        for (int q = 0; q < cnt; ++q) ep_loss += (double)h[q] * std::min<int64_t>(B, n - (st - cnt + 1 + q) * B);
      }
    }
    if (epoch_loss) epoch_loss[ep] = (float)(ep_loss / (double)n);
  }
  return cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "train_proposal");
}

// Training examples of one sketch: features F (R x 8) and labels y (R; 1 on
// the pivots of the plain QR, which runs on a private copy of Y).
extern "C" int idl_proposal_labels(idl_ctx* ctx, const float* Y, int64_t m, int64_t R, int64_t ldy, int64_t K,
                                   float* F, float* y) {
  TRY(ctx_ok(ctx));
  if (!Y || !F || !y || R < 2 || K < 1 || K >= R || K > m || ldy < m)
    return fail(ctx, IDL_EINVAL, "proposal_labels: bad arguments");
  TRY(launch_features(ctx, Y, m, R, ldy, K, F));
  float* Yc = (float*)ws_get(ctx, kWsPropCopy, sizeof(float) * (size_t)(ldy * R) + sizeof(int32_t) * K);
  if (!Yc) return IDL_ENOMEM;
  int32_t* J = (int32_t*)(Yc + (size_t)ldy * R);
  cudaError_t e = cudaMemcpyAsync(Yc, Y, sizeof(float) * (size_t)(ldy * R), cudaMemcpyDeviceToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(y, 0, sizeof(float) * (size_t)R, ctx->stream);
  TRY(cuda_check(ctx, e, "proposal_labels copy"));
  TRY(launch_cpqr(ctx, Yc, m, R, ldy, IDL_F32, K, J, nullptr));
  prop_labels_kernel<<<(unsigned)cdiv(K, 128), 128, 0, ctx->stream>>>(J, (int)K, (int)R, y), count_launch();
  return cuda_check(ctx, cudaGetLastError(), "proposal_labels");
}

// The QR stage through the column proposal on a given sketch (stage entry
// point of launch_proposal_qr).  proposal (host, optional): 1 certified,
// 2 rejected (the plain QR ran); reading it synchronises the stream.
extern "C" int idl_cpqr_proposal(idl_ctx* ctx, const float* Y2, float* Yf, int64_t m, int64_t R, int64_t ldy2,
                                 int64_t K, int mode, int cand_factor, int32_t* J, int* proposal) {
  TRY(ctx_ok(ctx));
  if (!Y2 || !Yf || !J || K < 1 || K >= R || K > m || ldy2 < m || R > 0x7fffffffLL || Y2 == Yf)
    return fail(ctx, IDL_EINVAL, "cpqr_proposal: bad arguments (Y2 and Yf must differ)");
  if (mode != IDL_PROPOSAL_MLP && mode != IDL_PROPOSAL_NORM) return fail(ctx, IDL_EINVAL, "cpqr_proposal: mode");
  TRY(cuda_check(ctx, cudaMemsetAsync(ctx->d_diag, 0, sizeof(double) * 16, ctx->stream), "diag clear"));
  TRY(launch_proposal_qr(ctx, Y2, Yf, m, R, ldy2, K, mode, cand_factor, J));
  if (proposal) {
    int f = 0;
    cudaError_t e = cudaMemcpyAsync(&f, ctx->d_status + 1, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    TRY(cuda_check(ctx, e, "cpqr_proposal readback"));
    *proposal = f ? 2 : 1;
  }
  return IDL_OK;
}
