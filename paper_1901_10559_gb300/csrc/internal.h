// internal.h -- host-side context and the launchers shared by the .cu files.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/idl.h"

struct idl_batch_state;
void idl_batch_state_free(idl_batch_state* b);

// A single-problem pipeline captured as a CUDA graph (idl_set_graphs).
struct PipeGraph {
  uint64_t key = 0;                // hash of the call's arguments
  std::string raw;                 // the arguments' bytes (compared in full before a replay)
  uint64_t gen = 0;                // workspace generation the graph's addresses belong to
  cudaGraphExec_t exec = nullptr;
  long long launches = 0;          // kernels in the graph (the launch counter adds them per replay)
  bool nocap = false;              // capture failed once: run these calls eagerly
};

struct idl_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t side = nullptr;     // the Gaussian draw runs here, overlapping the sketch (created on first use)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaStream_t copy = nullptr;     // host-array copies of the chunked CSR pipeline (created on first use)
  std::vector<cudaEvent_t> cevs;   // their events
  int graphs = 0;                  // idl_set_graphs: replay repeated pipeline calls as CUDA graphs
  uint64_t ws_gen = 1;             // bumped whenever a workspace slot is (re)allocated
  std::vector<PipeGraph> pgraphs;  // most recent last
  cudaStream_t gstream = nullptr;  // capture / replay stream (the legacy stream cannot be captured)
  cudaEvent_t gev_in = nullptr, gev_out = nullptr;
  int num_sms = 0;
  int smem_optin = 0;          // max dynamic shared memory per block (bytes)
  int* d_status = nullptr;     // device status word
  double* d_diag = nullptr;    // device diagnostics: [0] ||R22||^2, [1] ||Y2||^2, [2] explicit residual^2,
                               // [3] |r_11|, [4] |r_KK|
  std::string err;
  struct Buf { void* p = nullptr; size_t bytes = 0; };
  std::vector<Buf> slots;
  int last_cluster = 0;
  int gemm_simt = 0;           // 1: Gaussian stage on CUDA cores instead of tcgen05 (comparison / tests)
  int cpqr_smem_only = 0;      // 1: always use the shared-memory QR kernel (comparison / tests)
  idl_batch_state* batch = nullptr;   // batch graphs and tuning table
  int batch_no_graph = 0;      // 1: run batches without graph capture (tests)
  int batch_no_tune = 0;       // 1: skip the first-call tuning runs (tests)
  void* ts_tw = nullptr;       // FFT twiddle table of the TensorSketch kernels (built on first use)
  void* ts8_tw = nullptr;      // twiddle table of the L = 8192 TensorSketch kernels (built on first use)
  float* mlp = nullptr;        // proposal MLP: FP32 master weights | Adam first moments | second moments
  bool mlp_ready = false;
  long long mlp_step = 0;      // Adam steps taken since the weights were set
  bool poisoned = false;       // a bounded device wait expired: every later call returns IDL_ETIMEOUT
  size_t fail_alloc_at = 0;    // test hook: fail the n-th workspace allocation (0 = never)
  size_t alloc_count = 0;
  // per-stage CUDA-event profiling (idl_profile / idl_profile_read)
  bool prof_on = false;
  struct ProfPair { cudaEvent_t a = nullptr, b = nullptr; int stage = 0; };
  std::vector<ProfPair> prof;
  size_t prof_used = 0;
};

namespace idl {

// Workspace slots (each slot is one growable device buffer).
enum Slot {
  kWsH = 0, kWsS, kWsOmega, kWsBucketPtr, kWsRowList, kWsCursor, kWsBig, kWsY1, kWsPart,
  kWsY2, kWsOmegaConv, kWsRest, kWsA, kWsRowptr, kWsColidx, kWsVals, kWsJ, kWsT,
  kWsModeH, kWsModeS, kWsLam, kWsLamHat, kWsCpqrSync, kWsRinv, kWsBatch, kWsBatchTab, kWsYf, kWsProp,
  kWsPropGram, kWsPropTrain, kWsPropCopy, kWsBatchIn, kWsFactors, kWsModeSketch, kWsErrVec, kWsSrrqr, kWsCount
};

// Returns a device buffer of at least `bytes` for the slot (grown on demand), or
// nullptr with ctx->err set.
void* ws_get(idl_ctx* ctx, int slot, size_t bytes);

int fail(idl_ctx* ctx, int code, const std::string& msg);
// IDL_OK when ctx is non-null, not poisoned (see idl_ctx::poisoned) and its device is made current
int ctx_usable(idl_ctx* ctx);
// true for memory of a device (or managed memory); false for host memory and NULL
bool is_device_ptr(const void* p);
void ctx_add_launches(long long d);   // adjusts the process-wide launch counter (graph replays)
int cuda_check(idl_ctx* ctx, cudaError_t e, const char* where);
// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) only when kern needs more than
// was already allowed on this device (the attribute is per process and device;
// the driver call costs microseconds per launch).  Process-wide caches, locked.
cudaError_t ensure_smem(idl_ctx* ctx, const void* kern, size_t bytes);
// cudaFuncAttributeNonPortableClusterSizeAllowed, once per kernel
cudaError_t ensure_cluster_nonportable(idl_ctx* ctx, const void* kern);
// cudaOccupancyMaxActiveClusters, cached per (kernel, cluster size, threads, shared memory)
cudaError_t cluster_occupancy(idl_ctx* ctx, const void* kern, const cudaLaunchConfig_t& cfg, int* nclusters);

// draws.cu
cudaError_t launch_draw_countsketch(cudaStream_t st, uint64_t seed, int64_t I, int64_t L, int modified,
                                    int32_t* h, int8_t* s, int* status);
// h, s of rows i0 .. i0 + n - 1 of an I-row CountSketch, written to h[0 .. n), s[0 .. n)
cudaError_t launch_draw_countsketch_range(cudaStream_t st, uint64_t seed, int64_t I, int64_t i0, int64_t n, int64_t L,
                                          int modified, int32_t* h, int8_t* s, int* status);
cudaError_t launch_draw_gaussian(cudaStream_t st, uint64_t seed, int64_t m2, int64_t m1, double* Omega);
// the same Box-Muller pairs in FP32 arithmetic (FP32 pipelines and batches), stored as doubles
cudaError_t launch_draw_gaussian_f32(cudaStream_t st, uint64_t seed, int64_t m2, int64_t m1, double* Omega);
// the same draw from the stream of another tag (kTagGaussId, kTagGaussMode + n)
cudaError_t launch_draw_gaussian_tag(cudaStream_t st, uint64_t seed, uint32_t tag, int64_t m2, int64_t m1,
                                     double* Omega);
cudaError_t launch_draw_mode(cudaStream_t st, uint64_t seed, int n, int64_t In, int64_t L, int32_t* h,
                             int8_t* s);
int launch_bucket_offsets(idl_ctx* ctx, const int32_t* h, int64_t I, int64_t L, int32_t* bucket_ptr,
                          int32_t* row_list);

// countsketch.cu
// accum: add this block of rows' sketch to Y1 instead of writing it
int launch_countsketch_dense(idl_ctx* ctx, const void* A, int64_t I, int64_t R, int64_t lda, int dtype,
                             const int8_t* s, const int32_t* bucket_ptr, const int32_t* row_list,
                             int64_t L, void* Y1, int64_t ldy, bool accum = false);
int launch_countsketch_csr(idl_ctx* ctx, const int64_t* rowptr, const int32_t* colidx, const void* vals,
                           int64_t I, int64_t R, int64_t nnz, int dtype, const int8_t* s,
                           const int32_t* bucket_ptr, const int32_t* row_list, int64_t L, void* Y1,
                           int64_t ldy, bool accum = false);

// gaussian.cu
int launch_gaussian(idl_ctx* ctx, const double* Omega, int64_t m2, int64_t m1, const void* Y1, int64_t R,
                    int64_t ldy1, int dtype, int precision, void* Y2, int64_t ldy2);

// Y[l, r] = lambda_r prod_n G_n[l, r]: G holds N blocks of L x R column-major FP32 (ld L,
// block stride L R), Y column-major (ld L)
int launch_kr_product(idl_ctx* ctx, const float* G, int N, int64_t L, int64_t R, const double* lambda, float* Y);

// Y2 (column-major, ld ldy2) = or += Yp (column-major m x R, ld m)
int launch_add_sketch(idl_ctx* ctx, const void* Yp, int64_t m, int64_t R, int dtype, void* Y2, int64_t ldy2,
                      int accumulate);

int launch_gaussian_reduce(idl_ctx* ctx, const float* part, int splits, int64_t R, int MP, int64_t m2, float* Y2,
                           int64_t ldy2);
// gaussian_tc.cu
// y1_cm: Y1 column-major (column r at Y1 + r * ldy1) instead of row-major
int launch_gaussian_tc(idl_ctx* ctx, const double* Omega, int64_t m2, int64_t m1, const float* Y1, int64_t R,
                       int64_t ldy1, bool y1_cm, int precision, float* Y2, int64_t ldy2);

// cpqr.cu
// Extra roles of a QR launch (learned proposal): gate = fallback flag (run only
// when *gate != 0); colmap/Vout/Bout = candidate QR on a column subset in one
// CTA (max_cs = 1) with its reflectors recorded; diag = diagnostics base.
struct QrExtra {
  const int* gate = nullptr;
  const int32_t* colmap = nullptr;
  float* Vout = nullptr;
  float* Bout = nullptr;
  double* diag = nullptr;
  int max_cs = 16;
  const int32_t* force = nullptr;   // pivots given in order (register QR only; may alias J)
};
int launch_cpqr_ex(idl_ctx* ctx, const float* Yin, float* Yout, int64_t m, int64_t R, int64_t ld, int64_t K,
                   int32_t* J, double* rnorm, const QrExtra& x);
int launch_cpqr(idl_ctx* ctx, void* Y2, int64_t m, int64_t R, int64_t ld, int dtype, int64_t K, int32_t* J,
                double* rnorm);
// Gu-Eisenstat swaps after the pivoted QR (Fact 1; params.srrqr_f = f > 1): Yorig the
// sketch, Yf its factored form and J the pivots of the pivoted QR on entry; J, Yf, T and
// rest are those of the strong rank-revealing selection on exit.  Synchronises once
// per exchange considered.
int launch_srrqr(idl_ctx* ctx, const void* Yorig, void* Yf, int64_t m, int64_t R, int64_t ld, int dtype, int64_t K,
                 int32_t* J, double* T, int32_t* rest, float f);
int launch_t_solve(idl_ctx* ctx, const void* Y2, int64_t m, int64_t R, int64_t ld, int dtype, int64_t K,
                   const int32_t* J, double* T, int32_t* rest);
int launch_residual(idl_ctx* ctx, const void* Y2orig, const void* Y2fact, int64_t m, int64_t R, int64_t ld,
                    int dtype, int64_t K, const int32_t* J, const double* T, const int32_t* rest);
int launch_lambda_hat(idl_ctx* ctx, const double* lambda, const int32_t* J, const double* T, int64_t K,
                      int64_t R, double* lambda_hat);
int launch_transpose_to_colmajor(idl_ctx* ctx, const void* Y1, int64_t m, int64_t R, int64_t ldy1, int dtype,
                                 void* Y2, int64_t ldy2);

// errest.cu: ||A - A_J P||_2 / ||A||_2 by the power method (device pointers; synchronises)
int launch_id_error_dense(idl_ctx* ctx, const void* A, int64_t I, int64_t R, int64_t lda, int dtype,
                          const int32_t* J, const double* T, int64_t K, int iters, uint64_t seed, double* err);
int launch_id_error_csr(idl_ctx* ctx, const int64_t* rowptr, const int32_t* colidx, const void* vals, int64_t I,
                        int64_t R, int dtype, const int32_t* J, const double* T, int64_t K, int iters, uint64_t seed,
                        double* err);

// proposal.cu
int launch_features(idl_ctx* ctx, const float* Y, int64_t m, int64_t R, int64_t ld, int64_t K, float* F);
int launch_mlp_scores(idl_ctx* ctx, const float* F, int64_t n, float* s);
int launch_proposal_qr(idl_ctx* ctx, const float* Y2, float* Yf, int64_t m, int64_t R, int64_t ld, int64_t K,
                       int mode, int cand_factor, int32_t* J);

// tensorsketch.cu
const float2* ts_twiddles(idl_ctx* ctx);
const float2* ts8_twiddles(idl_ctx* ctx);
int launch_tensorsketch(idl_ctx* ctx, int N, const int64_t* dims, int64_t R, const void* const* factors,
                        const int64_t* ldf, const double* lambda, const int32_t* const* hs,
                        const int8_t* const* ss, int64_t L, float* Y, int64_t ldy, bool colmajor);

}  // namespace idl
