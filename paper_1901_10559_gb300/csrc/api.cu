// api.cu -- the C ABI of libidl: context, workspace, argument checks, the stage
// entry points and the three pipelines (Algorithm 2 and 3 with a Gaussian
// stage).  Host code only; every arithmetic step runs in the kernels of the
// other translation units.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <limits>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <string>

#include <atomic>

#include "common.cuh"
#include "internal.h"

using namespace idl;

namespace idl {

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void ctx_add_launches(long long d) { g_launches.fetch_add(d, std::memory_order_relaxed); }

int fail(idl_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

namespace {
std::mutex g_attr_mu;
std::map<std::pair<int, const void*>, int> g_smem_set;                      // (device, kernel) -> bytes allowed
std::map<std::pair<int, const void*>, bool> g_cluster_np;
std::map<std::tuple<int, const void*, int, int, size_t>, int> g_cluster_occ;  // (device, kernel, CS, threads, smem)
}  // namespace

cudaError_t ensure_smem(idl_ctx* ctx, const void* kern, size_t bytes) {
  std::lock_guard<std::mutex> lk(g_attr_mu);
  const auto key = std::make_pair(ctx->device, kern);
  auto it = g_smem_set.find(key);
  if (it != g_smem_set.end() && (size_t)it->second >= bytes) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) g_smem_set[key] = (int)bytes;
  return e;
}

cudaError_t ensure_cluster_nonportable(idl_ctx* ctx, const void* kern) {
  std::lock_guard<std::mutex> lk(g_attr_mu);
  const auto key = std::make_pair(ctx->device, kern);
  if (g_cluster_np.count(key)) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess) g_cluster_np[key] = true;
  return e;
}

cudaError_t cluster_occupancy(idl_ctx* ctx, const void* kern, const cudaLaunchConfig_t& cfg, int* nclusters) {
  int cs = 1;
  for (unsigned a = 0; a < cfg.numAttrs; ++a)
    if (cfg.attrs[a].id == cudaLaunchAttributeClusterDimension) cs = (int)cfg.attrs[a].val.clusterDim.x;
  const auto key = std::make_tuple(ctx->device, kern, cs, (int)cfg.blockDim.x, (size_t)cfg.dynamicSmemBytes);
  {
    std::lock_guard<std::mutex> lk(g_attr_mu);
    auto it = g_cluster_occ.find(key);
    if (it != g_cluster_occ.end()) { *nclusters = it->second; return cudaSuccess; }
  }
  const cudaError_t e = cudaOccupancyMaxActiveClusters(nclusters, kern, &cfg);
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> lk(g_attr_mu);
    g_cluster_occ[key] = *nclusters;
  }
  return e;
}

int cuda_check(idl_ctx* ctx, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return IDL_OK;
  if (ctx) ctx->err = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? IDL_ENOMEM : IDL_ECUDA;
}

void* ws_get(idl_ctx* ctx, int slot, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if ((int)ctx->slots.size() <= slot) ctx->slots.resize(slot + 1);
  idl_ctx::Buf& b = ctx->slots[slot];
  if (b.bytes >= bytes) return b.p;
  ++ctx->alloc_count;
  if (ctx->fail_alloc_at && ctx->alloc_count == ctx->fail_alloc_at) {
    ctx->err = "workspace allocation failed (injected)";
    return nullptr;
  }
  if (b.p) {
    cudaStreamSynchronize(ctx->stream);   // the old buffer may still be in use
    cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
  }
  ++ctx->ws_gen;                          // captured graphs hold the old addresses
  size_t want = bytes + bytes / 8;        // grow with headroom
  want = (want + 255) & ~(size_t)255;
  if (cudaMalloc(&b.p, want) != cudaSuccess) {
    (void)cudaGetLastError();
    b.p = nullptr;
    ctx->err = "workspace allocation of " + std::to_string(want) + " bytes failed";
    return nullptr;
  }
  b.bytes = want;
  return b.p;
}

}  // namespace idl

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
#define TRY(x)                         \
  do {                                 \
    int _rc = (x);                     \
    if (_rc != IDL_OK) return _rc;     \
  } while (0)
#define WS(ptr, type, slot, count)                                             \
  type* ptr = (type*)ws_get(ctx, slot, sizeof(type) * (size_t)(count));       \
  if (!ptr) return IDL_ENOMEM

// ---- per-stage event profiling ----
enum { kStDraw = 0, kStBucket, kStSketch, kStGauss, kStQR, kStSolve, kStCheck, kStCopy, kStCount };

// NVTX range names of the stages (header-only NVTX v3: a no-op unless a profiler is attached)
static const char* const kStageNames[kStCount] = {"idl:draws", "idl:buckets", "idl:sketch", "idl:gaussian",
                                                   "idl:cpqr",  "idl:tsolve",  "idl:check",  "idl:copy"};

static int prof_begin(idl_ctx* ctx, int stage) {
  if (!ctx->prof_on) return -1;
  if (ctx->prof_used == ctx->prof.size()) {
    idl_ctx::ProfPair pp;
    if (cudaEventCreate(&pp.a) != cudaSuccess || cudaEventCreate(&pp.b) != cudaSuccess) {
      (void)cudaGetLastError();
      return -1;
    }
    ctx->prof.push_back(pp);
  }
  idl_ctx::ProfPair& pp = ctx->prof[ctx->prof_used];
  pp.stage = stage;
  cudaEventRecord(pp.a, ctx->stream);
  return (int)ctx->prof_used++;
}
static void prof_end(idl_ctx* ctx, int idx) {
  if (idx >= 0) cudaEventRecord(ctx->prof[idx].b, ctx->stream);
}
#define STAGE(stage, expr)                  \
  do {                                      \
    nvtxRangePushA(kStageNames[stage]);     \
    int _pi = prof_begin(ctx, stage);       \
    int _rc = (expr);                       \
    prof_end(ctx, _pi);                     \
    nvtxRangePop();                         \
    if (_rc != IDL_OK) return _rc;          \
  } while (0)

namespace idl {
bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}
}  // namespace idl

static int dtype_size(int dtype) { return dtype == IDL_F64 ? 8 : 4; }

namespace idl {
int ctx_usable(idl_ctx* ctx) {
  if (!ctx) return IDL_EINVAL;
  if (ctx->poisoned)
    return fail(ctx, IDL_ETIMEOUT, "a bounded device wait expired on this context earlier; destroy it and create "
                                   "a new one (work that the timed-out kernel left in flight may still write its memory)");
  return cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
}
}  // namespace idl

static int check_ctx(idl_ctx* ctx) { return ctx_usable(ctx); }

// Copies a host array into a workspace slot (or returns the device pointer as is).
static const void* stage_in(idl_ctx* ctx, const void* p, size_t bytes, int slot, int* rc) {
  *rc = IDL_OK;
  if (is_device_ptr(p)) return p;
  void* d = ws_get(ctx, slot, bytes);
  if (!d) { *rc = IDL_ENOMEM; return nullptr; }
  const int pi = prof_begin(ctx, kStCopy);
  *rc = cuda_check(ctx, cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, ctx->stream), "copy in");
  prof_end(ctx, pi);
  return d;
}

static int clear_diag(idl_ctx* ctx) {
  return cuda_check(ctx, cudaMemsetAsync(ctx->d_diag, 0, sizeof(double) * 16, ctx->stream), "diag clear");
}

static int finish_info(idl_ctx* ctx, const idl_params* p, int precision, idl_info* info, int64_t K, int64_t R) {
  (void)K; (void)R;
  if (!info) return IDL_OK;
  double d[8];
  int stw[2] = {0, 0};
  cudaError_t e = cudaMemcpyAsync(d, ctx->d_diag, sizeof(d), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(stw, ctx->d_status, sizeof(stw), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  TRY(cuda_check(ctx, e, "info readback"));
  int st = stw[0];
  memset(info, 0, sizeof(*info));
  info->proposal = p->learned ? (stw[1] ? 2 : 1) : 0;
  info->y2_norm = std::sqrt(d[1]);
  info->rkk_ratio = d[3] > 0 ? d[4] / d[3] : 0.0;
  info->precision = precision;
  info->cluster = info->proposal == 1 ? 1 : ctx->last_cluster;
  const int mode = p->residual;
  if (mode == 1) info->residual = d[1] > 0 ? std::sqrt(d[0] / d[1]) : 0.0;
  else if (mode == 2) info->residual = d[1] > 0 ? std::sqrt(d[2] / d[1]) : 0.0;
  else info->residual = std::numeric_limits<double>::quiet_NaN();
  const double eps = precision == IDL_PREC_FP64 ? 2.220446049250313e-16 : 1.1920928955078125e-07;
  if (st == IDL_ETIMEOUT) ctx->poisoned = true;
  if (st == IDL_OK && !(d[4] > 64.0 * eps * d[3])) st = IDL_ERANK;
  info->status = st;
  int zero = 0;
  cudaMemcpyAsync(ctx->d_status, &zero, sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  return st;
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
extern "C" int idl_version(void) { return 100; }

extern "C" int idl_create(idl_ctx** out, int device) {
  if (!out) return IDL_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n <= device || device < 0) {
    (void)cudaGetLastError();
    return IDL_ECUDA;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return IDL_ECUDA;
  if (prop.major != 10 || prop.minor != 3) return IDL_ECUDA;   // built for sm_103a only
  if (cudaSetDevice(device) != cudaSuccess) return IDL_ECUDA;
  idl_ctx* c = new idl_ctx();
  c->device = device;
  c->num_sms = prop.multiProcessorCount;
  c->smem_optin = (int)prop.sharedMemPerBlockOptin;
  if (cudaMalloc(&c->d_status, sizeof(int) * 4) != cudaSuccess ||
      cudaMalloc(&c->d_diag, sizeof(double) * 16) != cudaSuccess) {
    delete c;
    return IDL_ENOMEM;
  }
  cudaMemset(c->d_status, 0, sizeof(int) * 4);
  cudaMemset(c->d_diag, 0, sizeof(double) * 16);
  *out = c;
  return IDL_OK;
}

extern "C" int idl_destroy(idl_ctx* ctx) {
  if (!ctx) return IDL_OK;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (auto& b : ctx->slots)
    if (b.p) cudaFree(b.p);
  for (auto& pp : ctx->prof) { cudaEventDestroy(pp.a); cudaEventDestroy(pp.b); }
  idl_batch_state_free(ctx->batch);
  if (ctx->mlp) cudaFree(ctx->mlp);
  if (ctx->ts_tw) cudaFree(ctx->ts_tw);
  if (ctx->ts8_tw) cudaFree(ctx->ts8_tw);
  if (ctx->side) { cudaStreamSynchronize(ctx->side); cudaStreamDestroy(ctx->side); }
  for (auto& g : ctx->pgraphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (ctx->gstream) { cudaStreamSynchronize(ctx->gstream); cudaStreamDestroy(ctx->gstream); }
  if (ctx->gev_in) cudaEventDestroy(ctx->gev_in);
  if (ctx->gev_out) cudaEventDestroy(ctx->gev_out);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->copy) { cudaStreamSynchronize(ctx->copy); cudaStreamDestroy(ctx->copy); }
  for (cudaEvent_t e : ctx->cevs) cudaEventDestroy(e);
  cudaFree(ctx->d_status);
  cudaFree(ctx->d_diag);
  delete ctx;
  return IDL_OK;
}

extern "C" int idl_set_stream(idl_ctx* ctx, void* stream) {
  if (!ctx) return IDL_EINVAL;
  ctx->stream = (cudaStream_t)stream;
  return IDL_OK;
}

extern "C" int idl_sync(idl_ctx* ctx) {
  TRY(check_ctx(ctx));
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  TRY(cuda_check(ctx, e, "idl_sync"));
  if (st == IDL_ETIMEOUT) ctx->poisoned = true;
  if (st != IDL_OK) {
    cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream);
    cudaStreamSynchronize(ctx->stream);
  }
  return st;
}

extern "C" const char* idl_last_error(idl_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" long long idl_launch_count(void) { return g_launches.load(); }

extern "C" int idl_profile(idl_ctx* ctx, int on) {
  if (!ctx) return IDL_EINVAL;
  ctx->prof_on = on != 0;
  return IDL_OK;
}

extern "C" int idl_profile_read(idl_ctx* ctx, double* ms, long long* calls, int nstages) {
  TRY(check_ctx(ctx));
  if (!ms || nstages < 1) return fail(ctx, IDL_EINVAL, "profile_read: bad arguments");
  TRY(cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "profile sync"));
  for (int q = 0; q < nstages; ++q) { ms[q] = 0.0; if (calls) calls[q] = 0; }
  for (size_t i = 0; i < ctx->prof_used; ++i) {
    const idl_ctx::ProfPair& pp = ctx->prof[i];
    float t = 0.f;
    if (cudaEventElapsedTime(&t, pp.a, pp.b) != cudaSuccess) { (void)cudaGetLastError(); continue; }
    if (pp.stage < nstages) { ms[pp.stage] += t; if (calls) calls[pp.stage] += 1; }
  }
  ctx->prof_used = 0;
  return IDL_OK;
}

// test hook (not in the public header): fail the n-th workspace allocation from now
extern "C" int idl_debug_fail_alloc(idl_ctx* ctx, int nth) {
  if (!ctx) return IDL_EINVAL;
  ctx->fail_alloc_at = nth > 0 ? ctx->alloc_count + (size_t)nth : 0;
  return IDL_OK;
}
extern "C" int idl_debug_gemm_path(idl_ctx* ctx, int simt) {
  if (!ctx) return IDL_EINVAL;
  ctx->gemm_simt = simt == 1;
  return IDL_OK;
}
extern "C" int idl_debug_cpqr_path(idl_ctx* ctx, int smem_only) {
  if (!ctx) return IDL_EINVAL;
  ctx->cpqr_smem_only = smem_only != 0;
  return IDL_OK;
}
extern "C" int idl_debug_release_workspace(idl_ctx* ctx) {
  TRY(check_ctx(ctx));
  cudaStreamSynchronize(ctx->stream);
  for (auto& b : ctx->slots) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
  }
  return IDL_OK;
}

// ---------------------------------------------------------------------------
// stage entry points
// ---------------------------------------------------------------------------
extern "C" int idl_draw_countsketch(idl_ctx* ctx, uint64_t seed, int64_t I, int64_t L, int modified, int32_t* h,
                                    int8_t* s) {
  TRY(check_ctx(ctx));
  if (I < 0 || L < 1 || L > 0x7fffffffLL || I > 0x7fffffffLL || (I > 0 && (!h || !s)))
    return fail(ctx, IDL_EINVAL, "draw_countsketch: bad sizes or null output");
  if (modified && !(L < I)) return fail(ctx, IDL_EINVAL, "draw_countsketch: modified map needs L < I");
  return cuda_check(ctx, launch_draw_countsketch(ctx->stream, seed, I, L, modified, h, s, ctx->d_status),
                    "draw_countsketch");
}

extern "C" int idl_draw_gaussian(idl_ctx* ctx, uint64_t seed, int64_t m2, int64_t m1, double* Omega) {
  TRY(check_ctx(ctx));
  if (m2 < 0 || m1 < 0 || (m2 * m1 > 0 && !Omega)) return fail(ctx, IDL_EINVAL, "draw_gaussian: bad arguments");
  return cuda_check(ctx, launch_draw_gaussian(ctx->stream, seed, m2, m1, Omega), "draw_gaussian");
}

extern "C" int idl_draw_gaussian_fp32(idl_ctx* ctx, uint64_t seed, int64_t m2, int64_t m1, double* Omega) {
  TRY(check_ctx(ctx));
  if (m2 < 0 || m1 < 0 || (m2 * m1 > 0 && !Omega)) return fail(ctx, IDL_EINVAL, "draw_gaussian_fp32: bad arguments");
  return cuda_check(ctx, launch_draw_gaussian_f32(ctx->stream, seed, m2, m1, Omega), "draw_gaussian_fp32");
}

extern "C" int idl_draw_mode(idl_ctx* ctx, uint64_t seed, int n, int64_t In, int64_t L, int32_t* h, int8_t* s) {
  TRY(check_ctx(ctx));
  if (n < 0 || In < 0 || L < 1 || L > 0x7fffffffLL || (In > 0 && (!h || !s)))
    return fail(ctx, IDL_EINVAL, "draw_mode: bad arguments");
  return cuda_check(ctx, launch_draw_mode(ctx->stream, seed, n, In, L, h, s), "draw_mode");
}

extern "C" int idl_bucket_offsets(idl_ctx* ctx, const int32_t* h, int64_t I, int64_t L, int32_t* bucket_ptr,
                                  int32_t* row_list) {
  TRY(check_ctx(ctx));
  if (I < 0 || I > 0x7fffffffLL || L < 1 || L > 0x7fffffffLL || !bucket_ptr || (I > 0 && (!h || !row_list)))
    return fail(ctx, IDL_EINVAL, "bucket_offsets: bad arguments");
  return launch_bucket_offsets(ctx, h, I, L, bucket_ptr, row_list);
}

extern "C" int idl_countsketch_dense(idl_ctx* ctx, const void* A, int64_t I, int64_t R, int64_t lda, int dtype,
                                     const int32_t* h, const int8_t* s, const int32_t* bucket_ptr,
                                     const int32_t* row_list, int64_t L, void* Y1, int64_t ldy) {
  (void)h;
  TRY(check_ctx(ctx));
  if ((dtype != IDL_F32 && dtype != IDL_F64) || I < 0 || R < 1 || lda < R || ldy < R || L < 1 || !Y1 || !s ||
      !bucket_ptr || (I > 0 && (!A || !row_list)))
    return fail(ctx, IDL_EINVAL, "countsketch_dense: bad arguments");
  return launch_countsketch_dense(ctx, A, I, R, lda, dtype, s, bucket_ptr, row_list, L, Y1, ldy);
}

extern "C" int idl_countsketch_csr(idl_ctx* ctx, const int64_t* rowptr, const int32_t* colidx, const void* vals,
                                   int64_t I, int64_t R, int64_t nnz, int dtype, const int32_t* h, const int8_t* s,
                                   const int32_t* bucket_ptr, const int32_t* row_list, int64_t L, void* Y1,
                                   int64_t ldy) {
  (void)h;
  TRY(check_ctx(ctx));
  if ((dtype != IDL_F32 && dtype != IDL_F64) || I < 0 || R < 1 || R > 0x7fffffffLL || nnz < 0 || ldy < R || L < 1 ||
      !Y1 || !rowptr || !bucket_ptr || (nnz > 0 && (!colidx || !vals)) || (I > 0 && (!s || !row_list)))
    return fail(ctx, IDL_EINVAL, "countsketch_csr: bad arguments");
  return launch_countsketch_csr(ctx, rowptr, colidx, vals, I, R, nnz, dtype, s, bucket_ptr, row_list, L, Y1, ldy);
}

static int tensorsketch_entry(idl_ctx* ctx, int N, const int64_t* dims, int64_t R, const void* const* factors,
                              const int64_t* ldf, const double* lambda, const int32_t* const* hs,
                              const int8_t* const* ss, int64_t L, float* Y, int64_t ldy, bool cm) {
  TRY(check_ctx(ctx));
  if (N < 1 || N > 8 || !dims || !factors || !ldf || !hs || !ss || !lambda || !Y || R < 1 || ldy < (cm ? L : R))
    return fail(ctx, IDL_EINVAL, "tensorsketch: bad arguments");
  for (int n = 0; n < N; ++n)
    if (dims[n] < 1 || ldf[n] < dims[n] || !factors[n] || !hs[n] || !ss[n])
      return fail(ctx, IDL_EINVAL, "tensorsketch: bad mode arguments");
  return launch_tensorsketch(ctx, N, dims, R, factors, ldf, lambda, hs, ss, L, Y, ldy, cm);
}

extern "C" int idl_tensorsketch(idl_ctx* ctx, int N, const int64_t* dims, int64_t R, const void* const* factors,
                                const int64_t* ldf, const double* lambda, const int32_t* const* hs,
                                const int8_t* const* ss, int64_t L, float* Y, int64_t ldy) {
  return tensorsketch_entry(ctx, N, dims, R, factors, ldf, lambda, hs, ss, L, Y, ldy, false);
}

extern "C" int idl_tensorsketch_colmajor(idl_ctx* ctx, int N, const int64_t* dims, int64_t R,
                                         const void* const* factors, const int64_t* ldf, const double* lambda,
                                         const int32_t* const* hs, const int8_t* const* ss, int64_t L, float* Y,
                                         int64_t ldy) {
  return tensorsketch_entry(ctx, N, dims, R, factors, ldf, lambda, hs, ss, L, Y, ldy, true);
}

extern "C" int idl_gaussian_stage(idl_ctx* ctx, const double* Omega, int64_t m2, int64_t m1, const void* Y1, int64_t R,
                                  int64_t ldy1, int dtype, int precision, void* Y2, int64_t ldy2) {
  TRY(check_ctx(ctx));
  if ((dtype != IDL_F32 && dtype != IDL_F64) || m2 < 1 || m1 < 1 || R < 1 || ldy1 < R || ldy2 < m2 || !Omega ||
      !Y1 || !Y2 || precision < 0 || precision > IDL_PREC_TF32X3 || (dtype == IDL_F64 && precision != IDL_PREC_FP64))
    return fail(ctx, IDL_EINVAL, "gaussian_stage: bad arguments");
  return launch_gaussian(ctx, Omega, m2, m1, Y1, R, ldy1, dtype, precision, Y2, ldy2);
}

extern "C" int idl_gaussian_stage_colmajor(idl_ctx* ctx, const double* Omega, int64_t m2, int64_t m1, const float* Y1,
                                           int64_t R, int64_t ldy1, int precision, float* Y2, int64_t ldy2) {
  TRY(check_ctx(ctx));
  if (m2 < 1 || m1 < 1 || R < 1 || ldy1 < m1 || ldy2 < m2 || !Omega || !Y1 || !Y2 ||
      (precision != IDL_PREC_FP32 && precision != IDL_PREC_BF16X3 && precision != IDL_PREC_BF16 &&
       precision != IDL_PREC_TF32X3))
    return fail(ctx, IDL_EINVAL, "gaussian_stage_colmajor: bad arguments");
  return launch_gaussian_tc(ctx, Omega, m2, m1, Y1, R, ldy1, true, precision, Y2, ldy2);
}

extern "C" int idl_cpqr(idl_ctx* ctx, void* Y2, int64_t m, int64_t R, int64_t ldy2, int dtype, int64_t K, int32_t* J,
                        double* rnorm) {
  TRY(check_ctx(ctx));
  if ((dtype != IDL_F32 && dtype != IDL_F64) || m < 1 || R < 1 || ldy2 < m || K < 1 || K > m || K > R || !Y2 || !J)
    return fail(ctx, IDL_EINVAL, "cpqr: bad arguments");
  TRY(clear_diag(ctx));
  return launch_cpqr(ctx, Y2, m, R, ldy2, dtype, K, J, rnorm);
}

extern "C" int idl_cpqr_srrqr(idl_ctx* ctx, const void* Y2, int64_t m, int64_t R, int64_t ldy2, int dtype, int64_t K,
                              float f, int32_t* J, double* T) {
  TRY(check_ctx(ctx));
  if ((dtype != IDL_F32 && dtype != IDL_F64) || m < 1 || R < 2 || ldy2 < m || K < 1 || K > m || K >= R || !Y2 || !J ||
      !T || !(f > 1.f))
    return fail(ctx, IDL_EINVAL, "cpqr_srrqr: bad arguments");
  const int es = dtype_size(dtype);
  void* Yf = ws_get(ctx, kWsYf, (size_t)es * (size_t)(R * ldy2));
  int32_t* rest = (int32_t*)ws_get(ctx, kWsRest, sizeof(int32_t) * (size_t)R);
  if (!Yf || !rest) return IDL_ENOMEM;
  TRY(cuda_check(ctx, cudaMemcpyAsync(Yf, Y2, (size_t)es * (size_t)(R * ldy2), cudaMemcpyDeviceToDevice, ctx->stream),
                 "copy"));
  TRY(clear_diag(ctx));
  TRY(launch_cpqr(ctx, Yf, m, R, ldy2, dtype, K, J, nullptr));
  return launch_srrqr(ctx, Y2, Yf, m, R, ldy2, dtype, K, J, T, rest, f);
}

extern "C" int idl_t_solve(idl_ctx* ctx, const void* Y2, int64_t m, int64_t R, int64_t ldy2, int dtype, int64_t K,
                           const int32_t* J, double* T, int32_t* rest) {
  TRY(check_ctx(ctx));
  if ((dtype != IDL_F32 && dtype != IDL_F64) || m < 1 || R < 1 || ldy2 < m || K < 1 || K > m || K >= R || !Y2 ||
      !J || !T)
    return fail(ctx, IDL_EINVAL, "t_solve: bad arguments");
  return launch_t_solve(ctx, Y2, m, R, ldy2, dtype, K, J, T, rest);
}

extern "C" int idl_lambda_hat(idl_ctx* ctx, const double* lambda, const int32_t* J, const double* T, int64_t K,
                              int64_t R, double* lambda_hat) {
  TRY(check_ctx(ctx));
  if (!lambda || !J || !T || !lambda_hat || K < 1 || K >= R) return fail(ctx, IDL_EINVAL, "lambda_hat: bad arguments");
  return launch_lambda_hat(ctx, lambda, J, T, K, R, lambda_hat);
}

// ---------------------------------------------------------------------------
// pipelines
// ---------------------------------------------------------------------------
static int check_params(idl_ctx* ctx, const idl_params* p, int dtype, int64_t I, int64_t R, int64_t K, bool tensor) {
  if (!p) return fail(ctx, IDL_EINVAL, "null params");
  if (dtype != IDL_F32 && dtype != IDL_F64) return fail(ctx, IDL_EINVAL, "dtype must be IDL_F32 or IDL_F64");
  if (p->precision < 0 || p->precision > IDL_PREC_TF32X3) return fail(ctx, IDL_EINVAL, "unknown precision");
  if (dtype == IDL_F64 && p->precision != IDL_PREC_FP64)
    return fail(ctx, IDL_EINVAL, "FP64 data needs precision IDL_PREC_FP64");
  if (dtype == IDL_F32 && p->precision == IDL_PREC_FP64)
    return fail(ctx, IDL_EINVAL, "FP32 data cannot use precision IDL_PREC_FP64");
  if (K < 1 || K >= R) return fail(ctx, IDL_EINVAL, "need 1 <= K < R");
  if (p->m1 < 1 || p->m1 > 0x7fffffffLL) return fail(ctx, IDL_EINVAL, "m1 out of range");
  if (K > p->m1) return fail(ctx, IDL_EINVAL, "need K <= m1");
  if (p->m2 < 0 || p->m2 > p->m1) return fail(ctx, IDL_EINVAL, "need 0 <= m2 <= m1");
  if (p->m2 > 0 && K > p->m2) return fail(ctx, IDL_EINVAL, "need K <= m2");
  if (!tensor && p->modified && !(p->m1 < I)) return fail(ctx, IDL_EINVAL, "modified CountSketch needs m1 < I");
  if (tensor && (p->m1 & (p->m1 - 1))) return fail(ctx, IDL_EINVAL, "TensorSketch length must be a power of two");
  if (p->residual < 0 || p->residual > 2) return fail(ctx, IDL_EINVAL, "residual mode must be 0, 1 or 2");
  if (R > 0x7fffffffLL || I > 0x7fffffffLL) return fail(ctx, IDL_ELIMIT, "I and R must fit in int32");
  if (p->learned < IDL_PROPOSAL_NONE || p->learned > IDL_PROPOSAL_NORM)
    return fail(ctx, IDL_EINVAL, "unknown proposal mode");
  if (p->learned && dtype != IDL_F32) return fail(ctx, IDL_EINVAL, "the column proposal needs FP32 data");
  if (p->cand_factor < 0 || p->cand_factor > 8) return fail(ctx, IDL_EINVAL, "cand_factor must be in 0..8");
  if (p->learned && ((p->m2 > 0 ? p->m2 : p->m1) > 128 || K > 128))
    return fail(ctx, IDL_ELIMIT, "the column proposal needs m <= 128 and K <= 128");
  if (!(p->srrqr_f == 0.f || p->srrqr_f > 1.f)) return fail(ctx, IDL_EINVAL, "srrqr_f must be 0 or > 1");
  if (p->srrqr_f > 0.f && p->learned) return fail(ctx, IDL_EINVAL, "srrqr_f and the column proposal exclude each other");
  return IDL_OK;
}

// The Gaussian matrix of the pipeline (m2 > 0): drawn on the context's side
// stream, forked from the main stream here -- after everything already queued,
// which may still read the Omega workspace -- so that the draw (FP64 Box-Muller,
// tens of microseconds) overlaps the sketch; finish_pipeline joins it before
// the Gaussian stage.  *Om = nullptr when m2 = 0.
static int fork_omega(idl_ctx* ctx, const idl_params* p, double** Om) {
  *Om = nullptr;
  if (p->m2 <= 0) return IDL_OK;
  double* o = (double*)ws_get(ctx, kWsOmega, sizeof(double) * (size_t)(p->m2 * p->m1));
  if (!o) return IDL_ENOMEM;
  if (!ctx->side) {
    cudaError_t e = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_check(ctx, e, "side stream");
  }
  TRY(cuda_check(ctx, cudaEventRecord(ctx->ev_fork, ctx->stream), "fork"));
  TRY(cuda_check(ctx, cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0), "fork wait"));
  TRY(cuda_check(ctx, p->precision == IDL_PREC_FP64 ? launch_draw_gaussian(ctx->side, p->seed, p->m2, p->m1, o)
                                                     : launch_draw_gaussian_f32(ctx->side, p->seed, p->m2, p->m1, o),
                 "draw gaussian"));
  TRY(cuda_check(ctx, cudaEventRecord(ctx->ev_join, ctx->side), "join"));
  *Om = o;
  return IDL_OK;
}

static int finish_from_y2(idl_ctx* ctx, const idl_params* p, int dtype, void* Y2, int64_t m, int64_t R, int64_t K,
                          int32_t* J, double* T, idl_info* info);

// The QR stage factors a copy of the sketch (kept beside it in the kWsY2 slot) for the
// explicit residual and for the strong rank-revealing exchanges.
static bool keeps_sketch(const idl_params* p) { return p->residual == 2 || p->srrqr_f > 0.f; }

// Sketch Y1 (m1 x R, row-major, ld = ldy1; column-major when y1_cm, which needs the
// tensor-core Gaussian stage) -> J, T, via the Gaussian stage and the QR stage.
// Om: the Gaussian matrix from fork_omega (joined here), or nullptr to draw it now.
static int finish_pipeline(idl_ctx* ctx, const idl_params* p, int dtype, void* Y1, int64_t ldy1, int64_t R,
                           int64_t K, int32_t* J, double* T, idl_info* info, bool y1_cm = false,
                           const double* Om = nullptr) {
  const int es = dtype_size(dtype);
  const int64_t m = p->m2 > 0 ? p->m2 : p->m1;
  const int64_t ld2 = m;
  void* Y2 = ws_get(ctx, kWsY2, (size_t)es * (size_t)(R * ld2) * (keeps_sketch(p) ? 2 : 1));
  if (!Y2) return IDL_ENOMEM;
  if (p->m2 > 0) {
    if (Om) {
      TRY(cuda_check(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0), "join wait"));
    } else {
      double* o = (double*)ws_get(ctx, kWsOmega, sizeof(double) * (size_t)(p->m2 * p->m1));
      if (!o) return IDL_ENOMEM;
      STAGE(kStDraw, cuda_check(ctx, p->precision == IDL_PREC_FP64
                                         ? launch_draw_gaussian(ctx->stream, p->seed, p->m2, p->m1, o)
                                         : launch_draw_gaussian_f32(ctx->stream, p->seed, p->m2, p->m1, o),
                                "draw gaussian"));
      Om = o;
    }
    if (y1_cm)
      STAGE(kStGauss, launch_gaussian_tc(ctx, Om, p->m2, p->m1, (const float*)Y1, R, ldy1, true, p->precision,
                                         (float*)Y2, ld2));
    else
      STAGE(kStGauss, launch_gaussian(ctx, Om, p->m2, p->m1, Y1, R, ldy1, dtype, p->precision, Y2, ld2));
  } else {
    STAGE(kStGauss, launch_transpose_to_colmajor(ctx, Y1, m, R, ldy1, dtype, Y2, ld2));
  }
  return finish_from_y2(ctx, p, dtype, Y2, m, R, K, J, T, info);
}

// The QR stage onwards from a sketch Y2 (m x R column-major, ld m, in the kWsY2 slot with
// room for a second copy when p->residual == 2): pivoted QR (or the column proposal),
// T solve, residual, outputs (staged back to host pointers), diagnostics.
static int finish_from_y2(idl_ctx* ctx, const idl_params* p, int dtype, void* Y2, int64_t m, int64_t R, int64_t K,
                          int32_t* J, double* T, idl_info* info) {
  const int es = dtype_size(dtype);
  const int64_t ld2 = m;
  const bool keep_orig = keeps_sketch(p);
  void* Yf = Y2;
  if (p->learned) {
    // the proposal reads the sketch and writes the factored copy; the fallback re-reads the sketch
    Yf = ws_get(ctx, kWsYf, (size_t)es * (size_t)(R * ld2));
    if (!Yf) return IDL_ENOMEM;
  } else if (keep_orig) {
    Yf = (char*)Y2 + (size_t)es * (size_t)(R * ld2);
    TRY(cuda_check(ctx, cudaMemcpyAsync(Yf, Y2, (size_t)es * R * ld2, cudaMemcpyDeviceToDevice, ctx->stream), "copy"));
  }
  const bool jdev = is_device_ptr(J), tdev = is_device_ptr(T);
  int32_t* Jd = J;
  double* Td = T;
  if (!jdev) { Jd = (int32_t*)ws_get(ctx, kWsJ, sizeof(int32_t) * (size_t)K); if (!Jd) return IDL_ENOMEM; }
  if (!tdev) { Td = (double*)ws_get(ctx, kWsT, sizeof(double) * (size_t)(K * (R - K))); if (!Td) return IDL_ENOMEM; }
  WS(rest, int32_t, kWsRest, R);
  TRY(clear_diag(ctx));
  if (p->learned)
    STAGE(kStQR, launch_proposal_qr(ctx, (const float*)Y2, (float*)Yf, m, R, ld2, K, p->learned, p->cand_factor, Jd));
  else
    STAGE(kStQR, launch_cpqr(ctx, Yf, m, R, ld2, dtype, K, Jd, nullptr));
  if (p->srrqr_f > 0.f)       // exchanges after the pivoted QR; ends with the T solve of the final selection
    STAGE(kStQR, launch_srrqr(ctx, Y2, Yf, m, R, ld2, dtype, K, Jd, Td, rest, p->srrqr_f));
  else
    STAGE(kStSolve, launch_t_solve(ctx, Yf, m, R, ld2, dtype, K, Jd, Td, rest));
  if (p->residual == 2) STAGE(kStCheck, launch_residual(ctx, Y2, Yf, m, R, ld2, dtype, K, Jd, Td, rest));
  if (!jdev)
    TRY(cuda_check(ctx, cudaMemcpyAsync(J, Jd, sizeof(int32_t) * K, cudaMemcpyDeviceToHost, ctx->stream), "copy J"));
  if (!tdev)
    TRY(cuda_check(ctx, cudaMemcpyAsync(T, Td, sizeof(double) * K * (R - K), cudaMemcpyDeviceToHost, ctx->stream),
                   "copy T"));
  if (info) return finish_info(ctx, p, p->precision, info, K, R);
  if (!jdev || !tdev) TRY(cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "sync"));
  return IDL_OK;
}

static int id_matrix_impl(idl_ctx* ctx, const void* A, int64_t I, int64_t R, int64_t lda, int dtype, int64_t K,
                         const idl_params* p, int32_t* J, double* T, idl_info* info) {
  TRY(check_ctx(ctx));
  TRY(check_params(ctx, p, dtype, I, R, K, false));
  if (I < 1 || lda < R || !A || !J || !T) return fail(ctx, IDL_EINVAL, "id_matrix: bad arguments");
  const int es = dtype_size(dtype);
  const int64_t m1 = p->m1;
  double* Om;
  TRY(fork_omega(ctx, p, &Om));
  int rc;
  const void* Ad = stage_in(ctx, A, (size_t)es * (size_t)((I - 1) * lda + R), kWsA, &rc);
  TRY(rc);
  WS(h, int32_t, kWsH, I);
  WS(s, int8_t, kWsS, I);
  WS(ptr, int32_t, kWsBucketPtr, m1 + 1);
  WS(rows, int32_t, kWsRowList, I);
  const int64_t ldy1 = round_up(R, 32);
  void* Y1 = ws_get(ctx, kWsY1, (size_t)es * (size_t)(m1 * ldy1));
  if (!Y1) return IDL_ENOMEM;
  STAGE(kStDraw, cuda_check(ctx, launch_draw_countsketch(ctx->stream, p->seed, I, m1, p->modified, h, s,
                                                         ctx->d_status), "draw countsketch"));
  STAGE(kStBucket, launch_bucket_offsets(ctx, h, I, m1, ptr, rows));
  STAGE(kStSketch, launch_countsketch_dense(ctx, Ad, I, R, lda, dtype, s, ptr, rows, m1, Y1, ldy1));
  return finish_pipeline(ctx, p, dtype, Y1, ldy1, R, K, J, T, info, false, Om);
}

// Host CSR arrays of a large matrix: the sketch is a sum over row blocks
// (Y1 = sum_c S[:, rows_c] A[rows_c, :]), so the rows are cut into chunks of about
// equal nonzeros, each chunk's column indices and values are copied on the context's
// copy stream, and the chunk is sketched (bucket offsets of its rows, CSR sketch added
// into Y1) as soon as its copy has arrived -- the copies of the next chunks overlap it.
constexpr int64_t kCsrChunkMinNnz = 1 << 22;
constexpr int kCsrChunks = 8;

static cudaEvent_t ctx_event(idl_ctx* ctx, size_t i) {
  while (ctx->cevs.size() <= i) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    ctx->cevs.push_back(e);
  }
  return ctx->cevs[i];
}

static int csr_chunked_sketch(idl_ctx* ctx, const int64_t* h_rowptr, const int32_t* h_colidx, const void* h_vals,
                              int64_t I, int64_t R, int64_t nnz, int dtype, const int64_t* d_rowptr, const int32_t* h,
                              const int8_t* s, int64_t m1, int32_t* ptr, int32_t* rows, void* Y1, int64_t ldy1) {
  const int es = dtype_size(dtype);
  int32_t* d_ci = (int32_t*)ws_get(ctx, kWsColidx, sizeof(int32_t) * (size_t)nnz);
  unsigned char* d_v = (unsigned char*)ws_get(ctx, kWsVals, (size_t)es * (size_t)nnz);
  if (!d_ci || !d_v) return IDL_ENOMEM;
  if (!ctx->copy) TRY(cuda_check(ctx, cudaStreamCreateWithFlags(&ctx->copy, cudaStreamNonBlocking), "copy stream"));
  cudaEvent_t e0 = ctx_event(ctx, 0);
  if (!e0) return fail(ctx, IDL_ECUDA, "event creation failed");
  // the copies start after the work queued before this call (which may still read these buffers)
  TRY(cuda_check(ctx, cudaEventRecord(e0, ctx->stream), "copy order"));
  TRY(cuda_check(ctx, cudaStreamWaitEvent(ctx->copy, e0, 0), "copy order"));
  int64_t r0 = 0;
  for (int c = 0; c < kCsrChunks && r0 < I; ++c) {
    // last row of the chunk: the first row whose rowptr reaches the chunk's share of nonzeros
    const int64_t target = nnz * (c + 1) / kCsrChunks;
    int64_t lo = r0 + 1, hi = I;
    while (lo < hi) {
      const int64_t mid = (lo + hi) / 2;
      if (h_rowptr[mid] >= target) hi = mid; else lo = mid + 1;
    }
    const int64_t r1 = c + 1 == kCsrChunks ? I : lo;
    const int64_t z0 = std::min(std::max<int64_t>(h_rowptr[r0], 0), nnz);
    const int64_t z1 = std::min(std::max<int64_t>(h_rowptr[r1], z0), nnz);
    if (z1 > z0) {
      TRY(cuda_check(ctx, cudaMemcpyAsync(d_ci + z0, h_colidx + z0, sizeof(int32_t) * (size_t)(z1 - z0),
                                          cudaMemcpyHostToDevice, ctx->copy), "copy in"));
      TRY(cuda_check(ctx, cudaMemcpyAsync(d_v + (size_t)es * z0, (const unsigned char*)h_vals + (size_t)es * z0,
                                          (size_t)es * (size_t)(z1 - z0), cudaMemcpyHostToDevice, ctx->copy),
                     "copy in"));
    }
    cudaEvent_t ec = ctx_event(ctx, (size_t)c + 1);
    if (!ec) return fail(ctx, IDL_ECUDA, "event creation failed");
    TRY(cuda_check(ctx, cudaEventRecord(ec, ctx->copy), "copy event"));
    const int64_t n = r1 - r0;
    STAGE(kStBucket, launch_bucket_offsets(ctx, h + r0, n, m1, ptr, rows));
    TRY(cuda_check(ctx, cudaStreamWaitEvent(ctx->stream, ec, 0), "chunk wait"));
    STAGE(kStSketch, launch_countsketch_csr(ctx, d_rowptr + r0, d_ci, d_v, n, R, nnz, dtype, s + r0, ptr, rows, m1,
                                            Y1, ldy1, c > 0));
    r0 = r1;
  }
  return IDL_OK;
}

static int id_matrix_csr_impl(idl_ctx* ctx, const int64_t* rowptr, const int32_t* colidx, const void* vals, int64_t I,
                             int64_t R, int64_t nnz, int dtype, int64_t K, const idl_params* p, int32_t* J, double* T,
                             idl_info* info) {
  TRY(check_ctx(ctx));
  TRY(check_params(ctx, p, dtype, I, R, K, false));
  if (I < 1 || nnz < 0 || !rowptr || !J || !T || (nnz > 0 && (!colidx || !vals)))
    return fail(ctx, IDL_EINVAL, "id_matrix_csr: bad arguments");
  const int es = dtype_size(dtype);
  const int64_t m1 = p->m1;
  double* Om;
  TRY(fork_omega(ctx, p, &Om));
  int rc;
  const int64_t* rp = (const int64_t*)stage_in(ctx, rowptr, sizeof(int64_t) * (size_t)(I + 1), kWsRowptr, &rc);
  TRY(rc);
  const bool chunked = nnz >= kCsrChunkMinNnz && !is_device_ptr(rowptr) && !is_device_ptr(colidx) &&
                       !is_device_ptr(vals);
  const int32_t* ci = colidx;
  const void* vv = vals;
  if (!chunked && nnz) {
    ci = (const int32_t*)stage_in(ctx, colidx, sizeof(int32_t) * (size_t)nnz, kWsColidx, &rc);
    TRY(rc);
    vv = stage_in(ctx, vals, (size_t)es * (size_t)nnz, kWsVals, &rc);
    TRY(rc);
  }
  WS(h, int32_t, kWsH, I);
  WS(s, int8_t, kWsS, I);
  WS(ptr, int32_t, kWsBucketPtr, m1 + 1);
  WS(rows, int32_t, kWsRowList, I);
  const int64_t ldy1 = round_up(R, 32);
  void* Y1 = ws_get(ctx, kWsY1, (size_t)es * (size_t)(m1 * ldy1));
  if (!Y1) return IDL_ENOMEM;
  STAGE(kStDraw, cuda_check(ctx, launch_draw_countsketch(ctx->stream, p->seed, I, m1, p->modified, h, s,
                                                         ctx->d_status), "draw countsketch"));
  if (chunked) {
    TRY(csr_chunked_sketch(ctx, rowptr, colidx, vals, I, R, nnz, dtype, rp, h, s, m1, ptr, rows, Y1, ldy1));
  } else {
    STAGE(kStBucket, launch_bucket_offsets(ctx, h, I, m1, ptr, rows));
    STAGE(kStSketch, launch_countsketch_csr(ctx, rp, ci, vv, I, R, nnz, dtype, s, ptr, rows, m1, Y1, ldy1));
  }
  return finish_pipeline(ctx, p, dtype, Y1, ldy1, R, K, J, T, info, false, Om);
}

// Host factor matrices are copied into one workspace buffer (each at a 256-byte
// offset, host_bytes in all); device ones are used in place.  fdev: N pointers.
static int stage_factors(idl_ctx* ctx, int N, const int64_t* dims, int64_t R, const void* const* factors,
                         const int64_t* ldf, size_t host_bytes, const void** fdev) {
  unsigned char* stg = host_bytes ? (unsigned char*)ws_get(ctx, kWsFactors, host_bytes) : nullptr;
  if (host_bytes && !stg) return IDL_ENOMEM;
  size_t off = 0;
  for (int n = 0; n < N; ++n) {
    fdev[n] = factors[n];
    if (is_device_ptr(factors[n])) continue;
    const size_t b = sizeof(float) * (size_t)((R - 1) * ldf[n] + dims[n]);
    const int pi = prof_begin(ctx, kStCopy);
    TRY(cuda_check(ctx, cudaMemcpyAsync(stg + off, factors[n], b, cudaMemcpyHostToDevice, ctx->stream), "copy in"));
    prof_end(ctx, pi);
    fdev[n] = stg + off;
    off += (b + 255) & ~(size_t)255;
  }
  return IDL_OK;
}

// Bytes of workspace the host factors need (0 when all are device pointers), and the
// argument checks shared by the two CP entry points.
static int cp_factor_args(idl_ctx* ctx, int N, const int64_t* dims, int64_t R, const void* const* factors,
                          const int64_t* ldf, size_t* host_bytes, int64_t* tot) {
  *host_bytes = 0;
  *tot = 0;
  for (int n = 0; n < N; ++n) {
    if (dims[n] < 1 || ldf[n] < dims[n] || !factors[n])
      return fail(ctx, IDL_EINVAL, "CP factors must be non-null with ldf >= dims");
    if (!is_device_ptr(factors[n]))
      *host_bytes += (sizeof(float) * (size_t)((R - 1) * ldf[n] + dims[n]) + 255) & ~(size_t)255;
    *tot += dims[n];
  }
  return IDL_OK;
}

static int id_cp_tensor_impl(idl_ctx* ctx, int N, const int64_t* dims, int64_t R, const void* const* factors,
                            const int64_t* ldf, const double* lambda, int64_t K, const idl_params* p, int32_t* J,
                            double* T, double* lambda_hat, idl_info* info) {
  TRY(check_ctx(ctx));
  TRY(check_params(ctx, p, IDL_F32, 1, R, K, true));
  if (N < 1 || N > 8 || !dims || !factors || !ldf || !lambda || !J || !T || !lambda_hat)
    return fail(ctx, IDL_EINVAL, "id_cp_tensor: bad arguments");
  const int64_t L = p->m1;
  int64_t maxdim = 0, tot = 0;
  size_t host_bytes = 0;
  for (int n = 0; n < N; ++n) {
    if (dims[n] < 1 || ldf[n] < dims[n] || !factors[n])
      return fail(ctx, IDL_EINVAL, "id_cp_tensor: factors must be non-null with ldf >= dims");
    if (!is_device_ptr(factors[n])) host_bytes += (sizeof(float) * (size_t)((R - 1) * ldf[n] + dims[n]) + 255) & ~(size_t)255;
    maxdim = std::max(maxdim, dims[n]);
    tot += dims[n];
  }
  double* Om;
  TRY(fork_omega(ctx, p, &Om));
  int rc;
  const void* fdev[8];
  TRY(stage_factors(ctx, N, dims, R, factors, ldf, host_bytes, fdev));
  factors = fdev;
  const double* lam = (const double*)stage_in(ctx, lambda, sizeof(double) * (size_t)R, kWsLam, &rc);
  TRY(rc);
  WS(hbuf, int32_t, kWsModeH, tot);
  WS(sbuf, int8_t, kWsModeS, tot);
  const int32_t* hs[8];
  const int8_t* ss[8];
  int64_t off = 0;
  for (int n = 0; n < N; ++n) {
    STAGE(kStDraw, cuda_check(ctx, launch_draw_mode(ctx->stream, p->seed, n, dims[n], L, hbuf + off, sbuf + off),
                              "draw mode"));
    hs[n] = hbuf + off;
    ss[n] = sbuf + off;
    off += dims[n];
  }
  // with a Gaussian stage on the tensor cores the sketch is written column-major (each
  // column contiguous for the FFT block that produces it and for the converter thread
  // that reads it); otherwise row-major
  const bool cm = p->m2 > 0 && !ctx->gemm_simt;
  const int64_t ldy1 = cm ? L : round_up(R, 32);
  float* Y1 = (float*)ws_get(ctx, kWsY1, sizeof(float) * (size_t)(cm ? R * L : L * ldy1));
  if (!Y1) return IDL_ENOMEM;
  STAGE(kStSketch, launch_tensorsketch(ctx, N, dims, R, factors, ldf, lam, hs, ss, L, Y1, ldy1, cm));
  // J and T on the device for lambda_hat; staged back if the caller passed host pointers
  const bool jdev = is_device_ptr(J), tdev = is_device_ptr(T), ldev = is_device_ptr(lambda_hat);
  int32_t* Jd = J;
  double* Td = T;
  if (!jdev) { Jd = (int32_t*)ws_get(ctx, kWsJ, sizeof(int32_t) * (size_t)K); if (!Jd) return IDL_ENOMEM; }
  if (!tdev) { Td = (double*)ws_get(ctx, kWsT, sizeof(double) * (size_t)(K * (R - K))); if (!Td) return IDL_ENOMEM; }
  TRY(finish_pipeline(ctx, p, IDL_F32, Y1, ldy1, R, K, Jd, Td, nullptr, cm, Om));
  double* lhd = lambda_hat;
  if (!ldev) { lhd = (double*)ws_get(ctx, kWsLamHat, sizeof(double) * (size_t)K); if (!lhd) return IDL_ENOMEM; }
  STAGE(kStCheck, launch_lambda_hat(ctx, lam, Jd, Td, K, R, lhd));
  if (!jdev) TRY(cuda_check(ctx, cudaMemcpyAsync(J, Jd, sizeof(int32_t) * K, cudaMemcpyDeviceToHost, ctx->stream), "J"));
  if (!tdev)
    TRY(cuda_check(ctx, cudaMemcpyAsync(T, Td, sizeof(double) * K * (R - K), cudaMemcpyDeviceToHost, ctx->stream), "T"));
  if (!ldev)
    TRY(cuda_check(ctx, cudaMemcpyAsync(lambda_hat, lhd, sizeof(double) * K, cudaMemcpyDeviceToHost, ctx->stream),
                   "lambda_hat"));
  if (info) return finish_info(ctx, p, p->precision, info, K, R);
  if (!jdev || !tdev || !ldev) TRY(cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "sync"));
  return IDL_OK;
}

// ---------------------------------------------------------------------------
// The sketch of a CP tensor without the QR stage: Y2 = Omega Y1 (m x R, column-major)
// with Y1 the TensorSketch of the columns lambda_r a_r^(1) o ... o a_r^(N) (Sec. 1.3,
// Eq. TA-formula).  Column r of the sketch depends on column r of the factors and on
// the maps of the modes only (drawn from seed, mode index, I_n and L), so a tensor
// whose R columns are split over ranks is sketched block by block and the blocks
// are gathered side by side: the column-sharded CP tensor ID.
// ---------------------------------------------------------------------------
extern "C" int idl_sketch_cp(idl_ctx* ctx, int N, const int64_t* dims, int64_t R, const void* const* factors,
                             const int64_t* ldf, const double* lambda, const idl_params* p, float* Y2,
                             int64_t ldy2) {
  TRY(check_ctx(ctx));
  if (!p || N < 1 || N > 8 || !dims || !factors || !ldf || !lambda || !Y2 || R < 1 || R > 0x7fffffffLL)
    return fail(ctx, IDL_EINVAL, "sketch_cp: bad arguments");
  if (p->precision < 0 || p->precision > IDL_PREC_TF32X3 || p->precision == IDL_PREC_FP64)
    return fail(ctx, IDL_EINVAL, "sketch_cp: FP32 data needs precision FP32, BF16X3, BF16 or TF32X3");
  if (p->m1 < 1 || p->m1 > 0x7fffffffLL || (p->m1 & (p->m1 - 1)))
    return fail(ctx, IDL_EINVAL, "TensorSketch length must be a power of two");
  if (p->m2 < 0 || p->m2 > p->m1 || p->m2 > 256) return fail(ctx, IDL_EINVAL, "need 0 <= m2 <= min(m1, 256)");
  const int64_t L = p->m1, m = p->m2 > 0 ? p->m2 : L;
  if (ldy2 < m) return fail(ctx, IDL_EINVAL, "sketch_cp: ldy2 < m");
  if (!is_device_ptr(Y2)) return fail(ctx, IDL_EINVAL, "sketch_cp: Y2 must be device memory");
  size_t host_bytes;
  int64_t tot;
  TRY(cp_factor_args(ctx, N, dims, R, factors, ldf, &host_bytes, &tot));
  double* Om;
  TRY(fork_omega(ctx, p, &Om));
  const void* fdev[8];
  TRY(stage_factors(ctx, N, dims, R, factors, ldf, host_bytes, fdev));
  int rc;
  const double* lam = (const double*)stage_in(ctx, lambda, sizeof(double) * (size_t)R, kWsLam, &rc);
  TRY(rc);
  WS(hbuf, int32_t, kWsModeH, tot);
  WS(sbuf, int8_t, kWsModeS, tot);
  const int32_t* hs[8];
  const int8_t* ss[8];
  int64_t off = 0;
  for (int n = 0; n < N; ++n) {
    STAGE(kStDraw, cuda_check(ctx, launch_draw_mode(ctx->stream, p->seed, n, dims[n], L, hbuf + off, sbuf + off),
                              "draw mode"));
    hs[n] = hbuf + off;
    ss[n] = sbuf + off;
    off += dims[n];
  }
  const bool cm = p->m2 > 0 && !ctx->gemm_simt;
  const int64_t ldy1 = cm ? L : round_up(R, 32);
  float* Y1 = (float*)ws_get(ctx, kWsY1, sizeof(float) * (size_t)(cm ? R * L : L * ldy1));
  if (!Y1) return IDL_ENOMEM;
  STAGE(kStSketch, launch_tensorsketch(ctx, N, dims, R, fdev, ldf, lam, hs, ss, L, Y1, ldy1, cm));
  if (p->m2 > 0) {
    TRY(cuda_check(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0), "join wait"));
    if (cm)
      STAGE(kStGauss, launch_gaussian_tc(ctx, Om, p->m2, L, Y1, R, ldy1, true, p->precision, Y2, ldy2));
    else
      STAGE(kStGauss, launch_gaussian(ctx, Om, p->m2, L, Y1, R, ldy1, IDL_F32, p->precision, Y2, ldy2));
  } else {
    STAGE(kStGauss, launch_transpose_to_colmajor(ctx, Y1, m, R, ldy1, IDL_F32, Y2, ldy2));
  }
  return IDL_OK;
}

// ---------------------------------------------------------------------------
// Row blocks (Sec. 1.3: S A = sum over row blocks of S[:, rows] A[rows, :]): the
// sketch Omega S[:, i0 .. i0+n) A[i0 .. i0+n, :] of one block of an I-row matrix,
// drawn with the whole matrix's maps, written or added into Y2; and the ID from a
// complete sketch.  Ranks that each hold a block of rows sum their partial
// sketches (one all-reduce of m x R) and run idl_id_from_sketch.
// ---------------------------------------------------------------------------
static int check_rows(idl_ctx* ctx, const idl_params* p, int dtype, int64_t n, int64_t i0, int64_t I, int64_t R,
                      const void* Y2, int64_t ldy2) {
  if (!p) return fail(ctx, IDL_EINVAL, "null params");
  if (dtype != IDL_F32 && dtype != IDL_F64) return fail(ctx, IDL_EINVAL, "dtype must be IDL_F32 or IDL_F64");
  if (p->precision < 0 || p->precision > IDL_PREC_TF32X3 || (dtype == IDL_F64) != (p->precision == IDL_PREC_FP64))
    return fail(ctx, IDL_EINVAL, "precision does not match the data type");
  if (p->m1 < 1 || p->m1 > 0x7fffffffLL || p->m2 < 0 || p->m2 > p->m1) return fail(ctx, IDL_EINVAL, "need 0 <= m2 <= m1");
  if (n < 1 || i0 < 0 || i0 + n > I || I > 0x7fffffffLL || R < 1 || R > 0x7fffffffLL || !Y2)
    return fail(ctx, IDL_EINVAL, "sketch_rows: need 0 <= i0, i0 + n <= I");
  if (p->modified && !(p->m1 < I)) return fail(ctx, IDL_EINVAL, "modified CountSketch needs m1 < I");
  if (ldy2 < (p->m2 > 0 ? p->m2 : p->m1)) return fail(ctx, IDL_EINVAL, "sketch_rows: ldy2 < m");
  if (!is_device_ptr(Y2)) return fail(ctx, IDL_EINVAL, "sketch_rows: Y2 must be device memory");
  return IDL_OK;
}

// shared tail: draws of the block's rows, bucket offsets, the sketch (dense or CSR), the
// Gaussian stage into a packed partial sketch, then Y2 (+)= it
template <typename SK>
static int sketch_rows_tail(idl_ctx* ctx, const idl_params* p, int dtype, int64_t n, int64_t i0, int64_t I, int64_t R,
                            void* Y2, int64_t ldy2, int accumulate, SK&& sketch) {
  const int es = dtype_size(dtype);
  const int64_t m1 = p->m1, m = p->m2 > 0 ? p->m2 : m1;
  WS(h, int32_t, kWsH, n);
  WS(s, int8_t, kWsS, n);
  WS(ptr, int32_t, kWsBucketPtr, m1 + 1);
  WS(rows, int32_t, kWsRowList, n);
  const int64_t ldy1 = round_up(R, 32);
  void* Y1 = ws_get(ctx, kWsY1, (size_t)es * (size_t)(m1 * ldy1));
  void* Yp = ws_get(ctx, kWsY2, (size_t)es * (size_t)(m * R));
  if (!Y1 || !Yp) return IDL_ENOMEM;
  STAGE(kStDraw, cuda_check(ctx, launch_draw_countsketch_range(ctx->stream, p->seed, I, i0, n, m1, p->modified, h, s,
                                                               ctx->d_status), "draw countsketch"));
  STAGE(kStBucket, launch_bucket_offsets(ctx, h, n, m1, ptr, rows));
  STAGE(kStSketch, sketch(s, ptr, rows, Y1, ldy1));
  if (p->m2 > 0) {
    double* Om = (double*)ws_get(ctx, kWsOmega, sizeof(double) * (size_t)(p->m2 * m1));
    if (!Om) return IDL_ENOMEM;
    STAGE(kStDraw, cuda_check(ctx, p->precision == IDL_PREC_FP64
                                       ? launch_draw_gaussian(ctx->stream, p->seed, p->m2, m1, Om)
                                       : launch_draw_gaussian_f32(ctx->stream, p->seed, p->m2, m1, Om),
                              "draw gaussian"));
    STAGE(kStGauss, launch_gaussian(ctx, Om, p->m2, m1, Y1, R, ldy1, dtype, p->precision, Yp, m));
  } else {
    STAGE(kStGauss, launch_transpose_to_colmajor(ctx, Y1, m, R, ldy1, dtype, Yp, m));
  }
  return launch_add_sketch(ctx, Yp, m, R, dtype, Y2, ldy2, accumulate);
}

extern "C" int idl_sketch_rows(idl_ctx* ctx, const void* A, int64_t n, int64_t R, int64_t lda, int dtype, int64_t i0,
                               int64_t I, const idl_params* p, void* Y2, int64_t ldy2, int accumulate) {
  TRY(check_ctx(ctx));
  TRY(check_rows(ctx, p, dtype, n, i0, I, R, Y2, ldy2));
  if (!A || lda < R) return fail(ctx, IDL_EINVAL, "sketch_rows: bad A");
  int rc;
  const void* Ad = stage_in(ctx, A, (size_t)dtype_size(dtype) * (size_t)((n - 1) * lda + R), kWsA, &rc);
  TRY(rc);
  return sketch_rows_tail(ctx, p, dtype, n, i0, I, R, Y2, ldy2, accumulate,
                          [&](const int8_t* s, const int32_t* ptr, const int32_t* rows, void* Y1, int64_t ldy1) {
                            return launch_countsketch_dense(ctx, Ad, n, R, lda, dtype, s, ptr, rows, p->m1, Y1, ldy1);
                          });
}

extern "C" int idl_sketch_rows_csr(idl_ctx* ctx, const int64_t* rowptr, const int32_t* colidx, const void* vals,
                                   int64_t n, int64_t R, int64_t nnz, int dtype, int64_t i0, int64_t I,
                                   const idl_params* p, void* Y2, int64_t ldy2, int accumulate) {
  TRY(check_ctx(ctx));
  TRY(check_rows(ctx, p, dtype, n, i0, I, R, Y2, ldy2));
  if (!rowptr || nnz < 0 || (nnz > 0 && (!colidx || !vals))) return fail(ctx, IDL_EINVAL, "sketch_rows_csr: bad CSR");
  int rc;
  const int64_t* rp = (const int64_t*)stage_in(ctx, rowptr, sizeof(int64_t) * (size_t)(n + 1), kWsRowptr, &rc);
  TRY(rc);
  const int32_t* ci = colidx;
  const void* vv = vals;
  if (nnz) {
    ci = (const int32_t*)stage_in(ctx, colidx, sizeof(int32_t) * (size_t)nnz, kWsColidx, &rc);
    TRY(rc);
    vv = stage_in(ctx, vals, (size_t)dtype_size(dtype) * (size_t)nnz, kWsVals, &rc);
    TRY(rc);
  }
  return sketch_rows_tail(ctx, p, dtype, n, i0, I, R, Y2, ldy2, accumulate,
                          [&](const int8_t* s, const int32_t* ptr, const int32_t* rows, void* Y1, int64_t ldy1) {
                            return launch_countsketch_csr(ctx, rp, ci, vv, n, R, nnz, dtype, s, ptr, rows, p->m1, Y1,
                                                          ldy1);
                          });
}

extern "C" int idl_id_from_sketch(idl_ctx* ctx, const void* Y2, int64_t m, int64_t R, int64_t ldy2, int dtype,
                                  int64_t K, const idl_params* p, int32_t* J, double* T, idl_info* info) {
  TRY(check_ctx(ctx));
  if (!p || !Y2 || !J || !T || (dtype != IDL_F32 && dtype != IDL_F64) || m < 1 || m > 256 || ldy2 < m || K < 1 ||
      K > m || K >= R || R > 0x7fffffffLL)
    return fail(ctx, IDL_EINVAL, "id_from_sketch: bad arguments (1 <= K <= m <= 256, K < R)");
  if (p->residual < 0 || p->residual > 2 || !(p->srrqr_f == 0.f || p->srrqr_f > 1.f) ||
      p->learned < IDL_PROPOSAL_NONE || p->learned > IDL_PROPOSAL_NORM || (p->learned && p->srrqr_f > 0.f))
    return fail(ctx, IDL_EINVAL, "id_from_sketch: bad params");
  if (p->learned && (dtype != IDL_F32 || m > 128 || K > 128))
    return fail(ctx, IDL_ELIMIT, "the column proposal needs FP32 data, m <= 128 and K <= 128");
  const int es = dtype_size(dtype);
  void* Yw = ws_get(ctx, kWsY2, (size_t)es * (size_t)(R * m) * (keeps_sketch(p) ? 2 : 1));
  if (!Yw) return IDL_ENOMEM;
  int rc;
  const void* Yd = stage_in(ctx, Y2, (size_t)es * (size_t)((R - 1) * ldy2 + m), kWsA, &rc);
  TRY(rc);
  TRY(cuda_check(ctx, cudaMemcpy2DAsync(Yw, (size_t)es * m, Yd, (size_t)es * ldy2, (size_t)es * m, R,
                                        cudaMemcpyDeviceToDevice, ctx->stream), "copy sketch"));
  return finish_from_y2(ctx, p, dtype, Yw, m, R, K, J, T, info);
}

// ---------------------------------------------------------------------------
// Gaussian ID, the comparison method (Sec. 1.2.1; Sec. 1.2.2 Eq. G-matrix):
// the sketch is a Gaussian matrix applied to A itself (matrix) or the
// Khatri-Rao structured Gaussian sketch of M (CP tensor); the QR stage and the
// T solve are the CountSketch pipelines'.
// ---------------------------------------------------------------------------
static int check_gaussian_id(idl_ctx* ctx, const idl_params* p, int dtype, int64_t R, int64_t K) {
  if (!p) return fail(ctx, IDL_EINVAL, "null params");
  if (dtype != IDL_F32 && dtype != IDL_F64) return fail(ctx, IDL_EINVAL, "dtype must be IDL_F32 or IDL_F64");
  if (p->precision < 0 || p->precision > IDL_PREC_TF32X3) return fail(ctx, IDL_EINVAL, "unknown precision");
  if ((dtype == IDL_F64) != (p->precision == IDL_PREC_FP64))
    return fail(ctx, IDL_EINVAL, "FP64 data needs precision IDL_PREC_FP64 and FP32 data another mode");
  if (K < 1 || K >= R) return fail(ctx, IDL_EINVAL, "need 1 <= K < R");
  if (p->m2 < K) return fail(ctx, IDL_EINVAL, "need K <= L = params.m2");
  if (p->m2 > (dtype == IDL_F64 ? 112 : 256)) return fail(ctx, IDL_ELIMIT, "Gaussian ID: L = params.m2 > 256 (112 in FP64)");
  if (p->residual < 0 || p->residual > 2) return fail(ctx, IDL_EINVAL, "residual mode must be 0, 1 or 2");
  if (p->learned < IDL_PROPOSAL_NONE || p->learned > IDL_PROPOSAL_NORM)
    return fail(ctx, IDL_EINVAL, "unknown proposal mode");
  if (p->learned && (dtype != IDL_F32 || p->m2 > 128 || K > 128))
    return fail(ctx, IDL_ELIMIT, "the column proposal needs FP32 data, m <= 128 and K <= 128");
  if (R > 0x7fffffffLL) return fail(ctx, IDL_ELIMIT, "R must fit in int32");
  if (!(p->srrqr_f == 0.f || p->srrqr_f > 1.f)) return fail(ctx, IDL_EINVAL, "srrqr_f must be 0 or > 1");
  if (p->srrqr_f > 0.f && p->learned) return fail(ctx, IDL_EINVAL, "srrqr_f and the column proposal exclude each other");
  return IDL_OK;
}

extern "C" int id_matrix_gaussian(idl_ctx* ctx, const void* A, int64_t I, int64_t R, int64_t lda, int dtype,
                                  int64_t K, const idl_params* p, int32_t* J, double* T, idl_info* info) {
  TRY(check_ctx(ctx));
  TRY(check_gaussian_id(ctx, p, dtype, R, K));
  if (I < 1 || I > 0x7fffffffLL || lda < R || !A || !J || !T) return fail(ctx, IDL_EINVAL, "id_matrix_gaussian: bad arguments");
  const int es = dtype_size(dtype);
  const int64_t L = p->m2;
  int rc;
  const void* Ad = stage_in(ctx, A, (size_t)es * (size_t)((I - 1) * lda + R), kWsA, &rc);
  TRY(rc);
  double* Om = (double*)ws_get(ctx, kWsOmega, sizeof(double) * (size_t)(L * I));
  if (!Om) return IDL_ENOMEM;
  void* Y2 = ws_get(ctx, kWsY2, (size_t)es * (size_t)(R * L) * (keeps_sketch(p) ? 2 : 1));
  if (!Y2) return IDL_ENOMEM;
  STAGE(kStDraw, cuda_check(ctx, launch_draw_gaussian_tag(ctx->stream, p->seed, kTagGaussId, L, I, Om), "draw"));
  STAGE(kStSketch, launch_gaussian(ctx, Om, L, I, Ad, R, lda, dtype, p->precision, Y2, L));
  return finish_from_y2(ctx, p, dtype, Y2, L, R, K, J, T, info);
}

extern "C" int id_cp_tensor_gaussian(idl_ctx* ctx, int N, const int64_t* dims, int64_t R, const void* const* factors,
                                     const int64_t* ldf, const double* lambda, int64_t K, const idl_params* p,
                                     int32_t* J, double* T, double* lambda_hat, idl_info* info) {
  TRY(check_ctx(ctx));
  TRY(check_gaussian_id(ctx, p, IDL_F32, R, K));
  if (N < 1 || N > 8 || !dims || !factors || !ldf || !lambda || !J || !T || !lambda_hat)
    return fail(ctx, IDL_EINVAL, "id_cp_tensor_gaussian: bad arguments");
  size_t host_bytes;
  int64_t tot;
  TRY(cp_factor_args(ctx, N, dims, R, factors, ldf, &host_bytes, &tot));
  const int64_t L = p->m2;
  int rc;
  const void* fdev[8];
  TRY(stage_factors(ctx, N, dims, R, factors, ldf, host_bytes, fdev));
  const double* lam = (const double*)stage_in(ctx, lambda, sizeof(double) * (size_t)R, kWsLam, &rc);
  TRY(rc);
  double* Om = (double*)ws_get(ctx, kWsOmega, sizeof(double) * (size_t)(L * tot));
  float* G = (float*)ws_get(ctx, kWsModeSketch, sizeof(float) * (size_t)(N * L * R));
  float* Y2 = (float*)ws_get(ctx, kWsY2, sizeof(float) * (size_t)(R * L) * (keeps_sketch(p) ? 2 : 1));
  if (!Om || !G || !Y2) return IDL_ENOMEM;
  int64_t off = 0;
  for (int n = 0; n < N; ++n) {     // Omega^(n)T (L x I_n, row-major), then G_n = Omega^(n)T A^(n)
    STAGE(kStDraw, cuda_check(ctx, launch_draw_gaussian_tag(ctx->stream, p->seed, kTagGaussMode + n, L, dims[n],
                                                            Om + off), "draw"));
    STAGE(kStSketch, launch_gaussian_tc(ctx, Om + off, L, dims[n], (const float*)fdev[n], R, ldf[n], true,
                                        p->precision, G + (size_t)n * L * R, L));
    off += L * dims[n];
  }
  STAGE(kStSketch, launch_kr_product(ctx, G, N, L, R, lam, Y2));
  const bool jdev = is_device_ptr(J), tdev = is_device_ptr(T), ldev = is_device_ptr(lambda_hat);
  int32_t* Jd = J;
  double* Td = T;
  if (!jdev) { Jd = (int32_t*)ws_get(ctx, kWsJ, sizeof(int32_t) * (size_t)K); if (!Jd) return IDL_ENOMEM; }
  if (!tdev) { Td = (double*)ws_get(ctx, kWsT, sizeof(double) * (size_t)(K * (R - K))); if (!Td) return IDL_ENOMEM; }
  TRY(finish_from_y2(ctx, p, IDL_F32, Y2, L, R, K, Jd, Td, nullptr));
  double* lhd = lambda_hat;
  if (!ldev) { lhd = (double*)ws_get(ctx, kWsLamHat, sizeof(double) * (size_t)K); if (!lhd) return IDL_ENOMEM; }
  STAGE(kStCheck, launch_lambda_hat(ctx, lam, Jd, Td, K, R, lhd));
  if (!jdev) TRY(cuda_check(ctx, cudaMemcpyAsync(J, Jd, sizeof(int32_t) * K, cudaMemcpyDeviceToHost, ctx->stream), "J"));
  if (!tdev)
    TRY(cuda_check(ctx, cudaMemcpyAsync(T, Td, sizeof(double) * K * (R - K), cudaMemcpyDeviceToHost, ctx->stream), "T"));
  if (!ldev)
    TRY(cuda_check(ctx, cudaMemcpyAsync(lambda_hat, lhd, sizeof(double) * K, cudaMemcpyDeviceToHost, ctx->stream),
                   "lambda_hat"));
  if (info) return finish_info(ctx, p, p->precision, info, K, R);
  if (!jdev || !tdev || !ldev) TRY(cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "sync"));
  return IDL_OK;
}

// ---------------------------------------------------------------------------
// ID error estimate (Sec. 6): ||A - A_J P||_2 / ||A||_2 by the power method on the
// device.  Host arrays are staged like the pipelines'; the call synchronises.
// ---------------------------------------------------------------------------
static int stage_jt(idl_ctx* ctx, const int32_t* J, const double* T, int64_t K, int64_t R, const int32_t** Jd,
                    const double** Td) {
  int rc;
  *Jd = (const int32_t*)stage_in(ctx, J, sizeof(int32_t) * (size_t)K, kWsJ, &rc);
  TRY(rc);
  *Td = (const double*)stage_in(ctx, T, sizeof(double) * (size_t)(K * (R - K)), kWsT, &rc);
  return rc;
}

extern "C" int idl_id_error(idl_ctx* ctx, const void* A, int64_t I, int64_t R, int64_t lda, int dtype,
                            const int32_t* J, const double* T, int64_t K, int32_t iters, uint64_t seed, double* err) {
  TRY(check_ctx(ctx));
  if ((dtype != IDL_F32 && dtype != IDL_F64) || I < 1 || R < 2 || lda < R || K < 1 || K >= R || !A || !J || !T ||
      !err || iters < 1 || iters > 1000 || R > 0x7fffffffLL)
    return fail(ctx, IDL_EINVAL, "id_error: bad arguments");
  int rc;
  const void* Ad = stage_in(ctx, A, (size_t)dtype_size(dtype) * (size_t)((I - 1) * lda + R), kWsA, &rc);
  TRY(rc);
  const int32_t* Jd;
  const double* Td;
  TRY(stage_jt(ctx, J, T, K, R, &Jd, &Td));
  return launch_id_error_dense(ctx, Ad, I, R, lda, dtype, Jd, Td, K, iters, seed, err);
}

extern "C" int idl_id_error_csr(idl_ctx* ctx, const int64_t* rowptr, const int32_t* colidx, const void* vals,
                                int64_t I, int64_t R, int64_t nnz, int dtype, const int32_t* J, const double* T,
                                int64_t K, int32_t iters, uint64_t seed, double* err) {
  TRY(check_ctx(ctx));
  if ((dtype != IDL_F32 && dtype != IDL_F64) || I < 1 || R < 2 || nnz < 0 || K < 1 || K >= R || !rowptr || !J ||
      !T || !err || (nnz > 0 && (!colidx || !vals)) || iters < 1 || iters > 1000 || R > 0x7fffffffLL)
    return fail(ctx, IDL_EINVAL, "id_error_csr: bad arguments");
  int rc;
  const int64_t* rp = (const int64_t*)stage_in(ctx, rowptr, sizeof(int64_t) * (size_t)(I + 1), kWsRowptr, &rc);
  TRY(rc);
  const int32_t* ci = nnz ? (const int32_t*)stage_in(ctx, colidx, sizeof(int32_t) * (size_t)nnz, kWsColidx, &rc)
                          : colidx;
  TRY(rc);
  const void* vv = nnz ? stage_in(ctx, vals, (size_t)dtype_size(dtype) * (size_t)nnz, kWsVals, &rc) : vals;
  TRY(rc);
  const int32_t* Jd;
  const double* Td;
  TRY(stage_jt(ctx, J, T, K, R, &Jd, &Td));
  return launch_id_error_csr(ctx, rp, ci, vv, I, R, dtype, Jd, Td, K, iters, seed, err);
}

// ---------------------------------------------------------------------------
// CUDA-graph replay of the pipelines (idl_set_graphs).  The first call with a
// given set of arguments runs eagerly (it sizes the workspace); the second is
// captured on a private stream and the graph launched; later calls replay it,
// ordered after the caller's stream and the caller's stream after it by events.
// A workspace reallocation (any call) makes the cached graphs stale.
// ---------------------------------------------------------------------------
namespace {
// The arguments of a pipeline call: an FNV-1a hash for the lookup and the raw
// bytes, compared in full before a cached graph is replayed.
struct KeyHash {
  uint64_t h = 1469598103934665603ull;                 // FNV-1a, 64-bit
  std::string raw;
  void add(const void* p, size_t n) {
    const unsigned char* c = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) { h ^= c[i]; h *= 1099511628211ull; }
    raw.append((const char*)p, n);
  }
  template <typename X> void v(const X& x) { add(&x, sizeof(X)); }
};
constexpr size_t kMaxPipeGraphs = 8;
}  // namespace

static int launch_pipe_graph(idl_ctx* ctx, const PipeGraph& g) {
  cudaError_t e = cudaEventRecord(ctx->gev_in, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->gstream, ctx->gev_in, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(g.exec, ctx->gstream);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->gev_out, ctx->gstream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->gev_out, 0);
  ctx_add_launches(g.launches);
  return cuda_check(ctx, e, "pipeline graph launch");
}

template <typename F>
static int graphed(idl_ctx* ctx, const KeyHash& k, F&& body) {
  const uint64_t key = k.h;
  PipeGraph* g = nullptr;
  for (auto& x : ctx->pgraphs)
    if (x.key == key && x.raw == k.raw) { g = &x; break; }
  if (g && g->exec && g->gen == ctx->ws_gen) return launch_pipe_graph(ctx, *g);
  if (!g || g->nocap || g->gen != ctx->ws_gen) {
    const int rc = body();                               // eager
    if (rc != IDL_OK) return rc;
    if (!g) {
      if (ctx->pgraphs.size() >= kMaxPipeGraphs) {
        if (ctx->pgraphs.front().exec) cudaGraphExecDestroy(ctx->pgraphs.front().exec);
        ctx->pgraphs.erase(ctx->pgraphs.begin());
      }
      ctx->pgraphs.push_back(PipeGraph{});
      g = &ctx->pgraphs.back();
      g->key = key;
      g->raw = k.raw;
    }
    if (g->exec) { cudaGraphExecDestroy(g->exec); g->exec = nullptr; }
    g->gen = ctx->ws_gen;                                // the workspace as this call left it
    return IDL_OK;
  }
  if (!ctx->gstream) {
    cudaError_t e = cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->gev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->gev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_check(ctx, e, "graph stream");
  }
  cudaStream_t user = ctx->stream;
  ctx->stream = ctx->gstream;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal);
  int rc = IDL_OK;
  const long long before = idl_launch_count();
  const uint64_t gen0 = ctx->ws_gen;
  if (e == cudaSuccess) {
    rc = body();
    e = cudaStreamEndCapture(ctx->gstream, &graph);
  }
  ctx->stream = user;
  const long long nl = idl_launch_count() - before;
  ctx_add_launches(-nl);                                 // counted when the graph runs
  if (e == cudaSuccess && rc == IDL_OK && ctx->ws_gen == gen0 && graph) {
    e = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e == cudaSuccess) {
      g->launches = nl;
      return launch_pipe_graph(ctx, *g);
    }
    g->exec = nullptr;
  } else if (graph) {
    cudaGraphDestroy(graph);
  }
  // nothing of the captured call ran: run it eagerly, and do not capture these arguments again
  (void)cudaGetLastError();
  ctx->err.clear();
  g->nocap = true;
  return body();
}

static bool graph_ok(idl_ctx* ctx, idl_info* info, std::initializer_list<const void*> ptrs) {
  if (!ctx || !ctx->graphs || info || ctx->prof_on) return false;
  for (const void* q : ptrs)
    if (q && !is_device_ptr(q)) return false;
  return true;
}

static void key_ctx(KeyHash& k, idl_ctx* ctx, const idl_params* p) {
  k.v(ctx->gemm_simt);
  k.v(ctx->cpqr_smem_only);
  if (p) k.v(*p);
}

extern "C" int id_matrix(idl_ctx* ctx, const void* A, int64_t I, int64_t R, int64_t lda, int dtype, int64_t K,
                         const idl_params* p, int32_t* J, double* T, idl_info* info) {
  auto body = [&] { return id_matrix_impl(ctx, A, I, R, lda, dtype, K, p, J, T, info); };
  if (!p || !graph_ok(ctx, info, {A, J, T})) return body();
  KeyHash k;
  k.v(1);
  k.v(A); k.v(I); k.v(R); k.v(lda); k.v(dtype); k.v(K); k.v(J); k.v(T);
  key_ctx(k, ctx, p);
  return graphed(ctx, k, body);
}

extern "C" int id_matrix_csr(idl_ctx* ctx, const int64_t* rowptr, const int32_t* colidx, const void* vals, int64_t I,
                             int64_t R, int64_t nnz, int dtype, int64_t K, const idl_params* p, int32_t* J, double* T,
                             idl_info* info) {
  auto body = [&] { return id_matrix_csr_impl(ctx, rowptr, colidx, vals, I, R, nnz, dtype, K, p, J, T, info); };
  if (!p || !graph_ok(ctx, info, {rowptr, colidx, vals, J, T})) return body();
  KeyHash k;
  k.v(2);
  k.v(rowptr); k.v(colidx); k.v(vals); k.v(I); k.v(R); k.v(nnz); k.v(dtype); k.v(K); k.v(J); k.v(T);
  key_ctx(k, ctx, p);
  return graphed(ctx, k, body);
}

extern "C" int id_cp_tensor(idl_ctx* ctx, int N, const int64_t* dims, int64_t R, const void* const* factors,
                            const int64_t* ldf, const double* lambda, int64_t K, const idl_params* p, int32_t* J,
                            double* T, double* lambda_hat, idl_info* info) {
  auto body = [&] { return id_cp_tensor_impl(ctx, N, dims, R, factors, ldf, lambda, K, p, J, T, lambda_hat, info); };
  if (!p || N < 1 || N > 8 || !dims || !factors || !ldf || !graph_ok(ctx, info, {lambda, J, T, lambda_hat}))
    return body();
  KeyHash k;
  k.v(3);
  k.v(N); k.v(R); k.v(lambda); k.v(K); k.v(J); k.v(T); k.v(lambda_hat);
  for (int n = 0; n < N; ++n) { k.v(dims[n]); k.v(factors[n]); k.v(ldf[n]); }
  key_ctx(k, ctx, p);
  return graphed(ctx, k, body);
}

extern "C" int idl_set_graphs(idl_ctx* ctx, int on) {
  if (!ctx) return IDL_EINVAL;
  ctx->graphs = on != 0;
  if (!on) {
    for (auto& g : ctx->pgraphs)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    ctx->pgraphs.clear();
  }
  return IDL_OK;
}
