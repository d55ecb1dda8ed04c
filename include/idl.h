/*
 * idl.h -- C ABI of libidl, a GB300 (sm_103a) implementation of the
 * CountSketch randomized interpolative decomposition (ID) of Malik & Becker,
 * "Fast randomized matrix and tensor interpolative decomposition using
 * CountSketch" (Adv. Comput. Math. 2020; arXiv 1901.10559).
 *
 * Conventions (all entry points):
 *   - Every call is asynchronous on the context's stream unless it says
 *     otherwise.  Returns IDL_OK or an IDL_E* code; no exception crosses the
 *     ABI.  idl_last_error() gives a one-line message for the last failure.
 *   - Indices are 0-based (the paper is 1-based).
 *   - "device pointer" arguments must point to memory of the context's device.
 *     The three pipeline calls (id_matrix, id_matrix_csr, id_cp_tensor) also
 *     accept host pointers (pinned or pageable) for their array arguments: the
 *     data are copied to the device inside the call, and host outputs are
 *     written back before the call returns (the call then synchronises).
 *   - Inputs are never modified.  Outputs are caller-allocated.
 *   - Dense matrices are row-major with a leading dimension (elements).
 *   - A sketch Y2 handed to or produced by the QR stage is column-major:
 *     element (j, r) at Y2[r * ldy2 + j], ldy2 >= m2.
 *   - No call falls back to the CPU: without a usable sm_103a device every
 *     call returns IDL_ECUDA.
 */
#ifndef IDL_H
#define IDL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define IDL_OK        0
#define IDL_EINVAL    1  /* invalid argument (checked on the host before any launch) */
#define IDL_ENOMEM    2  /* device workspace allocation failed */
#define IDL_ECUDA     3  /* CUDA runtime error (message in idl_last_error) */
#define IDL_ERANK     4  /* |r_KK| <= 64 eps |r_11|: sketch numerically rank deficient; J written, T undefined */
#define IDL_ETIMEOUT  5  /* a bounded device wait expired.  Once idl_sync (or an idl_info readback)
                            has reported it, the context is poisoned: every later call on it returns
                            IDL_ETIMEOUT, because tensor-core work or copies that the timed-out kernel
                            left in flight may still write the context's memory.  Destroy the context
                            and create a new one. */
#define IDL_EDATA     6  /* malformed input found on the device (CSR index out of range); bad entries skipped */
#define IDL_ELIMIT    7  /* problem exceeds an on-chip capacity of this build (see the entry point) */

/* ---- element types ---- */
#define IDL_F32 0
#define IDL_F64 1

/* ---- arithmetic of the Gaussian stage ---- */
#define IDL_PREC_FP64   0  /* FP64 operands, FP64 accumulation (CUDA cores)                        */
#define IDL_PREC_FP32   1  /* FP32-accurate: 3-way bf16 split of both operands, 6 tcgen05 products */
#define IDL_PREC_BF16X3 2  /* 2-way bf16 split, 3 tcgen05 products (hi*hi + hi*lo + lo*hi)         */
#define IDL_PREC_BF16   3  /* bf16 operands, FP32 accumulation, 1 tcgen05 product                   */
#define IDL_PREC_TF32X3 4  /* 2-way TF32 split of both operands (hi = top 11 significand bits, lo =
                              the top 11 of the rest, both by truncation), 3 tcgen05 kind::tf32
                              products (hi*hi + hi*lo + lo*hi): ~2^-21 relative per product.
                              Column-major FP32 Y1 is copied into shared memory as it is and only
                              the residual is formed (the fast mode of the column-major pipelines) */

typedef struct idl_ctx idl_ctx;

/* Parameters of one ID.  Zero-initialise and set what you need. */
typedef struct idl_params {
  int64_t  m1;        /* CountSketch rows (the sketch size L of Algorithm 2), or the TensorSketch length L of Algorithm 3 */
  int64_t  m2;        /* Gaussian-stage rows; 0 = no Gaussian stage (the paper's Algorithm 2/3 verbatim) */
  int32_t  modified;  /* 1 = modified CountSketch of Remark 2 (every bucket non-empty; needs m1 < I) */
  int32_t  precision; /* IDL_PREC_*; with IDL_F64 data only IDL_PREC_FP64 is accepted */
  uint64_t seed;      /* seed of the counter-based draws (h, s, the permutation, Omega) */
  int32_t  residual;  /* 0: none; 1: ||R22||_F / ||Y2||_F in FP64 (default); 2: explicit FP64 ||Y2_rest - Y2_J T||_F / ||Y2||_F */
  int32_t  learned;   /* QR stage column proposal: IDL_PROPOSAL_NONE (default), _MLP or _NORM (FP32 data, m <= 128) */
  int32_t  cand_factor; /* proposal candidates C = min(cand_factor * K, R); 0 = 2 (1..8) */
  float    srrqr_f;   /* 0: the pivoted QR's J (default); f > 1: Gu-Eisenstat exchanges after it until no
                         W_ij^2 + (gamma_j / omega_i)^2 exceeds f^2 (a strong rank-revealing QR, Fact 1 with
                         f = 2: |T_ij| <= f); single-item pipelines, not with a column proposal or batches */
  int64_t  reserved[3];
} idl_params;

/* Diagnostics of one ID (filled when a non-NULL pointer is passed; the call then synchronises). */
typedef struct idl_info {
  double   residual;   /* relative sketch residual selected by idl_params.residual (NaN if 0) */
  double   rkk_ratio;  /* |r_KK| / |r_11| of the pivoted QR */
  double   y2_norm;    /* ||Y2||_F */
  int32_t  status;     /* device status word (IDL_OK, IDL_ERANK, IDL_EDATA, IDL_ETIMEOUT) */
  int32_t  precision;  /* precision actually used */
  int32_t  cluster;    /* CTAs in the QR stage's thread-block cluster */
  int32_t  proposal;   /* 0: plain QR; 1: proposal certified; 2: proposal rejected, plain QR ran */
} idl_info;

/* ---------------------------------------------------------------------------
 * Context.  Owns the device workspace (grown on demand, reused across calls),
 * the status word and the stream.  One context per host thread at a time.
 *   idl_create: device = CUDA ordinal.  Fails with IDL_ECUDA if the device is
 *               not compute capability 10.3 (the library is built for sm_103a only).
 *   idl_set_stream: stream is a cudaStream_t (NULL = legacy default stream).
 *   idl_sync: waits for the stream and returns the device status word (then clears it).
 * ------------------------------------------------------------------------- */
int idl_create(idl_ctx** ctx, int device);
int idl_destroy(idl_ctx* ctx);
int idl_set_stream(idl_ctx* ctx, void* stream);
int idl_sync(idl_ctx* ctx);
const char* idl_last_error(idl_ctx* ctx);
int idl_version(void);

/* ---------------------------------------------------------------------------
 * Instrumentation (the paper averages wall time over runs, Sec. 6; this adds
 * device-side timing per stage).
 *   idl_launch_count: kernels this library has launched in the process so far.
 *   idl_profile: on != 0 makes every pipeline call record a CUDA event pair on
 *     the context's stream around each stage.
 *   idl_profile_read: waits for the stream, writes per-stage milliseconds summed
 *     over the calls since the last read (ms[0..nstages)) and how many pairs were
 *     summed (calls, may be NULL), then clears.  Stages: 0 draws, 1 bucket
 *     offsets, 2 sketch (CountSketch / TensorSketch), 3 Gaussian stage, 4 pivoted
 *     QR, 5 T solve, 6 checks (explicit residual, lambda_hat), 7 host->device copies.
 * ------------------------------------------------------------------------- */
long long idl_launch_count(void);
int idl_profile(idl_ctx* ctx, int on);
int idl_profile_read(idl_ctx* ctx, double* ms, long long* calls, int nstages);

/* ---------------------------------------------------------------------------
 * Draws (Sec. 1.3; Remark 2 and Sec. 7.2; Sec. 1.2.1).  Counter-based:
 *   u(seed, tag, i) = mix64(mix64(seed ^ tag*0xD1B54A32D192ED03) + (i+1)*0x9E3779B97F4A7C15)
 *   (mix64 = the SplitMix64 finaliser).  bounded(u, L) = (u*L) >> 64.
 *   tags: 1 buckets, 2 signs, 3 permutation round keys, 4 Gaussian, 16+n / 32+n per tensor mode.
 * idl_draw_countsketch: h[i] in [0, L) (int32), s[i] in {-1, +1} (int8) for i < I.
 *   modified = 1 uses h~(i) = pi(i) if pi(i) < L else bounded(u(seed,1,i), L), pi a
 *   4-round Feistel permutation of [I] with cycle walking; needs L < I.
 * idl_draw_gaussian: Omega (m2 x m1, row-major FP64), Box-Muller on pairs of the flat index.
 * idl_draw_mode: TensorSketch maps of mode n (plain iid maps, Sec. 1.3).
 * All outputs are device pointers.
 * ------------------------------------------------------------------------- */
int idl_draw_countsketch(idl_ctx* ctx, uint64_t seed, int64_t I, int64_t L, int modified,
                         int32_t* h, int8_t* s);
int idl_draw_gaussian(idl_ctx* ctx, uint64_t seed, int64_t m2, int64_t m1, double* Omega);
int idl_draw_mode(idl_ctx* ctx, uint64_t seed, int n, int64_t In, int64_t L, int32_t* h, int8_t* s);
/* idl_draw_gaussian_fp32: the Box-Muller pairs of idl_draw_gaussian from the same
 * uniforms, in FP32 arithmetic (ln U1 as log1pf(-(1 - U1)) for U1 > 1/2, the
 * angle reduced in integers), stored as FP64: within about 4e-7 (rho + |z|) of
 * idl_draw_gaussian.  The pipelines with FP32 data and the batches draw Omega
 * this way (GB300's FP64 pipes are narrow); FP64 data keeps idl_draw_gaussian. */
int idl_draw_gaussian_fp32(idl_ctx* ctx, uint64_t seed, int64_t m2, int64_t m1, double* Omega);

/* ---------------------------------------------------------------------------
 * Bucket offsets of Phi (Sec. 1.3): rows grouped by bucket, ascending within a
 * bucket.  bucket_ptr (L+1 int32) and row_list (I int32) are device outputs.
 * Every bucket lists its rows in increasing order, however many it holds (the
 * output is the stable counting sort of h, bit for bit).
 * ------------------------------------------------------------------------- */
int idl_bucket_offsets(idl_ctx* ctx, const int32_t* h, int64_t I, int64_t L,
                       int32_t* bucket_ptr, int32_t* row_list);

/* ---------------------------------------------------------------------------
 * Allocation-free bucket offsets.  The paper has no counterpart: this is a
 * service for callers that cannot allocate device memory when they need the
 * offsets -- code running while a stream is captured into a CUDA graph, code
 * under a memory budget that forbids allocations after start-up, or a
 * real-time loop that cannot afford a blocking cudaMalloc.  It computes the
 * same bucket_ptr / row_list as idl_bucket_offsets, but needs no context and
 * calls no cudaMalloc, cudaFree or allocating library routine: its scratch is
 * a fixed array of (2 * IDL_NOALLOC_MAX_BUCKETS + 6) int32 words (about
 * 512 KB) in the library's own device memory, which every GPU that loads the
 * library holds until the process exits.
 *   stream: cudaStream_t to launch on (NULL = legacy default stream); the
 *           device is the current device.  h, bucket_ptr, row_list as for
 *           idl_bucket_offsets (device pointers).
 *   Returns IDL_ELIMIT if L > IDL_NOALLOC_MAX_BUCKETS, IDL_EINVAL for bad
 *   sizes or null pointers, IDL_ECUDA on a CUDA error.
 *   The first call on each device looks up the scratch array's device address
 *   (cudaGetSymbolAddress, with that device current); make that first call
 *   before any stream capture.
 *   All calls on a device share the one scratch array and each call clears
 *   the parts that must start at zero, so calls that overlap on the GPU (on
 *   different streams or from different threads) race: serialise them.
 *   Entries of h outside [0, L) are skipped; then bucket_ptr[L] < I: the caller
 *   detects them by checking bucket_ptr[L] == I (no status word is kept).
 * ------------------------------------------------------------------------- */
#define IDL_NOALLOC_MAX_BUCKETS 65536
int idl_bucket_offsets_noalloc(void* stream, const int32_t* h, int64_t I, int64_t L,
                               int32_t* bucket_ptr, int32_t* row_list);

/* ---------------------------------------------------------------------------
 * CountSketch Y1 = S A (Sec. 1.3; the sketch step of Algorithm 2), as a segmented
 * reduction over the bucket offsets: Y1[b, :] = sum over rows i of bucket b of
 * s[i] * A[i, :].  A: I x R row-major (lda >= R), dtype IDL_F32 or IDL_F64;
 * Y1: L x R row-major (ldy >= R), same dtype.  All device pointers.
 * ------------------------------------------------------------------------- */
int idl_countsketch_dense(idl_ctx* ctx, const void* A, int64_t I, int64_t R, int64_t lda, int dtype,
                          const int32_t* h, const int8_t* s, const int32_t* bucket_ptr,
                          const int32_t* row_list, int64_t L, void* Y1, int64_t ldy);

/* Same for CSR A: rowptr (I+1, int64), colidx (nnz, int32), vals (nnz, dtype).
 * Duplicate (i, c) entries add; columns need not be sorted.  Entries with a
 * column outside [0, R) or rows with a decreasing rowptr are skipped and set
 * the status word to IDL_EDATA. */
int idl_countsketch_csr(idl_ctx* ctx, const int64_t* rowptr, const int32_t* colidx, const void* vals,
                        int64_t I, int64_t R, int64_t nnz, int dtype,
                        const int32_t* h, const int8_t* s, const int32_t* bucket_ptr,
                        const int32_t* row_list, int64_t L, void* Y1, int64_t ldy);

/* ---------------------------------------------------------------------------
 * TensorSketch of M = (Khatri-Rao of A^(1..N)) diag(lambda) (Sec. 1.3,
 * Eq. TA-formula; the sketch step of Algorithm 3): Y[:, r] = lambda_r * real(IFFT(prod_n
 * FFT(S^(n) a^(n)_r))).  factors[n]: device pointer to A^(n) stored column by
 * column (column r at factors[n] + r*ldf[n], ldf[n] >= dims[n]), IDL_F32.
 * lambda: R doubles (device).  hs[n], ss[n]: device maps of mode n (length
 * dims[n]).  Y: L x R row-major FP32 (ldy >= R).  L must be a power of two in
 * [16, 8192]; N <= 8.  The host arrays dims, factors, ldf, hs, ss are read
 * during the call only.
 * ------------------------------------------------------------------------- */
int idl_tensorsketch(idl_ctx* ctx, int N, const int64_t* dims, int64_t R,
                     const void* const* factors, const int64_t* ldf, const double* lambda,
                     const int32_t* const* hs, const int8_t* const* ss, int64_t L,
                     float* Y, int64_t ldy);

/* The same with Y column-major: column r at Y + r*ldy, ldy >= L.  id_cp_tensor
 * sketches in this layout when its Gaussian stage runs on the tensor cores
 * (each column is written contiguously by the block that transforms it). */
int idl_tensorsketch_colmajor(idl_ctx* ctx, int N, const int64_t* dims, int64_t R,
                              const void* const* factors, const int64_t* ldf, const double* lambda,
                              const int32_t* const* hs, const int8_t* const* ss, int64_t L,
                              float* Y, int64_t ldy);

/* ---------------------------------------------------------------------------
 * Gaussian stage Y2 = Omega Y1 (Sec. 1.2.1): Omega m2 x m1 row-major FP64
 * (device), Y1 m1 x R row-major (ldy1 >= R) of dtype, Y2 column-major
 * (R columns of ldy2 >= m2 entries) of dtype.  precision = IDL_PREC_*
 * (IDL_F64 requires IDL_PREC_FP64).  m2 <= 256.
 * ------------------------------------------------------------------------- */
int idl_gaussian_stage(idl_ctx* ctx, const double* Omega, int64_t m2, int64_t m1,
                       const void* Y1, int64_t R, int64_t ldy1, int dtype, int precision,
                       void* Y2, int64_t ldy2);

/* The same for FP32 Y1 stored column-major (column r at Y1 + r*ldy1, ldy1 >= m1),
 * on the tensor cores: precision IDL_PREC_FP32, IDL_PREC_BF16X3, IDL_PREC_BF16 or IDL_PREC_TF32X3. */
int idl_gaussian_stage_colmajor(idl_ctx* ctx, const double* Omega, int64_t m2, int64_t m1,
                                const float* Y1, int64_t R, int64_t ldy1, int precision,
                                float* Y2, int64_t ldy2);

/* ---------------------------------------------------------------------------
 * Rank-K column-pivoted Householder QR of Y2 (the pivoted QR of Algorithm 1; Golub & Van
 * Loan Alg. 5.4.1): K steps, each taking the column of largest remaining norm
 * (ties: smallest index).  Y2 (m x R column-major, ldy2 >= m, dtype) is
 * overwritten: rows 0..K-1 of every column hold the triangular factor R
 * (R11 on the pivot columns, R12 on the rest), rows K.. the trailing block.
 * J: K int32 (device), pivot order.  rnorm: K doubles (device) |r_tt|, or NULL.
 * Runs in one thread-block cluster with the matrix in distributed shared
 * memory: needs m <= 256 and m*R*sizeof(dtype) within the cluster's shared
 * memory (IDL_ELIMIT otherwise).
 * ------------------------------------------------------------------------- */
int idl_cpqr(idl_ctx* ctx, void* Y2, int64_t m, int64_t R, int64_t ldy2, int dtype, int64_t K,
             int32_t* J, double* rnorm);

/* ---------------------------------------------------------------------------
 * The QR stage with the strong rank-revealing exchanges of Fact 1 (Gu &
 * Eisenstat 1996): the pivoted QR of idl_cpqr, then, while some
 * rho_ij = W_ij^2 + (gamma_j / omega_i)^2 exceeds f^2 (W = R11^{-1} R12,
 * gamma_j the norm of R22's column j, 1 / omega_i the norm of row i of
 * R11^{-1}), skeleton column J[i] is exchanged for the j-th non-skeleton
 * column (largest rho; ties: smallest i, then j) and the sketch factored again
 * with J as given pivots; each exchange multiplies |det R11| by sqrt(rho).
 * Y2 (m x R column-major, ldy2 >= m, dtype, device) is read only; J (K int32)
 * and T (K x (R-K) FP64, the layout of idl_t_solve) are device outputs for the
 * final selection.  f > 1 (Fact 1 uses f = 2).  Synchronises once per exchange
 * considered; at most 256 exchanges.  The pipelines do the same with
 * idl_params.srrqr_f.
 * ------------------------------------------------------------------------- */
int idl_cpqr_srrqr(idl_ctx* ctx, const void* Y2, int64_t m, int64_t R, int64_t ldy2, int dtype, int64_t K, float f,
                   int32_t* J, double* T);

/* ---------------------------------------------------------------------------
 * T = R11^{-1} R12 in FP64 by back substitution (the solve step of Algorithm 1), from
 * the factored Y2 of idl_cpqr and its J.  T: K x (R-K) row-major FP64 (device);
 * column c of T belongs to the c-th non-skeleton column in ascending index.
 * rest (optional, R-K int32, device) receives those column indices.  K <= 128.
 * ------------------------------------------------------------------------- */
int idl_t_solve(idl_ctx* ctx, const void* Y2, int64_t m, int64_t R, int64_t ldy2, int dtype,
                int64_t K, const int32_t* J, double* T, int32_t* rest);

/* lambda_hat_k = lambda_{J[k]} * (1 + sum_c T[k, c])  (the s-value update of Algorithm 3), FP64, device. */
int idl_lambda_hat(idl_ctx* ctx, const double* lambda, const int32_t* J, const double* T,
                   int64_t K, int64_t R, double* lambda_hat);

/* ---------------------------------------------------------------------------
 * CUDA-graph replay of the pipeline calls (id_matrix, id_matrix_csr,
 * id_cp_tensor).  With on != 0, a call whose arguments (every pointer, size and
 * the params struct) equal an earlier call's is captured once and then replayed
 * as one CUDA graph: the same kernels on the same buffers, the draws from the
 * same seed, with the dependent-launch gaps of the single kernels removed.  Only
 * calls whose arrays are all device pointers, with info == NULL and without
 * stage profiling, are replayed; the others run as usual.  Contents of the
 * buffers may change between calls.  Replays are ordered on the context's
 * stream like eager calls.  Default off; off also frees the cached graphs.
 * ------------------------------------------------------------------------- */
int idl_set_graphs(idl_ctx* ctx, int on);

/* ---------------------------------------------------------------------------
 * Pipelines.  J: K int32, T: K x (R-K) FP64 row-major (see idl_t_solve),
 * lambda_hat: K FP64.  info may be NULL (then the call does not synchronise
 * unless host pointers are involved).
 *
 * id_matrix (Algorithm 2 with a Gaussian stage): dense A (I x R row-major,
 *   lda >= R), dtype IDL_F32 / IDL_F64.  Needs 1 <= K < R, K <= m1, K <= m2 when
 *   m2 > 0, m2 <= m1, m1 < I when modified.
 * id_matrix_csr: CSR A as in idl_countsketch_csr.
 * id_cp_tensor (Algorithm 3 with a Gaussian stage): CP tensor with N factor
 *   matrices (see idl_tensorsketch; device or host arrays), s-values lambda,
 *   params.m1 = the TensorSketch length L (power of two).
 * ------------------------------------------------------------------------- */
int id_matrix(idl_ctx* ctx, const void* A, int64_t I, int64_t R, int64_t lda, int dtype, int64_t K,
              const idl_params* p, int32_t* J, double* T, idl_info* info);
int id_matrix_csr(idl_ctx* ctx, const int64_t* rowptr, const int32_t* colidx, const void* vals,
                  int64_t I, int64_t R, int64_t nnz, int dtype, int64_t K, const idl_params* p,
                  int32_t* J, double* T, idl_info* info);
int id_cp_tensor(idl_ctx* ctx, int N, const int64_t* dims, int64_t R, const void* const* factors,
                 const int64_t* ldf, const double* lambda, int64_t K, const idl_params* p,
                 int32_t* J, double* T, double* lambda_hat, idl_info* info);

/* ---------------------------------------------------------------------------
 * Row blocks.  The sketch is linear in the rows of A (Sec. 1.3):
 *   Omega S A = sum over row blocks B of Omega S[:, B] A[B, :],
 * so a matrix split by rows over several GPUs (or streamed in pieces) is
 * sketched block by block and the partial sketches are summed.
 * idl_sketch_rows / idl_sketch_rows_csr: rows i0 .. i0+n-1 of an I-row matrix
 *   (A here holds just those n rows; the CSR rowptr has n + 1 entries indexing
 *   colidx / vals), sketched with the maps h, s, the permutation and Omega of
 *   the whole I-row matrix (params as for id_matrix; K is not needed), into
 *   the m x R column-major sketch Y2 (device memory, ldy2 >= m; m = params.m2,
 *   or params.m1 when m2 = 0): Y2 = partial (accumulate = 0) or Y2 += partial.
 *   A, rowptr, colidx, vals: device or host arrays.
 * idl_id_from_sketch: Algorithm 1 on a complete sketch Y2 (m x R column-major,
 *   device or host, ldy2 >= m, m <= 256): J, T (and info) as the pipelines
 *   give them; params.residual, learned, cand_factor and srrqr_f apply.
 * ------------------------------------------------------------------------- */
int idl_sketch_rows(idl_ctx* ctx, const void* A, int64_t n, int64_t R, int64_t lda, int dtype, int64_t i0, int64_t I,
                    const idl_params* p, void* Y2, int64_t ldy2, int accumulate);
int idl_sketch_rows_csr(idl_ctx* ctx, const int64_t* rowptr, const int32_t* colidx, const void* vals, int64_t n,
                        int64_t R, int64_t nnz, int dtype, int64_t i0, int64_t I, const idl_params* p, void* Y2,
                        int64_t ldy2, int accumulate);
int idl_id_from_sketch(idl_ctx* ctx, const void* Y2, int64_t m, int64_t R, int64_t ldy2, int dtype, int64_t K,
                       const idl_params* p, int32_t* J, double* T, idl_info* info);

/* Column blocks of a CP tensor.  Column r of the tensor's sketch depends only on
 * lambda_r, column r of every factor and the modes' maps h_n, s_n (drawn from
 * seed, n, I_n and L; Sec. 1.3, Eq. TA-formula), so a tensor whose R columns are
 * split over GPUs is sketched block by block and the blocks, gathered side by
 * side in column order, are the whole tensor's sketch (then idl_id_from_sketch
 * and idl_lambda_hat with the whole lambda).
 * idl_sketch_cp: Y2 = Omega Y1 (m x R column-major, device memory, ldy2 >= m;
 *   m = params.m2 <= 256, or L = params.m1 when m2 = 0) for the R columns given:
 *   factors, ldf, lambda as for id_cp_tensor (device or host arrays); params.m1
 *   = L a power of two, precision FP32, BF16X3, BF16 or TF32X3; K, residual, learned
 *   and srrqr_f are not used.  Returns without synchronising. */
int idl_sketch_cp(idl_ctx* ctx, int N, const int64_t* dims, int64_t R, const void* const* factors,
                  const int64_t* ldf, const double* lambda, const idl_params* p, float* Y2, int64_t ldy2);

/* ---------------------------------------------------------------------------
 * Gaussian ID, the comparison method of the paper (Sec. 1.2.1 and Sec. 1.2.2).
 * The sketch size is L = params.m2 (K <= L <= 256; L <= 112 for FP64 data);
 * params.m1 and params.modified are not used.  Outputs as for the pipelines
 * above; device or host arrays.
 * id_matrix_gaussian: Y = Omega A with Omega an L x I matrix of iid N(0,1)
 *   entries (the counter-based Box-Muller draw of idl_draw_gaussian with tag 5,
 *   row-major L x I), formed on the tensor cores in the precision mode of
 *   params.precision (FP64 data: CUDA cores), then the pivoted QR and T of
 *   Algorithm 1.  Dense A only (row-major, lda >= R).
 * id_cp_tensor_gaussian: the Khatri-Rao structured Gaussian sketch of Eq.
 *   G-matrix, y_lr = lambda_r prod_n <omega^(n)_:l, a^(n)_:r>, with Omega^(n)T
 *   the L x I_n draw of tag 48 + n; one tensor-core product per mode and an
 *   entrywise product; then Algorithm 1 and lambda_hat as in Algorithm 3.  FP32
 *   factors stored column by column (ldf[n] >= dims[n]).
 * ------------------------------------------------------------------------- */
int id_matrix_gaussian(idl_ctx* ctx, const void* A, int64_t I, int64_t R, int64_t lda, int dtype, int64_t K,
                       const idl_params* p, int32_t* J, double* T, idl_info* info);
int id_cp_tensor_gaussian(idl_ctx* ctx, int N, const int64_t* dims, int64_t R, const void* const* factors,
                          const int64_t* ldf, const double* lambda, int64_t K, const idl_params* p,
                          int32_t* J, double* T, double* lambda_hat, idl_info* info);

/* ---------------------------------------------------------------------------
 * ID error estimate of Sec. 6 (the randomized spectral-norm estimate of Woolfe
 * et al., Sec. 3.4): err = est ||A - A_J P||_2 / est ||A||_2, each estimate
 * `iters` steps of the power method on E^T E (E = A - A_J P) and on A^T A from
 * the counter-based Gaussian start vector of tag 6 (1 x R; seed for E, seed + 1
 * for A), FP64 vectors and accumulation.  The power method never overestimates a
 * spectral norm.  A dense (row-major, lda >= R) or CSR as for id_matrix_csr;
 * J (K int32) and T (K x (R-K) FP64, the pipelines' layout) from any pipeline.
 * Device or host arrays; err is a host double; the call synchronises.
 * 1 <= iters <= 1000.
 * ------------------------------------------------------------------------- */
int idl_id_error(idl_ctx* ctx, const void* A, int64_t I, int64_t R, int64_t lda, int dtype, const int32_t* J,
                 const double* T, int64_t K, int32_t iters, uint64_t seed, double* err);
int idl_id_error_csr(idl_ctx* ctx, const int64_t* rowptr, const int32_t* colidx, const void* vals, int64_t I,
                     int64_t R, int64_t nnz, int dtype, const int32_t* J, const double* T, int64_t K, int32_t iters,
                     uint64_t seed, double* err);

/* ---------------------------------------------------------------------------
 * Batches.  Many IDs of uneven sizes in one pass: every stage of the path is
 * one launch over all items, and the pivoted QR runs one thread-block cluster
 * per item in one launch.  The launch sequence of a batch shape is captured
 * once into a CUDA graph and replayed on later calls with the same shape.  On
 * the first call of a shape the dense sketch's block width, the Gaussian
 * stage's split-K rule (each item split to fill the SMs once or twice by
 * itself, or -- tune-file value 0 -- split only as far as the whole batch needs
 * for eight waves of CTAs), the QR stage's cluster sizes (16, 8 or 4 CTAs
 * per item) and its cap on threads per CTA (dense items 1024, 256 or 128; CP
 * items 1024, 512 or 320), dense and CP items separately, are chosen by timing
 * the candidates (the call then runs the batch several times); idl_tune_save /
 * idl_tune_load keep those choices in a text file (lines written before the
 * thread caps existed load with caps of 1024).  The QR stage groups the items
 * by the kernel shape each picks under those choices and launches the groups
 * concurrently, on side streams of the context.  In the bf16 precision modes the
 * TensorSketch of a CP item with L = 8192 writes the Gaussian stage's bf16
 * operand planes directly, in the tile layout the tensor cores read.
 *   Items: IDL_ITEM_DENSE (Algorithm 2 on a dense FP32 matrix) or IDL_ITEM_CP
 *   (Algorithm 3 on a CP tensor), FP32 data, one precision mode per batch
 *   (IDL_PREC_FP32 / BF16X3 / BF16 / TF32X3), Gaussian stage required with
 *   K <= m2 <= min(m1, 128), K <= 128.  CP factors are stored column by
 *   column (ldf = dims[n]).  Outputs as for the single-item calls.
 *   Either every array of the batch is device memory -- the call is then
 *   asynchronous after its first use of a shape, and idl_sync returns the
 *   device status word -- or every array is host memory (decided by the first
 *   item's A or first factor; pinned memory copies fastest): the call then
 *   copies the inputs into a device staging buffer on a copy stream of its own,
 *   the CP items' factors first and the dense matrices in eight groups of about
 *   equal bytes, and runs each group (the CP items, then each dense group)
 *   through every stage as soon as its own inputs have landed -- the results
 *   are those of the device-array call; it copies J, T and lambda_hat back and
 *   synchronises before it returns.  idl_batch_fallbacks then counts over all
 *   groups.
 * ------------------------------------------------------------------------- */
/* ---------------------------------------------------------------------------
 * Learned column proposal for the QR stage (not in the paper; an acceleration
 * of Algorithm 1's pivot search that never changes its result).
 *   With idl_params.learned = IDL_PROPOSAL_MLP the QR stage scores every
 *   column of the sketch Y2 (m x R) with a 3-layer MLP (width 128, bfloat16
 *   operands, FP32 accumulation) on 8 features per column: log and square root
 *   of the relative squared norm, three ridge leverage scores
 *   y^T (Y2 Y2^T + lambda I)^{-1} y with lambda = {1e-1, 1e-2, 1e-3} tr(Y2 Y2^T)/m,
 *   max |y_i| / ||y||, K/R and m/R.  The C = min(2K, R) best columns (ties:
 *   smaller index; cand_factor = 4 or 8 widens the set) go through the
 *   pivoted QR in one CTA; its reflectors are
 *   applied to every other column, and the certificate checks that no outside
 *   column's remaining norm reaches a step's pivot norm (squared norms within a
 *   relative margin of 1e-4).  If it holds, J and the factored sketch equal
 *   those of the plain QR; otherwise the plain QR runs (idl_info.proposal = 2).
 *   IDL_PROPOSAL_NORM is the ablation that scores columns by their norm.
 *   Needs FP32 data, m <= 128, K <= 128 (IDL_ELIMIT otherwise), and weights
 *   (idl_mlp_init, idl_mlp_set_weights or idl_load_weights) for _MLP.
 *
 * Parameters: IDL_MLP_NPARAM floats, flat: W1 (128 x 8 row-major), b1 (128),
 *   W2 (128 x 128 row-major), b2 (128), w3 (128), b3 (1); the context keeps
 *   them in FP32 (master copy for training) and rounds W1, W2, w3, the
 *   features and the first hidden layer to bfloat16 when it multiplies.
 * idl_mlp_set_weights / idl_mlp_get_weights: host or device pointer; setting
 *   resets the optimizer state.  idl_mlp_init: He-style random weights.
 * idl_save_weights / idl_load_weights: binary file "IDLMLP01", uint32 version
 *   1, 8, 128, IDL_MLP_NPARAM, the parameters (float32 little endian), uint64
 *   FNV-1a hash of the parameter bytes; a wrong layout or hash is IDL_EINVAL.
 * idl_proposal_features: F (R x 8 row-major FP32, device) of Y (m x R
 *   column-major, ldy >= m, FP32, device); m <= 128.
 * idl_mlp_scores: s[i] = MLP(F[i, :]) for n examples (device pointers).
 * idl_mlp_grad: mean loss over n examples with labels y in {0, 1}
 *   (pos_weight * y * softplus(-s) + (1 - y) * softplus(s)) and its gradient
 *   (IDL_MLP_NPARAM floats) with respect to the FP32 weights, treating the
 *   bfloat16 rounding as the identity; device pointers, no update.
 * idl_proposal_labels: training examples of one sketch: F as above and
 *   y[c] = 1 for the K pivots of the plain QR of Y (run on a copy), else 0.
 * idl_train_proposal: Adam (Kingma & Ba 2015) on the context's weights over
 *   n device-resident examples, minibatches of tp->batch in a seeded permuted
 *   order per epoch; epoch_loss (host, tp->epochs floats, optional) receives
 *   each epoch's mean minibatch loss.  Initialises the weights if none are set.
 * ------------------------------------------------------------------------- */
#define IDL_PROPOSAL_NONE 0
#define IDL_PROPOSAL_MLP  1
#define IDL_PROPOSAL_NORM 2
#define IDL_MLP_NPARAM 17793

typedef struct idl_train_params {
  int32_t  epochs;
  int32_t  batch;       /* examples per Adam step */
  float    lr;
  float    beta1, beta2, eps;   /* 0 = defaults 0.9, 0.999, 1e-8 */
  float    pos_weight;  /* weight of the positive (pivot) examples; 0 = 1 */
  int32_t  reserved0;
  uint64_t seed;        /* epoch orders (and the initial weights if none are set) */
} idl_train_params;

int idl_mlp_init(idl_ctx* ctx, uint64_t seed);
int idl_mlp_set_weights(idl_ctx* ctx, const float* theta);
int idl_mlp_get_weights(idl_ctx* ctx, float* theta);
int idl_save_weights(idl_ctx* ctx, const char* path);
int idl_load_weights(idl_ctx* ctx, const char* path);
int idl_proposal_features(idl_ctx* ctx, const float* Y, int64_t m, int64_t R, int64_t ldy, int64_t K, float* F);
int idl_mlp_scores(idl_ctx* ctx, const float* F, int64_t n, float* s);
int idl_mlp_grad(idl_ctx* ctx, const float* F, const float* y, int64_t n, float pos_weight, float* grad,
                 float* loss);
int idl_proposal_labels(idl_ctx* ctx, const float* Y, int64_t m, int64_t R, int64_t ldy, int64_t K,
                        float* F, float* y);
int idl_train_proposal(idl_ctx* ctx, const float* F, const float* y, int64_t n, const idl_train_params* tp,
                       float* epoch_loss);
/* The QR stage through the proposal on a given sketch: Y2 (m x R column-major,
 * ldy2 >= m, FP32, device, read only) -> Yf (same shape, the factored sketch
 * as idl_cpqr leaves it), J (K int32, device).  mode: IDL_PROPOSAL_MLP or
 * IDL_PROPOSAL_NORM; cand_factor as in idl_params.  proposal (host, optional): 1 certified, 2 rejected
 * (the plain QR ran); passing it synchronises the stream. */
int idl_cpqr_proposal(idl_ctx* ctx, const float* Y2, float* Yf, int64_t m, int64_t R, int64_t ldy2,
                      int64_t K, int mode, int cand_factor, int32_t* J, int* proposal);

#define IDL_ITEM_DENSE 0
#define IDL_ITEM_CP    2

typedef struct idl_batch_item {
  int32_t       kind;        /* IDL_ITEM_DENSE or IDL_ITEM_CP */
  int32_t       N;           /* CP: number of modes (1..8) */
  int64_t       I, R, lda;   /* dense: A is I x R row-major (lda >= R); CP: R = number of rank-1 terms */
  int64_t       K;           /* target rank */
  const float*  A;           /* dense matrix (device) */
  int64_t       dims[8];     /* CP: mode sizes */
  const float*  factors[8];  /* CP: factor matrices, column r of mode n at factors[n] + r*dims[n] (device) */
  const double* lambda;      /* CP: R s-values (device) */
  idl_params    params;      /* m1 (the TensorSketch length L for CP), m2, modified, precision, seed, learned */
  int32_t*      J;           /* out: K pivots (device) */
  double*       T;           /* out: K x (R-K) FP64 (device) */
  double*       lambda_hat;  /* out, CP: K s-values (device) */
} idl_batch_item;

int idl_batch_run(idl_ctx* ctx, const idl_batch_item* items, int n);
/* Items of the last idl_batch_run whose column proposal (params.learned) was
 * rejected by its certificate, so that the plain QR ran; synchronises the
 * stream.  Returns the count (>= 0) or minus an error code. */
int idl_batch_fallbacks(idl_ctx* ctx);
int idl_tune_save(idl_ctx* ctx, const char* path);
int idl_tune_load(idl_ctx* ctx, const char* path);

#ifdef __cplusplus
}
#endif
#endif /* IDL_H */
