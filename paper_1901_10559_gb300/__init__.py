"""GB300 (sm_103a) CountSketch interpolative decomposition -- Python binding.

A thin ctypes layer over ``libidl.so`` (C ABI declared in ``include/idl.h``):
the functions below have the C entry points' names and only marshal
arguments (torch CUDA tensors or numpy host arrays -> pointers).  Every step of
the method runs in the library's CUDA kernels; there is no CPU path here and
the import fails loudly when the library is missing.

Method: Malik & Becker, "Fast randomized matrix and tensor interpolative
decomposition using CountSketch" -- Algorithm 2 (CountSketch matrix ID) and
Algorithm 3 (TensorSketch tensor ID), each followed here by a Gaussian stage
(Sec. 1.2.1) before Algorithm 1's column-pivoted QR.
"""
from __future__ import annotations

import ctypes
import os
import re

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libidl.so")
# weights of the QR stage's column-proposal MLP, written by train_proposal.py
PROPOSAL_WEIGHTS = os.path.join(_HERE, "proposal_weights.bin")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "idl.h")

IDL_OK, IDL_EINVAL, IDL_ENOMEM, IDL_ECUDA, IDL_ERANK, IDL_ETIMEOUT, IDL_EDATA, IDL_ELIMIT = range(8)
IDL_F32, IDL_F64 = 0, 1
PREC_FP64, PREC_FP32, PREC_BF16X3, PREC_BF16, PREC_TF32X3 = 0, 1, 2, 3, 4
STAGES = ("draws", "buckets", "sketch", "gaussian", "cpqr", "tsolve", "check", "copy")
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ERANK", 5: "ETIMEOUT", 6: "EDATA", 7: "ELIMIT"}


class IdlError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"idl error {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("m1", ctypes.c_int64), ("m2", ctypes.c_int64), ("modified", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("seed", ctypes.c_uint64), ("residual", ctypes.c_int32),
                ("learned", ctypes.c_int32), ("cand_factor", ctypes.c_int32), ("srrqr_f", ctypes.c_float),
                ("reserved", ctypes.c_int64 * 3)]


class Info(ctypes.Structure):
    _fields_ = [("residual", ctypes.c_double), ("rkk_ratio", ctypes.c_double), ("y2_norm", ctypes.c_double),
                ("status", ctypes.c_int32), ("precision", ctypes.c_int32), ("cluster", ctypes.c_int32),
                ("proposal", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


PROPOSAL_NONE, PROPOSAL_MLP, PROPOSAL_NORM = 0, 1, 2
MLP_NPARAM = 17793


class TrainParams(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("pos_weight", ctypes.c_float), ("reserved0", ctypes.c_int32), ("seed", ctypes.c_uint64)]


IDL_ITEM_DENSE, IDL_ITEM_CP = 0, 2


class BatchItem(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("N", ctypes.c_int32), ("I", ctypes.c_int64), ("R", ctypes.c_int64),
                ("lda", ctypes.c_int64), ("K", ctypes.c_int64), ("A", ctypes.c_void_p),
                ("dims", ctypes.c_int64 * 8), ("factors", ctypes.c_void_p * 8), ("lambda_", ctypes.c_void_p),
                ("params", Params), ("J", ctypes.c_void_p), ("T", ctypes.c_void_p),
                ("lambda_hat", ctypes.c_void_p)]


_lib = None
_vp, _i64, _i32, _u64, _int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_int

_SIGS = {
    "idl_version": ([], _int),
    "idl_create": ([ctypes.POINTER(_vp), _int], _int),
    "idl_destroy": ([_vp], _int),
    "idl_set_stream": ([_vp, _vp], _int),
    "idl_sync": ([_vp], _int),
    "idl_last_error": ([_vp], ctypes.c_char_p),
    "idl_launch_count": ([], ctypes.c_longlong),
    "idl_profile": ([_vp, _int], _int),
    "idl_profile_read": ([_vp, _vp, _vp, _int], _int),
    "idl_debug_fail_alloc": ([_vp, _int], _int),
    "idl_debug_release_workspace": ([_vp], _int),
    "idl_debug_gemm_path": ([_vp, _int], _int),
    "idl_set_graphs": ([_vp, _int], _int),
    "idl_debug_cpqr_path": ([_vp, _int], _int),
    "idl_draw_countsketch": ([_vp, _u64, _i64, _i64, _int, _vp, _vp], _int),
    "idl_draw_gaussian": ([_vp, _u64, _i64, _i64, _vp], _int),
    "idl_draw_gaussian_fp32": ([_vp, _u64, _i64, _i64, _vp], _int),
    "idl_draw_mode": ([_vp, _u64, _int, _i64, _i64, _vp, _vp], _int),
    "idl_cpqr_srrqr": ([_vp, _vp, _i64, _i64, _i64, _int, _i64, ctypes.c_float, _vp, _vp], _int),
    "idl_bucket_offsets": ([_vp, _vp, _i64, _i64, _vp, _vp], _int),
    "idl_bucket_offsets_noalloc": ([_vp, _vp, _i64, _i64, _vp, _vp], _int),
    "idl_countsketch_dense": ([_vp, _vp, _i64, _i64, _i64, _int, _vp, _vp, _vp, _vp, _i64, _vp, _i64], _int),
    "idl_countsketch_csr": ([_vp, _vp, _vp, _vp, _i64, _i64, _i64, _int, _vp, _vp, _vp, _vp, _i64, _vp, _i64], _int),
    "idl_tensorsketch": ([_vp, _int, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _i64, _vp, _i64], _int),
    "idl_gaussian_stage": ([_vp, _vp, _i64, _i64, _vp, _i64, _i64, _int, _int, _vp, _i64], _int),
    "idl_tensorsketch_colmajor": ([_vp, _int, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _i64, _vp, _i64], _int),
    "idl_gaussian_stage_colmajor": ([_vp, _vp, _i64, _i64, _vp, _i64, _i64, _int, _vp, _i64], _int),
    "idl_cpqr": ([_vp, _vp, _i64, _i64, _i64, _int, _i64, _vp, _vp], _int),
    "idl_t_solve": ([_vp, _vp, _i64, _i64, _i64, _int, _i64, _vp, _vp, _vp], _int),
    "idl_lambda_hat": ([_vp, _vp, _vp, _vp, _i64, _i64, _vp], _int),
    "id_matrix": ([_vp, _vp, _i64, _i64, _i64, _int, _i64, ctypes.POINTER(Params), _vp, _vp,
                   ctypes.POINTER(Info)], _int),
    "id_matrix_csr": ([_vp, _vp, _vp, _vp, _i64, _i64, _i64, _int, _i64, ctypes.POINTER(Params), _vp, _vp,
                       ctypes.POINTER(Info)], _int),
    "id_cp_tensor": ([_vp, _int, _vp, _i64, _vp, _vp, _vp, _i64, ctypes.POINTER(Params), _vp, _vp, _vp,
                      ctypes.POINTER(Info)], _int),
    "id_matrix_gaussian": ([_vp, _vp, _i64, _i64, _i64, _int, _i64, ctypes.POINTER(Params), _vp, _vp,
                            ctypes.POINTER(Info)], _int),
    "id_cp_tensor_gaussian": ([_vp, _int, _vp, _i64, _vp, _vp, _vp, _i64, ctypes.POINTER(Params), _vp, _vp, _vp,
                               ctypes.POINTER(Info)], _int),
    "idl_id_error": ([_vp, _vp, _i64, _i64, _i64, _int, _vp, _vp, _i64, ctypes.c_int32, ctypes.c_uint64,
                      ctypes.POINTER(ctypes.c_double)], _int),
    "idl_id_error_csr": ([_vp, _vp, _vp, _vp, _i64, _i64, _i64, _int, _vp, _vp, _i64, ctypes.c_int32,
                          ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)], _int),
    "idl_sketch_rows": ([_vp, _vp, _i64, _i64, _i64, _int, _i64, _i64, ctypes.POINTER(Params), _vp, _i64, _int],
                        _int),
    "idl_sketch_rows_csr": ([_vp, _vp, _vp, _vp, _i64, _i64, _i64, _int, _i64, _i64, ctypes.POINTER(Params), _vp,
                             _i64, _int], _int),
    "idl_id_from_sketch": ([_vp, _vp, _i64, _i64, _i64, _int, _i64, ctypes.POINTER(Params), _vp, _vp,
                            ctypes.POINTER(Info)], _int),
    "idl_sketch_cp": ([_vp, _int, _vp, _i64, _vp, _vp, _vp, ctypes.POINTER(Params), _vp, _i64], _int),
    "idl_batch_run": ([_vp, ctypes.POINTER(BatchItem), _int], _int),
    "idl_tune_save": ([_vp, ctypes.c_char_p], _int),
    "idl_tune_load": ([_vp, ctypes.c_char_p], _int),
    "idl_debug_batch_mode": ([_vp, _int, _int], _int),
    "idl_debug_wait_probe": ([_vp, _int, ctypes.c_ulonglong], _int),
    "idl_debug_batch_timing": ([_vp, ctypes.POINTER(BatchItem), _int, ctypes.POINTER(ctypes.c_float)], _int),
    "idl_batch_fallbacks": ([_vp], _int),
    "idl_mlp_init": ([_vp, _u64], _int),
    "idl_mlp_set_weights": ([_vp, _vp], _int),
    "idl_mlp_get_weights": ([_vp, _vp], _int),
    "idl_save_weights": ([_vp, ctypes.c_char_p], _int),
    "idl_load_weights": ([_vp, ctypes.c_char_p], _int),
    "idl_proposal_features": ([_vp, _vp, _i64, _i64, _i64, _i64, _vp], _int),
    "idl_mlp_scores": ([_vp, _vp, _i64, _vp], _int),
    "idl_mlp_grad": ([_vp, _vp, _vp, _i64, ctypes.c_float, _vp, _vp], _int),
    "idl_proposal_labels": ([_vp, _vp, _i64, _i64, _i64, _i64, _vp, _vp], _int),
    "idl_train_proposal": ([_vp, _vp, _vp, _i64, ctypes.POINTER(TrainParams), _vp], _int),
    "idl_cpqr_proposal": ([_vp, _vp, _vp, _i64, _i64, _i64, _i64, _int, _int, _vp, ctypes.POINTER(ctypes.c_int)],
                          _int),
}


def header_symbols():
    """Function names declared in include/idl.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\**(\w+)\s*\(", txt, flags=re.M)))


def lib():
    """The loaded libidl.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_1901_10559_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            if hasattr(L, name):
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
        _lib = L
    return _lib


def _p(x):
    """Pointer of a torch tensor, numpy array, integer address or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return _vp(x)
    if hasattr(x, "data_ptr"):
        return _vp(x.data_ptr())
    if hasattr(x, "ctypes"):
        return _vp(x.ctypes.data)
    raise TypeError(f"cannot take a pointer of {type(x)}")


class Context:
    """An idl_ctx on one CUDA device (workspace, status word, stream)."""

    def __init__(self, device: int = 0):
        self.ptr = _vp()
        rc = lib().idl_create(ctypes.byref(self.ptr), device)
        if rc != IDL_OK:
            raise IdlError(rc, "idl_create failed (needs a compute capability 10.3 GPU)")
        self.device = device

    def check(self, rc):
        if rc != IDL_OK:
            raise IdlError(rc, lib().idl_last_error(self.ptr).decode())
        return rc

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
        h = 0 if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        self.check(lib().idl_set_stream(self.ptr, _vp(h)))

    def sync(self):
        return lib().idl_sync(self.ptr)

    def profile(self, on: bool):
        self.check(lib().idl_profile(self.ptr, int(on)))

    def profile_read(self):
        """Per-stage device milliseconds and event-pair counts since the last read."""
        ms = (ctypes.c_double * len(STAGES))()
        n = (ctypes.c_longlong * len(STAGES))()
        self.check(lib().idl_profile_read(self.ptr, ctypes.cast(ms, _vp), ctypes.cast(n, _vp), len(STAGES)))
        return {name: (ms[i], n[i]) for i, name in enumerate(STAGES)}

    def close(self):
        if self.ptr:
            lib().idl_destroy(self.ptr)
            self.ptr = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def launch_count() -> int:
    """Kernels the library has launched in this process."""
    return int(lib().idl_launch_count())


def make_params(m1, m2, seed, modified=True, precision=PREC_FP32, residual=1, learned=PROPOSAL_NONE,
                cand_factor=0, srrqr_f=0.0):
    p = Params()
    p.m1, p.m2, p.modified, p.precision, p.seed, p.residual = int(m1), int(m2), int(modified), int(precision), \
        int(seed), int(residual)
    p.learned, p.cand_factor, p.srrqr_f = int(learned), int(cand_factor), float(srrqr_f)
    return p


# ---------------------------------------------------------------- stage calls
def idl_draw_countsketch(ctx, seed, I, L, modified, h, s):
    return ctx.check(lib().idl_draw_countsketch(ctx.ptr, seed, I, L, int(modified), _p(h), _p(s)))


def idl_draw_gaussian(ctx, seed, m2, m1, Omega):
    return ctx.check(lib().idl_draw_gaussian(ctx.ptr, seed, m2, m1, _p(Omega)))


def idl_draw_gaussian_fp32(ctx, seed, m2, m1, Omega):
    return ctx.check(lib().idl_draw_gaussian_fp32(ctx.ptr, seed, m2, m1, _p(Omega)))


def idl_cpqr_srrqr(ctx, Y2, m, R, ldy2, dtype, K, f, J, T):
    return ctx.check(lib().idl_cpqr_srrqr(ctx.ptr, _p(Y2), m, R, ldy2, dtype, K, f, _p(J), _p(T)))


def idl_draw_mode(ctx, seed, n, In, L, h, s):
    return ctx.check(lib().idl_draw_mode(ctx.ptr, seed, n, In, L, _p(h), _p(s)))


def idl_bucket_offsets(ctx, h, I, L, bucket_ptr, row_list):
    return ctx.check(lib().idl_bucket_offsets(ctx.ptr, _p(h), I, L, _p(bucket_ptr), _p(row_list)))


def idl_bucket_offsets_noalloc(stream, h, I, L, bucket_ptr, row_list):
    """Allocation-free bucket offsets (no context; scratch in a fixed device array).
    stream: torch.cuda.Stream, raw cudaStream_t integer or None.  Returns the status code."""
    hs = 0 if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    return lib().idl_bucket_offsets_noalloc(_vp(hs), _p(h), I, L, _p(bucket_ptr), _p(row_list))


def idl_countsketch_dense(ctx, A, I, R, lda, dtype, h, s, bucket_ptr, row_list, L, Y1, ldy):
    return ctx.check(lib().idl_countsketch_dense(ctx.ptr, _p(A), I, R, lda, dtype, _p(h), _p(s), _p(bucket_ptr),
                                                 _p(row_list), L, _p(Y1), ldy))


def idl_countsketch_csr(ctx, rowptr, colidx, vals, I, R, nnz, dtype, h, s, bucket_ptr, row_list, L, Y1, ldy):
    return ctx.check(lib().idl_countsketch_csr(ctx.ptr, _p(rowptr), _p(colidx), _p(vals), I, R, nnz, dtype, _p(h),
                                               _p(s), _p(bucket_ptr), _p(row_list), L, _p(Y1), ldy))


def _arr(ctype, vals):
    return (ctype * len(vals))(*vals)


def idl_tensorsketch(ctx, factors, ldf, lam, hs, ss, L, Y, ldy, colmajor=False):
    """Y row-major (L x R, ldy >= R), or column-major (column r at Y + r*ldy,
    ldy >= L) with colmajor=True."""
    N = len(factors)
    dims = _arr(ctypes.c_int64, [int(f.shape[1]) for f in factors])   # factors given as (R, I_n) tensors
    R = int(factors[0].shape[0])
    fp = _arr(_vp, [f.data_ptr() for f in factors])
    lp = _arr(ctypes.c_int64, [int(x) for x in ldf])
    hp = _arr(_vp, [h.data_ptr() for h in hs])
    sp = _arr(_vp, [s.data_ptr() for s in ss])
    fn = lib().idl_tensorsketch_colmajor if colmajor else lib().idl_tensorsketch
    return ctx.check(fn(ctx.ptr, N, ctypes.cast(dims, _vp), R, ctypes.cast(fp, _vp), ctypes.cast(lp, _vp), _p(lam),
                        ctypes.cast(hp, _vp), ctypes.cast(sp, _vp), L, _p(Y), ldy))


def idl_gaussian_stage(ctx, Omega, m2, m1, Y1, R, ldy1, dtype, precision, Y2, ldy2):
    return ctx.check(lib().idl_gaussian_stage(ctx.ptr, _p(Omega), m2, m1, _p(Y1), R, ldy1, dtype, precision,
                                              _p(Y2), ldy2))


def idl_gaussian_stage_colmajor(ctx, Omega, m2, m1, Y1, R, ldy1, precision, Y2, ldy2):
    return ctx.check(lib().idl_gaussian_stage_colmajor(ctx.ptr, _p(Omega), m2, m1, _p(Y1), R, ldy1, precision,
                                                       _p(Y2), ldy2))


def idl_set_graphs(ctx, on=True):
    """Replay repeated pipeline calls (same arguments) as CUDA graphs."""
    return ctx.check(lib().idl_set_graphs(ctx.ptr, 1 if on else 0))


def idl_cpqr(ctx, Y2, m, R, ldy2, dtype, K, J, rnorm=None):
    return ctx.check(lib().idl_cpqr(ctx.ptr, _p(Y2), m, R, ldy2, dtype, K, _p(J), _p(rnorm)))


def idl_t_solve(ctx, Y2, m, R, ldy2, dtype, K, J, T, rest=None):
    return ctx.check(lib().idl_t_solve(ctx.ptr, _p(Y2), m, R, ldy2, dtype, K, _p(J), _p(T), _p(rest)))


def idl_lambda_hat(ctx, lam, J, T, K, R, lam_hat):
    return ctx.check(lib().idl_lambda_hat(ctx.ptr, _p(lam), _p(J), _p(T), K, R, _p(lam_hat)))


# ---------------------------------------------------------------- pipelines
def id_matrix(ctx, A, K, params, J, T, info=None, lda=None):
    """A: (I, R) torch tensor (CUDA or pinned/pageable CPU) or numpy array, float32/float64."""
    I, R = int(A.shape[0]), int(A.shape[1])
    dt = IDL_F64 if str(A.dtype).endswith("float64") else IDL_F32
    lda = R if lda is None else lda
    return ctx.check(lib().id_matrix(ctx.ptr, _p(A), I, R, lda, dt, K, ctypes.byref(params), _p(J), _p(T),
                                     ctypes.byref(info) if info is not None else None))


def id_matrix_csr(ctx, rowptr, colidx, vals, shape, K, params, J, T, info=None):
    I, R = int(shape[0]), int(shape[1])
    nnz = int(vals.shape[0])
    dt = IDL_F64 if str(vals.dtype).endswith("float64") else IDL_F32
    return ctx.check(lib().id_matrix_csr(ctx.ptr, _p(rowptr), _p(colidx), _p(vals), I, R, nnz, dt, K,
                                         ctypes.byref(params), _p(J), _p(T),
                                         ctypes.byref(info) if info is not None else None))


def id_cp_tensor(ctx, factors, lam, K, params, J, T, lam_hat, info=None, ldf=None):
    """factors: list of float32 tensors of shape (R, I_n) (A^(n) stored column by column), on the
    device or in host memory."""
    N = len(factors)
    R = int(factors[0].shape[0])
    dims = _arr(ctypes.c_int64, [int(f.shape[1]) for f in factors])
    ldf = [int(f.stride(0)) for f in factors] if ldf is None else ldf
    fp = _arr(_vp, [f.data_ptr() for f in factors])
    lp = _arr(ctypes.c_int64, ldf)
    return ctx.check(lib().id_cp_tensor(ctx.ptr, N, ctypes.cast(dims, _vp), R, ctypes.cast(fp, _vp),
                                        ctypes.cast(lp, _vp), _p(lam), K, ctypes.byref(params), _p(J), _p(T),
                                        _p(lam_hat), ctypes.byref(info) if info is not None else None))


def id_matrix_gaussian(ctx, A, K, params, J, T, info=None, lda=None):
    """Gaussian matrix ID (the comparison method): params.m2 = L."""
    I, R = int(A.shape[0]), int(A.shape[1])
    dt = IDL_F64 if str(A.dtype).endswith("float64") else IDL_F32
    lda = R if lda is None else lda
    return ctx.check(lib().id_matrix_gaussian(ctx.ptr, _p(A), I, R, lda, dt, K, ctypes.byref(params), _p(J), _p(T),
                                              ctypes.byref(info) if info is not None else None))


def id_cp_tensor_gaussian(ctx, factors, lam, K, params, J, T, lam_hat, info=None, ldf=None):
    """Gaussian (Khatri-Rao) tensor ID: factors as for id_cp_tensor, params.m2 = L."""
    N = len(factors)
    R = int(factors[0].shape[0])
    dims = _arr(ctypes.c_int64, [int(f.shape[1]) for f in factors])
    ldf = [int(f.stride(0)) for f in factors] if ldf is None else ldf
    fp = _arr(_vp, [f.data_ptr() for f in factors])
    lp = _arr(ctypes.c_int64, ldf)
    return ctx.check(lib().id_cp_tensor_gaussian(ctx.ptr, N, ctypes.cast(dims, _vp), R, ctypes.cast(fp, _vp),
                                                 ctypes.cast(lp, _vp), _p(lam), K, ctypes.byref(params), _p(J),
                                                 _p(T), _p(lam_hat), ctypes.byref(info) if info is not None else None))


def idl_id_error(ctx, A, J, T, K, iters=50, seed=1234, lda=None):
    """||A - A_J P||_2 / ||A||_2 estimated on the device (power method, Sec. 6)."""
    I, R = int(A.shape[0]), int(A.shape[1])
    dt = IDL_F64 if str(A.dtype).endswith("float64") else IDL_F32
    err = ctypes.c_double()
    ctx.check(lib().idl_id_error(ctx.ptr, _p(A), I, R, R if lda is None else lda, dt, _p(J), _p(T), K, iters, seed,
                                 ctypes.byref(err)))
    return err.value


def idl_id_error_csr(ctx, rowptr, colidx, vals, shape, J, T, K, iters=50, seed=1234):
    I, R = int(shape[0]), int(shape[1])
    dt = IDL_F64 if str(vals.dtype).endswith("float64") else IDL_F32
    err = ctypes.c_double()
    ctx.check(lib().idl_id_error_csr(ctx.ptr, _p(rowptr), _p(colidx), _p(vals), I, R, int(vals.shape[0]), dt, _p(J),
                                     _p(T), K, iters, seed, ctypes.byref(err)))
    return err.value


def _dt(x):
    return IDL_F64 if str(x.dtype).endswith("float64") else IDL_F32


def idl_sketch_rows(ctx, A_rows, i0, I, params, Y2, ldy2=None, accumulate=False, lda=None):
    """Y2 (+)= the sketch of rows i0 .. i0 + n - 1 (A_rows, n x R) of an I-row matrix."""
    n, R = int(A_rows.shape[0]), int(A_rows.shape[1])
    m = params.m2 if params.m2 > 0 else params.m1
    ctx.check(lib().idl_sketch_rows(ctx.ptr, _p(A_rows), n, R, R if lda is None else lda, _dt(A_rows), int(i0),
                                    int(I), ctypes.byref(params), _p(Y2), m if ldy2 is None else ldy2,
                                    int(bool(accumulate))))


def idl_sketch_rows_csr(ctx, rowptr, colidx, vals, n, R, i0, I, params, Y2, ldy2=None, accumulate=False):
    """The same for a CSR block of n rows (rowptr: n + 1 entries)."""
    m = params.m2 if params.m2 > 0 else params.m1
    ctx.check(lib().idl_sketch_rows_csr(ctx.ptr, _p(rowptr), _p(colidx), _p(vals), int(n), int(R),
                                        int(vals.shape[0]), _dt(vals), int(i0), int(I), ctypes.byref(params), _p(Y2),
                                        m if ldy2 is None else ldy2, int(bool(accumulate))))


def idl_id_from_sketch(ctx, Y2, m, R, K, params, J, T, info=None, ldy2=None):
    """Algorithm 1 on a complete m x R column-major sketch."""
    return ctx.check(lib().idl_id_from_sketch(ctx.ptr, _p(Y2), int(m), int(R), m if ldy2 is None else ldy2, _dt(Y2),
                                              int(K), ctypes.byref(params), _p(J), _p(T),
                                              ctypes.byref(info) if info is not None else None))


def idl_sketch_cp(ctx, factors, lam, params, Y2, ldy2=None):
    """Y2 = the m x R column-major sketch of the CP tensor's R columns given (factors:
    (R, I_n) tensors, lam: R float64), without the QR stage."""
    N = len(factors)
    R = int(factors[0].shape[0])
    dims = _arr(ctypes.c_int64, [int(f.shape[1]) for f in factors])
    fp = _arr(_vp, [f.data_ptr() for f in factors])
    lp = _arr(ctypes.c_int64, [int(f.stride(0)) for f in factors])
    m = params.m2 if params.m2 > 0 else params.m1
    return ctx.check(lib().idl_sketch_cp(ctx.ptr, N, ctypes.cast(dims, _vp), R, ctypes.cast(fp, _vp),
                                         ctypes.cast(lp, _vp), _p(lam), ctypes.byref(params), _p(Y2),
                                         m if ldy2 is None else ldy2))


# ---------------------------------------------------------------- batches
def dense_item(A, K, params, J, T, lda=None):
    """Batch item for a dense FP32 matrix A (I, R): a CUDA tensor, or a host (pinned)
    tensor with host J, T."""
    it = BatchItem()
    it.kind = IDL_ITEM_DENSE
    it.I, it.R = int(A.shape[0]), int(A.shape[1])
    it.lda = int(A.stride(0)) if lda is None else lda
    it.K = int(K)
    it.A = A.data_ptr()
    it.params = params
    it.J, it.T = J.data_ptr(), T.data_ptr()
    return it


def cp_item(factors, lam, K, params, J, T, lam_hat):
    """Batch item for a CP tensor: factors are float32 tensors (R, I_n), contiguous, on
    the device or (with every other array of the batch) in host memory."""
    it = BatchItem()
    it.kind = IDL_ITEM_CP
    it.N = len(factors)
    it.R = int(factors[0].shape[0])
    it.K = int(K)
    for n, f in enumerate(factors):
        it.dims[n] = int(f.shape[1])
        it.factors[n] = f.data_ptr()
    it.lambda_ = lam.data_ptr()
    it.params = params
    it.J, it.T, it.lambda_hat = J.data_ptr(), T.data_ptr(), lam_hat.data_ptr()
    return it


def batch_array(items):
    """A ctypes array of batch items (build it once and pass it to idl_batch_run on
    every call to save the per-call conversion)."""
    return (BatchItem * len(items))(*items)


def idl_batch_run(ctx, items):
    """items: a list of BatchItem or a batch_array.  All arrays of the batch are device
    memory, or all host memory (then the call copies them and synchronises)."""
    arr = items if isinstance(items, ctypes.Array) else batch_array(items)
    return ctx.check(lib().idl_batch_run(ctx.ptr, arr, len(arr)))


def idl_tune_save(ctx, path):
    return ctx.check(lib().idl_tune_save(ctx.ptr, str(path).encode()))


def idl_tune_load(ctx, path):
    return ctx.check(lib().idl_tune_load(ctx.ptr, str(path).encode()))


BATCH_STAGES = ("draws_buckets", "sketch_cp", "sketch_dense", "gaussian", "proposal", "cpqr", "tsolve")


def batch_stage_ms(ctx, items):
    """Milliseconds per stage group of one un-graphed, event-timed run of the batch
    (a dict keyed by BATCH_STAGES)."""
    arr = (BatchItem * len(items))(*items)
    ms = (ctypes.c_float * len(BATCH_STAGES))()
    ctx.check(lib().idl_debug_batch_timing(ctx.ptr, arr, len(items), ms))
    return {k: float(ms[i]) for i, k in enumerate(BATCH_STAGES)}


# ---------------------------------------------------------------- learned column proposal
def idl_mlp_init(ctx, seed):
    ctx.check(lib().idl_mlp_init(ctx.ptr, int(seed)))


def idl_mlp_set_weights(ctx, theta):
    """theta: IDL_MLP_NPARAM float32 values (numpy host array or CUDA tensor)."""
    ctx.check(lib().idl_mlp_set_weights(ctx.ptr, _p(theta)))


def idl_mlp_get_weights(ctx, theta):
    ctx.check(lib().idl_mlp_get_weights(ctx.ptr, _p(theta)))


def idl_save_weights(ctx, path):
    ctx.check(lib().idl_save_weights(ctx.ptr, os.fsencode(path)))


def idl_load_weights(ctx, path):
    ctx.check(lib().idl_load_weights(ctx.ptr, os.fsencode(path)))


def idl_proposal_features(ctx, Y, m, R, ldy, K, F):
    ctx.check(lib().idl_proposal_features(ctx.ptr, _p(Y), m, R, ldy, K, _p(F)))


def idl_mlp_scores(ctx, F, n, s):
    ctx.check(lib().idl_mlp_scores(ctx.ptr, _p(F), n, _p(s)))


def idl_mlp_grad(ctx, F, y, n, pos_weight, grad, loss):
    ctx.check(lib().idl_mlp_grad(ctx.ptr, _p(F), _p(y), n, float(pos_weight), _p(grad), _p(loss)))


def idl_proposal_labels(ctx, Y, m, R, ldy, K, F, y):
    ctx.check(lib().idl_proposal_labels(ctx.ptr, _p(Y), m, R, ldy, K, _p(F), _p(y)))


def idl_train_proposal(ctx, F, y, n, epochs, batch, lr, pos_weight=1.0, seed=0, beta1=0.9, beta2=0.999, eps=1e-8):
    """Returns the per-epoch mean loss (list of floats)."""
    tp = TrainParams()
    tp.epochs, tp.batch, tp.lr, tp.pos_weight, tp.seed = int(epochs), int(batch), float(lr), float(pos_weight), \
        int(seed)
    tp.beta1, tp.beta2, tp.eps = float(beta1), float(beta2), float(eps)
    out = (ctypes.c_float * int(epochs))()
    ctx.check(lib().idl_train_proposal(ctx.ptr, _p(F), _p(y), n, ctypes.byref(tp), ctypes.cast(out, _vp)))
    return list(out)


def idl_batch_fallbacks(ctx):
    """Items of the last idl_batch_run whose proposal certificate failed (synchronises)."""
    rc = lib().idl_batch_fallbacks(ctx.ptr)
    if rc < 0:
        raise IdlError(-rc, lib().idl_last_error(ctx.ptr).decode())
    return rc


def idl_cpqr_proposal(ctx, Y2, Yf, m, R, ldy2, K, mode, J, cand_factor=2, sync=True):
    """Returns 1 (certified) or 2 (rejected: the plain QR ran); None with sync=False."""
    out = ctypes.c_int(0)
    ctx.check(lib().idl_cpqr_proposal(ctx.ptr, _p(Y2), _p(Yf), m, R, ldy2, K, int(mode), int(cand_factor), _p(J),
                                      ctypes.byref(out) if sync else None))
    return out.value if sync else None
