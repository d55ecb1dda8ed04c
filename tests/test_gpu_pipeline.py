"""End-to-end GPU parity of the three pipelines (id_matrix, id_matrix_csr,
id_cp_tensor) against the FP64 oracle, at small ragged sizes and at the
workload sizes the bench runs; host-pointer calls; error codes."""
import numpy as np
import pytest
import torch

import paper_1901_10559_gb300 as idl
from oracle import countsketch as ocs
from oracle import draws as odr
from oracle import errors as oer
from oracle import idmethods as oid
from oracle.gaussian import BF16, FP32, FP64
from synth import cp_factors, gaussian_lowrank_dense, lowrank_dense, random_csr, sparse_plus_lowrank_csr
from tests.helpers import dev, host, pivots_well_separated, rel_fro

pytestmark = pytest.mark.gpu

RATIO = 1.1       # every ID's error within 1.1x the oracle's


def _outputs(K, R):
    return (torch.empty(K, dtype=torch.int32, device="cuda"),
            torch.empty(K * (R - K), dtype=torch.float64, device="cuda"))


def _check_id(J, T, Jw, Tw, info_w, err_fn, ttol):
    Jg = host(J)
    K = len(Jw)
    R = Tw.shape[1] + K
    Tg = host(T).reshape(K, R - K)
    assert len(set(Jg.tolist())) == K and Jg.min() >= 0 and Jg.max() < R
    e_w = err_fn(Jw, Tw)
    e_g = err_fn(Jg, Tg)
    if pivots_well_separated(info_w["gaps"]):
        assert np.array_equal(Jg, Jw)
        assert np.abs(Tg - Tw).max() <= ttol * max(1.0, np.abs(Tw).max())
    assert e_g <= RATIO * e_w + 1e-14, (e_g, e_w)
    return e_g, e_w


@pytest.mark.parametrize("dtype,I,R,K,m1,m2", [("f64", 4000, 2000, 20, 900, 30),     # plain FP64 workload
                                               ("f32", 3001, 517, 13, 200, 40),
                                               ("f64", 1500, 300, 10, 80, 0),        # Algorithm 2 verbatim
                                               ("f32", 1000, 64, 40, 100, 64)])
def test_id_matrix_dense(ctx, dtype, I, R, K, m1, m2):
    npdt = np.float64 if dtype == "f64" else np.float32
    A = lowrank_dense(I, R, 0.8, 1e-8, seed=20190130 + I, dtype=npdt)
    prec = idl.PREC_FP64 if dtype == "f64" else idl.PREC_FP32
    p = idl.make_params(m1, m2, seed=17, modified=True, precision=prec, residual=2)
    J, T = _outputs(K, R)
    info = idl.Info()
    idl.id_matrix(ctx, dev(A), K, p, J, T, info)
    assert info.status in (idl.IDL_OK, idl.IDL_ERANK)
    Jw, Tw, iw = oid.id_matrix(A, k=K, m1=m1, m2=m2, seed=17, modified=True,
                               precision=FP64 if dtype == "f64" else FP32)
    _check_id(J, T, Jw, Tw, iw, lambda j, t: oer.matrix_id_error(A, J=j, T=t),
              1e-7 if dtype == "f64" else 1e-2)
    # the FP64 residual check agrees with the oracle's sketch residual
    Y2 = iw["Y2"]
    Jg = host(J)
    rest = np.setdiff1d(np.arange(R), Jg)
    res_w = np.linalg.norm(Y2[:, rest] - Y2[:, Jg] @ host(T).reshape(K, R - K)) / np.linalg.norm(Y2)
    assert abs(info.residual - res_w) <= 1e-3 * max(res_w, 1e-12) + 1e-6


def test_numerically_rank_deficient_sketch_is_flagged(ctx):
    # sigma_61 / sigma_1 = 0.8**60 ~ 1.5e-6 is below 64 eps of FP32: IDL_ERANK, J still written
    A = lowrank_dense(1000, 64, 0.8, 1e-8, seed=5, dtype=np.float32)
    p = idl.make_params(100, 64, seed=17, modified=True, precision=idl.PREC_FP32)
    J, T = _outputs(60, 64)
    info = idl.Info()
    with pytest.raises(idl.IdlError) as ei:
        idl.id_matrix(ctx, dev(A), 60, p, J, T, info)
    assert ei.value.code == idl.IDL_ERANK and info.status == idl.IDL_ERANK
    Jg = host(J)
    assert len(set(Jg.tolist())) == 60 and Jg.max() < 64


def test_id_matrix_exact_rank_recovery(ctx):
    rng = np.random.default_rng(1)
    A = (rng.standard_normal((6000, 12)) @ rng.standard_normal((12, 700))).astype(np.float64)
    p = idl.make_params(120, 40, seed=3, modified=True, precision=idl.PREC_FP64)
    J, T = _outputs(12, 700)
    idl.id_matrix(ctx, dev(A), 12, p, J, T)
    err = oer.matrix_id_error(A, J=host(J), T=host(T).reshape(12, 688))
    assert err < 1e-12


@pytest.mark.parametrize("dtype,I,R,K,m1,m2,dens", [("f32", 20000, 1500, 25, 700, 35, 0.01),
                                                    ("f64", 8000, 400, 10, 150, 20, 0.03)])
def test_id_matrix_csr_small(ctx, dtype, I, R, K, m1, m2, dens):
    npdt = np.float64 if dtype == "f64" else np.float32
    c = sparse_plus_lowrank_csr(I, R, dens, rank=K, scale=10.0, dense_frac=0.01, seed=I, dtype=npdt)
    prec = idl.PREC_FP64 if dtype == "f64" else idl.PREC_FP32
    p = idl.make_params(m1, m2, seed=5, modified=True, precision=prec)
    J, T = _outputs(K, R)
    info = idl.Info()
    idl.id_matrix_csr(ctx, dev(c.rowptr), dev(c.colidx), dev(c.vals), c.shape, K, p, J, T, info)
    assert info.status == idl.IDL_OK
    csr = (c.rowptr, c.colidx, c.vals, c.shape)
    Jw, Tw, iw = oid.id_matrix(csr=csr, k=K, m1=m1, m2=m2, seed=5, modified=True,
                               precision=FP64 if dtype == "f64" else FP32)
    _check_id(J, T, Jw, Tw, iw, lambda j, t: oer.matrix_id_error(csr=csr, J=j, T=t, iters=40),
              1e-7 if dtype == "f64" else 1e-2)


@pytest.fixture(scope="module")
def cfg1():
    # sparse FP32 workload: 1e6 x 1e4, density 1e-3, rank-50 term of scale 10 on 1% of rows
    return sparse_plus_lowrank_csr(1_000_000, 10_000, 1e-3, rank=50, scale=10.0, dense_frac=0.01, seed=20190131)


def test_cfg1_sketch_full_size(ctx, cfg1):
    c = cfg1
    I, R = c.shape
    m1 = 3600
    h, s = torch.empty(I, dtype=torch.int32, device="cuda"), torch.empty(I, dtype=torch.int8, device="cuda")
    idl.idl_draw_countsketch(ctx, 20190131, I, m1, True, h, s)
    ptr = torch.empty(m1 + 1, dtype=torch.int32, device="cuda")
    rows = torch.empty(I, dtype=torch.int32, device="cuda")
    idl.idl_bucket_offsets(ctx, h, I, m1, ptr, rows)
    Y = torch.empty((m1, R), dtype=torch.float32, device="cuda")
    idl.idl_countsketch_csr(ctx, dev(c.rowptr), dev(c.colidx), dev(c.vals), I, R, c.nnz, idl.IDL_F32, h, s, ptr,
                            rows, m1, Y, R)
    hw, sw = odr.countsketch_maps(20190131, I, m1, True)
    want = ocs.countsketch_csr(c.rowptr, c.colidx, c.vals, R, hw, sw, m1)
    assert rel_fro(host(Y), want) <= 1e-5
    assert ctx.sync() == idl.IDL_OK


def test_cfg1_id_full_size(ctx, cfg1):
    c = cfg1
    I, R = c.shape
    K, m1, m2 = 50, 3600, 60
    p = idl.make_params(m1, m2, seed=20190131, modified=True, precision=idl.PREC_FP32)
    J, T = _outputs(K, R)
    info = idl.Info()
    idl.id_matrix_csr(ctx, dev(c.rowptr), dev(c.colidx), dev(c.vals), c.shape, K, p, J, T, info)
    assert info.status == idl.IDL_OK
    csr = (c.rowptr, c.colidx, c.vals, c.shape)
    Jw, Tw, iw = oid.id_matrix(csr=csr, k=K, m1=m1, m2=m2, seed=20190131, modified=True, precision=FP32)
    _check_id(J, T, Jw, Tw, iw, lambda j, t: oer.matrix_id_error(csr=csr, J=j, T=t, iters=25), 1e-2)


def test_cfg2_mixed_precision(ctx):
    # dense mixed precision, reduced rows (the full 131072-row case runs in the bench)
    I, R, K, m1, m2 = 32768, 4096, 100, 14400, 120
    A = gaussian_lowrank_dense(I, R, 100, 1e-4, seed=20190132)
    errs = {}
    for prec in (idl.PREC_FP32, idl.PREC_BF16X3, idl.PREC_BF16, idl.PREC_TF32X3):
        p = idl.make_params(m1, m2, seed=8, modified=True, precision=prec)
        J, T = _outputs(K, R)
        info = idl.Info()
        idl.id_matrix(ctx, dev(A), K, p, J, T, info)
        errs[prec] = oer.matrix_id_error(A, J=host(J), T=host(T).reshape(K, R - K), exact=False, iters=15)
    Jw, Tw, iw = oid.id_matrix(A, k=K, m1=m1, m2=m2, seed=8, modified=True, precision=FP64)
    e_or = oer.matrix_id_error(A, J=Jw, T=Tw, exact=False, iters=15)
    print(f"cfg2-shaped ID error: oracle FP64 {e_or:.3e}, FP32 {errs[idl.PREC_FP32]:.3e}, "
          f"BF16X3 {errs[idl.PREC_BF16X3]:.3e}, BF16 {errs[idl.PREC_BF16]:.3e}, TF32X3 {errs[idl.PREC_TF32X3]:.3e}")
    assert errs[idl.PREC_FP32] <= RATIO * e_or
    assert errs[idl.PREC_BF16X3] <= RATIO * e_or
    assert errs[idl.PREC_TF32X3] <= RATIO * e_or
    # plain bf16 operands (8-bit mantissa) put ~2^-9 relative noise on every sketch
    # entry, far above this matrix's 1e-4 noise floor: its error is stated, not gated
    # at 1.1x (it misses the 1e-3 level; BF16X3 is the mixed-precision mode that meets it)
    assert np.isfinite(errs[idl.PREC_BF16]) and errs[idl.PREC_BF16] < 0.2


def test_cfg2_full_size_mixed_precision(ctx):
    """The dense mixed-precision workload at full size (131072 x 4096, rank 100 plus
    1e-4 relative noise): FP32 and BF16X3 Gaussian stages against the FP64 oracle's
    ID, every error measured by the device estimate of Sec. 6 (the power method,
    parity-tested against the oracle's) on the same 2.1 GB matrix; both modes stay
    within 1.1x of the oracle's error."""
    I, R, K, m1, m2 = 131072, 4096, 100, 14400, 120
    A = gaussian_lowrank_dense(I, R, 100, 1e-4, seed=20190132)
    Ad = dev(A)
    errs = {}
    for prec in (idl.PREC_FP32, idl.PREC_BF16X3):
        p = idl.make_params(m1, m2, seed=8, modified=True, precision=prec)
        J, T = _outputs(K, R)
        idl.id_matrix(ctx, Ad, K, p, J, T)
        errs[prec] = idl.idl_id_error(ctx, Ad, J, T, K, iters=30, seed=5)
    Jw, Tw, _ = oid.id_matrix(A, k=K, m1=m1, m2=m2, seed=8, modified=True, precision=FP64)
    e_or = idl.idl_id_error(ctx, Ad, Jw.astype(np.int32), np.ascontiguousarray(Tw), K, iters=30, seed=5)
    print(f"cfg2 full size ID error: oracle FP64 {e_or:.3e}, FP32 {errs[idl.PREC_FP32]:.3e}, "
          f"BF16X3 {errs[idl.PREC_BF16X3]:.3e}")
    assert errs[idl.PREC_FP32] <= RATIO * e_or
    assert errs[idl.PREC_BF16X3] <= RATIO * e_or


@pytest.mark.parametrize("prec", [idl.PREC_FP32, idl.PREC_TF32X3])
def test_cfg3_cp_tensor(ctx, prec):
    dims, R, K, L, m2 = (1000, 1000, 1000), 1000, 50, 8192, 60
    facs, lam = cp_factors(dims, R, seed=20190133)
    fd = [dev(np.ascontiguousarray(F.T)) for F in facs]
    p = idl.make_params(L, m2, seed=9, modified=False, precision=prec)
    J, T = _outputs(K, R)
    lh = torch.empty(K, dtype=torch.float64, device="cuda")
    info = idl.Info()
    idl.id_cp_tensor(ctx, fd, dev(lam), K, p, J, T, lh, info)
    Jw, Tw, lhw, iw = oid.id_cp_tensor(facs, lam, k=K, L=L, m2=m2, seed=9, precision=FP32)
    e_w = oer.tensor_id_error(facs, lam, Jw, lhw)
    e_g = oer.tensor_id_error(facs, lam, host(J), host(lh))
    assert e_g <= RATIO * e_w
    if pivots_well_separated(iw["gaps"]):
        assert np.array_equal(host(J), Jw)
        assert np.allclose(host(lh), lhw, rtol=1e-3, atol=1e-6)
    # lambda_hat is Algorithm 3's update of the GPU's own J, T
    lh_ref = oid.lambda_hat(lam, host(J), host(T).reshape(K, R - K))
    assert np.allclose(host(lh), lh_ref, rtol=1e-12, atol=1e-14)


def test_cp_tensor_exact_rank(ctx):
    rng = np.random.default_rng(10)
    K, dims = 6, (30, 25, 20)
    base = [rng.standard_normal((d, K)) for d in dims]
    base = [F / np.linalg.norm(F, axis=0) for F in base]
    facs = [np.concatenate([F, F, F], axis=1).astype(np.float32) for F in base]     # R = 3K, M has rank K
    lam = rng.uniform(0.5, 1.5, 3 * K)
    fd = [dev(np.ascontiguousarray(F.T)) for F in facs]
    p = idl.make_params(256, 20, seed=2, modified=False, precision=idl.PREC_FP32)
    J, T = _outputs(K, 3 * K)
    lh = torch.empty(K, dtype=torch.float64, device="cuda")
    idl.id_cp_tensor(ctx, fd, dev(lam), K, p, J, T, lh)
    assert oer.tensor_id_error([F.astype(np.float64) for F in facs], lam, host(J), host(lh)) < 1e-5


def test_host_pointer_calls_match_device_calls(ctx):
    A = lowrank_dense(3000, 400, 0.85, 1e-6, seed=4, dtype=np.float32)
    K = 15
    p = idl.make_params(300, 30, seed=6, modified=True, precision=idl.PREC_FP32)
    Jd, Td = _outputs(K, 400)
    idl.id_matrix(ctx, dev(A), K, p, Jd, Td)
    Jh = np.empty(K, np.int32)
    Th = np.empty(K * (400 - K), np.float64)
    idl.id_matrix(ctx, A, K, p, Jh, Th)                       # pageable host memory
    assert np.array_equal(Jh, host(Jd)) and np.array_equal(Th, host(Td))
    Ap = torch.from_numpy(A).pin_memory()
    Jp = torch.empty(K, dtype=torch.int32).pin_memory()
    Tp = torch.empty(K * (400 - K), dtype=torch.float64).pin_memory()
    idl.id_matrix(ctx, Ap, K, p, Jp, Tp)                      # pinned host memory
    assert np.array_equal(Jp.numpy(), host(Jd)) and np.array_equal(Tp.numpy(), host(Td))
    c = random_csr(5000, 300, 0.02, seed=3)
    Jh2 = np.empty(K, np.int32)
    Th2 = np.empty(K * 285, np.float64)
    idl.id_matrix_csr(ctx, c.rowptr, c.colidx, c.vals, c.shape, K, p, Jh2, Th2)
    Jd2, Td2 = _outputs(K, 300)
    idl.id_matrix_csr(ctx, dev(c.rowptr), dev(c.colidx), dev(c.vals), c.shape, K, p, Jd2, Td2)
    # the CSR sketch adds nonzeros with shared-memory atomics: its summation order (and
    # so the last bits of T) may differ between calls; J and T agree to FP32 rounding
    assert np.array_equal(Jh2, host(Jd2))
    assert np.allclose(Th2, host(Td2), rtol=1e-4, atol=1e-6)
    # a large CSR matrix from host arrays: sketched in row chunks as their copies arrive
    cb = random_csr(200_000, 2000, 0.012, seed=5)
    assert cb.nnz >= (1 << 22)
    pb = idl.make_params(800, 40, seed=9, modified=True, precision=idl.PREC_FP32)
    Kb = 25
    Jd4, Td4 = _outputs(Kb, 2000)
    idl.id_matrix_csr(ctx, dev(cb.rowptr), dev(cb.colidx), dev(cb.vals), cb.shape, Kb, pb, Jd4, Td4)
    for pin in (False, True):
        arrs = [torch.from_numpy(a) for a in (cb.rowptr, cb.colidx, cb.vals)]
        if pin:
            arrs = [a.pin_memory() for a in arrs]
        Jh4 = np.full(Kb, -1, np.int32)
        Th4 = np.empty(Kb * (2000 - Kb), np.float64)
        idl.id_matrix_csr(ctx, *arrs, cb.shape, Kb, pb, Jh4, Th4)
        assert np.array_equal(Jh4, host(Jd4))
        assert np.allclose(Th4, host(Td4), rtol=1e-4, atol=1e-6)
    # CP tensor with host factors and s-values (pinned and pageable) and host outputs
    facs, lam = cp_factors((300, 200, 100), 120, seed=12)
    Kc = 10
    pc = idl.make_params(8192, 20, seed=3, modified=False, precision=idl.PREC_FP32)
    Jd3, Td3 = _outputs(Kc, 120)
    lhd = torch.empty(Kc, dtype=torch.float64, device="cuda")
    idl.id_cp_tensor(ctx, [dev(np.ascontiguousarray(F.T)) for F in facs], dev(lam), Kc, pc, Jd3, Td3, lhd)
    for pin in (False, True):
        fh = [torch.from_numpy(np.ascontiguousarray(F.T)) for F in facs]
        lam_h = torch.from_numpy(lam)
        if pin:
            fh, lam_h = [f.pin_memory() for f in fh], lam_h.pin_memory()
        Jh3 = np.full(Kc, -1, np.int32)
        Th3 = np.empty(Kc * (120 - Kc), np.float64)
        lhh = np.empty(Kc, np.float64)
        idl.id_cp_tensor(ctx, fh, lam_h, Kc, pc, Jh3, Th3, lhh)
        # colliding entries of a mode's CountSketch are summed by shared-memory atomics
        # (order not fixed): J equal, T and lambda_hat to FP32 rounding
        assert np.array_equal(Jh3, host(Jd3))
        assert np.allclose(Th3, host(Td3), rtol=1e-4, atol=1e-6)
        assert np.allclose(lhh, host(lhd), rtol=1e-4, atol=1e-9)


def test_argument_errors(ctx):
    A = dev(np.zeros((100, 20), np.float32))
    J, T = _outputs(5, 20)
    bad = [
        (idl.make_params(10, 5, 1, precision=idl.PREC_FP32), 6),        # K > m2
        (idl.make_params(10, 5, 1, precision=idl.PREC_FP32), 20),       # K >= R
        (idl.make_params(100, 5, 1, modified=True, precision=idl.PREC_FP32), 5),   # modified needs m1 < I
        (idl.make_params(10, 12, 1, precision=idl.PREC_FP32), 5),       # m2 > m1
        (idl.make_params(10, 5, 1, precision=idl.PREC_FP64), 5),        # FP64 precision with FP32 data
    ]
    for p, K in bad:
        with pytest.raises(idl.IdlError) as ei:
            idl.id_matrix(ctx, A, K, p, J, T)
        assert ei.value.code == idl.IDL_EINVAL
    with pytest.raises(idl.IdlError) as ei:
        idl.id_matrix(ctx, A, 5, idl.make_params(300, 299, 1, modified=False, precision=idl.PREC_FP32), J, T)
    assert ei.value.code == idl.IDL_ELIMIT                              # m2 > 256 (QR stage capacity)


def test_injected_allocation_failure_is_reported(ctx):
    lib = idl.lib()
    lib.idl_debug_release_workspace(ctx.ptr)
    lib.idl_debug_fail_alloc(ctx.ptr, 1)
    A = dev(np.random.default_rng(0).standard_normal((500, 50)).astype(np.float32))
    J, T = _outputs(5, 50)
    with pytest.raises(idl.IdlError) as ei:
        idl.id_matrix(ctx, A, 5, idl.make_params(40, 10, 1, precision=idl.PREC_FP32), J, T)
    assert ei.value.code == idl.IDL_ENOMEM
    lib.idl_debug_fail_alloc(ctx.ptr, 0)
    idl.id_matrix(ctx, A, 5, idl.make_params(40, 10, 1, precision=idl.PREC_FP32), J, T)   # recovers
    assert ctx.sync() == idl.IDL_OK


# ------------------------------------------------------------------ CUDA-graph replay
def test_graph_replay_matches_eager(ctx):
    """idl_set_graphs: the first call runs eagerly, the second is captured, later
    ones replay; every call reads the buffers' current contents (A is changed
    in place between calls, by powers of two), runs as many kernels as an eager
    call, and gives the eager call's J and T.  A call with other
    arguments in between (which regrows the workspace) invalidates the graph."""
    K, I, R, m1, m2 = 12, 3000, 400, 200, 30
    rng = np.random.default_rng(11)
    A0 = lowrank_dense(I, R, 0.7, 1e-9, seed=21).astype(np.float32)
    A = dev(A0)
    p = idl.make_params(m1, m2, seed=4, modified=True, precision=idl.PREC_FP32)
    J0, T0 = _outputs(K, R)
    idl.id_matrix(ctx, A, K, p, J0, T0)                     # eager reference
    Je, Te = host(J0).copy(), host(T0).copy()
    n_eager = None
    try:
        idl.idl_set_graphs(ctx, True)
        J, T = _outputs(K, R)
        for call in range(4):
            if call == 2:   # another problem that needs a larger workspace: the graph goes stale
                Ab = dev(lowrank_dense(2 * I, 2 * R, 0.7, 1e-9, seed=22).astype(np.float32))
                Jb, Tb = _outputs(K, 2 * R)
                idl.id_matrix(ctx, Ab, K, idl.make_params(2 * m1, m2, seed=5), Jb, Tb)
            scale = float(2.0 ** rng.integers(-3, 4))         # exact in FP32: J and T unchanged
            A.copy_(dev(A0 * np.float32(scale)))
            before = idl.lib().idl_launch_count()
            idl.id_matrix(ctx, A, K, p, J, T)
            torch.cuda.synchronize()
            n = idl.lib().idl_launch_count() - before
            if n_eager is None:
                n_eager = n
            assert n == n_eager, (call, n, n_eager)
            assert np.array_equal(host(J), Je), call          # J is scale invariant
            assert np.allclose(host(T), Te, rtol=1e-4, atol=1e-6), call
        assert ctx.sync() == idl.IDL_OK
    finally:
        idl.idl_set_graphs(ctx, False)


def test_graph_replay_cp_and_csr(ctx):
    """The CSR and CP pipelines replayed as graphs give the eager results."""
    K = 10
    c = random_csr(4000, 300, 0.02, seed=3)
    vals = (c.vals * (1.0 + 4.0 * c.colidx / 300.0)).astype(np.float32)   # column norms well apart
    p = idl.make_params(150, 25, seed=6, modified=True, precision=idl.PREC_FP32)
    rp, ci, vv = dev(c.rowptr), dev(c.colidx), dev(vals)
    dims, R = (60, 50, 40), 120
    facs, lam = cp_factors(dims, R, seed=8)
    fd = [dev(np.ascontiguousarray(F.T)) for F in facs]
    dl = dev(lam)
    pc = idl.make_params(1024, 25, seed=7, modified=False, precision=idl.PREC_FP32)
    outs = {}
    for graphs in (False, True):
        idl.idl_set_graphs(ctx, graphs)
        try:
            for rep in range(3):
                J, T = _outputs(K, 300)
                idl.id_matrix_csr(ctx, rp, ci, vv, c.shape, K, p, J, T)
                Jc, Tc = _outputs(K, R)
                lh = torch.empty(K, dtype=torch.float64, device="cuda")
                idl.id_cp_tensor(ctx, fd, dl, K, pc, Jc, Tc, lh)
                outs[(graphs, rep)] = (host(J), host(T), host(Jc), host(Tc), host(lh))
        finally:
            idl.idl_set_graphs(ctx, False)
    ref = outs[(False, 0)]
    for key, o in outs.items():
        assert np.array_equal(o[0], ref[0]) and np.array_equal(o[2], ref[2]), key
        for a, b in ((o[1], ref[1]), (o[3], ref[3]), (o[4], ref[4])):
            assert np.allclose(a, b, rtol=1e-4, atol=1e-6), key
    assert ctx.sync() == idl.IDL_OK


@pytest.mark.parametrize("kind", ["dense", "csr"])
def test_row_blocks_sum_to_the_whole_sketch(ctx, kind):
    """Sec. 1.3: the sketch is linear in the rows.  Three row blocks sketched with the
    whole matrix's maps and added (idl_sketch_rows*) give the oracle's sketch of the
    whole matrix, and idl_id_from_sketch on the sum gives the pipeline's J and T."""
    from paper_1901_10559_gb300 import sharded
    I, R, K, m1, m2 = 20000, 500, 15, 400, 40
    p = idl.make_params(m1, m2, seed=21, modified=True, precision=idl.PREC_FP32)
    Y2 = torch.zeros(m2 * R, dtype=torch.float32, device="cuda")
    J1, T1 = _outputs(K, R)
    if kind == "dense":
        A = lowrank_dense(I, R, 0.85, 1e-6, seed=9, dtype=np.float32)
        for b, (i0, i1) in enumerate(sharded.row_blocks(I, 3)):
            idl.idl_sketch_rows(ctx, dev(A[i0:i1]), i0, I, p, Y2, accumulate=b > 0)
        idl.id_matrix(ctx, dev(A), K, p, J1, T1)
        _, _, iw = oid.id_matrix(A, k=K, m1=m1, m2=m2, seed=21, modified=True, precision=FP32)
    else:
        c = sparse_plus_lowrank_csr(I, R, 0.02, rank=10, scale=5.0, dense_frac=0.02, seed=4)
        for b, (i0, i1) in enumerate(sharded.row_blocks(I, 3)):
            rp, ci, v = sharded.csr_row_block(c.rowptr, c.colidx, c.vals, i0, i1)
            idl.idl_sketch_rows_csr(ctx, dev(rp), dev(ci), dev(v), i1 - i0, R, i0, I, p, Y2, accumulate=b > 0)
        idl.id_matrix_csr(ctx, dev(c.rowptr), dev(c.colidx), dev(c.vals), c.shape, K, p, J1, T1)
        _, _, iw = oid.id_matrix(csr=(c.rowptr, c.colidx, c.vals, c.shape), k=K, m1=m1, m2=m2, seed=21,
                                 modified=True, precision=FP32)
    got = host(Y2).reshape(R, m2).T
    assert rel_fro(got, iw["Y2"]) <= 1e-5
    J2, T2 = _outputs(K, R)
    idl.idl_id_from_sketch(ctx, Y2, m2, R, K, p, J2, T2)
    assert np.array_equal(host(J2), host(J1))
    assert np.allclose(host(T2), host(T1), rtol=1e-3, atol=1e-6)
    assert ctx.sync() == idl.IDL_OK


@pytest.mark.parametrize("L,m2", [(8192, 40), (1024, 40), (256, 0)])
def test_cp_column_blocks_gather_to_the_whole_sketch(ctx, L, m2):
    """Column r of a CP tensor's sketch depends on column r of the factors and the
    modes' maps only (Sec. 1.3, Eq. TA-formula): column blocks sketched apart by
    idl_sketch_cp and placed side by side equal the oracle's sketch of the whole
    tensor, and Algorithm 1 + the s-value update on the gathered sketch give
    id_cp_tensor's J and lambda_hat."""
    from paper_1901_10559_gb300 import sharded
    dims, R, K = (70, 50, 40), 333, 12
    facs, lam = cp_factors(dims, R, seed=31)
    p = idl.make_params(L, m2, seed=17, modified=False, precision=idl.PREC_FP32)
    m = m2 if m2 > 0 else L
    Y2 = torch.full((m * R,), float("nan"), dtype=torch.float32, device="cuda")
    for c0, c1 in sharded.column_blocks(R, 3):
        fd = [dev(np.ascontiguousarray(F[:, c0:c1].T)) for F in facs]
        idl.idl_sketch_cp(ctx, fd, dev(lam[c0:c1]), p, Y2[c0 * m:c1 * m])
    Jw, Tw, lhw, iw = oid.id_cp_tensor(facs, lam, k=K, L=L, m2=m2, seed=17, precision=FP32)
    got = host(Y2).reshape(R, m).T
    assert rel_fro(got, iw["Y2"]) <= 1e-5
    J1, T1 = _outputs(K, R)
    lh1 = torch.empty(K, dtype=torch.float64, device="cuda")
    idl.id_cp_tensor(ctx, [dev(np.ascontiguousarray(F.T)) for F in facs], dev(lam), K, p, J1, T1, lh1)
    J2, T2 = _outputs(K, R)
    lh2 = torch.empty(K, dtype=torch.float64, device="cuda")
    idl.idl_id_from_sketch(ctx, Y2, m, R, K, p, J2, T2)
    idl.idl_lambda_hat(ctx, dev(lam), J2, T2, K, R, lh2)
    if pivots_well_separated(iw["gaps"]):
        assert np.array_equal(host(J2), Jw) and np.array_equal(host(J1), Jw)
        assert np.allclose(host(lh2), host(lh1), rtol=1e-3, atol=1e-6)
    e_w = oer.tensor_id_error(facs, lam, Jw, lhw)
    assert oer.tensor_id_error(facs, lam, host(J2), host(lh2)) <= RATIO * e_w
    assert ctx.sync() == idl.IDL_OK


def test_sketch_cp_argument_errors(ctx):
    facs, lam = cp_factors((20, 20), 30, seed=1)
    fd = [dev(np.ascontiguousarray(F.T)) for F in facs]
    Y2 = torch.empty(40 * 30, dtype=torch.float32, device="cuda")
    for kw, code in [(dict(m1=100, m2=20), idl.IDL_EINVAL),                        # L not a power of two
                     (dict(m1=256, m2=20, precision=idl.PREC_FP64), idl.IDL_EINVAL)]:
        p = idl.make_params(kw["m1"], kw["m2"], seed=1, modified=False, precision=kw.get("precision", idl.PREC_FP32))
        with pytest.raises(idl.IdlError) as e:
            idl.idl_sketch_cp(ctx, fd, dev(lam), p, Y2)
        assert e.value.code == code
    p = idl.make_params(256, 20, seed=1, modified=False, precision=idl.PREC_FP32)
    with pytest.raises(idl.IdlError) as e:
        idl.idl_sketch_cp(ctx, fd, dev(lam), p, torch.empty(20 * 30, dtype=torch.float32))   # host Y2
    assert e.value.code == idl.IDL_EINVAL
    assert ctx.sync() == idl.IDL_OK
