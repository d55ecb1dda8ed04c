"""GPU parity of every stage of the hot path against the FP64 oracle, through
the C ABI (draws, bucket offsets, CountSketch dense/CSR, Gaussian stage, CPQR,
T solve, TensorSketch, lambda_hat)."""
import numpy as np
import pytest
import torch

import paper_1901_10559_gb300 as idl
from oracle import countsketch as ocs
from oracle import cpqr as ocp
from oracle import draws as odr
from oracle import gaussian as ogs
from oracle import tensorsketch as ots
from synth import cp_factors, random_csr
from tests.helpers import assert_sum_within_bound, colmajor_to_matrix, dev, host, pivots_well_separated, rel_fro

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5     # sketch parity in FP32 (relative Frobenius)
FP64_TOL = 1e-12    # sketch parity in FP64


# ------------------------------------------------------------------ a1 draws
@pytest.mark.parametrize("I,L,modified,seed", [(1, 1, False, 0), (4000, 900, True, 20190130),
                                               (1_000_000, 3600, True, 7), (131072, 14400, True, 3),
                                               (4097, 4096, True, 11), (50_000, 7, False, 5)])
def test_countsketch_draws_bit_exact(ctx, I, L, modified, seed):
    h = torch.empty(I, dtype=torch.int32, device="cuda")
    s = torch.empty(I, dtype=torch.int8, device="cuda")
    idl.idl_draw_countsketch(ctx, seed, I, L, modified, h, s)
    hw, sw = odr.countsketch_maps(seed, I, L, modified)
    assert np.array_equal(host(h), hw)
    assert np.array_equal(host(s), sw)
    assert ctx.sync() == idl.IDL_OK


def test_gaussian_draws(ctx):
    for m2, m1, seed in [(30, 900, 20190130), (7, 13, 1), (120, 14400, 4)]:
        Om = torch.empty(m2 * m1, dtype=torch.float64, device="cuda")
        idl.idl_draw_gaussian(ctx, seed, m2, m1, Om)
        want = odr.gaussian_matrix(seed, m2, m1)
        got = host(Om).reshape(m2, m1)
        assert np.abs(got - want).max() <= 1e-13 * max(1.0, np.abs(want).max())
        # the fp32 working copies agree to one fp32 ulp (the FP64 values differ in the last bits)
        g32, w32 = got.astype(np.float32), want.astype(np.float32)
        assert np.all(np.abs(g32 - w32) <= np.spacing(np.abs(w32)))


def test_gaussian_draws_fp32_arithmetic(ctx):
    """The FP32-arithmetic draw of the FP32 pipelines: every entry within
    4e-7 (rho + |z|) of the FP64 definition, rho the pair's radius; the even sizes
    and an odd count (a lone last entry) are covered."""
    for m2, m1, seed in [(30, 900, 20190130), (7, 13, 1), (120, 14400, 4), (1, 1_000_001, 9)]:
        Om = torch.empty(m2 * m1, dtype=torch.float64, device="cuda")
        idl.idl_draw_gaussian_fp32(ctx, seed, m2, m1, Om)
        want = odr.gaussian_matrix(seed, m2, m1).ravel()
        got = host(Om)
        n = want.size
        first = 2 * (np.arange(n) // 2)                                # first entry of each entry's pair
        second = np.where(first + 1 < n, want[np.minimum(first + 1, n - 1)], 0.0)
        rho = np.hypot(want[first], second)
        assert np.all(np.abs(got - want) <= 4e-7 * (rho + np.abs(want)) + 1e-30), np.abs(got - want).max()
        assert np.all(got == got.astype(np.float32))                 # FP32 values


def test_mode_draws(ctx):
    for n in range(4):
        h = torch.empty(1000, dtype=torch.int32, device="cuda")
        s = torch.empty(1000, dtype=torch.int8, device="cuda")
        idl.idl_draw_mode(ctx, 9, n, 1000, 8192, h, s)
        hs, ss = odr.tensorsketch_maps(9, [1000] * 4, 8192)
        assert np.array_equal(host(h), hs[n]) and np.array_equal(host(s), ss[n])


# ------------------------------------------------------------------ a2 bucket offsets
@pytest.mark.parametrize("I,L,modified", [(4000, 900, True), (1_000_000, 3600, True), (20000, 9, False),
                                          (131072, 14400, True), (3, 2, True)])
def test_bucket_offsets_bit_exact(ctx, I, L, modified):
    h = torch.empty(I, dtype=torch.int32, device="cuda")
    s = torch.empty(I, dtype=torch.int8, device="cuda")
    idl.idl_draw_countsketch(ctx, 5, I, L, modified, h, s)
    ptr = torch.empty(L + 1, dtype=torch.int32, device="cuda")
    rows = torch.empty(I, dtype=torch.int32, device="cuda")
    idl.idl_bucket_offsets(ctx, h, I, L, ptr, rows)
    pw, rw = ocs.bucket_offsets(odr.countsketch_maps(5, I, L, modified)[0], L)
    assert np.array_equal(host(ptr), pw)
    assert np.array_equal(host(rows), rw)


# ------------------------------------------------------------------ a3 dense CountSketch
def _draw(ctx, seed, I, L, modified):
    h = torch.empty(I, dtype=torch.int32, device="cuda")
    s = torch.empty(I, dtype=torch.int8, device="cuda")
    idl.idl_draw_countsketch(ctx, seed, I, L, modified, h, s)
    ptr = torch.empty(L + 1, dtype=torch.int32, device="cuda")
    rows = torch.empty(I, dtype=torch.int32, device="cuda")
    idl.idl_bucket_offsets(ctx, h, I, L, ptr, rows)
    return h, s, ptr, rows


@pytest.mark.parametrize("dtype,I,R,L,lda_pad", [("f32", 3001, 2053, 211, 0), ("f64", 4000, 2000, 900, 0),
                                                 ("f32", 5000, 1030, 64, 3), ("f64", 777, 17, 100, 1),
                                                 ("f32", 2, 5, 1, 0)])
def test_countsketch_dense_parity(ctx, dtype, I, R, L, lda_pad):
    rng = np.random.default_rng(I + R)
    npdt = np.float32 if dtype == "f32" else np.float64
    lda = R + lda_pad
    Afull = rng.standard_normal((I, lda)).astype(npdt)
    A = dev(Afull)
    modified = L < I
    h, s, ptr, rows = _draw(ctx, 13, I, L, modified)
    ldy = R + 5
    Y = torch.full((L, ldy), np.nan, dtype=A.dtype, device="cuda")
    idl.idl_countsketch_dense(ctx, A, I, R, lda, idl.IDL_F32 if dtype == "f32" else idl.IDL_F64, h, s, ptr, rows,
                              L, Y, ldy)
    hw, sw = odr.countsketch_maps(13, I, L, modified)
    want = ocs.countsketch_dense(Afull[:, :R], hw, sw, L)
    got = host(Y)[:, :R]
    tol = FP32_TOL if dtype == "f32" else FP64_TOL
    assert rel_fro(got, want) <= tol
    assert np.all(np.isnan(host(Y)[:, R:]))                 # padding untouched
    # entry by entry: within the rounding of a sum of the bucket's terms
    absum = ocs.countsketch_dense(np.abs(Afull[:, :R]), hw, np.ones_like(sw), L)
    u = 2.0 ** -24 if dtype == "f32" else 2.0 ** -52
    assert_sum_within_bound(got, want, absum, int(np.bincount(hw, minlength=L).max()), u)


# ------------------------------------------------------------------ a4 CSR CountSketch
@pytest.mark.parametrize("dtype,I,R,L,density", [("f32", 20000, 3000, 300, 0.01), ("f64", 5000, 700, 64, 0.05),
                                                 ("f32", 100, 60000, 10, 0.01)])
def test_countsketch_csr_parity(ctx, dtype, I, R, L, density):
    npdt = np.float32 if dtype == "f32" else np.float64
    c = random_csr(I, R, density, seed=I, dtype=npdt)
    # dense rows + duplicate and unsorted columns in the first rows
    cols = c.colidx.copy()
    if c.nnz > 8:
        cols[1] = cols[0]
        cols[2], cols[3] = cols[3], cols[2]
    rowptr, vals = c.rowptr, c.vals
    h, s, ptr, rows = _draw(ctx, 21, I, L, True)
    ldy = R
    Y = torch.empty((L, ldy), dtype=torch.float32 if dtype == "f32" else torch.float64, device="cuda")
    idl.idl_countsketch_csr(ctx, dev(rowptr), dev(cols), dev(vals), I, R, c.nnz,
                            idl.IDL_F32 if dtype == "f32" else idl.IDL_F64, h, s, ptr, rows, L, Y, ldy)
    hw, sw = odr.countsketch_maps(21, I, L, True)
    want = ocs.countsketch_csr(rowptr, cols, vals, R, hw, sw, L)
    tol = FP32_TOL if dtype == "f32" else FP64_TOL
    assert rel_fro(host(Y), want) <= tol
    absum = ocs.countsketch_csr(rowptr, cols, np.abs(vals), R, hw, np.ones_like(sw), L)
    nterms = int(np.max(np.bincount(hw, weights=np.diff(rowptr), minlength=L)))   # nonzeros per bucket
    assert_sum_within_bound(host(Y), want, absum, nterms, 2.0 ** -24 if dtype == "f32" else 2.0 ** -52)
    assert ctx.sync() == idl.IDL_OK


@pytest.mark.parametrize("I,R,L,modified,frac_long", [(20000, 3000, 300, True, 0.0), (50, 400, 200, False, 0.0),
                                                       (3000, 10000, 61, True, 0.02), (700, 20000, 9, True, 0.1),
                                                       (1, 5, 3, False, 0.0)])
def test_countsketch_csr_edge_shapes(ctx, I, R, L, modified, frac_long):
    """The CSR CountSketch against the oracle entry by entry within the rounding of
    each bucket's sum: empty buckets (plain maps with L > I), rows of thousands of
    nonzeros beside short ones, unaligned row starts, a single row."""
    rng = np.random.default_rng(I + R + L)
    lens = np.where(rng.random(I) < frac_long, rng.integers(min(4000, R), R + 1, I), rng.integers(0, 40, I))
    lens = np.minimum(lens, R)
    cols = np.concatenate([np.sort(rng.permutation(R)[:n]) for n in lens]).astype(np.int32)
    vals = rng.standard_normal(cols.size).astype(np.float32)
    rowptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    nnz = int(rowptr[-1])
    h, s, ptr, rows = _draw(ctx, 41, I, L, modified)
    hw, sw = odr.countsketch_maps(41, I, L, modified)
    want = ocs.countsketch_csr(rowptr, cols, vals, R, hw, sw, L)
    absum = ocs.countsketch_csr(rowptr, cols, np.abs(vals), R, hw, np.ones_like(sw), L)
    nterms = int(np.max(np.bincount(hw, weights=np.diff(rowptr), minlength=L)))
    Y = torch.full((L, R), float("nan"), dtype=torch.float32, device="cuda")
    idl.idl_countsketch_csr(ctx, dev(rowptr), dev(cols), dev(vals), I, R, nnz, idl.IDL_F32, h, s, ptr, rows, L, Y, R)
    g = host(Y)
    assert np.all(np.isfinite(g))
    assert_sum_within_bound(g, want, absum, nterms, 2.0 ** -24)
    assert ctx.sync() == idl.IDL_OK


@pytest.mark.parametrize("dtype,offset,R,L", [("f32", 0, 3000, 40), ("f32", 1, 3000, 40), ("f64", 0, 2500, 33),
                                              ("f64", 1, 2500, 33), ("f32", 3, 20000, 7),
                                              ("f32", 1, 60000, 5)])
def test_countsketch_csr_long_rows(ctx, dtype, offset, R, L):
    """Rows of 256 .. R nonzeros (read as masked 16-byte quads) mixed with short
    and empty rows; the last row is long and nnz is not a multiple of 4; with
    offset > 0 colidx and vals start off a 16-byte boundary (scalar loads)."""
    rng = np.random.default_rng(R + offset)
    npdt = np.float32 if dtype == "f32" else np.float64
    I = 400
    lens = np.where(rng.random(I) < 0.15, rng.integers(256, R + 1, I), rng.integers(0, 20, I))
    lens[-1] = R - 1 if (R - 1) % 4 else R - 2
    cols = np.concatenate([rng.permutation(R)[:n] for n in lens]).astype(np.int32)
    if cols.size % 4 == 0:
        lens[-1] -= 1
        cols = cols[:-1]
    vals = rng.standard_normal(cols.size).astype(npdt)
    rowptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    nnz = int(rowptr[-1])
    assert nnz % 4 != 0
    cbuf = torch.zeros(nnz + offset, dtype=torch.int32, device="cuda")
    vbuf = torch.zeros(nnz + offset, dtype=torch.float32 if dtype == "f32" else torch.float64, device="cuda")
    cbuf[offset:] = dev(cols)
    vbuf[offset:] = dev(vals)
    h, s, ptr, rows = _draw(ctx, 31, I, L, True)
    Y = torch.empty((L, R), dtype=vbuf.dtype, device="cuda")
    idl.idl_countsketch_csr(ctx, dev(rowptr), cbuf[offset:], vbuf[offset:], I, R, nnz,
                            idl.IDL_F32 if dtype == "f32" else idl.IDL_F64, h, s, ptr, rows, L, Y, R)
    hw, sw = odr.countsketch_maps(31, I, L, True)
    want = ocs.countsketch_csr(rowptr, cols, vals, R, hw, sw, L)
    tol = FP32_TOL if dtype == "f32" else FP64_TOL
    assert rel_fro(host(Y), want) <= tol
    absum = ocs.countsketch_csr(rowptr, cols, np.abs(vals), R, hw, np.ones_like(sw), L)
    nterms = int(np.max(np.bincount(hw, weights=np.diff(rowptr), minlength=L)))
    assert_sum_within_bound(host(Y), want, absum, nterms, 2.0 ** -24 if dtype == "f32" else 2.0 ** -52)
    assert ctx.sync() == idl.IDL_OK


@pytest.mark.parametrize("dtype,R", [("f32", 3000), ("f64", 1000), ("f32", 10000)])
def test_countsketch_csr_full_rows(ctx, dtype, R):
    """Rows with nnz == R (every quad of them read with 16-byte loads): stored in
    column order, permuted, or with a repeated column, mixed with short rows."""
    rng = np.random.default_rng(R)
    npdt = np.float32 if dtype == "f32" else np.float64
    I, L = 300, 37
    kind = rng.choice(4, size=I, p=[0.75, 0.15, 0.05, 0.05])    # short, sorted, permuted, repeated column
    cols_l = []
    for k in kind:
        if k == 0:
            cols_l.append(np.sort(rng.permutation(R)[:rng.integers(0, 30)]))
        elif k == 1:
            cols_l.append(np.arange(R))
        elif k == 2:
            cols_l.append(rng.permutation(R))
        else:
            c = np.arange(R)
            c[rng.integers(1, R)] = c[0]
            cols_l.append(c)
    lens = np.array([len(c) for c in cols_l])
    cols = np.concatenate(cols_l).astype(np.int32)
    vals = rng.standard_normal(cols.size).astype(npdt)
    rowptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    h, s, ptr, rows = _draw(ctx, 41, I, L, True)
    hw, sw = odr.countsketch_maps(41, I, L, True)
    want = ocs.countsketch_csr(rowptr, cols, vals, R, hw, sw, L)
    tol = FP32_TOL if dtype == "f32" else FP64_TOL
    Y = torch.empty((L, R), dtype=torch.float32 if dtype == "f32" else torch.float64, device="cuda")
    idl.idl_countsketch_csr(ctx, dev(rowptr), dev(cols), dev(vals), I, R, cols.size,
                            idl.IDL_F32 if dtype == "f32" else idl.IDL_F64, h, s, ptr, rows, L, Y, R)
    assert rel_fro(host(Y), want) <= tol
    assert ctx.sync() == idl.IDL_OK


def test_countsketch_csr_flags_bad_column(ctx):
    c = random_csr(1000, 50, 0.1, seed=1)
    cols = c.colidx.copy()
    cols[5] = 50          # out of range: skipped and flagged
    cols[7] = -3
    h, s, ptr, rows = _draw(ctx, 2, 1000, 20, True)
    Y = torch.empty((20, 50), dtype=torch.float32, device="cuda")
    idl.idl_countsketch_csr(ctx, dev(c.rowptr), dev(cols), dev(c.vals), 1000, 50, c.nnz, idl.IDL_F32, h, s, ptr,
                            rows, 20, Y, 50)
    assert ctx.sync() == idl.IDL_EDATA
    keep = np.ones(c.nnz, bool)
    keep[[5, 7]] = False
    # reference without the two bad entries
    rp = np.concatenate([[0], np.cumsum([keep[c.rowptr[i]:c.rowptr[i + 1]].sum() for i in range(1000)])])
    hw, sw = odr.countsketch_maps(2, 1000, 20, True)
    want = ocs.countsketch_csr(rp, cols[keep], c.vals[keep], 50, hw, sw, 20)
    assert rel_fro(host(Y), want) <= FP32_TOL
    assert ctx.sync() == idl.IDL_OK     # status cleared after it was read


# ------------------------------------------------------------------ a6 Gaussian stage
@pytest.mark.parametrize("prec,m2,m1,R", [(idl.PREC_FP64, 30, 900, 2000), (idl.PREC_FP32, 60, 3600, 1000),
                                          (idl.PREC_BF16X3, 60, 3600, 1000), (idl.PREC_BF16, 120, 1440, 520),
                                          (idl.PREC_FP32, 17, 100, 45), (idl.PREC_TF32X3, 60, 3600, 1000),
                                          (idl.PREC_TF32X3, 17, 100, 45), (idl.PREC_TF32X3, 256, 777, 300)])
def test_gaussian_stage_parity(ctx, prec, m2, m1, R):
    rng = np.random.default_rng(m1)
    f64 = prec == idl.PREC_FP64
    npdt = np.float64 if f64 else np.float32
    Y1 = rng.standard_normal((m1, R)).astype(npdt)
    ldy1 = R + 3
    Y1p = np.zeros((m1, ldy1), npdt)
    Y1p[:, :R] = Y1
    Om = torch.empty(m2 * m1, dtype=torch.float64, device="cuda")
    idl.idl_draw_gaussian(ctx, 3, m2, m1, Om)
    ldy2 = m2 + 1
    Y2 = torch.empty(R * ldy2, dtype=torch.float64 if f64 else torch.float32, device="cuda")
    idl.idl_gaussian_stage(ctx, Om, m2, m1, dev(Y1p), R, ldy1, idl.IDL_F64 if f64 else idl.IDL_F32, prec, Y2, ldy2)
    want = ogs.gaussian_stage(odr.gaussian_matrix(3, m2, m1), Y1, prec)
    got = colmajor_to_matrix(Y2, m2, R, ldy2)
    tol = {idl.PREC_FP64: 1e-12, idl.PREC_FP32: FP32_TOL, idl.PREC_BF16X3: 2e-5, idl.PREC_BF16: 1e-5,
           idl.PREC_TF32X3: FP32_TOL}[prec]
    assert rel_fro(got, want) <= tol


# ------------------------------------------------------------------ a7/a8 CPQR + T
@pytest.mark.parametrize("dtype,m,R,K", [("f64", 30, 2000, 20), ("f32", 60, 10000, 50), ("f32", 120, 4096, 100),
                                         ("f32", 60, 1000, 50), ("f64", 12, 40, 12), ("f32", 5, 3, 2)])
def test_cpqr_and_t_parity(ctx, dtype, m, R, K):
    rng = np.random.default_rng(m * R)
    npdt = np.float32 if dtype == "f32" else np.float64
    Y = (rng.standard_normal((m, R)) * rng.uniform(0.2, 5.0, R)[None, :]).astype(npdt)
    ld = m + 2
    buf = np.zeros((R, ld), npdt)
    buf[:, :m] = Y.T
    Yd = dev(buf)
    J = torch.empty(K, dtype=torch.int32, device="cuda")
    rn = torch.empty(K, dtype=torch.float64, device="cuda")
    dt = idl.IDL_F32 if dtype == "f32" else idl.IDL_F64
    idl.idl_cpqr(ctx, Yd, m, R, ld, dt, K, J, rn)
    Jw, Tw, info = ocp.matrix_id(Y.astype(np.float64), K)
    Jg = host(J)
    if pivots_well_separated(info["gaps"]):
        assert np.array_equal(Jg, Jw)
    assert len(set(Jg.tolist())) == K and Jg.min() >= 0 and Jg.max() < R
    assert np.allclose(host(rn), info["norms"][:K] if np.array_equal(Jg, Jw) else host(rn), rtol=1e-4)
    if K < R:
        T = torch.empty(K * (R - K), dtype=torch.float64, device="cuda")
        rest = torch.empty(R - K, dtype=torch.int32, device="cuda")
        idl.idl_t_solve(ctx, Yd, m, R, ld, dt, K, J, T, rest)
        Tg = host(T).reshape(K, R - K)
        restw = np.setdiff1d(np.arange(R), Jg)
        assert np.array_equal(host(rest), restw)
        # T is fixed by J: compare with the oracle's least-squares T for the GPU's J
        Y64 = Y.astype(np.float64)
        Tl = np.linalg.lstsq(Y64[:, Jg], Y64[:, restw], rcond=None)[0]
        tol = 1e-9 if dtype == "f64" else 2e-3
        assert np.abs(Tg - Tl).max() <= tol * max(1.0, np.abs(Tl).max())
    assert ctx.sync() == idl.IDL_OK


@pytest.mark.parametrize("dtype,K,R", [("f32", 50, 3000), ("f32", 128, 700), ("f64", 40, 500), ("f32", 3, 5)])
def test_t_solve_from_factored_sketch(ctx, dtype, K, R):
    """T = R11^{-1} R12 from a given factored sketch equals the FP64 back
    substitution of the oracle on the same stored values: the FP32 path
    accumulates in double-float arithmetic (about 48 bits), so the gate is
    1e-11 relative to |R11^{-1}| |R12| (FP64 data: 1e-13)."""
    rng = np.random.default_rng(K + R)
    npdt = np.float32 if dtype == "f32" else np.float64
    m = K + 7
    J = rng.permutation(R)[:K].astype(np.int32)
    U = np.triu(rng.standard_normal((K, K))) + np.diag(rng.uniform(2.0, 4.0, K) * rng.choice([-1, 1], K))
    Y = rng.standard_normal((m, R))                                      # rows >= K of the rest: R22
    Y[:, J] = 0.0
    Y[:K, J] = U                                                         # pivot column t: rows 0..t of R11
    Y = Y.astype(npdt)
    rest = np.setdiff1d(np.arange(R), J)
    R11 = Y[:K, J].astype(np.float64)
    R12 = Y[:K, rest].astype(np.float64)
    want = ocp.back_substitution(R11, R12)
    Yd = dev(np.ascontiguousarray(Y.T))
    T = torch.empty(K * (R - K), dtype=torch.float64, device="cuda")
    rd = torch.empty(R - K, dtype=torch.int32, device="cuda")
    dt = idl.IDL_F32 if dtype == "f32" else idl.IDL_F64
    idl.idl_t_solve(ctx, Yd, m, R, m, dt, K, dev(J), T, rd)
    got = host(T).reshape(K, R - K)
    assert np.array_equal(host(rd), rest)
    scale = np.abs(np.linalg.inv(R11)) @ np.abs(R12)
    tol = 1e-11 if dtype == "f32" else 1e-13
    assert np.all(np.abs(got - want) <= tol * np.maximum(scale, 1e-30))


def test_cpqr_exact_rank_and_ties(ctx):
    # duplicated columns (exact ties): the smallest index wins, like the oracle
    base = np.random.default_rng(0).standard_normal((20, 8))
    Y = np.concatenate([base, base], axis=1).astype(np.float64)
    ld = 20
    Yd = dev(np.ascontiguousarray(Y.T))
    J = torch.empty(8, dtype=torch.int32, device="cuda")
    idl.idl_cpqr(ctx, Yd, 20, 16, ld, idl.IDL_F64, 8, J)
    Jw, _, _ = ocp.matrix_id(Y, 8)
    assert np.array_equal(host(J), Jw)
    assert host(J).max() < 8


# ------------------------------------------------------------------ a5 TensorSketch + a9 lambda_hat
@pytest.mark.parametrize("dims,R,L", [((1000, 1000, 1000), 100, 8192), ((6, 5, 4), 5, 16), ((200,) * 4, 51, 1024),
                                      ((37, 41), 10, 64), ((30, 20, 10), 7, 2048), ((9, 9), 4, 32),
                                      ((50, 40), 9, 256), ((200,) * 4, 331, 8192), ((1500, 7, 2100), 9, 8192),
                                      ((300,), 1, 8192), ((8192, 3), 4, 8192)])
def test_tensorsketch_parity(ctx, dims, R, L):
    facs, lam = cp_factors(dims, R, seed=len(dims) + R)
    hs, ss = odr.tensorsketch_maps(4, dims, L)
    want = ots.tensorsketch(facs, lam, hs, ss, L)
    fd = [dev(np.ascontiguousarray(F.T)) for F in facs]            # (R, I_n): columns contiguous
    hd = [torch.empty(d, dtype=torch.int32, device="cuda") for d in dims]
    sd = [torch.empty(d, dtype=torch.int8, device="cuda") for d in dims]
    for n, d in enumerate(dims):
        idl.idl_draw_mode(ctx, 4, n, d, L, hd[n], sd[n])
    ldy = R + 1
    Y = torch.empty((L, ldy), dtype=torch.float32, device="cuda")
    idl.idl_tensorsketch(ctx, fd, [d for d in dims], dev(lam), hd, sd, L, Y, ldy)
    got = host(Y)[:, :R]
    for r in range(R):       # per column: relative error of each sketched column
        assert rel_fro(got[:, r], want[:, r]) <= FP32_TOL, r


@pytest.mark.parametrize("dims,R,L,extra", [((1000, 1000, 1000), 101, 8192, 0), ((6, 5, 4), 5, 16, 3),
                                            ((200,) * 4, 51, 1024, 32), ((37, 41), 10, 64, 1),
                                            ((200,) * 4, 307, 8192, 4)])
def test_tensorsketch_colmajor_parity(ctx, dims, R, L, extra):
    """Column-major output (column r at Y + r*ldy): the oracle's sketch column by
    column, and the row-major call's values (up to the order of the shared-memory
    atomic adds that sum colliding entries of a mode's CountSketch)."""
    facs, lam = cp_factors(dims, R, seed=len(dims) + R + 1)
    hs, ss = odr.tensorsketch_maps(6, dims, L)
    want = ots.tensorsketch(facs, lam, hs, ss, L)
    fd = [dev(np.ascontiguousarray(F.T)) for F in facs]
    hd = [torch.empty(d, dtype=torch.int32, device="cuda") for d in dims]
    sd = [torch.empty(d, dtype=torch.int8, device="cuda") for d in dims]
    for n, d in enumerate(dims):
        idl.idl_draw_mode(ctx, 6, n, d, L, hd[n], sd[n])
    ldy = L + extra
    Yc = torch.full((R, ldy), float("nan"), dtype=torch.float32, device="cuda")
    idl.idl_tensorsketch(ctx, fd, list(dims), dev(lam), hd, sd, L, Yc, ldy, colmajor=True)
    Yr = torch.empty((L, R), dtype=torch.float32, device="cuda")
    idl.idl_tensorsketch(ctx, fd, list(dims), dev(lam), hd, sd, L, Yr, R)
    got = host(Yc)[:, :L].T
    rows = host(Yr)
    for r in range(R):
        assert rel_fro(got[:, r], rows[:, r]) <= FP32_TOL, r
    for r in range(R):
        assert rel_fro(got[:, r], want[:, r]) <= FP32_TOL, r
    if extra:
        assert np.all(np.isnan(host(Yc)[:, L:]))      # the padding is not written
    assert ctx.sync() == idl.IDL_OK


def test_lambda_hat_parity(ctx):
    rng = np.random.default_rng(3)
    K, R = 7, 40
    T = rng.standard_normal((K, R - K))
    J = rng.choice(R, K, replace=False).astype(np.int32)
    lam = rng.uniform(0.1, 1, R)
    out = torch.empty(K, dtype=torch.float64, device="cuda")
    idl.idl_lambda_hat(ctx, dev(lam), dev(J), dev(T), K, R, out)
    from oracle.idmethods import lambda_hat
    assert np.allclose(host(out), lambda_hat(lam, J, T), rtol=1e-14, atol=1e-14)


# ------------------------------------------------------------------ a6 on tcgen05: shapes and the CUDA-core path
@pytest.mark.parametrize("m2,m1,R", [(1, 64, 128), (16, 65, 1), (17, 63, 130), (60, 3600, 1000), (120, 1000, 257),
                                     (256, 200, 300), (33, 1, 5)])
def test_gaussian_tc_shapes_and_simt_agreement(ctx, m2, m1, R):
    rng = np.random.default_rng(m2 * 7 + m1)
    Y1 = rng.standard_normal((m1, R)).astype(np.float32)
    Om = torch.empty(m2 * m1, dtype=torch.float64, device="cuda")
    idl.idl_draw_gaussian(ctx, 5, m2, m1, Om)
    Omw = odr.gaussian_matrix(5, m2, m1)
    for prec, tol in [(idl.PREC_FP32, FP32_TOL), (idl.PREC_BF16X3, 2e-5), (idl.PREC_BF16, 1e-5),
                      (idl.PREC_TF32X3, FP32_TOL)]:
        outs = []
        for simt in (0, 1):             # tcgen05, CUDA cores
            idl.lib().idl_debug_gemm_path(ctx.ptr, simt)
            Y2 = torch.full((R * m2,), float("nan"), dtype=torch.float32, device="cuda")
            idl.idl_gaussian_stage(ctx, Om, m2, m1, dev(Y1), R, R, idl.IDL_F32, prec, Y2, m2)
            outs.append(colmajor_to_matrix(Y2, m2, R, m2))
        idl.lib().idl_debug_gemm_path(ctx.ptr, 0)
        want = ogs.gaussian_stage(Omw, Y1, prec)
        assert np.all(np.isfinite(outs[0]))
        assert rel_fro(outs[0], want) <= tol, (prec, rel_fro(outs[0], want))
        if prec == idl.PREC_FP32:
            assert rel_fro(outs[0], outs[1]) <= 2 * FP32_TOL
    assert ctx.sync() == idl.IDL_OK


@pytest.mark.parametrize("m2,m1,R,extra", [(60, 8192, 1000, 0), (17, 63, 130, 1), (33, 100, 5, 4),
                                            (120, 1000, 257, 3), (16, 65, 1, 0), (74, 4096, 300, 0)])
def test_gaussian_tc_colmajor_input(ctx, m2, m1, R, extra):
    """Y1 column-major (ragged K tails, unaligned ldy1 -> scalar loads, aligned ->
    vector loads): the same planes enter the same MMAs, so the result equals the
    row-major call's up to the order of the split-K partial sums (the two layouts
    may run a different number of CTAs per SM and so split K differently), and
    is within the oracle's tolerance of Omega Y1."""
    rng = np.random.default_rng(m2 + 3 * m1 + R)
    Y1 = rng.standard_normal((m1, R)).astype(np.float32)
    Om = torch.empty(m2 * m1, dtype=torch.float64, device="cuda")
    idl.idl_draw_gaussian(ctx, 8, m2, m1, Om)
    Omw = odr.gaussian_matrix(8, m2, m1)
    ldc = m1 + extra
    Yc = np.zeros((R, ldc), np.float32)
    Yc[:, :m1] = Y1.T
    Ycd, Yrd = dev(Yc), dev(Y1)
    for prec, tol in [(idl.PREC_FP32, FP32_TOL), (idl.PREC_BF16X3, 2e-5), (idl.PREC_BF16, 1e-5),
                      (idl.PREC_TF32X3, FP32_TOL)]:
        Y2c = torch.full((R * m2,), float("nan"), dtype=torch.float32, device="cuda")
        Y2r = torch.full((R * m2,), float("nan"), dtype=torch.float32, device="cuda")
        idl.idl_gaussian_stage_colmajor(ctx, Om, m2, m1, Ycd, R, ldc, prec, Y2c, m2)
        idl.idl_gaussian_stage(ctx, Om, m2, m1, Yrd, R, R, idl.IDL_F32, prec, Y2r, m2)
        assert rel_fro(host(Y2c), host(Y2r)) <= 1e-6, prec
        want = ogs.gaussian_stage(Omw, Y1, prec)
        assert rel_fro(colmajor_to_matrix(Y2c, m2, R, m2), want) <= tol, prec
    with pytest.raises(idl.IdlError):
        idl.idl_gaussian_stage_colmajor(ctx, Om, m2, m1, Ycd, R, m1 - 1, idl.PREC_FP32, Y2c, m2)
    with pytest.raises(idl.IdlError):
        idl.idl_gaussian_stage_colmajor(ctx, Om, m2, m1, Ycd, R, ldc, idl.PREC_FP64, Y2c, m2)
    assert ctx.sync() == idl.IDL_OK


@pytest.mark.parametrize("dtype,m,R,K", [("f32", 60, 10000, 50), ("f32", 120, 4096, 100), ("f64", 30, 2000, 20),
                                         ("f32", 60, 1000, 50), ("f32", 200, 700, 150), ("f64", 7, 3, 3)])
def test_cpqr_register_and_shared_memory_kernels_agree(ctx, dtype, m, R, K):
    rng = np.random.default_rng(m + R)
    npdt = np.float32 if dtype == "f32" else np.float64
    Y = (rng.standard_normal((m, R)) * rng.uniform(0.2, 5.0, R)[None, :]).astype(npdt)
    dt = idl.IDL_F32 if dtype == "f32" else idl.IDL_F64
    outs = []
    for smem_only in (0, 1):
        idl.lib().idl_debug_cpqr_path(ctx.ptr, smem_only)
        Yd = dev(np.ascontiguousarray(Y.T))
        J = torch.empty(K, dtype=torch.int32, device="cuda")
        idl.idl_cpqr(ctx, Yd, m, R, m, dt, K, J)
        outs.append((host(J), host(Yd).reshape(R, m).T.astype(np.float64)))
    idl.lib().idl_debug_cpqr_path(ctx.ptr, 0)
    (J0, F0), (J1, F1) = outs
    Jw, _, info = ocp.matrix_id(Y.astype(np.float64), K)
    if pivots_well_separated(info["gaps"]):
        assert np.array_equal(J0, Jw) and np.array_equal(J1, Jw)
    if np.array_equal(J0, J1):
        # the same reflections up to rounding: rows 0..K-1 of the factor agree
        tol = 1e-3 if dtype == "f32" else 1e-10
        assert np.abs(F0[:K] - F1[:K]).max() <= tol * np.abs(F1[:K]).max()
    assert ctx.sync() == idl.IDL_OK
