"""Pins of the oracle's CountSketch and TensorSketch (Sec. 1.3, Eq. TA-formula,
Lemma 1, Eq. MTM-formula) -- CPU only."""
import numpy as np
import pytest

from oracle import countsketch as cs
from oracle import draws
from oracle import errors
from oracle import tensorsketch as ts
from oracle.gaussian import BF16, FP32, gaussian_stage, round_bf16
from synth import random_csr


def _csr_to_dense(c):
    I, R = c.shape
    A = np.zeros((I, R))
    for i in range(I):
        a, b = c.rowptr[i], c.rowptr[i + 1]
        np.add.at(A[i], c.colidx[a:b], c.vals[a:b].astype(np.float64))
    return A


@pytest.mark.parametrize("modified", [False, True])
def test_hashed_equals_explicit_S_bit_exact(modified):
    rng = np.random.default_rng(1)
    I, R, L = 300, 17, 40
    A = rng.integers(-1000, 1000, size=(I, R)).astype(np.float64)   # integers: exact sums
    h, s = draws.countsketch_maps(7, I, L, modified)
    S = cs.explicit_S(h, s, L)
    assert np.array_equal(S @ A, cs.countsketch_dense(A, h, s, L))
    assert np.array_equal(cs.countsketch_dense_rows(A, h, s, [0, 5, L - 1]),
                          (S @ A)[[0, 5, L - 1]])


def test_csr_sketch_equals_explicit():
    c = random_csr(500, 60, 0.05, seed=3, dtype=np.float64)
    c.vals = np.round(c.vals * 64)                                  # integer-valued
    A = _csr_to_dense(c)
    h, s = draws.countsketch_maps(5, 500, 37, True)
    Y = cs.countsketch_csr(c.rowptr, c.colidx, c.vals, 60, h, s, 37)
    assert np.array_equal(Y, cs.explicit_S(h, s, 37) @ A)
    assert np.array_equal(cs.countsketch_csr_rows(c.rowptr, c.colidx, c.vals, 60, h, s, [3, 36]),
                          Y[[3, 36]])


def test_csr_duplicates_add():
    rowptr = np.array([0, 3, 3, 5])
    colidx = np.array([1, 1, 0, 2, 2])
    vals = np.array([1.0, 2.0, 4.0, 8.0, 16.0])
    h = np.array([0, 1, 0])
    s = np.array([1, 1, -1], dtype=np.int8)
    Y = cs.countsketch_csr(rowptr, colidx, vals, 3, h, s, 2)
    assert np.array_equal(Y, np.array([[4.0, 3.0, -24.0], [0, 0, 0]]))


def test_bucket_offsets_group_rows_stably():
    h = np.array([2, 0, 2, 1, 0, 2, 2])
    ptr, rows = cs.bucket_offsets(h, 4)
    assert list(ptr) == [0, 2, 3, 7, 7]
    assert list(rows) == [1, 4, 3, 0, 2, 5, 6]


def test_lemma1_C_equals_identity_plus_E():
    """(S U)^T (S U) = I + E with E the off-diagonal collision sum (Lemma 1)."""
    rng = np.random.default_rng(2)
    I, K, L = 40, 3, 7
    U, _ = np.linalg.qr(rng.standard_normal((I, K)))
    h, s = draws.countsketch_maps(8, I, L, False)
    S = cs.explicit_S(h, s, L)
    C = (S @ U).T @ (S @ U)
    E = np.zeros((K, K))
    for i in range(I):
        for j in range(I):
            if i != j and h[i] == h[j]:
                E += s[i] * s[j] * np.outer(U[i], U[j])
    assert np.allclose(C, np.eye(K) + E, atol=1e-13)


def _tiny_cp(seed, dims=(3, 5, 4), R=5):
    rng = np.random.default_rng(seed)
    facs = [rng.standard_normal((d, R)) for d in dims]
    facs = [F / np.linalg.norm(F, axis=0) for F in facs]
    lam = rng.uniform(0.5, 2.0, R)
    return facs, lam


def test_tensorsketch_equals_explicit_khatri_rao():
    """Eq. TA-formula against the explicitly built T (H, S of Sec. 1.3) applied to
    the explicitly built M (Eq. M-matrix)."""
    facs, lam = _tiny_cp(0)
    dims, L = [F.shape[0] for F in facs], 16
    hs, ss = draws.tensorsketch_maps(6, dims, L)
    Y = ts.tensorsketch(facs, lam, hs, ss, L)
    M = ts.khatri_rao(facs) * lam[None, :]
    T = ts.explicit_T(dims, hs, ss, L)
    assert np.abs(Y - T @ M).max() <= 1e-13 * np.abs(T @ M).max()


def test_tensorsketch_is_circular_convolution():
    facs, lam = _tiny_cp(1, dims=(6, 5), R=3)
    L = 16
    hs, ss = draws.tensorsketch_maps(2, [6, 5], L)
    C = ts.mode_sketches(facs, hs, ss, L)
    Y = ts.tensorsketch(facs, lam, hs, ss, L)
    for r in range(3):
        direct = ts.circular_convolution(C[0][:, r], C[1][:, r]) * lam[r]
        assert np.allclose(Y[:, r], direct, atol=1e-13)


def test_gram_identity():
    """M^T M = Hadamard product of A^(n)T A^(n) (Eq. MTM-formula)."""
    facs, _ = _tiny_cp(3)
    M = ts.khatri_rao(facs)
    assert np.allclose(M.T @ M, errors.gram(facs), atol=1e-13)


def test_tensor_error_matches_explicit_tensor():
    facs, lam = _tiny_cp(4)
    M = ts.khatri_rao(facs)
    J = np.array([0, 3])
    lam_hat = np.array([1.3, -0.4])
    X = M @ lam
    Xh = M[:, J] @ lam_hat
    want = np.linalg.norm(Xh - X) / np.linalg.norm(X)
    assert abs(errors.tensor_id_error(facs, lam, J, lam_hat) - want) < 1e-13


def test_round_bf16_is_nearest_even():
    x = np.array([1.0, 1.00390625, 1.005859375, 1.0078125 + 2**-9, -3.14159265, 1e-30,
                  65504.0, 3.0e38], dtype=np.float32)
    r = round_bf16(x)
    for xi, ri in zip(x, r):
        # bf16 grid around xi: 8 significant bits
        e = np.floor(np.log2(abs(float(xi))))
        ulp = 2.0 ** (e - 7)
        lo = np.floor(float(xi) / ulp) * ulp
        cands = [lo, lo + ulp]
        d = [abs(c - float(xi)) for c in cands]
        if d[0] == d[1]:   # tie: even mantissa
            want = cands[0] if int(round(cands[0] / ulp)) % 2 == 0 else cands[1]
        else:
            want = cands[int(np.argmin(d))]
        assert float(ri) == want, (xi, ri, want)
    # exactly representable values survive
    assert np.array_equal(round_bf16(np.array([0.5, -2.0, 1.5], np.float32)), [0.5, -2.0, 1.5])


def test_gaussian_stage_modes():
    rng = np.random.default_rng(5)
    Om = draws.gaussian_matrix(1, 6, 50)
    Y1 = rng.standard_normal((50, 9))
    exact = Om @ Y1
    assert np.allclose(gaussian_stage(Om, Y1), exact, rtol=0, atol=1e-12)
    assert np.abs(gaussian_stage(Om, Y1, FP32) - exact).max() < 1e-5 * np.abs(exact).max()
    bf = gaussian_stage(Om, Y1, BF16)
    assert np.abs(bf - exact).max() < 5e-2 * np.abs(exact).max()
    assert not np.allclose(bf, exact, atol=1e-6)
