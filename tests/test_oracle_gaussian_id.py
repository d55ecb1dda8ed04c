"""Pins of the Gaussian ID comparators (Sec. 1.2.1; Sec. 1.2.2, Eq. G-matrix)."""
import numpy as np
import pytest

from oracle import draws, errors, gaussian_id as gid
from oracle import tensorsketch as ots
from synth import cp_factors, lowrank_dense, random_csr


def test_khatri_rao_sketch_equals_the_explicit_product():
    """y_lr = lambda_r prod_n <omega^(n)_:l, a^(n)_:r> is Omega M with the explicitly
    built Omega = (Khatri-Rao of Omega^(n))^T and M = (Khatri-Rao of A^(n)) diag(lambda)."""
    dims, R, L = (3, 4, 2), 5, 7
    facs, lam = cp_factors(dims, R, seed=3)
    facs = [F.astype(np.float64) for F in facs]
    Oms = gid.mode_gaussians(11, dims, L)
    Om_full = ots.khatri_rao(Oms).T                    # L x prod(dims)
    M = ots.khatri_rao(facs) * lam[None, :]            # prod(dims) x R
    want = Om_full @ M
    got = gid.khatri_rao_gaussian_sketch(facs, lam, L, 11)
    assert np.allclose(got, want, rtol=1e-13, atol=1e-14)


def test_mode_gaussians_are_the_transposed_tagged_draws():
    Oms = gid.mode_gaussians(5, (6, 4), 3)
    for n, (Om, In) in enumerate(zip(Oms, (6, 4))):
        assert Om.shape == (In, 3)
        assert np.array_equal(Om.T, draws.gaussian_matrix(5, 3, In, tag=draws.TAG_GAUSS_MODE + n))
    # other tags are other streams
    assert not np.allclose(draws.gaussian_matrix(5, 3, 6, tag=draws.TAG_GAUSS_ID), Oms[0].T)


def test_dense_and_csr_sketches_agree():
    c = random_csr(300, 40, 0.05, seed=2, dtype=np.float64)
    A = np.zeros((300, 40))
    for i in range(300):
        for q in range(c.rowptr[i], c.rowptr[i + 1]):
            A[i, c.colidx[q]] += c.vals[q]
    Yd = gid.gaussian_sketch_matrix(A, L=12, seed=4)
    Yc = gid.gaussian_sketch_matrix(csr=(c.rowptr, c.colidx, c.vals, c.shape), L=12, seed=4)
    assert np.allclose(Yd, Yc, rtol=1e-12, atol=1e-12)


def test_norm_preserved_in_expectation():
    """E ||Omega a||^2 = L ||a||^2 for iid N(0,1) Omega (Sec. 1.2.1); mean over seeds within 5 sigma."""
    rng = np.random.default_rng(0)
    a = rng.standard_normal((50, 1))
    L, n = 20, 300
    vals = [float(np.sum(gid.gaussian_sketch_matrix(a, L=L, seed=s) ** 2)) for s in range(n)]
    ratio = np.mean(vals) / (L * float(np.sum(a * a)))
    assert abs(ratio - 1.0) <= 5.0 * np.sqrt(2.0 / (n * L))


def test_khatri_rao_entries_have_unit_second_moment():
    """With unit-norm factor columns, each <omega^(n)_:l, a^(n)_:r> is N(0, 1) and the
    modes are independent, so E y_lr^2 = lambda_r^2."""
    facs, lam = cp_factors((30, 20, 10), 8, seed=1, lam=np.ones(8))
    ys = np.concatenate([gid.khatri_rao_gaussian_sketch(facs, lam, 50, s).ravel() for s in range(40)])
    m = np.mean(ys ** 2)
    # var(y^2) = E y^4 - 1 = 3^3 - 1 for a product of three independent N(0,1)
    assert abs(m - 1.0) <= 5.0 * np.sqrt((27.0 - 1.0) / ys.size)


def test_gaussian_matrix_id_recovers_exact_rank():
    A = lowrank_dense(400, 60, 0.7, 0.0, seed=5, rank=8)
    J, T, _ = gid.gaussian_id_matrix(A, k=8, L=18, seed=3)
    assert errors.matrix_id_error(A, J=J, T=T, exact=True) < 1e-12


def test_gaussian_tensor_id_recovers_exact_rank():
    rng = np.random.default_rng(10)
    K, dims = 5, (12, 9, 7)
    base = [rng.standard_normal((d, K)) for d in dims]
    base = [F / np.linalg.norm(F, axis=0) for F in base]
    facs = [np.concatenate([F, F], axis=1) for F in base]          # R = 2K, M has rank K
    lam = rng.uniform(0.5, 1.5, 2 * K)
    J, T, lh, _ = gid.gaussian_id_tensor(facs, lam, k=K, L=K + 6, seed=2)
    assert errors.tensor_id_error(facs, lam, J, lh) < 1e-10
