"""Pins of the oracle's Algorithm 1/2/3 (Sec. 1.2.1, Sec. 3, Sec. 4, Fact 1,
Prop. 1) -- CPU only."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import cpqr, draws, errors, idmethods
from oracle import countsketch as cs
from oracle.gaussian import gaussian_stage
from synth import lowrank_dense, random_csr


def _distinct_norm_matrix(seed, m, n):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((m, n)) * rng.uniform(0.5, 3.0, n)[None, :]


@pytest.mark.parametrize("seed,m,n,K", [(0, 30, 80, 10), (1, 12, 40, 12), (2, 60, 200, 25)])
def test_pivots_and_R_match_lapack_geqp3(seed, m, n, K):
    """The greedy max-norm Householder CPQR is LAPACK's dgeqp3 (scipy qr with
    pivoting): same pivots, same |R| rows (signs per row may differ)."""
    Y = _distinct_norm_matrix(seed, m, n)
    f = cpqr.cpqr(Y, K)
    Qs, Rs, Ps = sla.qr(Y, pivoting=True, mode="economic")
    assert np.array_equal(f["perm"][:K], Ps[:K])
    sgn = np.sign(np.diag(Rs)[:K]) * np.sign(np.diag(f["R"])[:K])
    Rl = Rs[:K, :] * sgn[:, None]
    # columns of LAPACK's R are in its own permutation; put both in original order
    ours = np.zeros((K, n)); ours[:, f["perm"]] = f["R"]
    theirs = np.zeros((K, n)); theirs[:, Ps] = Rl
    assert np.allclose(ours, theirs, atol=1e-11 * np.abs(Rs).max())


def test_T_is_least_squares_solution():
    Y = _distinct_norm_matrix(3, 40, 120)
    J, T, info = cpqr.matrix_id(Y, 15)
    rest = cpqr.rest_columns(J, 120)
    Tl = np.linalg.lstsq(Y[:, J], Y[:, rest], rcond=None)[0]
    assert np.abs(T - Tl).max() <= 1e-10 * max(1.0, np.abs(Tl).max())
    assert np.array_equal(info["rest"], rest)


def test_back_substitution_matches_lapack():
    rng = np.random.default_rng(4)
    U = np.triu(rng.standard_normal((9, 9))) + 5 * np.eye(9)
    B = rng.standard_normal((9, 13))
    assert np.allclose(cpqr.back_substitution(U, B), sla.solve_triangular(U, B), atol=1e-13)


def test_P_structure_and_full_rank_exactness():
    """Fact 1 (i): the skeleton columns of P form I_K; Fact 1 (v): K = rank gives
    A_J P = A."""
    rng = np.random.default_rng(5)
    G = rng.standard_normal((30, 6)) @ rng.standard_normal((6, 50))
    J, T, _ = cpqr.matrix_id(G, 6)
    P = cpqr.build_P(J, T, 50)
    assert np.array_equal(P[:, J], np.eye(6))
    assert np.linalg.norm(G - G[:, J] @ P) <= 1e-12 * np.linalg.norm(G)


def test_scale_and_permutation_invariance():
    Y = _distinct_norm_matrix(6, 25, 70)
    J, T, _ = cpqr.matrix_id(Y, 8)
    J2, T2, _ = cpqr.matrix_id(3.7 * Y, 8)
    assert np.array_equal(J, J2) and np.allclose(T, T2, atol=1e-12)
    p = np.random.default_rng(7).permutation(70)
    J3, _, _ = cpqr.matrix_id(Y[:, p], 8)
    assert np.array_equal(p[J3], J)


def test_ties_go_to_smallest_index():
    Y = np.eye(4)[:, [0, 1, 2, 3]] * np.array([1.0, 2.0, 2.0, 1.0])
    f = cpqr.cpqr(Y, 2)
    assert list(f["perm"][:2]) == [1, 2]


def test_brute_force_tiny():
    """On tiny matrices the ID error is within Fact 1 (vi)'s sqrt(4K(R-K)+1)
    sigma_{K+1} factor and close to the best K-subset (exhaustive search)."""
    rng = np.random.default_rng(8)
    for trial in range(6):
        I, R, K = 12, 8, 2 + trial % 2
        A = rng.standard_normal((I, 4)) @ rng.standard_normal((4, R)) + 0.05 * rng.standard_normal((I, R))
        J, T, _ = cpqr.matrix_id(A, K)
        err = errors.matrix_id_error(A, J=J, T=T)
        sig = np.linalg.svd(A, compute_uv=False)
        assert err * sig[0] <= np.sqrt(4 * K * (R - K) + 1) * sig[K] * (1 + 1e-12)
        best = errors.best_subset_error(A, K)
        assert best <= err * (1 + 1e-12)
        assert err <= 3.0 * best


def test_exact_rank_k_recovery_dense():
    """Exactly rank-K input: the sketched ID is exact up to rounding (Fact 1 (v),
    cf. the ~1e-15 errors of Table 3 at K = rank)."""
    rng = np.random.default_rng(9)
    A = rng.standard_normal((2000, 10)) @ rng.standard_normal((10, 300))
    for m2 in (0, 20):
        J, T, _ = idmethods.id_matrix(A, k=10, m1=60, m2=m2, seed=1)
        assert errors.matrix_id_error(A, J=J, T=T) < 1e-12


def test_exact_rank_k_recovery_csr():
    c = random_csr(3000, 40, 0.02, seed=2, dtype=np.float64)
    # make it exactly rank 5 by replacing columns with combinations of 5 of them
    A = np.zeros((3000, 40))
    for i in range(3000):
        a, b = c.rowptr[i], c.rowptr[i + 1]
        A[i, c.colidx[a:b]] += c.vals[a:b]
    rng = np.random.default_rng(3)
    A = A[:, :5] @ rng.standard_normal((5, 40))
    rows, cols = np.nonzero(A)
    rowptr = np.zeros(3001, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    csr = (rowptr, cols.astype(np.int32), A[rows, cols], (3000, 40))
    J, T, _ = idmethods.id_matrix(csr=csr, k=5, m1=50, m2=15, seed=4)
    assert errors.matrix_id_error(csr=csr, J=J, T=T) < 1e-12
    assert errors.matrix_id_error(A, J=J, T=T) < 1e-12


def test_m2_zero_is_algorithm2_verbatim():
    A = lowrank_dense(500, 60, 0.8, 1e-8, seed=3)
    J, T, info = idmethods.id_matrix(A, k=8, m1=40, m2=0, seed=5)
    h, s = draws.countsketch_maps(5, 500, 40, True)
    J2, T2, _ = cpqr.matrix_id(cs.countsketch_dense(A, h, s, 40), 8)
    assert np.array_equal(J, J2) and np.array_equal(T, T2)


def test_gaussian_scale_invariance():
    A = lowrank_dense(400, 50, 0.8, 1e-8, seed=4)
    h, s = draws.countsketch_maps(2, 400, 60, True)
    Y1 = cs.countsketch_dense(A, h, s, 60)
    Om = draws.gaussian_matrix(2, 20, 60)
    J, T, _ = cpqr.matrix_id(gaussian_stage(Om, Y1), 8)
    J2, T2, _ = cpqr.matrix_id(gaussian_stage(5.0 * Om, Y1), 8)
    assert np.array_equal(J, J2) and np.allclose(T, T2, atol=1e-10)


def test_prop1_bound_holds_loosely():
    """||A_J P - A|| <~ 2 sigma_{K+1} sqrt(K I R) (Prop. 1), on a decaying spectrum."""
    I, R, K = 1500, 120, 10
    A = lowrank_dense(I, R, 0.7, 0.0, seed=6)
    J, T, _ = idmethods.id_matrix(A, k=K, m1=K + 10, m2=0, seed=7)
    sig = np.linalg.svd(A, compute_uv=False)
    err = errors.matrix_id_error(A, J=J, T=T) * sig[0]
    assert err <= 2 * sig[K] * np.sqrt(K * I * R)
    assert err <= 100 * sig[K]      # and in practice within a modest factor


def test_power_iteration_estimate_never_overestimates():
    A = lowrank_dense(300, 40, 0.8, 1e-3, seed=8)
    J, T, _ = cpqr.matrix_id(A, 5)
    exact = errors.matrix_id_error(A, J=J, T=T, exact=True)
    est = errors.matrix_id_error(A, J=J, T=T, exact=False, iters=200)
    assert est <= exact * (1 + 1e-9) and est >= 0.5 * exact


def test_tensor_id_exact_when_M_has_rank_K():
    """Duplicate rank-1 terms make M (Eq. M-matrix) rank K: Algorithm 3 recovers X
    exactly and lambda_hat merges the duplicates' s-values."""
    rng = np.random.default_rng(10)
    K, dims = 4, (7, 6, 5)
    base = [rng.standard_normal((d, K)) for d in dims]
    base = [F / np.linalg.norm(F, axis=0) for F in base]
    facs = [np.concatenate([F, F], axis=1) for F in base]         # R = 2K
    lam = rng.uniform(0.5, 1.5, 2 * K)
    J, T, lam_hat, _ = idmethods.id_cp_tensor(facs, lam, k=K, L=64, m2=12, seed=3)
    assert errors.tensor_id_error(facs, lam, J, lam_hat) < 1e-12
    assert np.allclose(np.sort(lam_hat), np.sort(lam[:K] + lam[K:]), atol=1e-12)


def test_lambda_hat_reconstructs_explicit_tensor():
    """X_hat = sum_k lambda_hat_k X^(j_k) (Eq. X-star) built explicitly equals
    M_J P lambda-weighted sum (Algorithm 3 lambda update)."""
    from oracle import tensorsketch as ts
    rng = np.random.default_rng(11)
    dims, R = (4, 3, 5), 6
    facs = [rng.standard_normal((d, R)) for d in dims]
    facs = [F / np.linalg.norm(F, axis=0) for F in facs]
    lam = rng.uniform(0.5, 1.5, R)
    J, T, lam_hat, _ = idmethods.id_cp_tensor(facs, lam, k=3, L=32, m2=0, seed=1)
    M = ts.khatri_rao(facs) * lam[None, :]
    P = cpqr.build_P(J, T, R)
    X_id = (M[:, J] @ P).sum(axis=1)                               # sum_r (M_J P)_{:r}
    X_hat = ts.khatri_rao(facs)[:, J] @ lam_hat
    assert np.allclose(X_id, X_hat, atol=1e-12)
