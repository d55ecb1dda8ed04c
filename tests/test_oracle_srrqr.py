"""Pins of the strong rank-revealing QR refinement (Sec. 1.2.1, Fact 1; Gu &
Eisenstat 1996): determinant growth per exchange, local optimality by brute
force, Fact 1's bounds, and a Kahan matrix on which column pivoting fails."""
import itertools

import numpy as np
import pytest

from oracle import cpqr, errors
from oracle import srrqr


def kahan(n, theta, eps=1e-10):
    """Kahan's matrix diag(s^i) (I - c N), N strictly upper triangular ones, with the
    columns scaled by (1 - eps)^j so that column pivoting keeps the natural order."""
    s, c = np.sin(theta), np.cos(theta)
    U = np.eye(n) - c * np.triu(np.ones((n, n)), 1)
    return np.diag(s ** np.arange(n)) @ U @ np.diag((1.0 - eps) ** np.arange(n))


def absdet(Y, J):
    """|det R11| of the selection J, from the Gram determinant (no QR)."""
    YJ = Y[:, np.asarray(J)]
    return float(np.sqrt(abs(np.linalg.det(YJ.T @ YJ))))


def test_pivoted_qr_fails_on_kahan_and_the_swaps_repair_it():
    A = kahan(30, 1.2)
    K = 29
    J, T, _ = cpqr.matrix_id(A, K)
    assert np.abs(T).max() > 100.0                   # Fact 1 (ii) fails for plain pivoting
    J2, T2, info = srrqr.srrqr_id(A, K, f=2.0)
    assert len(info["swaps"]) >= 1
    assert np.abs(T2).max() <= 2.0


def test_each_exchange_multiplies_the_determinant_by_sqrt_rho():
    """Gu-Eisenstat: exchanging J[i] for rest[j] scales |det R11| by sqrt(rho_ij)."""
    A = np.vstack([kahan(20, 1.1), 1e-3 * np.random.default_rng(0).standard_normal((4, 20))])
    J0, _, _ = cpqr.matrix_id(A, 12)
    J = np.array(J0)
    c = srrqr.criterion(A, J)
    for i in range(3):
        for j in (0, 3, 5):
            J2 = J.copy()
            J2[i] = c["rest"][j]
            assert absdet(A, J2) / absdet(A, J) == pytest.approx(np.sqrt(c["rho"][i, j]), rel=1e-6)


@pytest.mark.parametrize("seed,f", [(1, 1.05), (2, 1.5), (3, 2.0)])
def test_no_single_exchange_grows_the_determinant_by_more_than_f(seed, f):
    """Local optimality at termination, by brute force over every exchange."""
    rng = np.random.default_rng(seed)
    A = kahan(14, 1.0 + 0.1 * seed) + 1e-6 * rng.standard_normal((14, 14))
    K = 7
    J, T, info = srrqr.srrqr_id(A, K, f=f)
    d0 = absdet(A, J)
    rest = np.setdiff1d(np.arange(14), J)
    for i, j in itertools.product(range(K), rest):
        J2 = J.copy()
        J2[i] = j
        assert absdet(A, J2) <= f * d0 * (1 + 1e-9)


@pytest.mark.parametrize("seed", [4, 5, 6])
def test_fact1_bounds_with_f_two(seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((25, 18)) @ np.diag(0.6 ** np.arange(18)) @ rng.standard_normal((18, 40))
    K, R = 6, 40
    J, T, info = srrqr.srrqr_id(A, K, f=2.0)
    P = np.zeros((K, R))
    P[np.arange(K), J] = 1.0
    P[:, info["rest"]] = T
    sv = np.linalg.svd(A, compute_uv=False)
    assert np.abs(T).max() <= 2.0 + 1e-12                                       # (ii)
    assert np.linalg.norm(P, 2) <= np.sqrt(4 * K * (R - K) + 1)                  # (iii)
    assert np.linalg.svd(P, compute_uv=False).min() >= 1.0 - 1e-12               # (iv)
    err = np.linalg.norm(A[:, J] @ P - A, 2)
    assert err <= sv[K] * np.sqrt(4 * K * (R - K) + 1)                           # (v)
    assert errors.matrix_id_error(A, J=J, T=T, exact=True) == pytest.approx(err / sv[0], rel=1e-10)
