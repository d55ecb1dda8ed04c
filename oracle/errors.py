"""Error of an ID, for judging results (Sec. 6).

TEST INFRASTRUCTURE (see ``oracle/__init__``).

Matrix: relative spectral-norm error ||A - A_J P||_2 / ||A||_2.  Exact (LAPACK
SVD) for small A; otherwise 50 steps of the power method on E^T E from a seeded
Gaussian start, which never overestimates ||E||_2 -- the same one-sided
behaviour as the randomized estimate the paper uses (Sec. 6, after Woolfe et
al. Sec. 3.4).  The start vector is the counter-based Gaussian draw with tag
ERR_START (1 x n, seed ``seed`` for E and ``seed + 1`` for A), so that the
device estimator can start from the same vector.

CP tensor: relative Frobenius error ||X_hat - X||_F / ||X||_F, exact, from the
Gram identity M^T M = Hadamard product of A^(n)T A^(n) (Eq. MTM-formula):
X_hat - X = sum_r c_r X^(r) with c = scatter(lambda_hat at J) - lambda, so
||X_hat - X||_F^2 = c^T G c with G = M^T M / (lambda lambda^T) entrywise, i.e.
G = Hadamard product of the factor Gram matrices.
"""
from __future__ import annotations

import numpy as np

from . import draws
from .cpqr import build_P


def _power(matvec, rmatvec, n: int, iters: int, seed: int) -> float:
    x = draws.gaussian_matrix(seed, 1, n, tag=draws.TAG_ERR_START)[0]
    x /= np.linalg.norm(x)
    est = 0.0
    for _ in range(iters):
        y = rmatvec(matvec(x))
        ny = np.linalg.norm(y)
        if ny == 0.0:
            return 0.0
        est = np.sqrt(ny)
        x = y / ny
    return float(est)


def _as_operator(A=None, csr=None):
    if A is not None:
        A64 = np.asarray(A, dtype=np.float64)
        return (lambda x: A64 @ x), (lambda y: A64.T @ y), A64.shape
    import scipy.sparse as sp
    rowptr, colidx, vals, shape = csr
    M = sp.csr_matrix((np.asarray(vals, dtype=np.float64), np.asarray(colidx, dtype=np.int64),
                       np.asarray(rowptr, dtype=np.int64)), shape=shape)
    MT = M.T.tocsr()
    return (lambda x: M @ x), (lambda y: MT @ y), shape


def matrix_id_error(A=None, csr=None, *, J, T, exact=None, iters: int = 50, seed: int = 1234) -> float:
    """||A - A_J P||_2 / ||A||_2."""
    mv, rmv, (I, R) = _as_operator(A, csr)
    P = build_P(J, T, R)
    J = np.asarray(J)
    if exact is None:
        exact = A is not None and I * R <= 4_000_000
    if exact:
        A64 = np.asarray(A, dtype=np.float64)
        E = A64 - A64[:, J] @ P
        return float(np.linalg.norm(E, 2) / np.linalg.norm(A64, 2))

    def emv(x):
        px = P @ x                   # K
        z = np.zeros(R)
        z[J] = px
        return mv(x) - mv(z)

    def ermv(y):
        aty = rmv(y)                 # R
        return aty - P.T @ aty[J]

    num = _power(emv, ermv, R, iters, seed)
    den = _power(mv, rmv, R, iters, seed + 1)
    return num / den


def best_subset_error(A, K: int) -> float:
    """min over all K-subsets J of ||A - A_J A_J^+ A||_2 / ||A||_2 (brute force)."""
    import itertools
    A = np.asarray(A, dtype=np.float64)
    nA = np.linalg.norm(A, 2)
    best = np.inf
    for J in itertools.combinations(range(A.shape[1]), K):
        AJ = A[:, J]
        E = A - AJ @ np.linalg.lstsq(AJ, A, rcond=None)[0]
        best = min(best, np.linalg.norm(E, 2))
    return best / nA


def gram(factors) -> np.ndarray:
    """Hadamard product of the factor Gram matrices A^(n)T A^(n) (Eq. MTM-formula)."""
    G = None
    for F in factors:
        F64 = np.asarray(F, dtype=np.float64)
        g = F64.T @ F64
        G = g if G is None else G * g
    return G


def tensor_id_error(factors, lam, J, lam_hat) -> float:
    """||X_hat - X||_F / ||X||_F for CP tensors sharing the rank-1 terms X^(r)."""
    G = gram(factors)
    lam = np.asarray(lam, dtype=np.float64)
    c = -lam.copy()
    np.add.at(c, np.asarray(J), np.asarray(lam_hat, dtype=np.float64))
    num = float(c @ G @ c)
    den = float(lam @ G @ lam)
    return float(np.sqrt(max(num, 0.0) / den))
