"""Algorithm 1: matrix ID via a rank-K column-pivoted QR.

TEST INFRASTRUCTURE (see ``oracle/__init__``).

Algorithm 1 (Sec. 1.2.1):
  * rank-K QR with column pivoting  Y Pi ~ Q R  (the paper uses column-pivoted
    QR in practice instead of SRRQR, Sec. 1.2.1 after Fact 1);
  * j = the first K pivots;
  * R11 = first K columns of R (K x K, upper triangular), R12 = the rest;
  * P^T = Pi [I_K, R11^{-1} R12]^T.

The QR is Householder QR with column pivoting (Golub & Van Loan, Matrix
Computations, Alg. 5.4.1): at step t the column of largest remaining 2-norm
(rows t..m-1) is moved to position t and a Householder reflection zeroes it
below row t.  Norms are recomputed exactly at every step (no downdating).
Ties go to the smallest original column index.

Output convention: J (length K, pivot order); T = R11^{-1} R12 of shape
K x (R-K) whose column c belongs to the c-th non-skeleton column in ascending
original index; P (K x R) has P[:, J[i]] = e_i and P[:, rest[c]] = T[:, c].
"""
from __future__ import annotations

import numpy as np


def householder(x: np.ndarray):
    """v, beta, alpha with (I - beta v v^T) x = alpha e_1, |alpha| = ||x||_2.
    alpha takes the sign opposite to x_0 (no cancellation in v_0)."""
    nrm = np.sqrt(np.dot(x, x))
    v = x.copy()
    if nrm == 0.0:
        return v * 0.0, 0.0, 0.0
    alpha = -nrm if x[0] >= 0 else nrm
    v[0] = x[0] - alpha
    vtv = np.dot(v, v)
    beta = 2.0 / vtv if vtv > 0 else 0.0
    return v, beta, alpha


def cpqr(Y: np.ndarray, K: int):
    """Rank-K Householder QR with column pivoting of Y (m x n), float64.

    Returns dict with
      perm  : the column permutation (perm[t] = original index at position t)
      R     : K x n, rows 0..K-1 of the triangular factor in permuted order
      gaps  : per step, (best - second best) / best of the squared norms
      norms : per step, the winning column's norm |r_tt|
    """
    A = np.array(Y, dtype=np.float64, copy=True)
    m, n = A.shape
    if not (1 <= K <= min(m, n)):
        raise ValueError("need 1 <= K <= min(m, n)")
    perm = np.arange(n)
    gaps, piv_norms = [], []
    for t in range(K):
        nrm2 = np.sum(A[t:, t:] ** 2, axis=0)
        best = nrm2.max()
        cands = np.nonzero(nrm2 == best)[0]
        j = t + cands[np.argmin(perm[t + cands])]          # tie -> smallest index
        rest = np.delete(nrm2, j - t)
        second = rest.max() if rest.size else 0.0
        gaps.append((best - second) / best if best > 0 else 0.0)
        piv_norms.append(np.sqrt(best))
        if j != t:
            A[:, [t, j]] = A[:, [j, t]]
            perm[[t, j]] = perm[[j, t]]
        v, beta, alpha = householder(A[t:, t])
        if beta != 0.0:
            w = beta * (v @ A[t:, t:])
            A[t:, t:] -= np.outer(v, w)
            A[t + 1:, t] = 0.0
            A[t, t] = alpha
    return dict(perm=perm, R=np.triu(A[:K, :]), gaps=np.array(gaps),
                norms=np.array(piv_norms), R22=A[K:, K:].copy())


def back_substitution(U: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X = U^{-1} B for upper-triangular U (K x K), by rows from the bottom up."""
    K = U.shape[0]
    X = np.array(B, dtype=np.float64, copy=True)
    for i in range(K - 1, -1, -1):
        if i + 1 < K:
            X[i] -= U[i, i + 1:] @ X[i + 1:]
        X[i] /= U[i, i]
    return X


def matrix_id(Y: np.ndarray, K: int):
    """Algorithm 1 on Y: returns (J, T, info)."""
    f = cpqr(Y, K)
    perm = f["perm"]
    R11 = f["R"][:, :K]
    R12 = f["R"][:, K:]
    J = perm[:K].copy()
    rest = perm[K:]
    Tp = back_substitution(R11, R12)
    order = np.argsort(rest, kind="stable")
    T = Tp[:, order]
    info = dict(gaps=f["gaps"], norms=f["norms"], rest=rest[order],
                R11=R11, R22_fro=float(np.linalg.norm(f["R22"])))
    return J, T, info


def build_P(J, T, n: int) -> np.ndarray:
    """The K x n coefficient matrix P of Algorithm 1 from (J, T)."""
    K = len(J)
    P = np.zeros((K, n), dtype=np.float64)
    P[np.arange(K), np.asarray(J)] = 1.0
    rest = np.setdiff1d(np.arange(n), np.asarray(J))
    P[:, rest] = T
    return P


def rest_columns(J, n: int) -> np.ndarray:
    """Non-skeleton columns in ascending order."""
    return np.setdiff1d(np.arange(n), np.asarray(J))
