"""Gaussian ID, the comparison method of the paper (Sec. 1.2.1 and Sec. 1.2.2).

TEST INFRASTRUCTURE (see ``oracle/__init__``).

Matrix (Sec. 1.2.1, the randomized ID of Martinsson et al.): Y = Omega A with
Omega an L x I matrix of iid N(0,1) entries, then the ID of Y (Algorithm 1);
the same J and P are an ID of A.  Omega is the counter-based Gaussian draw with
tag GAUSS_ID (row-major L x I).

CP tensor (Sec. 1.2.2, Eq. G-matrix, after Biagioni et al.): the sketch
Y = Omega M of M = (Khatri-Rao of A^(n)) diag(lambda) with
Omega = (Khatri-Rao of Omega^(n))^T, each Omega^(n) an I_n x L matrix of iid
N(0,1) entries, formed without Omega or M:
    y_lr = lambda_r prod_n < omega^(n)_:l , a^(n)_:r >.
Omega^(n) is the transpose of the counter-based draw with tag GAUSS_MODE + n,
row-major L x I_n.  Then the ID of Y (Algorithm 1) and
lambda_hat_k = lambda_{j_k} (1 + sum_c T_kc) as in Algorithm 3.
"""
from __future__ import annotations

import numpy as np

from . import draws
from .cpqr import matrix_id
from .idmethods import lambda_hat


def gaussian_sketch_matrix(A=None, csr=None, *, L: int, seed: int) -> np.ndarray:
    """Y = Omega A (L x R), float64."""
    if A is not None:
        I = A.shape[0]
        Om = draws.gaussian_matrix(seed, L, I, tag=draws.TAG_GAUSS_ID)
        return Om @ np.asarray(A, dtype=np.float64)
    import scipy.sparse as sp
    rowptr, colidx, vals, (I, R) = csr
    M = sp.csr_matrix((np.asarray(vals, dtype=np.float64), np.asarray(colidx, dtype=np.int64),
                       np.asarray(rowptr, dtype=np.int64)), shape=(I, R))
    Om = draws.gaussian_matrix(seed, L, I, tag=draws.TAG_GAUSS_ID)
    return np.asarray((M.T @ Om.T).T)


def mode_gaussians(seed: int, dims, L: int):
    """Omega^(n) (I_n x L) for every mode: the transposes of the L x I_n draws."""
    return [draws.gaussian_matrix(seed, L, In, tag=draws.TAG_GAUSS_MODE + n).T for n, In in enumerate(dims)]


def khatri_rao_gaussian_sketch(factors, lam, L: int, seed: int) -> np.ndarray:
    """Y (L x R) with y_lr = lambda_r prod_n <omega^(n)_:l, a^(n)_:r> (Eq. G-matrix)."""
    dims = [F.shape[0] for F in factors]
    Oms = mode_gaussians(seed, dims, L)
    Y = np.ones((L, factors[0].shape[1]), dtype=np.float64)
    for Om, F in zip(Oms, factors):
        Y *= Om.T @ np.asarray(F, dtype=np.float64)
    return Y * np.asarray(lam, dtype=np.float64)[None, :]


def gaussian_id_matrix(A=None, csr=None, *, k: int, L: int, seed: int):
    """Gaussian matrix ID.  Returns (J, T, info)."""
    Y = gaussian_sketch_matrix(A, csr, L=L, seed=seed)
    J, T, info = matrix_id(Y, k)
    info["Y2"] = Y
    return J, T, info


def gaussian_id_tensor(factors, lam, *, k: int, L: int, seed: int):
    """Gaussian tensor ID through the Khatri-Rao structured sketch.  Returns
    (J, T, lambda_hat, info)."""
    Y = khatri_rao_gaussian_sketch(factors, lam, L, seed)
    J, T, info = matrix_id(Y, k)
    info["Y2"] = Y
    return J, T, lambda_hat(lam, J, T), info
