"""Strong rank-revealing QR refinement of Algorithm 1's pivots (Sec. 1.2.1, Fact 1;
Gu & Eisenstat 1996).

TEST INFRASTRUCTURE (see ``oracle/__init__``).

Fact 1 states its bounds for an ID whose QR step is a strong rank-revealing QR
(SRRQR): no entry of P exceeds f (the paper's f = 2) and
||A_J P - A|| <= sigma_{K+1} sqrt(f^2 K (R - K) + 1).  Gu and Eisenstat reach it
from any K-column selection J by swaps: with R11 the triangular factor of the
selected columns (in J's order), R12 = Q^T A_rest, R22 = A_rest - Q R12,
    W = R11^{-1} R12,  omega_i = 1 / ||e_i^T R11^{-1}||,  gamma_j = ||R22 e_j||,
while some rho_ij = W_ij^2 + (gamma_j / omega_i)^2 exceeds f^2, the skeleton
column J[i] is exchanged with the non-skeleton column rest[j]; each exchange
multiplies |det R11| by sqrt(rho_ij) > f, so the loop ends.

Here: the start is the column-pivoted QR's J (``cpqr.matrix_id``); each step
takes the largest rho (ties: smallest i, then smallest j) and recomputes every
quantity from scratch (Householder QR of A_J by LAPACK -- a library primitive --
and triangular solves), in float64.  T = W for the final J (rest ascending), the
output convention of ``cpqr.matrix_id``.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .cpqr import matrix_id


def criterion(Y: np.ndarray, J) -> dict:
    """rho (K x (R-K)), W, omega, gamma and rest (ascending) for the selection J."""
    Y = np.asarray(Y, dtype=np.float64)
    J = np.asarray(J)
    R = Y.shape[1]
    rest = np.setdiff1d(np.arange(R), J)
    Q, R11 = np.linalg.qr(Y[:, J])                    # reduced: m x K, K x K
    R12 = Q.T @ Y[:, rest]
    R22 = Y[:, rest] - Q @ R12
    Rinv = sla.solve_triangular(R11, np.eye(len(J)))
    W = Rinv @ R12
    inv_omega = np.linalg.norm(Rinv, axis=1)           # 1 / omega_i
    gamma = np.linalg.norm(R22, axis=0)
    rho = W ** 2 + (gamma[None, :] * inv_omega[:, None]) ** 2
    return dict(rho=rho, W=W, inv_omega=inv_omega, gamma=gamma, rest=rest)


def srrqr_id(Y: np.ndarray, K: int, f: float = 2.0, max_swaps: int = 256):
    """Algorithm 1 with Gu-Eisenstat swaps after the pivoted QR.  Returns (J, T, info)
    with info["swaps"] the exchanges made and info["gaps"] the pivoted QR's gaps."""
    if not f > 1.0:
        raise ValueError("need f > 1")
    J0, _, info0 = matrix_id(Y, K)
    J = np.array(J0)
    swaps = []
    for _ in range(max_swaps + 1):
        c = criterion(Y, J)
        rho = c["rho"]
        q = int(np.argmax(rho))                         # first maximum in row-major order
        i, j = divmod(q, rho.shape[1])
        if rho[i, j] <= f * f or len(swaps) == max_swaps:
            break
        swaps.append((i, int(c["rest"][j]), float(rho[i, j])))
        J[i] = c["rest"][j]
    c = criterion(Y, J)
    info = dict(swaps=swaps, gaps=info0["gaps"], rho_max=float(c["rho"].max()), rest=c["rest"])
    return J, c["W"], info
