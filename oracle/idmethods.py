"""Algorithm 2 (CountSketch matrix ID) and Algorithm 3 (TensorSketch tensor ID).

TEST INFRASTRUCTURE (see ``oracle/__init__``).

Matrix ID (Algorithm 2, Sec. 3), with the Gaussian stage of Sec. 1.2.1 placed
after the CountSketch:
  1. draw S (h, s), with the modified map of Remark 2 when ``modified``;
  2. Y1 = S A                                (m1 x R)
  3. Y2 = Omega Y1 if m2 > 0 else Y1          (m2 x R)
  4. [P, j] = Algorithm 1 (Y2, K).
With m2 = 0 this is the paper's Algorithm 2 verbatim.

Tensor ID (Algorithm 3, Sec. 4):
  1. draw T (h_n, s_n per mode);
  2. Y = T M by Eq. TA-formula (M never formed);
  3. Y2 = Omega Y if m2 > 0;
  4. [P, j] = Algorithm 1 (Y2, K);
  5. lambda_hat_k = lambda_{j_k} * sum_r p_kr = lambda_{j_k} (1 + sum_c T_kc)
     (Algorithm 3; the identity columns of P contribute the 1).
"""
from __future__ import annotations

import numpy as np

from . import countsketch as cs
from . import draws
from . import gaussian as gs
from . import tensorsketch as ts
from .cpqr import matrix_id


def sketch_matrix(A=None, csr=None, *, m1: int, seed: int, modified: bool = True):
    """Y1 = S A for dense A (I x R) or csr = (rowptr, colidx, vals, (I, R))."""
    if A is not None:
        I = A.shape[0]
        h, s = draws.countsketch_maps(seed, I, m1, modified)
        return cs.countsketch_dense(A, h, s, m1)
    rowptr, colidx, vals, shape = csr
    I, R = shape
    h, s = draws.countsketch_maps(seed, I, m1, modified)
    return cs.countsketch_csr(rowptr, colidx, vals, R, h, s, m1)


def id_matrix(A=None, csr=None, *, k: int, m1: int, m2: int, seed: int,
              modified: bool = True, precision: int = gs.FP64):
    """Algorithm 2 with the Gaussian stage.  Returns (J, T, info)."""
    Y1 = sketch_matrix(A, csr, m1=m1, seed=seed, modified=modified)
    if m2 > 0:
        Om = draws.gaussian_matrix(seed, m2, m1)
        Y2 = gs.gaussian_stage(Om, Y1, precision)
    else:
        Y2 = Y1
    J, T, info = matrix_id(Y2, k)
    info["Y1"] = Y1
    info["Y2"] = Y2
    return J, T, info


def lambda_hat(lam, J, T) -> np.ndarray:
    """lambda_hat_k = lambda_{j_k} * sum_r p_kr (Algorithm 3)."""
    lam = np.asarray(lam, dtype=np.float64)
    return lam[np.asarray(J)] * (1.0 + np.asarray(T).sum(axis=1))


def id_cp_tensor(factors, lam, *, k: int, L: int, m2: int, seed: int,
                 precision: int = gs.FP64):
    """Algorithm 3 with the Gaussian stage.  Returns (J, T, lambda_hat, info)."""
    dims = [F.shape[0] for F in factors]
    hs, ss = draws.tensorsketch_maps(seed, dims, L)
    Y = ts.tensorsketch(factors, lam, hs, ss, L)
    if m2 > 0:
        Om = draws.gaussian_matrix(seed, m2, L)
        Y2 = gs.gaussian_stage(Om, Y, precision)
    else:
        Y2 = Y
    J, T, info = matrix_id(Y2, k)
    info["Y1"] = Y
    info["Y2"] = Y2
    return J, T, lambda_hat(lam, J, T), info
