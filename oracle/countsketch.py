"""CountSketch Y = S A, S = Phi D in R^{L x I} (Sec. 1.3; the sketch step of Algorithm 2).

TEST INFRASTRUCTURE (see ``oracle/__init__``).

Applying S adds row i of A, multiplied by d_ii = s(i), into row h(i) of Y.
Everything is accumulated in float64.
"""
from __future__ import annotations

import numpy as np


def explicit_S(h: np.ndarray, s: np.ndarray, L: int) -> np.ndarray:
    """The L x I matrix S = Phi D itself: phi_{h(i), i} = 1, D = diag(s)."""
    I = len(h)
    S = np.zeros((L, I), dtype=np.float64)
    S[np.asarray(h), np.arange(I)] = np.asarray(s, dtype=np.float64)
    return S


def countsketch_dense(A: np.ndarray, h: np.ndarray, s: np.ndarray, L: int) -> np.ndarray:
    """Y[h(i), :] += s(i) * A[i, :] for every row i; float64 result."""
    A = np.asarray(A, dtype=np.float64)
    Y = np.zeros((L, A.shape[1]), dtype=np.float64)
    np.add.at(Y, np.asarray(h), np.asarray(s, dtype=np.float64)[:, None] * A)
    return Y


def countsketch_dense_rows(A: np.ndarray, h: np.ndarray, s: np.ndarray, rows) -> np.ndarray:
    """Selected rows b of Y = S A: Y[b, :] = sum over {i : h(i) = b} of s(i) A[i, :]."""
    h = np.asarray(h)
    out = np.zeros((len(rows), A.shape[1]), dtype=np.float64)
    for t, b in enumerate(rows):
        members = np.nonzero(h == b)[0]
        if len(members):
            out[t] = (np.asarray(s[members], dtype=np.float64)[:, None]
                      * np.asarray(A[members], dtype=np.float64)).sum(axis=0)
    return out


def countsketch_csr(rowptr, colidx, vals, R: int, h, s, L: int) -> np.ndarray:
    """Y = S A for A in CSR form: each nonzero a_ic adds s(i) a_ic into
    Y[h(i), c] (cost O(nnz(A)), Sec. 1.3).  Duplicate (i, c) entries add."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    I = len(rowptr) - 1
    row_of = np.repeat(np.arange(I, dtype=np.int64), np.diff(rowptr))
    flat = np.asarray(h, dtype=np.int64)[row_of] * R + np.asarray(colidx, dtype=np.int64)
    w = np.asarray(s, dtype=np.float64)[row_of] * np.asarray(vals, dtype=np.float64)
    return np.bincount(flat, weights=w, minlength=L * R).reshape(L, R)


def countsketch_csr_rows(rowptr, colidx, vals, R: int, h, s, rows) -> np.ndarray:
    """Selected rows b of Y = S A for CSR A (one bucket at a time)."""
    h = np.asarray(h)
    out = np.zeros((len(rows), R), dtype=np.float64)
    for t, b in enumerate(rows):
        for i in np.nonzero(h == b)[0]:
            a, e = int(rowptr[i]), int(rowptr[i + 1])
            np.add.at(out[t], np.asarray(colidx[a:e], dtype=np.int64),
                      float(s[i]) * np.asarray(vals[a:e], dtype=np.float64))
    return out


def bucket_offsets(h: np.ndarray, L: int):
    """Rows grouped by bucket: bucket_ptr[b] .. bucket_ptr[b+1] index into
    row_list, rows listed in ascending order within each bucket (a stable
    counting sort of h).  This is the row-to-bucket map of Phi read column-wise."""
    h = np.asarray(h, dtype=np.int64)
    counts = np.bincount(h, minlength=L)
    ptr = np.zeros(L + 1, dtype=np.int64)
    ptr[1:] = np.cumsum(counts)
    row_list = np.argsort(h, kind="stable")
    return ptr, row_list
