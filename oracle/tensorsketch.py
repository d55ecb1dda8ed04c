"""TensorSketch of the Khatri-Rao matrix of CP factors (Sec. 1.3, Eq. TA-formula).

TEST INFRASTRUCTURE (see ``oracle/__init__``).

For M = (Khatri-Rao product of A^(1..N)) diag(lambda) (Eq. M-matrix), the
sketch T M is formed without M: per mode the CountSketch S^(n) A^(n) (L x R),
then T A = IFFT( Hadamard product over n of FFT(S^(n) A^(n)) ) (Eq.
TA-formula), then column r scaled by lambda_r.  The FFT is numpy's (a library
primitive); the real part of the inverse transform is the sketch.

The explicit forms (``khatri_rao``, ``explicit_T``) build H and S of Sec. 1.3
over all tuples and are used only at tiny sizes to pin the FFT formula.
"""
from __future__ import annotations

import itertools

import numpy as np

from .countsketch import countsketch_dense


def mode_sketches(factors, hs, ss, L: int):
    """C_n = S^(n) A^(n), each L x R, float64."""
    return [countsketch_dense(F, h, s, L) for F, h, s in zip(factors, hs, ss)]


def tensorsketch(factors, lam, hs, ss, L: int) -> np.ndarray:
    """Y = T M (L x R) via Eq. TA-formula, float64."""
    Cs = mode_sketches(factors, hs, ss, L)
    prod = np.ones((L, Cs[0].shape[1]), dtype=np.complex128)
    for C in Cs:
        prod *= np.fft.fft(C, axis=0)
    Y = np.real(np.fft.ifft(prod, axis=0))
    return Y * np.asarray(lam, dtype=np.float64)[None, :]


def tuples(dims):
    """All index tuples (i_1, ..., i_N), first mode fastest (the row order of
    the Khatri-Rao product used by ``khatri_rao``)."""
    for t in itertools.product(*[range(d) for d in reversed(dims)]):
        yield tuple(reversed(t))


def khatri_rao(factors) -> np.ndarray:
    """Explicit Khatri-Rao matrix: row for tuple (i_1..i_N) in ``tuples``
    order, column r = product over n of A^(n)[i_n, r]."""
    dims = [F.shape[0] for F in factors]
    R = factors[0].shape[1]
    rows = []
    for t in tuples(dims):
        v = np.ones(R, dtype=np.float64)
        for n, i in enumerate(t):
            v = v * np.asarray(factors[n][i], dtype=np.float64)
        rows.append(v)
    return np.array(rows)


def explicit_T(dims, hs, ss, L: int) -> np.ndarray:
    """The L x prod(dims) TensorSketch matrix: column of tuple i has the single
    entry S(i) = prod s_n(i_n) in row H(i) = (sum h_n(i_n)) mod L (0-based)."""
    cols = []
    for t in tuples(dims):
        H = sum(int(hs[n][i]) for n, i in enumerate(t)) % L
        S = 1
        for n, i in enumerate(t):
            S *= int(ss[n][i])
        c = np.zeros(L)
        c[H] = S
        cols.append(c)
    return np.array(cols).T


def circular_convolution(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Direct O(L^2) cyclic convolution (c)_l = sum_m a_m b_{(l - m) mod L}."""
    L = len(a)
    c = np.zeros(L, dtype=np.float64)
    for l in range(L):
        for m in range(L):
            c[l] += a[m] * b[(l - m) % L]
    return c
