"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the tests, the bench and the oracle's callers.  It
holds NONE of the method's arithmetic: no CountSketch, no Gaussian stage, no
pivoted QR, no TensorSketch, no draws of the sketching operators (those are
drawn by each side from the counter-based generator defined in the draws
specification).  It only builds the matrices and CP tensors that the method is
applied to, with numpy's PCG64 generator.

Workloads (sizes follow the paper's experiments, Sec. 6):
  * ``lowrank_dense``   -- A = U diag(sigma) V^T + noise, U, V Haar-orthonormal
                           (Mezzadri's sign-fixed QR of a Gaussian matrix).
  * ``sparse_plus_lowrank_csr`` -- sparse uniform-position N(0,1) entries plus
                           a scaled rank-r dense term on a fraction of the rows,
                           stored as CSR with sorted, de-duplicated columns
                           (Sec. 6.1.1 uses sparse synthetic matrices).
  * ``gaussian_lowrank_dense`` -- A = G1 G2^T + E with ||E||_F fixed relative to
                           ||G1 G2^T||_F.
  * ``cp_factors``      -- N(0,1) factor matrices with unit-norm columns and a
                           given s-value schedule (Eq. def-X-tensor, Sec. 1.1).
"""
from __future__ import annotations

import dataclasses

import numpy as np

__all__ = [
    "CSR",
    "haar_orthonormal",
    "lowrank_dense",
    "sparse_plus_lowrank_csr",
    "gaussian_lowrank_dense",
    "cp_factors",
    "random_csr",
    "batch_matrix_specs",
]


@dataclasses.dataclass
class CSR:
    """Compressed sparse row matrix: int64 rowptr, int32 colidx, values."""

    rowptr: np.ndarray
    colidx: np.ndarray
    vals: np.ndarray
    shape: tuple

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def haar_orthonormal(n: int, p: int, rng: np.random.Generator) -> np.ndarray:
    """n x p matrix with Haar-distributed orthonormal columns.

    QR of an n x p standard Gaussian matrix, with the columns' signs fixed so
    that diag(R) > 0 (Mezzadri 2007, "How to generate random matrices from the
    classical compact groups").
    """
    g = rng.standard_normal((n, p))
    q, r = np.linalg.qr(g)
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d[None, :]


def lowrank_dense(I: int, R: int, decay: float, noise: float, seed: int,
                  dtype=np.float64, rank: int | None = None) -> np.ndarray:
    """A = U diag(sigma) V^T + noise * N(0,1), sigma_i = decay**i (i = 1..).

    ``rank`` limits the number of nonzero singular values (default min(I, R)).
    Row-major (C-contiguous) output in ``dtype``.
    """
    rng = _rng(seed)
    p = min(I, R) if rank is None else rank
    U = haar_orthonormal(I, p, rng)
    V = haar_orthonormal(R, p, rng)
    sig = decay ** np.arange(1, p + 1, dtype=np.float64)
    A = (U * sig[None, :]) @ V.T
    if noise:
        A += noise * rng.standard_normal((I, R))
    return np.ascontiguousarray(A.astype(dtype))


def gaussian_lowrank_dense(I: int, R: int, rank: int, rel_noise: float, seed: int,
                           dtype=np.float32, block: int = 8192) -> np.ndarray:
    """A = G1 G2^T + E, G1 (I x rank), G2 (R x rank) N(0,1), E Gaussian with
    ||E||_F = rel_noise * ||G1 G2^T||_F.  Built in row blocks to bound memory."""
    rng = _rng(seed)
    G1 = rng.standard_normal((I, rank)).astype(np.float32)
    G2 = rng.standard_normal((R, rank)).astype(np.float32)
    A = np.empty((I, R), dtype=dtype)
    # ||G1 G2^T||_F^2 = trace((G1^T G1)(G2^T G2))
    fro2 = float(np.sum((G1.T.astype(np.float64) @ G1) * (G2.T.astype(np.float64) @ G2)))
    sd = rel_noise * np.sqrt(fro2 / (I * R))
    for r0 in range(0, I, block):
        r1 = min(I, r0 + block)
        blk = G1[r0:r1] @ G2.T
        blk += (sd * rng.standard_normal((r1 - r0, R))).astype(np.float32)
        A[r0:r1] = blk
    return A


def random_csr(I: int, R: int, density: float, seed: int, dtype=np.float32) -> CSR:
    """Uniform random positions, N(0,1) values; duplicates summed, columns sorted."""
    rng = _rng(seed)
    counts = rng.binomial(R, density, size=I).astype(np.int64)
    n = int(counts.sum())
    rows = np.repeat(np.arange(I, dtype=np.int64), counts)
    cols = rng.integers(0, R, size=n, dtype=np.int64)
    vals = rng.standard_normal(n)
    return _coo_to_csr(rows, cols, vals, I, R, dtype)


def _coo_to_csr(rows, cols, vals, I, R, dtype) -> CSR:
    key = rows * R + cols
    order = np.argsort(key, kind="stable")
    key = key[order]
    vals = vals[order]
    uk, start = np.unique(key, return_index=True)
    summed = np.add.reduceat(vals, start) if len(vals) else vals
    r = uk // R
    c = uk % R
    rowptr = np.zeros(I + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    return CSR(rowptr, c.astype(np.int32), summed.astype(dtype), (I, R))


def sparse_plus_lowrank_csr(I: int, R: int, density: float, rank: int, scale: float,
                            dense_frac: float, seed: int, dtype=np.float32) -> CSR:
    """Sparse N(0,1) matrix at ``density`` plus ``scale * U V^T / sqrt(rank)``
    (U, V N(0,1)) on a uniformly chosen ``dense_frac`` of the rows.

    The dense rows are stored fully (all R columns); the sparse entries that fall
    on them are added in.  Columns are sorted within each row.
    """
    rng = _rng(seed)
    sp = random_csr(I, R, density, seed + 7919, dtype=np.float64)
    nd = int(round(dense_frac * I))
    drows = np.sort(rng.choice(I, size=nd, replace=False)).astype(np.int64)
    U = rng.standard_normal((nd, rank))
    V = rng.standard_normal((R, rank))
    D = (scale / np.sqrt(rank)) * (U @ V.T)          # nd x R, float64
    # add the sparse entries of the dense rows into D
    for j, r in enumerate(drows):
        a, b = sp.rowptr[r], sp.rowptr[r + 1]
        if b > a:
            D[j, sp.colidx[a:b]] += sp.vals[a:b]
    isdense = np.zeros(I, dtype=bool)
    isdense[drows] = True
    counts = np.diff(sp.rowptr)
    counts[isdense] = R
    rowptr = np.zeros(I + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(counts)
    nnz = int(rowptr[-1])
    colidx = np.empty(nnz, dtype=np.int32)
    vals = np.empty(nnz, dtype=dtype)
    # sparse rows: contiguous copy of their entries
    sp_row_of = np.repeat(np.arange(I, dtype=np.int64), np.diff(sp.rowptr))
    keep = ~isdense[sp_row_of]
    src = np.nonzero(keep)[0]
    dst = rowptr[sp_row_of[src]] + (src - sp.rowptr[sp_row_of[src]])
    colidx[dst] = sp.colidx[src]
    vals[dst] = sp.vals[src].astype(dtype)
    ar = np.arange(R, dtype=np.int32)
    for j, r in enumerate(drows):
        a = rowptr[r]
        colidx[a:a + R] = ar
        vals[a:a + R] = D[j].astype(dtype)
    return CSR(rowptr, colidx, vals, (I, R))


def cp_factors(dims, R: int, seed: int, lam=None, dtype=np.float32):
    """CP tensor in the form of Eq. def-X-tensor: factor matrices A^(n) (I_n x R)
    with N(0,1) entries, columns scaled to unit 2-norm, and s-values ``lam``.

    Returns (factors, lam) with factors[n] of shape (I_n, R) in ``dtype`` and lam
    float64 of length R.  ``lam`` defaults to 0.9**r, r = 1..R.
    """
    rng = _rng(seed)
    facs = []
    for In in dims:
        F = rng.standard_normal((In, R))
        F /= np.linalg.norm(F, axis=0, keepdims=True)
        facs.append(np.ascontiguousarray(F.astype(dtype)))
    if lam is None:
        lam = 0.9 ** np.arange(1, R + 1, dtype=np.float64)
    return facs, np.asarray(lam, dtype=np.float64)


def batch_matrix_specs(n: int, seed: int):
    """Uneven batch of low-rank problems: rows log-uniform in [2048, 65536],
    cols log-uniform in [256, 2048], rank r ~ U{8..64}, decay d ~ U[0.7, 0.95].
    Returns a list of dicts (I, R, rank, decay, seed)."""
    rng = _rng(seed)
    out = []
    for b in range(n):
        I = int(round(np.exp(rng.uniform(np.log(2048), np.log(65536)))))
        R = int(round(np.exp(rng.uniform(np.log(256), np.log(2048)))))
        r = int(rng.integers(8, 65))
        d = float(rng.uniform(0.7, 0.95))
        out.append(dict(I=I, R=R, rank=r, decay=d, seed=int(seed * 1000 + b)))
    return out


def batch_dense_item(spec: dict, seed: int, dtype=np.float32) -> np.ndarray:
    """One dense matrix of the batched workload (numpy, host): A = U diag(sigma) V^T
    + noise with U (I x r), V (R x r) N(0,1) scaled by 1/sqrt(I), 1/sqrt(R),
    sigma_i = d^i (i = 1..r) and N(0,1) noise of scale 1e-6 d / sqrt(max(I, R)).
    The GPU bench draws the same recipe with torch on the device."""
    rng = _rng(seed)
    I, R, r, d = spec["I"], spec["R"], spec["rank"], spec["decay"]
    U = rng.standard_normal((I, r)) / np.sqrt(I)
    V = rng.standard_normal((R, r)) / np.sqrt(R)
    sig = d ** np.arange(1, r + 1, dtype=np.float64)
    A = (U * sig[None, :]) @ V.T
    A += (1e-6 * d / np.sqrt(max(I, R))) * rng.standard_normal((I, R))
    return np.ascontiguousarray(A.astype(dtype))


def batch_cp_lambda(R: int, K: int) -> np.ndarray:
    """s-values of a CP item of the batched workload: 10^(-6 r / K) for r < K
    (0-based), 1e-6 beyond (a paper-shaped decay to the target rank K)."""
    r = np.arange(R, dtype=np.float64)
    return np.where(r < K, 10.0 ** (-6.0 * r / K), 1e-6)


def batch_cp_item(b: int, seed: int, dims=(200, 200, 200, 200), R: int = 5000):
    """CP item b of the batched workload (numpy, host): N(0,1) unit-norm factor
    columns, K cycling over (16, 32, 48, 64), s-values batch_cp_lambda(R, K).
    Returns (factors (I_n x R each, float32), lam, K)."""
    K = (16, 32, 48, 64)[b % 4]
    facs, lam = cp_factors(dims, R, seed=seed, lam=batch_cp_lambda(R, K))
    return facs, lam, K
