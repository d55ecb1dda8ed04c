"""FP64 CPU oracle for the CountSketch interpolative decomposition.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
library under ``paper_1901_10559_gb300`` never imports it and shares no code,
tables or constants with it.

Every function is a plain, slow, readable statement of what the method
computes, in float64, following the paper (Malik & Becker, "Fast randomized
matrix and tensor interpolative decomposition using CountSketch"):

  draws.py        -- the sketching operators' random maps (Sec. 1.3, Remark 2)
                     from the counter-based draws specification
  countsketch.py  -- Y = S A for dense and CSR A, and the explicit S (Sec. 1.3)
  gaussian.py     -- the Gaussian stage Omega Y (Sec. 1.2.1) and the
                     bfloat16 rounding used by the mixed-precision path
  cpqr.py         -- Algorithm 1 (matrix ID via rank-K column-pivoted QR)
  tensorsketch.py -- Eq. TA-formula and the explicit TensorSketch (Sec. 1.3)
  idmethods.py    -- Algorithm 2 (matrix) and Algorithm 3 (tensor, with the
                     s-value update lambda_hat)
  errors.py       -- ID error evaluation (spectral norm, Gram identity
                     Eq. MTM-formula for CP tensors)
  proposal.py     -- the learned column proposal for the QR stage: column
                     features, the scoring MLP (forward, backward, Adam),
                     top-C candidates and the certificate

Parity status: every function is pinned by tests in ``tests/test_oracle_*``
(closed forms, invariants, brute force, independent library routines).  The
exact skeleton set J under near-tied pivots is not unique; there only the ID
error is compared ("parity unpinned" for J under near ties).
"""
