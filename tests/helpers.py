"""Shared helpers of the GPU parity tests: move data, compare to the oracle."""
import numpy as np
import torch


def dev(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel_fro(got, want):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    d = np.linalg.norm(want)
    return np.linalg.norm(got - want) / (d if d > 0 else 1.0)


def colmajor_to_matrix(Y2, m, R, ld):
    """Column-major device buffer (R columns of ld) -> m x R numpy array."""
    return host(Y2).reshape(R, ld)[:, :m].T.astype(np.float64)


def pivots_well_separated(gaps, tol=1e-3):
    return bool(np.all(np.asarray(gaps) > tol))


def assert_sum_within_bound(got, want, abs_sum, nterms, u):
    """Entry by entry: |got - want| <= (nterms + 1) u sum|terms| (a recursive sum of
    nterms terms in unit roundoff u; the want side exact to float64), so that a
    dropped, doubled or sign-flipped term of any entry fails unless it is below the
    rounding of that entry."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    bound = (nterms + 1) * u * np.asarray(abs_sum, dtype=np.float64) + 1e-300
    bad = np.abs(got - want) > bound
    assert not bad.any(), (int(bad.sum()), float(np.max(np.abs(got - want) / bound)))
