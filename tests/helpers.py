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
