"""The device ID error estimate (Sec. 6: power method on E^T E, E = A - A_J P)
against the oracle's power method from the same counter-based start vector,
and against the exact spectral norm at small sizes."""
import numpy as np
import pytest
import torch

import paper_1901_10559_gb300 as idl
from oracle import errors as oer
from synth import lowrank_dense, random_csr
from tests.helpers import dev, host

pytestmark = pytest.mark.gpu


def _id(ctx, A, K, m1, m2, prec):
    R = A.shape[1]
    J = torch.empty(K, dtype=torch.int32, device="cuda")
    T = torch.empty(K * (R - K), dtype=torch.float64, device="cuda")
    idl.id_matrix(ctx, dev(A), K, idl.make_params(m1, m2, seed=5, modified=True, precision=prec), J, T)
    return J, T


@pytest.mark.parametrize("dtype,I,R,K", [("f64", 3000, 400, 15), ("f32", 5003, 777, 21), ("f32", 700, 65, 40)])
def test_dense_estimate_matches_the_oracle_power_method(ctx, dtype, I, R, K):
    npdt = np.float64 if dtype == "f64" else np.float32
    A = lowrank_dense(I, R, 0.85, 1e-6, seed=I, dtype=npdt)
    J, T = _id(ctx, A, K, min(10 * K, I // 2), K + 10, idl.PREC_FP64 if dtype == "f64" else idl.PREC_FP32)
    got = idl.idl_id_error(ctx, dev(A), J, T, K, iters=50, seed=1234)
    want = oer.matrix_id_error(A, J=host(J), T=host(T).reshape(K, R - K), exact=False, iters=50, seed=1234)
    assert abs(got - want) <= 1e-8 * want, (got, want)
    # host arrays give the same estimate
    got_h = idl.idl_id_error(ctx, A, host(J), host(T), K, iters=50, seed=1234)
    assert abs(got_h - got) <= 1e-12 * got


def test_csr_estimate_matches_the_oracle_power_method(ctx):
    c = random_csr(20000, 500, 0.01, seed=8)
    K = 30
    J = torch.empty(K, dtype=torch.int32, device="cuda")
    T = torch.empty(K * (500 - K), dtype=torch.float64, device="cuda")
    idl.id_matrix_csr(ctx, dev(c.rowptr), dev(c.colidx), dev(c.vals), c.shape, K,
                      idl.make_params(400, 60, seed=2, modified=True, precision=idl.PREC_FP32), J, T)
    got = idl.idl_id_error_csr(ctx, dev(c.rowptr), dev(c.colidx), dev(c.vals), c.shape, J, T, K, iters=30, seed=77)
    want = oer.matrix_id_error(csr=(c.rowptr, c.colidx, c.vals, c.shape), J=host(J),
                               T=host(T).reshape(K, 500 - K), iters=30, seed=77)
    assert abs(got - want) <= 1e-8 * want, (got, want)


def test_estimate_never_exceeds_the_exact_norm_ratio_at_small_sizes(ctx):
    A = lowrank_dense(300, 80, 0.7, 1e-4, seed=3)
    K = 10
    J, T = _id(ctx, A, K, 60, 20, idl.PREC_FP64)
    Jh, Th = host(J), host(T).reshape(K, 80 - K)
    exact_num = np.linalg.norm(A - A[:, Jh] @ np.hstack([np.eye(K), Th])[:, np.argsort(
        np.concatenate([Jh, np.setdiff1d(np.arange(80), Jh)]))], 2)
    exact = exact_num / np.linalg.norm(A, 2)
    assert abs(exact - oer.matrix_id_error(A, J=Jh, T=Th, exact=True)) <= 1e-12 * exact
    est = idl.idl_id_error(ctx, dev(A), J, T, K, iters=200, seed=9)
    # the numerator is never overestimated, the denominator converges from below:
    # the ratio lies within a small band around the exact value after 200 steps
    assert 0.9 * exact <= est <= 1.01 * exact, (est, exact)
