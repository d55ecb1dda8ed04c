"""The strong rank-revealing exchanges (Fact 1; Gu & Eisenstat 1996) on the GPU
against the oracle's: Kahan's matrix (columns scaled by (1 - 1e-3)^j, so that
column pivoting takes them in order with a clear margin at every step), on
which column pivoting leaves |T| in the thousands and one exchange repairs it;
Kahan-type matrices with a tight f; and the pipelines with params.srrqr_f."""
import numpy as np
import pytest
import torch

import paper_1901_10559_gb300 as idl
from oracle import errors as oer
from oracle import idmethods as oid
from oracle import srrqr as osr
from oracle.gaussian import FP32, FP64
from synth import lowrank_dense
from tests.helpers import dev, host, pivots_well_separated

pytestmark = pytest.mark.gpu


def kahan(n, theta, eps=1e-3):
    s, c = np.sin(theta), np.cos(theta)
    U = np.eye(n) - c * np.triu(np.ones((n, n)), 1)
    return np.diag(s ** np.arange(n)) @ U @ np.diag((1.0 - eps) ** np.arange(n))


def _run(ctx, Y, K, f, dtype):
    m, R = Y.shape
    Yd = dev(np.ascontiguousarray(Y.T).astype(np.float64 if dtype == idl.IDL_F64 else np.float32))   # column-major
    J = torch.empty(K, dtype=torch.int32, device="cuda")
    T = torch.empty(K * (R - K), dtype=torch.float64, device="cuda")
    idl.idl_cpqr_srrqr(ctx, Yd, m, R, m, dtype, K, f, J, T)
    return host(J), host(T).reshape(K, R - K)


@pytest.mark.parametrize("n,theta,dtype", [(30, 1.2, idl.IDL_F64), (40, 1.0, idl.IDL_F64), (30, 1.2, idl.IDL_F32)])
def test_kahan_matrix_exchange(ctx, n, theta, dtype):
    A = kahan(n, theta)
    K = n - 1
    Jw, Tw, info = osr.srrqr_id(A, K, f=2.0)
    assert len(info["swaps"]) >= 1
    Jg, Tg = _run(ctx, A, K, 2.0, dtype)
    assert np.array_equal(Jg, Jw)
    tol = 1e-9 if dtype == idl.IDL_F64 else 1e-3
    assert np.abs(Tg - Tw).max() <= tol * max(1.0, np.abs(Tw).max())
    assert np.abs(Tg).max() <= 2.0 * (1 + 1e-4)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_tight_f_matches_the_oracle_criterion(ctx, seed):
    """f = 1.05 on Kahan-type matrices plus noise: the GPU's final selection satisfies
    the oracle's FP64 criterion (no rho above f^2 beyond rounding) and, where the
    pivoted QR's steps and every exchange were decided with a clear margin, equals
    the oracle's."""
    rng = np.random.default_rng(seed)
    A = kahan(24, 1.0 + 0.1 * seed) + 1e-6 * rng.standard_normal((24, 24))
    A = np.vstack([A, 1e-4 * rng.standard_normal((8, 24))])
    K = 12
    Jg, Tg = _run(ctx, A, K, 1.05, idl.IDL_F64)
    c = osr.criterion(A, Jg)
    assert c["rho"].max() <= 1.05 ** 2 * (1 + 1e-5)
    Jw, Tw, info = osr.srrqr_id(A, K, f=1.05)
    if pivots_well_separated(info["gaps"]) and all(abs(r - 1.05 ** 2) > 1e-3 for _, _, r in info["swaps"]):
        assert np.array_equal(Jg, Jw)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_pipeline_with_srrqr(ctx, dtype):
    npdt = np.float64 if dtype == "f64" else np.float32
    A = lowrank_dense(3000, 400, 0.85, 1e-8, seed=11, dtype=npdt)
    K, m1, m2 = 20, 300, 30
    prec = idl.PREC_FP64 if dtype == "f64" else idl.PREC_FP32
    p = idl.make_params(m1, m2, seed=3, modified=True, precision=prec, srrqr_f=2.0)
    J = torch.empty(K, dtype=torch.int32, device="cuda")
    T = torch.empty(K * (400 - K), dtype=torch.float64, device="cuda")
    info = idl.Info()
    idl.id_matrix(ctx, dev(A), K, p, J, T, info)
    Jg, Tg = host(J), host(T).reshape(K, 400 - K)
    assert np.abs(Tg).max() <= 2.0 * (1 + 1e-3)
    _, _, iw = oid.id_matrix(A, k=K, m1=m1, m2=m2, seed=3, modified=True,
                             precision=FP64 if dtype == "f64" else FP32)
    Jw, Tw, _ = osr.srrqr_id(iw["Y2"], K, f=2.0)
    e_g = oer.matrix_id_error(A, J=Jg, T=Tg)
    e_w = oer.matrix_id_error(A, J=Jw, T=Tw)
    assert e_g <= 1.1 * e_w + 1e-14, (e_g, e_w)


def test_srrqr_argument_errors(ctx):
    A = dev(np.zeros((100, 20), np.float32))
    J = torch.empty(5, dtype=torch.int32, device="cuda")
    T = torch.empty(5 * 15, dtype=torch.float64, device="cuda")
    with pytest.raises(idl.IdlError):
        idl.id_matrix(ctx, A, 5, idl.make_params(10, 8, 1, precision=idl.PREC_FP32, srrqr_f=0.5), J, T)
    with pytest.raises(idl.IdlError):
        idl.id_matrix(ctx, A, 5, idl.make_params(10, 8, 1, precision=idl.PREC_FP32, srrqr_f=2.0,
                                                 learned=idl.PROPOSAL_NORM), J, T)
