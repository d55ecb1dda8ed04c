"""Gaussian ID comparators on the GPU (Sec. 1.2.1; Sec. 1.2.2 Eq. G-matrix) against
the oracle's Gaussian ID: pivots where every oracle pivot step is well
separated, T to the working precision, and the ID error within 1.1x the
oracle's."""
import numpy as np
import pytest
import torch

import paper_1901_10559_gb300 as idl
from oracle import errors as oer
from oracle import gaussian_id as ogid
from synth import cp_factors, lowrank_dense
from tests.helpers import dev, host, pivots_well_separated

pytestmark = pytest.mark.gpu

RATIO = 1.1


@pytest.mark.parametrize("dtype,I,R,K,L", [("f64", 1500, 300, 12, 22), ("f32", 3001, 517, 13, 40),
                                           ("f32", 700, 129, 30, 64)])
def test_gaussian_matrix_id(ctx, dtype, I, R, K, L):
    npdt = np.float64 if dtype == "f64" else np.float32
    A = lowrank_dense(I, R, 0.8, 1e-8, seed=7 + I, dtype=npdt)
    prec = idl.PREC_FP64 if dtype == "f64" else idl.PREC_FP32
    p = idl.make_params(0, L, seed=23, modified=False, precision=prec)
    J = torch.empty(K, dtype=torch.int32, device="cuda")
    T = torch.empty(K * (R - K), dtype=torch.float64, device="cuda")
    info = idl.Info()
    idl.id_matrix_gaussian(ctx, dev(A), K, p, J, T, info)
    assert info.status in (idl.IDL_OK, idl.IDL_ERANK)
    Jw, Tw, iw = ogid.gaussian_id_matrix(A, k=K, L=L, seed=23)
    Jg, Tg = host(J), host(T).reshape(K, R - K)
    if pivots_well_separated(iw["gaps"]):
        assert np.array_equal(Jg, Jw)
        tol = 1e-7 if dtype == "f64" else 1e-2
        assert np.abs(Tg - Tw).max() <= tol * max(1.0, np.abs(Tw).max())
    e_g = oer.matrix_id_error(A, J=Jg, T=Tg)
    e_w = oer.matrix_id_error(A, J=Jw, T=Tw)
    assert e_g <= RATIO * e_w + 1e-14, (e_g, e_w)


@pytest.mark.parametrize("dims,R,K,L", [((40, 30, 20), 300, 16, 26), ((200,) * 4, 1000, 32, 42),
                                        ((7, 300), 65, 8, 18)])
def test_gaussian_tensor_id(ctx, dims, R, K, L):
    facs, lam = cp_factors(dims, R, seed=R + len(dims), lam=10.0 ** (-6.0 * np.minimum(np.arange(R), K) / K))
    p = idl.make_params(0, L, seed=31, modified=False, precision=idl.PREC_FP32)
    J = torch.empty(K, dtype=torch.int32, device="cuda")
    T = torch.empty(K * (R - K), dtype=torch.float64, device="cuda")
    lh = torch.empty(K, dtype=torch.float64, device="cuda")
    fd = [dev(np.ascontiguousarray(F.T)) for F in facs]
    idl.id_cp_tensor_gaussian(ctx, fd, dev(lam), K, p, J, T, lh)
    Jw, Tw, lhw, iw = ogid.gaussian_id_tensor(facs, lam, k=K, L=L, seed=31)
    Jg = host(J)
    if pivots_well_separated(iw["gaps"]):
        assert np.array_equal(Jg, Jw)
        assert np.allclose(host(lh), lhw, rtol=1e-3, atol=1e-9)
    e_g = oer.tensor_id_error(facs, lam, Jg, host(lh))
    e_w = oer.tensor_id_error(facs, lam, Jw, lhw)
    assert e_g <= RATIO * e_w + 1e-7, (e_g, e_w)
    assert ctx.sync() == idl.IDL_OK


def test_gaussian_id_argument_errors(ctx):
    A = dev(np.zeros((100, 20), np.float32))
    J = torch.empty(5, dtype=torch.int32, device="cuda")
    T = torch.empty(5 * 15, dtype=torch.float64, device="cuda")
    for L, K in [(4, 5), (300, 5)]:                                   # L < K; L above the limit
        with pytest.raises(idl.IdlError):
            idl.id_matrix_gaussian(ctx, A, K, idl.make_params(0, L, 1, precision=idl.PREC_FP32), J, T)
