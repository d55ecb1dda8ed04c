"""Failure detection without a GPU fault: a bounded device wait that is made to
run out.  The probe kernel waits, through the same bounded mbarrier wait as the
tensor-core Gaussian stage, for a phase that completes only if the host asks
for the arrival; without it the wait gives up after a short limit, the kernel
records IDL_ETIMEOUT and returns.  Nothing traps, faults or hangs."""
import time

import numpy as np
import pytest
import torch

import paper_1901_10559_gb300 as idl
from synth import lowrank_dense
from tests.helpers import dev

pytestmark = pytest.mark.gpu


def _small_id(ctx):
    A = lowrank_dense(2000, 300, 0.8, 1e-6, seed=1, dtype=np.float32)
    J = torch.empty(10, dtype=torch.int32, device="cuda")
    T = torch.empty(10 * 290, dtype=torch.float64, device="cuda")
    p = idl.make_params(200, 20, seed=1, modified=True, precision=idl.PREC_FP32)
    idl.id_matrix(ctx, dev(A), 10, p, J, T)
    return J


def test_bounded_wait_completes_when_the_phase_arrives():
    c = idl.Context(0)
    assert idl.lib().idl_debug_wait_probe(c.ptr, 1, 1_000_000) == idl.IDL_OK
    assert c.sync() == idl.IDL_OK
    _small_id(c)
    assert c.sync() == idl.IDL_OK
    c.close()


def test_bounded_wait_expires_poisons_the_context_and_a_new_one_works():
    c = idl.Context(0)
    t0 = time.perf_counter()
    assert idl.lib().idl_debug_wait_probe(c.ptr, 0, 2_000_000) == idl.IDL_OK      # 2 ms limit
    assert c.sync() == idl.IDL_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    # the context refuses further work: a timed-out tensor-core stage may leave work in flight
    assert idl.lib().idl_debug_wait_probe(c.ptr, 1, 1_000_000) == idl.IDL_ETIMEOUT
    with pytest.raises(idl.IdlError) as ei:
        _small_id(c)
    assert ei.value.code == idl.IDL_ETIMEOUT
    c.close()
    # the GPU context itself is intact: a new library context runs a pipeline cleanly
    c2 = idl.Context(0)
    J = _small_id(c2)
    assert c2.sync() == idl.IDL_OK
    assert len(set(J.cpu().tolist())) == 10
    c2.close()


def test_wait_probe_rejects_limits_outside_one_microsecond_to_one_second(ctx):
    assert idl.lib().idl_debug_wait_probe(ctx.ptr, 0, 10) == idl.IDL_EINVAL
    assert idl.lib().idl_debug_wait_probe(ctx.ptr, 0, 5_000_000_000) == idl.IDL_EINVAL
