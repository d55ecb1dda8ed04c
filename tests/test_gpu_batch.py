"""Batched IDs (one launch per stage over all items, QR clusters per item, CUDA
graph replay, first-call tuning) against the single-item calls and the oracle."""
import numpy as np
import pytest
import torch

import paper_1901_10559_gb300 as idl
from oracle import errors as oer
from oracle import idmethods as oid
from oracle.gaussian import BF16, BF16X3, FP32
from synth import cp_factors, lowrank_dense
from tests.helpers import dev, host

pytestmark = pytest.mark.gpu


def _dense_problems(seed):
    rng = np.random.default_rng(seed)
    probs = []
    for b, (I, R) in enumerate([(3000, 300), (5000, 700), (2048, 256), (7000, 1025), (4100, 513)]):
        r = int(rng.integers(8, 30))
        A = lowrank_dense(I, R, float(rng.uniform(0.7, 0.95)), 1e-6, seed=seed * 100 + b, dtype=np.float32, rank=r)
        m2 = r + 10
        probs.append(dict(A=A, K=r, m1=min(m2 * m2, I // 2), m2=m2, seed=1000 + b))
    return probs


def _cp_problems(seed):
    probs = []
    # L = 1024 (per-pair blocks) and L = 8192 (persistent blocks; one item with modes of
    # uneven size and an odd column count)
    for b, (dims, R, K, L) in enumerate([((40, 30, 20), 300, 16, 1024), ((50, 50, 50, 50), 501, 32, 8192),
                                         ((400, 30, 300), 257, 8, 8192)]):
        facs, lam = cp_factors(dims, R, seed=seed + b, lam=10.0 ** (-6.0 * np.minimum(np.arange(R), K) / K))
        probs.append(dict(facs=facs, lam=lam, K=K, L=L, m2=K + 10, seed=2000 + b))
    return probs


def _outputs(K, R, cp=False):
    J = torch.empty(K, dtype=torch.int32, device="cuda")
    T = torch.empty(K * (R - K), dtype=torch.float64, device="cuda")
    lh = torch.empty(K, dtype=torch.float64, device="cuda") if cp else None
    return J, T, lh


def _build(dense, cps, prec=idl.PREC_FP32, learned=(idl.PROPOSAL_NONE,)):
    items, outs, keep = [], [], []
    for b, pr in enumerate(dense):
        A = dev(pr["A"])
        J, T, _ = _outputs(pr["K"], pr["A"].shape[1])
        p = idl.make_params(pr["m1"], pr["m2"], seed=pr["seed"], modified=True, precision=prec,
                            learned=learned[b % len(learned)])
        items.append(idl.dense_item(A, pr["K"], p, J, T))
        outs.append((J, T, None))
        keep.append(A)
    for pr in cps:
        fd = [dev(np.ascontiguousarray(F.T)) for F in pr["facs"]]
        lam = dev(pr["lam"])
        R = pr["facs"][0].shape[1]
        J, T, lh = _outputs(pr["K"], R, cp=True)
        p = idl.make_params(pr["L"], pr["m2"], seed=pr["seed"], modified=False, precision=prec,
                            learned=learned[-1])
        items.append(idl.cp_item(fd, lam, pr["K"], p, J, T, lh))
        outs.append((J, T, lh))
        keep.append((fd, lam))
    return items, outs, keep


# the oracle's mode of each precision (TF32X3 has FP32's definition)
_ORACLE_PREC = {idl.PREC_FP32: FP32, idl.PREC_TF32X3: FP32, idl.PREC_BF16X3: BF16X3, idl.PREC_BF16: BF16}


# FP32, BF16X3 and BF16 take the pre-tiled operand planes for the L = 8192 CP item
# (R = 501: an odd last column and a partial last column tile); TF32X3 the FP32 sketch
@pytest.mark.parametrize("graph,tune,prec", [(0, 0, idl.PREC_FP32), (1, 1, idl.PREC_FP32), (1, 0, idl.PREC_TF32X3),
                                             (1, 1, idl.PREC_BF16X3), (0, 1, idl.PREC_BF16)])
def test_batch_matches_single_item_calls(ctx, graph, tune, prec):
    dense, cps = _dense_problems(3), _cp_problems(5)
    oprec = _ORACLE_PREC[prec]
    idl.lib().idl_debug_batch_mode(ctx.ptr, int(not graph), int(not tune))
    items, outs, keep = _build(dense, cps, prec=prec)
    for _ in range(2):                                   # second call replays the graph
        idl.idl_batch_run(ctx, items)
    assert ctx.sync() == idl.IDL_OK
    idl.lib().idl_debug_batch_mode(ctx.ptr, 0, 0)
    for pr, (J, T, _) in zip(dense, outs[:len(dense)]):
        K, R = pr["K"], pr["A"].shape[1]
        Js, Ts, _ = _outputs(K, R)
        p = idl.make_params(pr["m1"], pr["m2"], seed=pr["seed"], modified=True, precision=prec)
        idl.id_matrix(ctx, dev(pr["A"]), K, p, Js, Ts)
        assert np.array_equal(host(J), host(Js))
        # T agrees to FP32 rounding of the sketch amplified by cond(R11); the batch may split
        # the Gaussian product's K range differently, so compare the ID errors instead
        # and the oracle's error gate
        Jw, Tw, _ = oid.id_matrix(pr["A"], k=K, m1=pr["m1"], m2=pr["m2"], seed=pr["seed"], precision=oprec)
        e_g = oer.matrix_id_error(pr["A"], J=host(J), T=host(T).reshape(K, R - K), exact=False, iters=30)
        e_w = oer.matrix_id_error(pr["A"], J=Jw, T=Tw, exact=False, iters=30)
        assert e_g <= 1.1 * e_w + 1e-7
    for pr, (J, T, lh) in zip(cps, outs[len(dense):]):
        K, R = pr["K"], pr["facs"][0].shape[1]
        Js, Ts, lhs = _outputs(K, R, cp=True)
        p = idl.make_params(pr["L"], pr["m2"], seed=pr["seed"], modified=False, precision=prec)
        fd = [dev(np.ascontiguousarray(F.T)) for F in pr["facs"]]
        idl.id_cp_tensor(ctx, fd, dev(pr["lam"]), K, p, Js, Ts, lhs)
        assert np.array_equal(host(J), host(Js))
        assert np.allclose(host(lh), host(lhs), rtol=1e-3, atol=1e-9)
        Jw, Tw, lhw, _ = oid.id_cp_tensor(pr["facs"], pr["lam"], k=K, L=pr["L"], m2=pr["m2"], seed=pr["seed"],
                                          precision=oprec)
        e_g = oer.tensor_id_error(pr["facs"], pr["lam"], host(J), host(lh))
        e_w = oer.tensor_id_error(pr["facs"], pr["lam"], Jw, lhw)
        assert e_g <= 1.1 * e_w + 1e-7


def test_batch_graph_replay_reads_new_data(ctx):
    dense = _dense_problems(7)[:3]
    items, outs, keep = _build(dense, [])
    idl.idl_batch_run(ctx, items)                        # captures the graph
    # new contents in the same buffers: the replayed graph must see them
    for b, A in enumerate(keep):
        g = torch.Generator(device="cuda").manual_seed(b)
        perm = torch.randperm(A.shape[1], device="cuda", generator=g)
        A.copy_(A[:, perm].contiguous())
    idl.idl_batch_run(ctx, items)                        # replays it
    assert ctx.sync() == idl.IDL_OK
    for b, pr in enumerate(dense):
        K, R = pr["K"], pr["A"].shape[1]
        Js, Ts, _ = _outputs(K, R)
        p = idl.make_params(pr["m1"], pr["m2"], seed=pr["seed"], modified=True, precision=idl.PREC_FP32)
        idl.id_matrix(ctx, keep[b], K, p, Js, Ts)
        assert np.array_equal(host(outs[b][0]), host(Js))


def test_batch_tuning_save_load(ctx, tmp_path):
    dense = _dense_problems(11)[:2]
    items, outs, keep = _build(dense, [], prec=idl.PREC_BF16X3)
    idl.idl_batch_run(ctx, items)
    path = tmp_path / "tune.txt"
    idl.idl_tune_save(ctx, path)
    lines = [l for l in path.read_text().splitlines() if not l.startswith("#")]
    assert len(lines) >= 1
    c2 = idl.Context(0)
    idl.idl_tune_load(c2, path)
    J2, T2, _ = _outputs(dense[0]["K"], dense[0]["A"].shape[1])
    items2 = list(items)
    items2[0] = idl.dense_item(keep[0], dense[0]["K"], items[0].params, J2, T2)
    idl.idl_batch_run(c2, items2)
    assert c2.sync() == idl.IDL_OK
    assert np.array_equal(host(J2), host(outs[0][0]))
    c2.close()


@pytest.mark.parametrize("split,cs_dense,cap_dense,cap_cp", [(0, 16, 1024, 1024), (1, 8, 128, 320), (2, 4, 256, 512)])
def test_batch_forced_tunings(ctx, tmp_path, split, cs_dense, cap_dense, cap_cp):
    """Every choice the first-call tuner may make, forced through a tune file: the
    Gaussian stage's K split (0 = only as far as the whole batch needs), the dense QR
    cluster size and the QR thread caps.  Pivots match the tuned run's; the ID errors
    stay within 1.1x of it (the choices reorder roundings only)."""
    dense, cps = _dense_problems(13)[:3], _cp_problems(15)
    items, outs, keep = _build(dense, cps, prec=idl.PREC_BF16X3)
    idl.idl_batch_run(ctx, items)
    assert ctx.sync() == idl.IDL_OK
    path = tmp_path / "tune.txt"
    idl.idl_tune_save(ctx, path)
    key = [l for l in path.read_text().splitlines() if not l.startswith("#")][-1].split()[0]
    path.write_text(f"{key} 256 {split} {cs_dense} 16 {cap_dense} {cap_cp}\n")
    c2 = idl.Context(0)
    try:
        idl.idl_tune_load(c2, path)
        items2, outs2, keep2 = _build(dense, cps, prec=idl.PREC_BF16X3)
        idl.idl_batch_run(c2, items2)
        assert c2.sync() == idl.IDL_OK
    finally:
        c2.close()
    for pr, (J, T, _), (J2, T2, _) in zip(dense, outs, outs2):
        K, R = pr["K"], pr["A"].shape[1]
        assert np.array_equal(host(J2), host(J))
        e1 = oer.matrix_id_error(pr["A"], J=host(J), T=host(T).reshape(K, R - K), exact=False, iters=30)
        e2 = oer.matrix_id_error(pr["A"], J=host(J2), T=host(T2).reshape(K, R - K), exact=False, iters=30)
        assert e2 <= 1.1 * e1 + 1e-7
    for pr, (J, T, lh), (J2, T2, lh2) in zip(cps, outs[len(dense):], outs2[len(dense):]):
        assert np.array_equal(host(J2), host(J))
        e1 = oer.tensor_id_error(pr["facs"], pr["lam"], host(J), host(lh))
        e2 = oer.tensor_id_error(pr["facs"], pr["lam"], host(J2), host(lh2))
        assert e2 <= 1.1 * e1 + 1e-7


def test_batch_rejects_mixed_precision(ctx):
    dense = _dense_problems(13)[:2]
    items, outs, keep = _build(dense, [])
    items[1].params.precision = idl.PREC_BF16
    with pytest.raises(idl.IdlError) as ei:
        idl.idl_batch_run(ctx, items)
    assert ei.value.code == idl.IDL_EINVAL


@pytest.mark.parametrize("graph", [0, 1])
def test_batch_with_proposal_matches_plain(ctx, graph):
    """Items that take the column proposal (norm scores, MLP scores with random
    weights) get the plain QR's pivots and T, certified or through the gated
    fallback; the fallback count is reported."""
    from oracle import proposal as opr
    idl.idl_mlp_set_weights(ctx, opr.flatten(opr.init_params(3)).astype(np.float32))
    dense, cps = _dense_problems(7), _cp_problems(9)
    idl.lib().idl_debug_batch_mode(ctx.ptr, int(not graph), 1)
    items0, outs0, keep0 = _build(dense, cps)
    idl.idl_batch_run(ctx, items0)
    assert ctx.sync() == idl.IDL_OK
    modes = (idl.PROPOSAL_NORM, idl.PROPOSAL_NONE, idl.PROPOSAL_MLP)
    items1, outs1, keep1 = _build(dense, cps, learned=modes)
    for _ in range(2):
        idl.idl_batch_run(ctx, items1)
    assert ctx.sync() == idl.IDL_OK
    nfb = idl.idl_batch_fallbacks(ctx)
    idl.lib().idl_debug_batch_mode(ctx.ptr, 0, 0)
    nprop = sum(1 for b in range(len(dense)) if modes[b % 3] != idl.PROPOSAL_NONE) + len(cps)
    assert 0 <= nfb <= nprop
    for (J0, T0, l0), (J1, T1, l1) in zip(outs0, outs1):
        assert np.array_equal(host(J0), host(J1))
        # same sketch, same pivots; the factor rows differ by FP32 rounding (another
        # reduction layout), which T = R11^-1 R12 amplifies by cond(R11)
        t0, t1 = host(T0), host(T1)
        assert np.linalg.norm(t1 - t0) <= 1e-2 * np.linalg.norm(t0)
        if l0 is not None:
            assert np.allclose(host(l0), host(l1), rtol=1e-2, atol=1e-9)


def test_batch_host_arrays_match_device_arrays(ctx):
    """The same batch with every array in pinned host memory: idl_batch_run stages the
    inputs (the TensorSketch waits only for the CP factors, the dense sketch for each
    group of matrices) and copies the outputs back; results equal the device call's."""
    dense, cps = _dense_problems(17), _cp_problems(19)
    items, outs, keep = _build(dense, cps)
    idl.idl_batch_run(ctx, items)
    assert ctx.sync() == idl.IDL_OK
    hitems, houts = [], []
    for it, pr in zip(items[:len(dense)], dense):
        A = torch.from_numpy(pr["A"]).pin_memory()
        K, R = pr["K"], pr["A"].shape[1]
        J = torch.full((K,), -1, dtype=torch.int32).pin_memory()
        T = torch.empty(K * (R - K), dtype=torch.float64).pin_memory()
        hitems.append(idl.dense_item(A, K, it.params, J, T))
        houts.append((J, T, None, A))
    for it, pr in zip(items[len(dense):], cps):
        fs = [torch.from_numpy(np.ascontiguousarray(F.T)).pin_memory() for F in pr["facs"]]
        lam = torch.from_numpy(pr["lam"]).pin_memory()
        K, R = pr["K"], pr["facs"][0].shape[1]
        J = torch.full((K,), -1, dtype=torch.int32).pin_memory()
        T = torch.empty(K * (R - K), dtype=torch.float64).pin_memory()
        lh = torch.empty(K, dtype=torch.float64).pin_memory()
        hitems.append(idl.cp_item(fs, lam, K, it.params, J, T, lh))
        houts.append((J, T, lh, fs, lam))
    for _ in range(2):                                   # the second call reuses the staging buffer
        idl.idl_batch_run(ctx, hitems)
        for (Jd, Td, ld), (Jh, Th, lh, *_) in zip(outs, houts):
            assert np.array_equal(host(Jd), Jh.numpy())
            assert np.array_equal(host(Td), Th.numpy())
            if ld is not None:
                assert np.array_equal(host(ld), lh.numpy())
    assert ctx.sync() == idl.IDL_OK


@pytest.mark.parametrize("which", ["dense", "cp"])
def test_batch_host_arrays_single_kind(ctx, which):
    """Host-array batches of one kind only (the item groups are then the CP items alone,
    or the dense groups alone): results equal the device-array call's."""
    dense, cps = (_dense_problems(23)[:3], []) if which == "dense" else ([], _cp_problems(29))
    items, outs, keep = _build(dense, cps)
    idl.idl_batch_run(ctx, items)
    assert ctx.sync() == idl.IDL_OK
    hitems, houts = [], []
    for it, pr in zip(items[:len(dense)], dense):
        A = torch.from_numpy(pr["A"]).pin_memory()
        K, R = pr["K"], pr["A"].shape[1]
        J = torch.full((K,), -1, dtype=torch.int32).pin_memory()
        T = torch.empty(K * (R - K), dtype=torch.float64).pin_memory()
        hitems.append(idl.dense_item(A, K, it.params, J, T))
        houts.append((J, T, None, A))
    for it, pr in zip(items[len(dense):], cps):
        fs = [torch.from_numpy(np.ascontiguousarray(F.T)).pin_memory() for F in pr["facs"]]
        lam = torch.from_numpy(pr["lam"]).pin_memory()
        K, R = pr["K"], pr["facs"][0].shape[1]
        J = torch.full((K,), -1, dtype=torch.int32).pin_memory()
        T = torch.empty(K * (R - K), dtype=torch.float64).pin_memory()
        lh = torch.empty(K, dtype=torch.float64).pin_memory()
        hitems.append(idl.cp_item(fs, lam, K, it.params, J, T, lh))
        houts.append((J, T, lh, fs, lam))
    idl.idl_batch_run(ctx, hitems)
    for (Jd, Td, ld), (Jh, Th, lh, *_) in zip(outs, houts):
        assert np.array_equal(host(Jd), Jh.numpy())
        if which == "dense":       # the CP sketch's shared-memory atomics may reorder colliding entries
            assert np.array_equal(host(Td), Th.numpy())
        else:
            assert np.allclose(host(Td), Th.numpy(), rtol=1e-4, atol=1e-6)
            assert np.allclose(host(ld), lh.numpy(), rtol=1e-4, atol=1e-9)
    assert ctx.sync() == idl.IDL_OK
