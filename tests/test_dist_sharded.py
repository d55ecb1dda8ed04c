"""Sharded IDs (paper_1901_10559_gb300.sharded) with two gloo ranks on CPU: a
matrix split by rows (all-reduce) and a CP tensor split by columns (all-gather).

Each rank holds a contiguous block of rows; its partial sketch is
Omega S[:, B] A[B, :] with the maps of the whole matrix; one all-reduce sums the
partial sketches and every rank runs Algorithm 1 on the sum.  On CPU the partial
sketch and the ID of the sketch are the oracle's (passed in), so the test checks
the partition, the block slicing, the all-reduce and that the summed sketch and
the resulting J, T equal the oracle's for the whole matrix (Sec. 1.3: the sketch
is linear in the rows)."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
I, R, K, M1, M2, SEED = 6000, 300, 12, 400, 30, 77


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from oracle import countsketch as ocs
    from oracle import cpqr as ocp
    from oracle import draws as odr
    from oracle import gaussian as ogs
    from paper_1901_10559_gb300 import sharded
    from synth import sparse_plus_lowrank_csr

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        c = sparse_plus_lowrank_csr(I, R, 0.02, rank=8, scale=5.0, dense_frac=0.05, seed=3)
        i0, i1 = sharded.row_blocks(I, ws)[rank]
        # float64 values: the summed sketch is then compared in float64
        rp, ci, v = sharded.csr_row_block(c.rowptr, c.colidx, c.vals.astype(np.float64), i0, i1)
        h, s = odr.countsketch_maps(SEED, I, M1, True)          # the whole matrix's maps
        Om = odr.gaussian_matrix(SEED, M2, M1)

        def sketch_rows(blk, i0_, I_, params_, Y2):
            rp_, ci_, v_ = blk
            n = rp_.shape[0] - 1
            Y1 = ocs.countsketch_csr(rp_, ci_, v_, R, h[i0_:i0_ + n], s[i0_:i0_ + n], M1)
            Y2.copy_(torch.from_numpy(np.ascontiguousarray(ogs.gaussian_stage(Om, Y1, ogs.FP64).T).ravel()))

        def id_from_sketch(Y2, m, R_, K_, params_, J, T):
            Jw, Tw, _ = ocp.matrix_id(Y2.numpy().reshape(R_, m).T, K_)
            J[:] = Jw
            T[:] = Tw.ravel()

        params = type("P", (), {"m1": M1, "m2": M2})()
        J = np.empty(K, np.int64)
        T = np.empty(K * (R - K))
        Y2 = sharded.sharded_id((rp, ci, v), i0, I, R, K, params, J, T, sketch_rows=sketch_rows,
                                id_from_sketch=id_from_sketch)
        q.put((rank, (i0, i1), Y2.numpy().copy(), J.copy(), T.copy()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_sum_to_the_whole_matrix_sketch_and_id():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(2):
        rank, *rest = q.get(timeout=120)
        out[rank] = rest
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sys.path.insert(0, ROOT)
    from oracle import idmethods as oid
    from oracle.gaussian import FP64
    from synth import sparse_plus_lowrank_csr
    c = sparse_plus_lowrank_csr(I, R, 0.02, rank=8, scale=5.0, dense_frac=0.05, seed=3)
    Jw, Tw, iw = oid.id_matrix(csr=(c.rowptr, c.colidx, c.vals.astype(np.float64), c.shape), k=K, m1=M1, m2=M2,
                               seed=SEED,
                               modified=True, precision=FP64)
    want = iw["Y2"]
    assert out[0][0] == (0, I // 2) and out[1][0] == (I // 2, I)
    for rank in (0, 1):
        _, Y2, J, T = out[rank]
        got = Y2.reshape(R, M2).T
        assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)
        assert np.array_equal(J, Jw)
        assert np.abs(T - Tw.ravel()).max() <= 1e-9 * max(1.0, np.abs(Tw).max())


def test_row_blocks_partition_and_csr_slices():
    sys.path.insert(0, ROOT)
    from paper_1901_10559_gb300 import sharded
    from synth import random_csr
    for I_, w in [(10, 3), (7, 7), (1000, 4)]:
        b = sharded.row_blocks(I_, w)
        assert b[0][0] == 0 and b[-1][1] == I_
        assert all(b[g][1] == b[g + 1][0] for g in range(w - 1))
        assert max(x[1] - x[0] for x in b) - min(x[1] - x[0] for x in b) <= 1
    c = random_csr(50, 20, 0.2, seed=1)
    rp, ci, v = sharded.csr_row_block(c.rowptr, c.colidx, c.vals, 10, 30)
    assert rp[0] == 0 and rp.shape[0] == 21
    assert np.array_equal(ci, c.colidx[c.rowptr[10]:c.rowptr[30]])
    assert np.array_equal(rp, c.rowptr[10:31] - c.rowptr[10])


DIMS, RC, KC, LC, M2C = (30, 40, 25), 301, 10, 256, 24


def _cp_worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from oracle import cpqr as ocp
    from oracle import draws as odr
    from oracle import gaussian as ogs
    from oracle import idmethods as oid
    from oracle import tensorsketch as ots
    from paper_1901_10559_gb300 import sharded
    from synth import cp_factors

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        factors, lam = cp_factors(DIMS, RC, seed=4, dtype=np.float64)
        c0, c1 = sharded.column_blocks(RC, ws)[rank]
        mine = [torch.from_numpy(np.ascontiguousarray(F[:, c0:c1].T)) for F in factors]   # (columns, I_n)
        hs, ss = odr.tensorsketch_maps(SEED, DIMS, LC)
        Om = odr.gaussian_matrix(SEED, M2C, LC)

        def sketch_cols(f_, lam_, params_, Y2_):
            Fs = [t.numpy().T for t in f_]
            Y = ots.tensorsketch(Fs, lam_, hs, ss, LC)
            Y2_[:Y.shape[1] * M2C] = torch.from_numpy(np.ascontiguousarray((Om @ Y).T).ravel()).to(Y2_.dtype)

        def id_from_sketch(Y2_, m_, R_, K_, params_, J_, T_):
            Jw, Tw, _ = ocp.matrix_id(Y2_.double().numpy().reshape(R_, m_).T, K_)
            J_[:] = Jw
            T_[:] = Tw.ravel()

        def lambda_hat(lam_, J_, T_, K_, R_, out_):
            out_[:] = oid.lambda_hat(lam_, J_, T_.reshape(K_, R_ - K_))

        params = type("P", (), {"m1": LC, "m2": M2C})()
        J = np.empty(KC, np.int64)
        T = np.empty(KC * (RC - KC))
        lh = np.empty(KC)
        Y2 = sharded.sharded_cp_id(mine, lam[c0:c1], lam, RC, KC, params, J, T, lh, sketch_cols=sketch_cols,
                                   id_from_sketch=id_from_sketch, lambda_hat=lambda_hat)
        q.put((rank, (c0, c1), Y2.double().numpy().copy(), J.copy(), T.copy(), lh.copy()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_gather_cp_column_blocks_to_the_whole_tensor_id():
    """Column blocks of a CP tensor sketched apart and gathered give the whole
    tensor's sketch (FP32 pieces: 2^-24 relative per entry), and Algorithm 3 on
    it gives the oracle's J, T and lambda_hat for the whole tensor."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_cp_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(2):
        rank, *rest = q.get(timeout=120)
        out[rank] = rest
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sys.path.insert(0, ROOT)
    from oracle import idmethods as oid
    from synth import cp_factors
    factors, lam = cp_factors(DIMS, RC, seed=4, dtype=np.float64)
    Jw, Tw, lw, info = oid.id_cp_tensor(factors, lam, k=KC, L=LC, m2=M2C, seed=SEED)
    want = info["Y2"]
    assert out[0][0] == (0, RC // 2) and out[1][0] == (RC // 2, RC)
    for rank in (0, 1):
        _, Y2, J, T, lh = out[rank]
        got = Y2.reshape(RC, M2C).T
        assert np.abs(got - want).max() <= 2.0 ** -23 * np.abs(want).max()
        assert np.array_equal(J, Jw)
        assert np.abs(T - Tw.ravel()).max() <= 1e-4 * max(1.0, np.abs(Tw).max())
        assert np.allclose(lh, lw, rtol=1e-4, atol=0)
