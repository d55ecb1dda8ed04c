"""Sharded IDs over several GPUs, one process per GPU (torch.distributed): a
matrix split by rows (one all-reduce of the m x R sketch) and a CP tensor split
by columns (one all-gather of the m x R sketch).

The sketch is linear in the rows of A (Sec. 1.3):

    Omega S A = sum over ranks g of Omega S[:, B_g] A[B_g, :],

so every rank sketches its own contiguous block of rows B_g with the maps of the
whole matrix (idl_sketch_rows: the draws are indexed by the global row), one
all-reduce (sum) of the m x R sketch follows, and every rank runs the QR stage
and the T solve on the summed sketch (idl_id_from_sketch) -- the same J and T on
every rank, no further exchange.  The m x R sketch (m = params.m2) is the only
data that crosses ranks: 60 x 1e4 FP32 = 2.4 MB for the sparse workload.

The partial sketch and the ID from the sketch are the library's calls by
default; `sketch_rows` / `id_from_sketch` may be replaced (the multi-process
tests on CPU pass functions of their own there).
"""
from __future__ import annotations


def row_blocks(I: int, world: int):
    """Contiguous, balanced row ranges [(i0, i1)] of an I-row matrix, one per rank."""
    if I < world:
        raise ValueError("fewer rows than ranks")
    return [(I * g // world, I * (g + 1) // world) for g in range(world)]


def csr_row_block(rowptr, colidx, vals, i0: int, i1: int):
    """The CSR arrays of rows i0 .. i1 - 1 (rowptr rebased to 0)."""
    a, b = int(rowptr[i0]), int(rowptr[i1])
    return rowptr[i0:i1 + 1] - rowptr[i0], colidx[a:b], vals[a:b]


def sharded_id(block, i0: int, I: int, R: int, K: int, params, J, T, *, group=None, sketch_rows=None,
               id_from_sketch=None, info=None, ctx=None, device=None):
    """This rank's rows i0 .. i0 + n - 1 (``block``: a dense (n, R) tensor, or a
    (rowptr, colidx, vals) CSR triple) of an I-row matrix; J, T receive the ID of
    the whole matrix on every rank.  Returns the summed sketch (m x R column-major,
    as a flat tensor)."""
    import torch
    import torch.distributed as dist
    m = params.m2 if params.m2 > 0 else params.m1
    if sketch_rows is None or id_from_sketch is None:
        import paper_1901_10559_gb300 as idl
        if ctx is None:
            raise ValueError("a library context is needed for the default sketch and ID calls")
        if sketch_rows is None:
            def sketch_rows(blk, i0_, I_, params_, Y2_):
                if isinstance(blk, tuple):
                    rp, ci, v = blk
                    idl.idl_sketch_rows_csr(ctx, rp, ci, v, rp.shape[0] - 1, R, i0_, I_, params_, Y2_)
                else:
                    idl.idl_sketch_rows(ctx, blk, i0_, I_, params_, Y2_)
        if id_from_sketch is None:
            def id_from_sketch(Y2_, m_, R_, K_, params_, J_, T_):
                idl.idl_id_from_sketch(ctx, Y2_, m_, R_, K_, params_, J_, T_, info)
    vals = block[2] if isinstance(block, tuple) else block
    dtype = vals.dtype if isinstance(vals, torch.Tensor) else torch.from_numpy(vals[:0]).dtype
    Y2 = torch.zeros(m * R, dtype=dtype, device=device)
    sketch_rows(block, i0, I, params, Y2)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(Y2, op=dist.ReduceOp.SUM, group=group)
    id_from_sketch(Y2, m, R, K, params, J, T)
    return Y2


def column_blocks(R: int, world: int):
    """Contiguous, balanced column ranges [(c0, c1)] of an R-column CP tensor, one per rank."""
    return row_blocks(R, world)


def sharded_cp_id(factors, lam_block, lam_all, R: int, K: int, params, J, T, lam_hat, *, group=None,
                  sketch_cols=None, id_from_sketch=None, lambda_hat=None, info=None, ctx=None, device=None):
    """Column-sharded CP tensor ID.  This rank holds columns c0 .. c1 - 1 of every
    factor (``factors``: (c1 - c0, I_n) tensors) and their weights ``lam_block``;
    ``lam_all`` holds the R weights of the whole tensor.  Column r of the sketch
    depends on column r of the factors and the modes' maps alone (Sec. 1.3, Eq.
    TA-formula), so every rank sketches its own columns (idl_sketch_cp), one
    all-gather places the blocks side by side (m x R column-major: rank g's block
    at columns c0_g .. c1_g - 1), and every rank runs Algorithm 1 on the whole
    sketch and the s-value update of Algorithm 3 with the whole lambda: the same
    J, T and lambda_hat on every rank.  Returns the gathered sketch (flat)."""
    import torch
    import torch.distributed as dist
    m = params.m2 if params.m2 > 0 else params.m1
    if sketch_cols is None or id_from_sketch is None or lambda_hat is None:
        import paper_1901_10559_gb300 as idl
        if ctx is None:
            raise ValueError("a library context is needed for the default sketch and ID calls")
        if sketch_cols is None:
            def sketch_cols(f_, lam_, params_, Y2_):
                idl.idl_sketch_cp(ctx, f_, lam_, params_, Y2_)
        if id_from_sketch is None:
            def id_from_sketch(Y2_, m_, R_, K_, params_, J_, T_):
                idl.idl_id_from_sketch(ctx, Y2_, m_, R_, K_, params_, J_, T_, info)
        if lambda_hat is None:
            def lambda_hat(lam_, J_, T_, K_, R_, out_):
                idl.idl_lambda_hat(ctx, lam_, J_, T_, K_, R_, out_)
    world = dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1
    rank = dist.get_rank(group) if world > 1 else 0
    blocks = column_blocks(R, world)
    c0, c1 = blocks[rank]
    if int(factors[0].shape[0]) != c1 - c0:
        raise ValueError(f"rank {rank} holds {int(factors[0].shape[0])} columns, its block is {c1 - c0}")
    width = max(b - a for a, b in blocks)
    # equal-size pieces for the all-gather (the last columns of a short block are padding)
    piece = torch.zeros(m * width, dtype=torch.float32, device=device)
    sketch_cols(factors, lam_block, params, piece)
    if world > 1:
        parts = [torch.empty_like(piece) for _ in range(world)]
        dist.all_gather(parts, piece, group=group)
    else:
        parts = [piece]
    Y2 = torch.cat([parts[g][:m * (b - a)] for g, (a, b) in enumerate(blocks)])
    id_from_sketch(Y2, m, R, K, params, J, T)
    lambda_hat(lam_all, J, T, K, R, lam_hat)
    return Y2
