"""Row-sharded matrix ID: a matrix split by rows over several GPUs, one process
per GPU (torch.distributed).

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
