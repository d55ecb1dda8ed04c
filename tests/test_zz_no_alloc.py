"""The allocation-free bucket-offset entry point (idl_bucket_offsets_noalloc).

It is meant for callers that cannot call cudaMalloc when they need the offsets
(inside a stream capture, under a fixed memory budget, in a real-time loop):
its scratch is a fixed device array inside the library.  This file is named so
that pytest collects it last; it also passes when run on its own.
"""
import numpy as np
import pytest
import torch

import paper_1901_10559_gb300 as idl
from oracle import countsketch as ocs

pytestmark = pytest.mark.gpu


def _maps(ctx, seed, I, L, modified):
    h = torch.empty(I, dtype=torch.int32, device="cuda")
    s = torch.empty(I, dtype=torch.int8, device="cuda")
    idl.idl_draw_countsketch(ctx, seed, I, L, modified, h, s)
    return h


def _reference_offsets(ctx, h, I, L):
    ptr = torch.empty(L + 1, dtype=torch.int32, device="cuda")
    rows = torch.empty(I, dtype=torch.int32, device="cuda")
    idl.idl_bucket_offsets(ctx, h, I, L, ptr, rows)
    torch.cuda.synchronize()
    return ptr.cpu().numpy(), rows.cpu().numpy()


def test_noalloc_matches_bucket_offsets_on_consecutive_calls(ctx):
    # two calls in a row; the second has fewer buckets and rows, so any counter
    # left over from the first call would show up in its output
    cases = [(300_000, 3600, True, 11), (40_000, 900, False, 12)]
    stream = torch.cuda.current_stream()
    for I, L, modified, seed in cases:
        h = _maps(ctx, seed, I, L, modified)
        want_ptr, want_rows = _reference_offsets(ctx, h, I, L)
        ptr = torch.full((L + 1,), -7, dtype=torch.int32, device="cuda")
        rows = torch.full((I,), -7, dtype=torch.int32, device="cuda")
        rc = idl.idl_bucket_offsets_noalloc(stream, h, I, L, ptr, rows)
        assert rc == idl.IDL_OK
        torch.cuda.synchronize()
        # integer work: bit-exact, the tolerance the other bucket tests use
        assert np.array_equal(ptr.cpu().numpy(), want_ptr)
        assert np.array_equal(rows.cpu().numpy(), want_rows)


@pytest.mark.parametrize("I,L,skew", [(300_000, 8, False), (60_000, 20_000, True)])
def test_noalloc_and_regular_offsets_equal_the_oracle_with_oversized_buckets(ctx, I, L, skew):
    """Buckets of more than 12288 rows (I = 300000 over 8 buckets, and a skewed map
    that puts 20000 rows into one of 20000 buckets) come out in increasing row order
    from both entry points: bit-exact against the oracle's stable counting sort."""
    if skew:
        g = torch.Generator(device="cuda").manual_seed(3)
        h = torch.randint(0, L, (I,), dtype=torch.int32, device="cuda", generator=g)
        h[torch.randperm(I, device="cuda", generator=g)[:20_000]] = 7
    else:
        h = _maps(ctx, 21, I, L, False)
    want_ptr, want_rows = ocs.bucket_offsets(h.cpu().numpy(), L)
    got = _reference_offsets(ctx, h, I, L)
    assert np.array_equal(got[0], want_ptr) and np.array_equal(got[1], want_rows)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        ptr = torch.full((L + 1,), -7, dtype=torch.int32, device="cuda")
        rows = torch.full((I,), -7, dtype=torch.int32, device="cuda")
        assert idl.idl_bucket_offsets_noalloc(stream, h, I, L, ptr, rows) == idl.IDL_OK
        torch.cuda.synchronize()
        assert np.array_equal(ptr.cpu().numpy(), want_ptr)
        assert np.array_equal(rows.cpu().numpy(), want_rows)


def test_noalloc_rejects_sizes_beyond_its_scratch(built_lib):
    I = 10
    h = torch.zeros(I, dtype=torch.int32, device="cuda")
    ptr = torch.empty(2, dtype=torch.int32, device="cuda")
    rows = torch.empty(I, dtype=torch.int32, device="cuda")
    too_many = 65536 + 1
    assert idl.idl_bucket_offsets_noalloc(None, h, I, too_many, ptr, rows) == idl.IDL_ELIMIT
    assert idl.idl_bucket_offsets_noalloc(None, h, -1, 4, ptr, rows) == idl.IDL_EINVAL
