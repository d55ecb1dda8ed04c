"""The multi-rank host logic of bench.py with two gloo ranks on CPU.

Under torchrun every rank solves its own instance (its own draws) with no
collective on the data path; the job's time is the slowest rank's, its value
the solves of all ranks over that time, and the reference arm runs on rank 0
only.  These tests run the same helpers bench.py calls in two processes joined
by a gloo process group (127.0.0.1)."""
import os
import socket
import sys
import types

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        env = bench.dist_env()
        t_max = bench.max_over_ranks(0.5 + rank, dist, "cpu")          # rank 1 is the slow one
        seed = bench.rank_seed(bench.WORKLOADS["sparse"], rank)
        value = bench.job_value(ws, 10, 1, t_max)
        args = types.SimpleNamespace(workload="sparse", steps=3, warmup=3)
        ref = bench.run_reference(args, ws, rank) if rank != 0 else "skipped"
        dist.barrier()
        q.put((rank, env, t_max, seed, value, ref))
    finally:
        dist.destroy_process_group()


def _run(ws):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(ws):
        rank, *rest = q.get(timeout=120)
        out[rank] = rest
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return out


def test_two_gloo_ranks_max_time_seeds_and_rank0_reference():
    out = _run(2)
    for rank, (env, t_max, seed, value, ref) in out.items():
        assert env == (2, rank, rank)
        assert t_max == 1.5                          # the slowest rank's time on every rank
        assert value == 2 * 10 / 1.5                 # solves of both ranks over that time
        if rank:
            assert ref is None                       # the reference arm: rank 0 alone works
    seeds = [out[r][2] for r in range(2)]
    assert seeds[0] != seeds[1]
    # independent draws per rank: the two ranks' CountSketch maps differ
    from oracle import draws as odr
    h0, s0 = odr.countsketch_maps(seeds[0], 5000, 300, True)
    h1, s1 = odr.countsketch_maps(seeds[1], 5000, 300, True)
    assert not np.array_equal(h0, h1) and not np.array_equal(s0, s1)


def test_single_process_helpers_without_a_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
    assert bench.rank_seed({"seed": 7}, 0) == 7 and bench.rank_seed({"seed": 7}, 2) == 2007
    assert bench.job_value(1, 4, 320, 2.0) == 640.0
