"""The benchmark's multi-GPU host logic on CPU with two gloo ranks: every rank gets its own
consecutive slice of one seeded trace stream (weak scaling, no data exchange), and the step time is
the maximum over ranks."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    d = bench.dist_init(world, use_cuda=False)
    fib = synth.gen_fib(500, seed=7)
    xh, xl = bench.rank_shard(fib, n, seed=9, rank=rank)
    t = bench.max_over_ranks(d, float(rank + 1) * 0.5, use_cuda=False)
    bench.barrier(d)
    q.put((rank, xh, xl, t))
    d.destroy_process_group()


def test_two_gloo_ranks_shard_one_stream_and_reduce_max():
    world, n = 2, 10_000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    fib = synth.gen_fib(500, seed=7)
    full_h, full_l = synth.gen_trace(fib, world * n, seed=10)
    for rank, xh, xl, t in res:
        assert np.array_equal(xh, full_h[rank * n:(rank + 1) * n])
        assert np.array_equal(xl, full_l[rank * n:(rank + 1) * n])
        assert t == world * 0.5                     # the slowest rank's time
    assert not np.array_equal(res[0][1], res[1][1])
