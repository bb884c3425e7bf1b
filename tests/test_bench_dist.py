"""Multi-process path of bench.py on CPU (gloo, world size 2): the timing
reductions take the maximum time and the summed work over ranks, and ranks
meet at the barriers that bracket the timed region."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    import torch.distributed as dist
    bench.init_dist(world, "gloo")
    bench.barrier(world)
    t = bench.reduce_max(1.0 + rank, world)
    s = bench.reduce_sum(10.0 * (rank + 1), world)
    bench.barrier(world)
    out[rank] = (t, s)
    dist.destroy_process_group()


def test_reductions_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert out[0] == out[1] == (2.0, 30.0)


def test_single_rank_helpers_are_identity():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.reduce_sum(2.0, 1) == 2.0
    bench.barrier(1)


def test_factor_work_counts():
    import bench
    # one 2x2 pivot of a 4x4 block: t = 2 trailing rows -> 2*2*3 + 8*2 flops
    assert bench._pair_flops(4, 1) == 2 * 2 * 3 + 8 * 2
    fl, by = bench.factor_work(10, 20, 400, 4)
    fe, be = bench.elem_factor_work(10, 20, 400, 4)
    assert fl > fe and by > be
