"""Multi-process replica logic on CPU (gloo, world size 2): the benchmark's
whole-job value is the sum of the ranks' atom-steps over the slowest rank's
time, and the ranks exchange nothing but those two numbers."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    sec = [2.0, 3.0][rank]                  # rank 1 is the slowest
    atom_steps = [1e9, 1e9][rank]
    sec_max = bench.max_over_ranks(sec, world)
    total = bench.sum_over_ranks(atom_steps, world)
    out[rank] = (sec_max, total, total / sec_max)
    bench.barrier(world)
    dist.destroy_process_group()


def test_replica_throughput_is_sum_over_max_time():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        sec_max, total, value = res[r]
        assert sec_max == 3.0 and total == 2e9
        assert value == pytest.approx(2e9 / 3.0)


def test_single_process_reductions_are_identity():
    import bench
    assert bench.max_over_ranks(1.5, 1) == 1.5
    assert bench.sum_over_ranks(7.0, 1) == 7.0
