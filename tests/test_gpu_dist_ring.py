"""The multi-process slice ring with the library's CUDA slice kernel on
device buffers (dsea_example_heat1d through ring_dist.heat1d_slice_kernel):
one process, and two processes that share cuda:0 and pass slices through host
memory over gloo (their kernels never wait on each other).  Results equal,
bit for bit, the same steps on the whole rod in FP32 on the host."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2507_11289_gb300 import ring_dist
from tests.test_dist_ring import A, _free_port, initial, whole_rod

pytestmark = pytest.mark.gpu

POINTS = 4096


def _worker(rank, world, port, n_slices, steps, k_per, out_q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        u0 = initial(n_slices, POINTS).view(n_slices, POINTS)
        local = {j: u0[j].to("cuda") for j in range(n_slices) if j % world == rank}
        plan = ring_dist.RingPlan(n_slices, steps, world, k_per, 1)
        stream = torch.cuda.current_stream()
        kernel = ring_dist.heat1d_slice_kernel(A, POINTS, stream)
        send, recv, flush = ring_dist.torch_transport(staged=True)

        def k_sync(j, s, ins):   # the staged sends read the result on the host
            out = kernel(j, s, ins)
            torch.cuda.current_stream().synchronize()
            return out

        mine = ring_dist.run(plan, local, k_sync, rank, send, recv,
                             lambda: torch.empty(POINTS, dtype=torch.float32, device="cuda"), flush)
        torch.cuda.synchronize()
        out_q.put((rank, {j: t.cpu().numpy() for j, t in mine.items()}))
    finally:
        dist.destroy_process_group()


def _run(world, n_slices, steps, k_per):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_slices, steps, k_per, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(world):
        rank, part = q.get(timeout=300)
        got.update(part)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return np.stack([got[j] for j in range(n_slices)])


@pytest.mark.parametrize("world,k_per", [(1, 2), (2, 1), (2, 2)])
def test_device_slices_through_the_ring(world, k_per):
    n_slices, steps = 12 if k_per == 1 else 8, 9
    ring = _run(world, n_slices, steps, k_per)
    ref = whole_rod(initial(n_slices, POINTS), steps).numpy().reshape(n_slices, POINTS)
    assert np.array_equal(ring, ref)
