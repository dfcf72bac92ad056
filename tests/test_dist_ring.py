"""The multi-process slice ring (Sec. 3.1 data flow, Sec. 3.4 round-robin
loading and storing, Eq. 1) on CPU processes over gloo: two or three
processes exchange real slice buffers point to point and the final slices
equal, bit for bit, the single-process run and a plain sweep of the whole
rod.  The slice kernel is a host stand-in with the rounding of the library's
example kernel (u' = u + a (u[i-1] - 2 u[i] + u[i+1]), every operation
rounded in FP32)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2507_11289_gb300 import ring_dist

A = 0.2


def heat_step(left, mid, right):
    """One explicit heat step of one slice from its two neighbour slices."""
    u_l = torch.cat([left[-1:], mid[:-1]])
    u_r = torch.cat([mid[1:], right[:1]])
    t = u_l - 2.0 * mid
    t = t + u_r
    return mid + torch.tensor(A, dtype=torch.float32) * t


def whole_rod(u0, steps):
    """The same steps on the rod in one piece (periodic)."""
    u = u0.clone()
    for _ in range(steps):
        t = torch.roll(u, 1) - 2.0 * u
        t = t + torch.roll(u, -1)
        u = u + torch.tensor(A, dtype=torch.float32) * t
    return u


def initial(n_slices, points, seed=5):
    rng = np.random.Generator(np.random.PCG64(seed))
    return torch.from_numpy(rng.uniform(-1.0, 1.0, n_slices * points).astype(np.float32))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n_slices, points, steps, k_per, out_q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        u0 = initial(n_slices, points).view(n_slices, points)
        local = {j: u0[j].clone() for j in range(n_slices) if j % world == rank}
        plan = ring_dist.RingPlan(n_slices, steps, world, k_per, 1)
        send, recv, flush = ring_dist.torch_transport()
        mine = ring_dist.run(plan, local, lambda j, s, ins: heat_step(*ins), rank, send, recv,
                             lambda: torch.empty(points, dtype=torch.float32), flush)
        out_q.put((rank, {j: t.numpy().copy() for j, t in mine.items()}))
    finally:
        dist.destroy_process_group()


def _run_world(world, n_slices, points, steps, k_per):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_slices, points, steps, k_per, q))
             for r in range(world)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(world):
        rank, part = q.get(timeout=120)
        for j, a in part.items():
            assert j % world == rank          # stored round-robin
            got[j] = a
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return np.stack([got[j] for j in range(n_slices)])


@pytest.mark.parametrize("world,n_slices,k_per,steps", [(2, 8, 2, 11), (2, 12, 1, 7), (3, 12, 1, 10)])
def test_ring_across_processes_equals_one_process(world, n_slices, k_per, steps):
    points = 64
    ring = _run_world(world, n_slices, points, steps, k_per)
    single = _run_world(1, n_slices, points, steps, k_per)
    ref = whole_rod(initial(n_slices, points), steps).numpy().reshape(n_slices, points)
    assert np.array_equal(ring, single)
    assert np.array_equal(ring, ref)


def test_plan_follows_the_data_flow():
    plan = ring_dist.RingPlan(n_slices=8, n_steps=11, n_processes=2, workers_per_process=2, o_in=1)
    # workers 0,1 on process 0, workers 2,3 on process 1; super-cycles of 4 levels
    assert [plan.process_of_level(s) for s in range(9)] == [0, 0, 1, 1, 0, 0, 1, 1, 0]
    msgs = plan.messages()
    # a level crosses a link only where its worker and the next are on different processes
    assert sorted({(s, a, b) for s, _, a, b in msgs}) == [(2, 0, 1), (4, 1, 0), (6, 0, 1), (8, 1, 0), (10, 0, 1)]
    assert len(msgs) == 5 * 8                 # every slice of each crossing level, one message each
    # each level's sweep starts one slice (O_in + O_out) further than the previous one
    assert plan.sweep(0)[:3] == [0, 1, 2] and plan.sweep(3)[:3] == [3, 4, 5]
    assert plan.holder_of_final() == 1        # level 10 runs on process 1


def test_eq1_bounds_the_process_count():
    assert ring_dist.max_processes(596, 1, 1, 1) == 149   # the paper's 10^9-molecule case
    assert ring_dist.max_processes(8, 2, 1) == 2
    with pytest.raises(ValueError):
        ring_dist.RingPlan(n_slices=8, n_steps=4, n_processes=3, workers_per_process=2, o_in=1)
