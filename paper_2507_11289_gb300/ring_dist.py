"""The multi-process slice ring (Sec. 3.1 data flow, Sec. 3.4 program
structure, Eq. 1): N_GPU processes in a ring, N_wGPU workers per process.

Worker w (w = 0 .. N_w - 1, N_w = N_GPU N_wGPU) advances the time levels
s = w, w + N_w, w + 2 N_w, ...: one full sweep of the slices per level, so the
dataset passes every worker once per super-cycle of N_w steps.  Process r
owns the workers r N_wGPU .. r N_wGPU + N_wGPU - 1; the output of its last
worker (every slice of the level it finishes) is sent to process r + 1 (mod
N_GPU) point to point, one slice per message, as soon as the slice is final.
Inside a process the levels pass from worker to worker without a copy.

The domain is periodic along the slice axis.  The paper requires a
non-periodic axis for its pipeline; here each level sweeps the slices from
an offset that advances R = O_in + O_out slices per level (the time-skewed
cyclic order of the single-GPU ring), so the slice a worker takes at sweep
position i needs the previous level's slices up to position i + 2 R of the
previous sweep only, and the periodic seam never stalls the pipeline.

Loading and storing follow Sec. 3.4: process i holds slices j N_GPU + i; at
the start it sends them to the process of the first worker, and at the end
the process of the last level sends slice k back to process k mod N_GPU.

Only O_out = 0 kernels run through this driver (every unit writes its own
slice only); the Lennard-Jones step (O_out = 1) runs in the single-GPU ring
of the C library.  The slice kernel is a callback; on GPUs,
`heat1d_slice_kernel` runs the library's CUDA example kernel on device
tensors, and point-to-point messages go through NCCL.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass


def max_processes(n_slices: int, workers_per_process: int, o_in: int, o_out: int = 0) -> int:
    """Eq. 1: the largest number of processes that keep every worker busy,
    N_max = N_S / (2 + N_wGPU (O_in + O_out)) (rounded down)."""
    return n_slices // (2 + workers_per_process * (o_in + o_out))


@dataclass(frozen=True)
class RingPlan:
    """Who does what in the multi-process ring (no communication; the same
    on every process)."""
    n_slices: int
    n_steps: int
    n_processes: int
    workers_per_process: int
    o_in: int

    def __post_init__(self):
        if self.n_slices < 2 * self.o_in + 1 or self.o_in < 0:
            raise ValueError("need n_slices >= 2 O_in + 1")
        if self.n_steps < 0 or self.n_processes < 1 or self.workers_per_process < 1:
            raise ValueError("invalid ring size")
        if self.n_processes > max(1, max_processes(self.n_slices, self.workers_per_process, self.o_in)):
            raise ValueError(f"{self.n_processes} processes exceed Eq. 1's N_max = "
                             f"{max_processes(self.n_slices, self.workers_per_process, self.o_in)}")

    @property
    def n_workers(self) -> int:
        return self.n_processes * self.workers_per_process

    def process_of_level(self, s: int) -> int:
        """Process whose worker advances level s to s + 1."""
        return (s % self.n_workers) // self.workers_per_process

    def sweep(self, s: int) -> list[int]:
        """Slices of level s in the order its worker takes them."""
        n, R = self.n_slices, self.o_in
        return [(i + R * s) % n for i in range(n)]

    def holder_of_final(self) -> int:
        """Process that holds the last level when the run ends (the worker of
        level n_steps - 1; the loading process when there are no steps)."""
        return self.process_of_level(self.n_steps - 1) if self.n_steps > 0 else self.process_of_level(0)

    def messages(self) -> list[tuple[int, int, int, int]]:
        """Every ring message (level, slice, from, to) of the run, in send order
        per sender (loading and storing excluded)."""
        out = []
        for s in range(self.n_steps - 1):
            a, b = self.process_of_level(s), self.process_of_level(s + 1)
            if a != b:
                out.extend((s + 1, j, a, b) for j in self.sweep(s))
        return out


def run(plan: RingPlan, local_slices: dict, kernel, rank: int, send, recv, new_buffer, flush=lambda: None):
    """Run plan on this process.

    local_slices: {slice j: buffer} of the slices this process loads (j mod
    N_GPU == rank).  kernel(slice, step, [2 O_in + 1 input buffers]) returns
    the slice's buffer at step + 1.  send(buffer, dst) starts moving one slice
    point to point without waiting for the receiver (the paper's output
    thread; the buffer is never written again); recv(buffer, src) fills a
    buffer from new_buffer() and returns when it is complete; flush() waits
    for every send started.  Sends must not wait for their receiver: with one
    worker per process, neighbouring processes send to each other at the same
    time.  Returns {slice j: buffer} of the final level for the slices this
    process stores (j mod N_GPU == rank).
    """
    N, n = plan.n_processes, plan.n_slices
    R = plan.o_in
    first = plan.process_of_level(0)
    # loading (Sec. 3.4): every process sends its round-robin share to the
    # process of the first worker, which receives them in slice order
    if rank != first:
        for j in sorted(local_slices):
            send(local_slices[j], first)
        cur = {}
    else:
        cur = dict(local_slices)
        for j in range(n):
            if j % N != rank:
                buf = new_buffer()
                recv(buf, j % N)
                cur[j] = buf
    level = 0
    if rank != first:
        cur = None   # this process does not hold level 0
    for s in range(plan.n_steps):
        p = plan.process_of_level(s)
        if p != rank:
            continue
        if cur is None or level != s:
            # level s arrives from the previous process, slice by slice in the
            # order its last worker finished them (the sweep order of s - 1)
            src = plan.process_of_level(s - 1)
            pending = iter(plan.sweep(s - 1))
            cur = {}
        else:
            pending = None
        nxt = {}
        hand_on = plan.process_of_level(s + 1) if s + 1 < plan.n_steps else rank
        for j in plan.sweep(s):
            need = [(j + d) % n for d in range(-R, R + 1)]
            while pending is not None and any(k not in cur for k in need):
                k = next(pending)
                buf = new_buffer()
                recv(buf, src)
                cur[k] = buf
            out = kernel(j, s, [cur[k] for k in need])
            if hand_on != rank:
                send(out, hand_on)   # final at once: O_out = 0
            else:
                nxt[j] = out
        cur = nxt if hand_on == rank else None
        level = s + 1
    # storing (Sec. 3.4): the holder of the last level sends slice k to
    # process k mod N_GPU
    holder = plan.holder_of_final()
    mine = {}
    if rank == holder:
        for j in range(n):
            if j % N == rank:
                mine[j] = cur[j]
            else:
                send(cur[j], j % N)
    else:
        for j in range(n):
            if j % N == rank:
                buf = new_buffer()
                recv(buf, holder)
                mine[j] = buf
    flush()
    return mine


def torch_transport(group=None, staged=False):
    """send / recv / flush over torch.distributed: sends are started with
    isend and kept until flush; messages between a pair of processes arrive
    in the order sent.  Device tensors go over NCCL as they are, or, with
    `staged`, through host memory (a copy to the host before the send and back
    to the device after the receive), which any backend carries (gloo, or
    processes that share one GPU)."""
    import torch
    import torch.distributed as dist
    pending = []

    def send(t, dst):
        if staged and t.is_cuda:
            t = t.to("cpu")
        pending.append((dist.isend(t, dst, group=group), t))

    def recv(t, src):
        if staged and t.is_cuda:
            h = torch.empty(t.shape, dtype=t.dtype)
            dist.recv(h, src, group=group)
            t.copy_(h)
        else:
            dist.recv(t, src, group=group)

    def flush():
        for work, _ in pending:
            work.wait()
        pending.clear()

    return send, recv, flush


def heat1d_slice_kernel(a: float, points: int, stream=None):
    """A kernel callback for device tensors that runs the library's CUDA
    example slice kernel (dsea_example_heat1d: one explicit FP32 heat step,
    O_in = 1) on the three input slices and returns the new slice."""
    import torch

    from . import dsea
    lib = dsea.load()
    user = ctypes.c_float(a)
    sh = dsea._stream_handle(stream)

    def kernel(j, s, ins):
        out = torch.empty(points, dtype=torch.float32, device=ins[0].device)
        in_ptrs = (ctypes.c_void_p * 3)(*[t.data_ptr() for t in ins])
        out_ptrs = (ctypes.c_void_p * 1)(out.data_ptr())
        rc = lib.dsea_example_heat1d(ctypes.byref(user), j, s, in_ptrs, out_ptrs, points * 4, sh)
        if rc != dsea.OK:
            raise dsea.DseaError(rc, "dsea_example_heat1d")
        return out

    return kernel
