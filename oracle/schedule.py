"""Slice-streaming schedule oracle (Sec. 3.1, 3.3, Table 1, Eq. 1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Three things, each written from the paper's statement:

* ``one_worker_table(n_s)`` -- the stage-by-stage operation of one worker
  with O_in = O_out = 1 (Sec. 3.3): in each stage one slice can be received
  into the input buffer and one finalised slice sent from the output buffer;
  the worker fires on slice w when slices w-1, w, w+1 (those that exist) are
  stored in the input buffer, contributes to w-1, w, w+1 of the output
  buffer, and a slice is finalised when the worker will not contribute to it
  in the next stage.  Slices leave the input buffer only when a new slice
  arrives and they are no longer needed.  The rows are derived by
  simulating those rules, not written out.
* ``n_max(n_s, n_wgpu, o_in, o_out)`` -- Eq. 1.
* ``ring_dependencies(j, s, n_s)`` -- on a ring of slices that is periodic in
  x (the reading taken for the periodic workloads), the update of slice j
  at time level s reads slices j-1, j, j+1 at level s, and slice k at level s
  is complete once the updates of k-1, k, k+1 at level s-1 have written to it
  (O_in = O_out = 1, Sec. 4); so unit (j, s) depends on units
  (j-2 .. j+2, s-1), indices modulo n_s.
"""
from __future__ import annotations


def n_max(n_s: int, n_wgpu: int = 1, o_in: int = 1, o_out: int = 1) -> float:
    """Eq. 1: the largest number of processes that can work in parallel."""
    return n_s / (2 + n_wgpu * (o_in + o_out))


def one_worker_table(n_s: int):
    """Rows (stage, store, receive, worker, partial, send) for one worker.

    Sets are returned as sorted tuples; `receive`, `worker`, `send` are a slice
    number or None.  Slices are numbered 1..n_s, stages from 1."""
    if n_s < 3:
        raise ValueError("the table needs at least three slices")
    rows = []
    stored: list[int] = []          # input buffer content usable in this stage
    next_recv = 1                   # next slice to arrive
    next_work = 1                   # next slice the worker will process
    contributed: set[int] = set()   # output slices with contributions, not yet finalised
    finalised: list[int] = []       # finalised slices waiting to be sent
    stage = 0
    while True:
        stage += 1
        # receive: one slice per stage (becomes usable from the next stage)
        receive = next_recv if next_recv <= n_s else None
        # the worker fires if its 2*O_in+1 inputs (those that exist) are stored
        need = [k for k in (next_work - 1, next_work, next_work + 1) if 1 <= k <= n_s]
        worker = None
        if next_work <= n_s and all(k in stored for k in need):
            worker = next_work
            contributed.update(k for k in (worker - 1, worker, worker + 1) if 1 <= k <= n_s)
            # a slice is final if the worker will not contribute to it next stage
            nxt = worker + 1
            for k in sorted(contributed):
                if nxt > n_s or k < nxt - 1:
                    finalised.append(k)
            contributed.difference_update(finalised)
            next_work += 1
        store_col = tuple(sorted(stored))
        send = finalised.pop(0) if finalised else None
        # the output buffer holds contributed slices and finalised ones not yet sent
        partial = tuple(sorted(contributed.union(finalised)))
        rows.append((stage, store_col, receive, worker, partial, send))
        # end of stage: the received slice becomes usable; evict slices that
        # are no longer needed, but only when a new slice arrives
        if receive is not None:
            stored.append(receive)
            next_recv += 1
            still_needed = next_work - 1
            stored = [k for k in stored if k >= still_needed]
        elif next_work > n_s:
            stored = []
        if receive is None and worker is None and send is None:
            rows.pop()
            break
    return rows


def ring_dependencies(j: int, s: int, n_s: int):
    """Units (slice, level) that must be complete before unit (j, s) may run
    on a periodic ring of n_s >= 3 slices (no dependency for s == 0)."""
    if s <= 0:
        return []
    return sorted({((j + d) % n_s, s - 1) for d in (-2, -1, 0, 1, 2)})
