"""Checkpoint / resume through the C ABI, host-side fault injection through a
failing allocator, and determinism (the same run twice gives the same bits).

Resume: the paper loads slices at the start and stores them at the end; here
a run is stored by reading positions and velocities back in atom-ID order and
resumed by creating a new box from them.  The resumed trajectory is the
uninterrupted one up to rounding (the velocity half-kicks of the two runs
are grouped differently) and matches the FP64 oracle's uninterrupted run.

Fault injection: an allocator callback that fails once, at each allocation
point in turn, makes the failing call report DSEA_ERR_OOM and leave the box
as it was, so that the same call succeeds when retried; the run then ends
with the bits of a run without failures, and every allocation is released."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2507_11289_gb300 import dsea, inputs

pytestmark = pytest.mark.gpu


def _wrap_diff(a, b, box):
    d = a - b
    return d - box * np.round(d / box)


@pytest.mark.parametrize("precision, tol", [(dsea.FP64, 1e-10), (dsea.MIXED, 1e-5)])
def test_resume_from_read_back_state(precision, tol):
    pos, vel, box = inputs.SMALL_4K.state()
    with dsea.Box(pos, vel, box, n_slices=4, precision=precision) as b:
        b.advance(60)
        r_whole = b.positions()
    with dsea.Box(pos, vel, box, n_slices=4, precision=precision) as b:
        b.advance(30)
        r_mid, v_mid = b.positions(), b.velocities()
    with dsea.Box(r_mid, v_mid, box, n_slices=4, precision=precision) as b:
        b.advance(30)
        r_res, obs = b.positions(), b.observables()
    assert obs["step"] == 30
    assert np.abs(_wrap_diff(r_res, r_whole, box)).max() <= tol
    if precision == dsea.FP64:
        r_ora, _, _, _ = oracle.run(pos, vel, box, steps=60)
        assert np.abs(_wrap_diff(r_res, r_ora, box)).max() <= 1e-9


class _FailOnce(dsea.TorchAllocator):
    """Torch's caching allocator, except that allocation number `fail_at`
    (counting from 0) returns NULL once; records the live allocations."""

    def __init__(self, fail_at=None):
        super().__init__()
        self.fail_at = fail_at
        self.count = 0
        self.live = {}

    def _do_alloc(self, nbytes, ctx):
        k = self.count
        self.count += 1
        if k == self.fail_at:
            return None
        p = super()._do_alloc(nbytes, ctx)
        if p:
            self.live[p] = nbytes
        return p

    def _do_free(self, ptr, ctx):
        self.live.pop(ptr, None)
        super()._do_free(ptr, ctx)


def _run_with(alloc, pos, vel, box, precision, steps):
    """create, register, advance twice, read back; a call that fails with
    DSEA_ERR_OOM is retried once.  Returns (positions, failed call or None)."""
    failed = None

    def attempt(name, fn):
        nonlocal failed
        try:
            return fn()
        except dsea.DseaError as e:
            assert e.code == dsea.ERR_OOM, (name, e.code)
            assert failed is None
            failed = name
            return fn()

    h = attempt("create", lambda: dsea.box_create(pos, vel, box, 4, None, alloc))
    try:
        attempt("register", lambda: dsea.register_kernel(h, dsea.make_params(precision=precision)))
        attempt("advance", lambda: dsea.advance(h, steps))
        attempt("advance 2", lambda: dsea.advance(h, 1030))   # grows the ring plan arrays (1024)
        r = attempt("read", lambda: dsea.read_positions(h))
        v = attempt("read v", lambda: dsea.read_velocities(h))
    finally:
        dsea.box_destroy(h)
    return r, v, failed


@pytest.mark.parametrize("precision", [dsea.MIXED, dsea.FP64])
def test_failing_allocator_at_every_point(precision):
    import torch
    pos, vel, box = inputs.SMALL_4K.state()
    clean = _FailOnce()
    r0, v0, none = _run_with(clean, pos, vel, box, precision, 20)
    assert none is None and not clean.live
    n_allocs = clean.count
    assert n_allocs >= 10
    seen = set()
    for k in range(n_allocs):
        alloc = _FailOnce(fail_at=k)
        r, v, failed = _run_with(alloc, pos, vel, box, precision, 20)
        assert failed is not None, k
        seen.add(failed)
        assert np.array_equal(r, r0) and np.array_equal(v, v0), (k, failed)
        assert not alloc.live, (k, failed)            # every allocation was released
    assert {"create", "register", "advance", "advance 2", "read"} <= seen
    torch.cuda.synchronize()


def test_same_run_twice_gives_the_same_bits():
    """Races in the ring (ticket order, dependency waits, arrival slots) would
    show as runs that differ; 108,000 atoms over 100 steps in both forms."""
    pos, box = inputs.fcc_lattice(30, 0.8)
    vel = inputs.maxwell_boltzmann(len(pos), 1.5, 17)
    for precision in (dsea.MIXED, dsea.FP64):
        runs = []
        for _ in range(2):
            with dsea.Box(pos, vel, box, precision=precision) as b:
                b.advance(100 if precision == dsea.MIXED else 20)
                runs.append((b.positions(), b.velocities(), b.forces(), b.observables()))
        (r0, v0, f0, o0), (r1, v1, f1, o1) = runs
        assert np.array_equal(r0, r1) and np.array_equal(v0, v1) and np.array_equal(f0, f1)
        assert o0 == o1
