"""Failure detection without any GPU fault: bounded device waits that expire
on a withheld dependency, cell-capacity overflow and over-long migration are
reported as status codes, and the CUDA context stays usable afterwards."""
import numpy as np
import pytest

from paper_2507_11289_gb300 import dsea, inputs

pytestmark = pytest.mark.gpu


def _still_usable():
    pos, vel, box = inputs.SMALL_4K.state()
    with dsea.Box(pos, vel, box, n_slices=4, precision=dsea.MIXED) as b:
        b.advance(3)
        assert b.observables()["step"] == 3


def test_withheld_slice_times_out():
    pos, vel, box = inputs.SMALL_4K.state()
    b = dsea.Box(pos, vel, box, n_slices=4, precision=dsea.MIXED)
    try:
        dsea.debug_set(b.h, dsea.DEBUG_WAIT_LIMIT_NS, 200_000_000)   # 0.2 s
        dsea.debug_set(b.h, dsea.DEBUG_WITHHOLD_SLICE, 1)
        b.advance(5)
        with pytest.raises(dsea.DseaError) as e:
            b.sync()
        assert e.value.code == dsea.ERR_TIMEOUT
        with pytest.raises(dsea.DseaError):
            b.advance(1)                  # the box stays failed
    finally:
        b.close()
    _still_usable()


def test_cell_capacity_overflow_is_reported():
    pos, vel, box = inputs.SMALL_4K.state()
    with pytest.raises(dsea.DseaError) as e:
        dsea.Box(pos, vel, box, n_slices=4, cell_capacity=8)   # ~28 atoms per cell
    assert e.value.code == dsea.ERR_CAPACITY
    _still_usable()


def test_migration_beyond_one_slice_is_reported():
    pos, vel, box = inputs.SMALL_4K.state()
    vel = vel.copy()
    vel[0] = [2000.0, 0.0, 0.0]        # 10 sigma in one step: more than one 4.3-sigma slice
    with dsea.Box(pos, vel, box, n_slices=4) as b:
        b.advance(1)
        with pytest.raises(dsea.DseaError) as e:
            b.sync()
        assert e.value.code == dsea.ERR_MIGRATION
    _still_usable()


def test_invalid_calls():
    pos, vel, box = inputs.SMALL_4K.state()
    with pytest.raises(dsea.DseaError) as e:
        dsea.Box(pos, vel, np.array([4.0, 17.0, 17.0]))      # fewer than 3 cells along x
    assert e.value.code == dsea.ERR_INVALID_ARG
    with pytest.raises(dsea.DseaError):
        dsea.Box(pos, vel, box, n_slices=8)                  # slices thinner than rc
    h = dsea.box_create(pos, vel, box, 4)
    try:
        with pytest.raises(dsea.DseaError) as e:
            dsea.advance(h, 1)                               # no kernel registered
        assert e.value.code == dsea.ERR_STATE
        with pytest.raises(dsea.DseaError):
            dsea.register_kernel(h, kind=2)
    finally:
        dsea.box_destroy(h)
