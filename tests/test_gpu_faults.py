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


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_non_finite_positions_are_rejected_at_create(bad):
    """dsea_box_create copies the caller's arrays to the device and checks
    them there before it returns."""
    pos, vel, box = inputs.SMALL_4K.state()
    pos = pos.copy()
    pos[1234, 2] = bad
    with pytest.raises(dsea.DseaError) as e:
        dsea.box_create(pos, vel, box, 4)
    assert e.value.code == dsea.ERR_INVALID_ARG
    _still_usable()


def test_caller_arrays_may_change_after_create():
    """The box owns its device copy of the initial state once create returns:
    the caller's arrays can be overwritten before registration, and the copy
    is released once the atoms are binned."""
    pos, vel, box = inputs.SMALL_4K.state()
    p, v = pos.copy(), vel.copy()
    n = len(pos)
    h = dsea.box_create(p, v, box, 4)
    h0 = dsea.box_create(p, None, box, 4)           # no velocities: no velocity copy
    try:
        assert dsea.box_get_info(h)["device_bytes"] == 2 * 24 * n
        assert dsea.box_get_info(h0)["device_bytes"] == 24 * n
        p[:] = 0.5
        v[:] = 7.0
        for x in (h, h0):
            dsea.register_kernel(x, dsea.make_params(precision=dsea.FP64))
        assert np.array_equal(dsea.read_positions(h), pos)
        assert np.array_equal(dsea.read_velocities(h), vel)
        assert np.all(dsea.read_velocities(h0) == 0.0)
        assert dsea.box_get_info(h)["device_bytes"] == dsea.box_get_info(h0)["device_bytes"]
    finally:
        dsea.box_destroy(h)
        dsea.box_destroy(h0)


@pytest.mark.parametrize("precision", [dsea.MIXED, dsea.FP64])
def test_thermostat_energy_beyond_its_range_is_reported(precision):
    """The slice thermostat sums kinetic energies exactly in fixed point; a
    chunk of home atoms at 1024 epsilon or more is outside that range and is
    reported as DSEA_ERR_RANGE (here one atom at 50 sigma/tau, 1250 epsilon,
    alone in its cell).  The same state without the thermostat runs."""
    from tests.test_oracle_nvt import _gas
    pos, vel, box, _, _ = _gas(60, [1.0, 1.0, 1.0])
    vel = vel.copy()
    vel[0] = [50.0, 0.0, 0.0]
    with dsea.Box(pos, vel, box, n_slices=3, precision=precision, temperature=1.0) as b:
        b.advance(2)
        with pytest.raises(dsea.DseaError) as e:
            b.sync()
        assert e.value.code == dsea.ERR_RANGE
    with dsea.Box(pos, vel, box, n_slices=3, precision=precision) as b:
        b.advance(2)
        b.sync()
    _still_usable()
