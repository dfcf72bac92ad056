"""GPU parity with mirror walls along x (DSEA_BOUNDARY_MIRROR) against the
oracle's walls.  Same tolerances as the periodic parity tests:
  FP64 forces       rms_i |F_gpu - F_oracle| <= 1e-12 rms_i |F_oracle|
  FP64 trajectory   max |r_gpu - r_oracle| <= 1e-9 sigma after 100 steps
  mixed forces      rms_i |F_gpu - F_oracle| <= 2e-6 rms_i |F_oracle|
"""
import numpy as np
import pytest

import oracle
from paper_2507_11289_gb300 import dsea, inputs

pytestmark = pytest.mark.gpu

RC = 2.5


def rms(a):
    return float(np.sqrt((np.asarray(a) ** 2).sum(-1).mean()))


def yz_image(d, box):
    """Minimum image along y and z only (x is bounded by walls)."""
    d = np.array(d, dtype=np.float64)
    d[..., 1:] -= box[1:] * np.round(d[..., 1:] / box[1:])
    return d


@pytest.mark.parametrize("precision,tol", [(dsea.FP64, 1e-12), (dsea.MIXED, 2e-6)])
@pytest.mark.parametrize("schedule", [dsea.SCHED_RING, dsea.SCHED_STEPWISE])
def test_forces_with_walls_match_oracle(precision, tol, schedule, melted_4k):
    pos, vel, box = melted_4k
    Fo, Uo, Wo = oracle.forces(pos, box, RC, "cells", walls=True)
    Fp, _, _ = oracle.forces(pos, box, RC, "cells")
    assert rms(Fo - Fp) > 0.01 * rms(Fo)          # the walls change the forces near them
    with dsea.Box(pos, vel, box, n_slices=4, precision=precision, schedule=schedule, walls=True) as b:
        assert b.info()["boundary_x"] == dsea.BOUNDARY_MIRROR
        Fg = b.forces()
        ob = b.observables()
    e = rms(Fg - Fo) / rms(Fo)
    print(f"precision {precision} walls: force error rms {e:.3e} of rms force")
    assert e <= tol
    scale = (1e-12 if precision == dsea.FP64 else 2e-6) * len(pos) * rms(Fo)
    assert abs(ob["U"] - Uo) <= scale and abs(ob["W"] - Wo) <= scale


def test_fp64_trajectory_with_walls_100_steps(melted_4k):
    pos, vel, box = melted_4k
    ro, vo, Fo, obs = oracle.run(pos, vel, box, steps=100, walls=True)
    # atoms met the walls on the way: some x velocities were reversed by them
    rp, vp, _, _ = oracle.run(pos, vel, box, steps=100)
    with dsea.Box(pos, vel, box, n_slices=4, precision=dsea.FP64, walls=True) as b:
        b.advance(60)
        b.advance(40)
        rg, vg, og = b.positions(), b.velocities(), b.observables()
    dr = np.abs(yz_image(rg - ro, box)).max()
    dv = np.abs(vg - vo).max()
    print(f"walls FP64: max |dr| {dr:.3e}, max |dv| {dv:.3e}")
    assert dr <= 1e-9 and dv <= 1e-8
    assert np.all((rg[:, 0] >= 0) & (rg[:, 0] < box[0]))
    assert og["U"] == pytest.approx(obs[-1, 0], rel=1e-10)
    assert og["KE"] == pytest.approx(obs[-1, 2], rel=1e-10)
    assert np.abs(vp - vo).max() > 0.1             # the periodic run differs: walls were hit


@pytest.mark.parametrize("precision", [dsea.FP64, dsea.MIXED])
def test_free_flight_into_both_walls(precision):
    box = np.array([12.0, 12.0, 12.0])
    pos = np.array([[0.3, 5.0, 6.0], [11.7, 2.0, 3.0]])
    vel = np.array([[-1.5, 0.25, -0.5], [1.5, 0.0, 0.0]])
    steps, dt = 80, 0.005
    ro, vo, _, _ = oracle.run(pos, vel, box, steps=steps, dt=dt, walls=True)
    with dsea.Box(pos, vel, box, precision=precision, walls=True) as b:
        b.advance(steps)
        rg, vg = b.positions(), b.velocities()
    t = steps * dt
    assert rg[0, 0] == pytest.approx(abs(0.3 - 1.5 * t), abs=1e-6)
    assert rg[1, 0] == pytest.approx(2 * 12.0 - (11.7 + 1.5 * t), abs=1e-6)
    assert np.allclose(vg[:, 0], [1.5, -1.5], atol=1e-6)
    tol = 1e-12 if precision == dsea.FP64 else 1e-6
    assert np.abs(rg - ro).max() <= tol and np.abs(vg - vo).max() <= tol


def test_no_pair_across_the_walls():
    box = np.array([9.0, 9.0, 9.0])
    pos = np.array([[0.3, 1.0, 4.0], [8.6, 1.0, 4.0]])
    for prec in (dsea.FP64, dsea.MIXED):
        with dsea.Box(pos, None, box, precision=prec, walls=True) as b:
            assert np.all(b.forces() == 0) and b.observables()["U"] == 0.0
        with dsea.Box(pos, None, box, precision=prec) as b:
            assert np.abs(b.forces()).max() > 1.0


@pytest.mark.parametrize("precision", [dsea.FP64, dsea.MIXED])
def test_ring_equals_stepwise_with_walls(precision, melted_4k):
    pos, vel, box = melted_4k
    out = []
    for sched in (dsea.SCHED_RING, dsea.SCHED_STEPWISE):
        with dsea.Box(pos, vel, box, n_slices=4, precision=precision, schedule=sched, walls=True) as b:
            b.advance(30)
            out.append((b.positions(), b.velocities(), b.observables()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]


def test_mixed_energy_drift_with_walls_1000_steps(melted_4k):
    pos, vel, box = melted_4k
    n = len(pos)
    e_gpu = []
    with dsea.Box(pos, vel, box, n_slices=4, precision=dsea.MIXED, walls=True) as b:
        for _ in range(100):
            o = b.observables()
            e_gpu.append((o["U"] + o["KE"]) / n)
            b.advance(10)
        o = b.observables()
        e_gpu.append((o["U"] + o["KE"]) / n)
        assert np.all((b.positions()[:, 0] >= 0) & (b.positions()[:, 0] < box[0]))
    _, _, _, obs = oracle.run(pos, vel, box, steps=1000, walls=True)
    e_ora = (obs[::10, 0] + obs[::10, 2]) / n
    e_gpu = np.array(e_gpu)
    drift_gpu = abs(e_gpu[-10:].mean() - e_gpu[:10].mean())
    drift_ora = abs(e_ora[-10:].mean() - e_ora[:10].mean())
    print(f"walls: drift per atom over 1000 steps: mixed {drift_gpu:.3e}, oracle FP64 {drift_ora:.3e}")
    assert drift_gpu <= max(1e-4, 2.0 * drift_ora)


@pytest.mark.parametrize("precision", [dsea.MIXED, dsea.FP64])
def test_walls_box_in_a_batch_equals_alone(precision, melted_4k):
    """A box with mirror walls and periodic boxes in one persistent launch:
    each box keeps its own boundary, and ends bit for bit where it ends
    alone."""
    pos, vel, box = melted_4k
    others = [s.state() for s in inputs.batch_specs(n_boxes=2, seed=12, n_max=5000)]
    kinds = [((pos, vel, box), True), (others[0], False), (others[1], False)]
    steps = [25, 18, 25]
    alone = []
    for (st, walls), n in zip(kinds, steps):
        with dsea.Box(*st, n_slices=4 if walls else 0, precision=precision, walls=walls) as b:
            b.advance(n)
            alone.append((b.positions(), b.velocities(), b.observables()))
    boxes = [dsea.Box(*st, n_slices=4 if walls else 0, precision=precision, walls=walls) for st, walls in kinds]
    try:
        bt = dsea.batch_create([b.h for b in boxes])
        dsea.batch_advance(bt, steps)
        dsea.batch_destroy(bt)
        for b, (r, v, o) in zip(boxes, alone):
            assert np.array_equal(b.positions(), r) and np.array_equal(b.velocities(), v)
            assert b.observables() == o
        assert np.all((boxes[0].positions()[:, 0] >= 0) & (boxes[0].positions()[:, 0] < box[0]))
    finally:
        for b in boxes:
            b.close()
