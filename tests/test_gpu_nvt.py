"""GPU parity of the slice thermostat (NVT) and of the per-slice profiles with
the oracle (oracle.run_nvt, oracle.profiles).  Tolerances as in the NVE
parity tests: FP64 trajectory 1e-9 sigma after 100 steps; FP64 profile sums
1e-12 relative; mixed forms hold the target temperature.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2507_11289_gb300 import dsea, inputs
from tests.test_oracle_nvt import _gas

pytestmark = pytest.mark.gpu

RC = 2.5


def slices_of(b):
    inf = b.info()
    return inf["cells"][0], inf["cells_per_slice_x"]


def min_image(d, box):
    return d - box * np.round(d / box)


def test_fp64_nvt_trajectory_matches_oracle(melted_4k):
    pos, vel, box = melted_4k
    T0 = 1.1
    with dsea.Box(pos, vel, box, n_slices=4, precision=dsea.FP64, temperature=T0) as b:
        ncx, cps = slices_of(b)
        b.advance(55)
        b.advance(45)
        rg, vg, og = b.positions(), b.velocities(), b.observables()
    ro, vo, Fo, obs, st = oracle.run_nvt(pos, vel, box, 100, ncx, cps, T0)
    dr = np.abs(min_image(rg - ro, box)).max()
    dv = np.abs(vg - vo).max()
    print(f"NVT FP64: max |dr| {dr:.3e}, max |dv| {dv:.3e}")
    assert dr <= 1e-9 and dv <= 1e-8
    assert og["KE"] == pytest.approx(obs[-1, 2], rel=1e-10)


def test_fp64_nvt_with_walls_matches_oracle(melted_4k):
    """The slice thermostat and mirror walls together (the paper's validation
    runs combine its thermostat with the walls at the x ends): 100 FP64
    steps against the oracle's, then the per-slice profiles."""
    pos, vel, box = melted_4k
    T0 = 1.3
    with dsea.Box(pos, vel, box, n_slices=4, precision=dsea.FP64, temperature=T0, walls=True) as b:
        ncx, cps = slices_of(b)
        b.advance(60)
        b.advance(40)
        rg, vg, og = b.positions(), b.velocities(), b.observables()
        pg = b.profiles()
    ro, vo, Fo, obs, st = oracle.run_nvt(pos, vel, box, 100, ncx, cps, T0, walls=True)
    assert rg[:, 0].min() >= 0.0 and rg[:, 0].max() < box[0]   # nothing crossed a wall
    d = rg - ro                       # no periodic image along x; y and z stay periodic
    d[:, 1:] = min_image(d[:, 1:], box[1:])
    dr = np.abs(d).max()
    dv = np.abs(vg - vo).max()
    print(f"NVT + walls FP64: max |dr| {dr:.3e}, max |dv| {dv:.3e}")
    assert dr <= 1e-9 and dv <= 1e-8
    assert og["KE"] == pytest.approx(obs[-1, 2], rel=1e-10)
    po = oracle.profiles(rg, vg, box, ncx, cps, walls=True)
    assert np.array_equal(pg["N"], po[:, 3].astype(np.int64))
    assert np.allclose(pg["KE"], po[:, 2], rtol=1e-10)


@pytest.mark.parametrize("precision,tol", [(dsea.FP64, 1e-13), (dsea.MIXED, 1e-6)])
def test_ideal_gas_slices_reach_the_target_in_one_scaling(precision, tol):
    temps = [2.0, 0.5, 1.2]
    pos, vel, box, ncx, cps = _gas(60, temps)
    with dsea.Box(pos, vel, box, n_slices=3, precision=precision, temperature=1.0) as b:
        assert slices_of(b) == (ncx, cps)
        b.advance(40)
        vg = b.velocities()
        prof = b.profiles()
    for j, T in enumerate(temps):
        sl = slice(60 * j, 60 * (j + 1))
        assert np.allclose(vg[sl], vel[sl] * math.sqrt(1.0 / T), rtol=tol, atol=tol)
    assert np.all(prof["N"] == 60)
    assert np.allclose(2 * prof["KE"] / (3 * prof["N"]), 1.0, rtol=10 * tol)


@pytest.mark.parametrize("precision", [dsea.FP64, dsea.MIXED])
def test_ring_equals_stepwise_with_thermostat(precision, melted_4k):
    pos, vel, box = melted_4k
    out = []
    for sched in (dsea.SCHED_RING, dsea.SCHED_STEPWISE):
        with dsea.Box(pos, vel, box, n_slices=4, precision=precision, schedule=sched, temperature=1.2) as b:
            b.advance(20)
            b.advance(17)
            out.append((b.positions(), b.velocities()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_mixed_slices_hold_the_target(melted_4k):
    pos, vel, box = melted_4k
    T0 = 0.9
    temps = []
    with dsea.Box(pos, vel, box, n_slices=4, precision=dsea.MIXED, temperature=T0) as b:
        b.advance(150)
        for _ in range(15):
            b.advance(10)
            p = b.profiles()
            temps.append(2 * p["KE"] / (3 * p["N"]))
    late = np.mean(temps, axis=0)
    print("mixed NVT slice temperatures", late)
    assert np.allclose(late, T0, rtol=0.02)


@pytest.mark.parametrize("precision", [dsea.FP64, dsea.MIXED])
def test_profiles_match_oracle(precision, melted_4k):
    pos, vel, box = melted_4k
    with dsea.Box(pos, vel, box, n_slices=4, precision=precision) as b:
        ncx, cps = slices_of(b)
        pg = b.profiles()
        ob = b.observables()
    po = oracle.profiles(pos, vel, box, ncx, cps)
    assert np.array_equal(pg["N"], po[:, 3].astype(np.int64))
    tol = 1e-12 if precision == dsea.FP64 else 2e-6
    F, _, _ = oracle.forces(pos, box, RC)
    frms = float(np.sqrt((F ** 2).sum(1).mean()))
    for k, col in (("U", 0), ("W", 1)):
        assert np.abs(pg[k] - po[:, col]).max() <= tol * len(pos) * frms / 4
    assert np.allclose(pg["KE"], po[:, 2], rtol=1e-12 if precision == dsea.FP64 else 1e-6)
    assert pg["U"].sum() == pytest.approx(ob["U"], rel=1e-12)
    # FP64: after steps too (cells are decided in FP64 like the oracle's slices)
    if precision == dsea.FP64:
        with dsea.Box(pos, vel, box, n_slices=4, precision=precision) as b:
            b.advance(30)
            pg = b.profiles()
            rg, vg = b.positions(), b.velocities()
        po = oracle.profiles(rg, vg, box, ncx, cps)
        assert np.array_equal(pg["N"], po[:, 3].astype(np.int64))
        assert np.allclose(pg["U"], po[:, 0], rtol=1e-11)


@pytest.mark.parametrize("precision", [dsea.MIXED, dsea.FP64])
def test_thermostat_box_in_a_batch_equals_alone(precision, melted_4k):
    """A box under the slice thermostat beside an NVE box in one persistent
    launch: each keeps its own ensemble and ends bit for bit where it ends
    alone (slice factors are per box and per step parity)."""
    pos, vel, box = melted_4k
    other = inputs.batch_specs(n_boxes=1, seed=21, n_max=5000)[0].state()
    kinds = [((pos, vel, box), 1.2, 4), (other, 0.0, 0)]
    steps = [30, 21]
    alone = []
    for (st, T0, ns), n in zip(kinds, steps):
        with dsea.Box(*st, n_slices=ns, precision=precision, temperature=T0) as b:
            b.advance(n)
            alone.append((b.positions(), b.velocities(), b.observables(), b.profiles()))
    boxes = [dsea.Box(*st, n_slices=ns, precision=precision, temperature=T0) for st, T0, ns in kinds]
    try:
        bt = dsea.batch_create([b.h for b in boxes])
        dsea.batch_advance(bt, steps)
        dsea.batch_destroy(bt)
        for b, (r, v, o, p) in zip(boxes, alone):
            assert np.array_equal(b.positions(), r) and np.array_equal(b.velocities(), v)
            assert b.observables() == o
            q = b.profiles()
            assert all(np.array_equal(q[k], p[k]) for k in p)
    finally:
        for b in boxes:
            b.close()


@pytest.mark.parametrize("walls", [False, True])
def test_fp64_nvt_two_layer_slices_anisotropic_box(walls):
    """The slice thermostat where each slice holds two cell layers, in a box
    with three different edges and cell counts (6 x 4 x 3 cells): 60 FP64
    steps and the per-slice profiles against the oracle's."""
    box = np.array([21.7, 13.4, 10.6])
    g = [np.arange(k) * (L / k) + 0.25 for k, L in zip((18, 11, 9), box)]
    pos = np.stack(np.meshgrid(*g, indexing="ij"), axis=-1).reshape(-1, 3)
    pos = inputs.jitter(pos, box, 0.08, seed=43)
    vel = inputs.maxwell_boltzmann(len(pos), 0.9, seed=44)
    T0 = 1.4
    with dsea.Box(pos, vel, box, n_slices=3, precision=dsea.FP64, temperature=T0, walls=walls) as b:
        ncx, cps = slices_of(b)
        assert (ncx, cps) == (6, 2)
        b.advance(60)
        rg, vg = b.positions(), b.velocities()
        pg = b.profiles()
    ro, vo, Fo, obs, st = oracle.run_nvt(pos, vel, box, 60, ncx, cps, T0, walls=walls)
    d = rg - ro
    d[:, 1:] = min_image(d[:, 1:], box[1:])
    if not walls:
        d[:, 0] -= box[0] * np.round(d[:, 0] / box[0])
    dr, dv = np.abs(d).max(), np.abs(vg - vo).max()
    print(f"NVT FP64, two-layer slices, walls {walls}: max |dr| {dr:.3e}, max |dv| {dv:.3e}")
    assert dr <= 1e-9 and dv <= 1e-8
    po = oracle.profiles(rg, vg, box, ncx, cps, walls=walls)
    assert np.array_equal(pg["N"], po[:, 3].astype(np.int64))
    assert np.allclose(pg["KE"], po[:, 2], rtol=1e-10)
