"""GPU parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Tolerances (written from the stated targets):
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


def min_image(d, box):
    return d - box * np.round(d / box)


def rms(a):
    return float(np.sqrt((np.asarray(a) ** 2).sum(-1).mean()))


def force_err(Fg, Fo):
    return rms(Fg - Fo) / rms(Fo), float(np.sqrt(((Fg - Fo) ** 2).sum(-1)).max() / rms(Fo))


def jittered_4k(amp=0.12, seed=7):
    pos, vel, box = inputs.SMALL_4K.state()
    return inputs.jitter(pos, box, amp, seed), vel, box


@pytest.mark.parametrize("schedule", [dsea.SCHED_RING, dsea.SCHED_STEPWISE])
@pytest.mark.parametrize("tiles", [(4, 4), (2, 3), (6, 6)])
def test_fp64_forces_match_oracle(schedule, tiles):
    pos, vel, box = jittered_4k()
    Fo, Uo, Wo = oracle.forces(pos, box, RC, "cells")
    with dsea.Box(pos, vel, box, n_slices=4, precision=dsea.FP64, schedule=schedule,
                  tile_y=tiles[0], tile_z=tiles[1]) as b:
        Fg = b.forces()
        ob = b.observables()
        rg = b.positions()
    e_rms, e_max = force_err(Fg, Fo)
    assert e_rms <= 1e-12, (e_rms, e_max)
    assert ob["U"] == pytest.approx(Uo, rel=1e-12)
    assert ob["W"] == pytest.approx(Wo, rel=1e-12)
    assert ob["KE"] == pytest.approx(0.5 * (vel ** 2).sum(), rel=1e-12)
    assert np.abs(min_image(rg - pos, box)).max() < 1e-12


def test_mixed_forces_match_oracle(melted_4k):
    pos, vel, box = melted_4k
    Fo, Uo, Wo = oracle.forces(pos, box, RC, "cells")
    with dsea.Box(pos, vel, box, n_slices=4, precision=dsea.MIXED) as b:
        Fg = b.forces()
        ob = b.observables()
    e_rms, e_max = force_err(Fg, Fo)
    print(f"mixed force error: rms {e_rms:.3e}  max {e_max:.3e} (of rms force)")
    assert e_rms <= 2e-6
    # U and W are sums of FP32 pair terms that cancel (W of a liquid is a small
    # difference of terms ~ F * sigma): hold them to 2e-6 of N * F_rms * sigma
    scale = 2e-6 * len(pos) * rms(Fo)
    assert abs(ob["U"] - Uo) <= scale
    assert abs(ob["W"] - Wo) <= scale


@pytest.mark.parametrize("precision", [dsea.FP64, dsea.MIXED])
def test_first_config_trajectory_100_steps(precision):
    """4,000-atom fcc start, T* 1.5, 4 slices, 100 velocity-Verlet steps."""
    spec = inputs.SMALL_4K
    pos, vel, box = spec.state()
    ro, vo, Fo, obs = oracle.run(pos, vel, box, steps=spec.steps)
    with dsea.Box(pos, vel, box, n_slices=spec.n_slices, precision=precision) as b:
        b.advance(spec.steps)
        rg, vg, Fg, og = b.positions(), b.velocities(), b.forces(), b.observables()
    dr = np.abs(min_image(rg - ro, box)).max()
    dv = np.abs(vg - vo).max()
    print(f"precision {precision}: max |dr| {dr:.3e}, max |dv| {dv:.3e}")
    assert og["step"] == spec.steps
    if precision == dsea.FP64:
        assert dr <= 1e-9 and dv <= 1e-8
        assert force_err(Fg, Fo)[0] <= 1e-10
        assert og["U"] == pytest.approx(obs[-1, 0], rel=1e-10)
        assert og["W"] == pytest.approx(obs[-1, 1], rel=1e-10)
        assert og["KE"] == pytest.approx(obs[-1, 2], rel=1e-10)
    else:
        # mixed: trajectories separate chaotically; they stay close over 100 steps
        assert dr <= 1e-4
        assert og["U"] + og["KE"] == pytest.approx(obs[-1, 0] + obs[-1, 2], abs=1e-3 * len(pos))


@pytest.mark.parametrize("precision", [dsea.FP64, dsea.MIXED])
def test_ring_equals_stepwise_bitwise(precision, melted_4k):
    pos, vel, box = melted_4k
    out = []
    for sched in (dsea.SCHED_RING, dsea.SCHED_STEPWISE):
        with dsea.Box(pos, vel, box, n_slices=4, precision=precision, schedule=sched) as b:
            b.advance(25)
            b.advance(15)
            out.append((b.positions(), b.velocities(), b.observables()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]


@pytest.mark.parametrize("precision", [dsea.MIXED, dsea.FP64])
@pytest.mark.parametrize("temperature", [0.0, 1.2])
def test_unit_shape_does_not_change_results(melted_4k, precision, temperature):
    """The unit shape only groups home cells: each atom's force is summed in an
    order fixed by the state, the observables and profiles are fixed-order
    sums of per-cell partials, and the thermostat sums kinetic energies in
    exact fixed point.  Every result is bitwise the same for every shape."""
    pos, vel, box = melted_4k
    ref = None
    for ty, tz in [(1, 1), (2, 5), (4, 4), (6, 6)]:
        with dsea.Box(pos, vel, box, n_slices=4, precision=precision, tile_y=ty, tile_z=tz,
                      temperature=temperature) as b:
            b.advance(20 if precision == dsea.MIXED else 8)
            got = (b.positions(), b.velocities(), b.observables(), b.profiles())
        if ref is None:
            ref = got
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), (ty, tz)
        assert got[2] == ref[2], (ty, tz)
        assert all(np.array_equal(got[3][k], ref[3][k]) for k in ref[3]), (ty, tz)


@pytest.mark.parametrize("precision", [dsea.MIXED, dsea.FP64])
def test_stage_count_does_not_change_results(precision):
    """The ring's stage count (CTAs of the persistent launch) only changes
    which stage takes which unit: one CTA, a few, the default rule and every
    resident CTA give the same bits on a 62,500-atom box (17 slices, where
    the default rule runs about half the resident stages)."""
    import torch
    pos, box = inputs.fcc_lattice(25, 0.8)
    vel = inputs.maxwell_boltzmann(len(pos), 1.5, 8)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ref = None
    for ctas in (1, 3, 0, sms * (4 if precision == dsea.MIXED else 2)):
        with dsea.Box(pos, vel, box, precision=precision, ctas=ctas) as b:
            b.advance(12 if precision == dsea.MIXED else 4)
            got = (b.positions(), b.velocities(), b.observables())
        if ref is None:
            ref = got
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), ctas
        assert got[2] == ref[2], ctas


@pytest.mark.parametrize("n_slices", [3, 4, 6])
def test_slice_count_fp64_parity(n_slices, melted_4k):
    pos, vel, box = melted_4k
    ro, vo, _, _ = oracle.run(pos, vel, box, steps=30)
    with dsea.Box(pos, vel, box, n_slices=n_slices, precision=dsea.FP64) as b:
        assert b.info()["n_slices"] == n_slices
        b.advance(30)
        rg = b.positions()
    assert np.abs(min_image(rg - ro, box)).max() <= 1e-9


def test_mixed_energy_drift_1000_steps(melted_4k):
    """NVE drift of the mixed form over 1000 steps, next to the oracle's own."""
    pos, vel, box = melted_4k
    n = len(pos)
    e_gpu = []
    with dsea.Box(pos, vel, box, n_slices=4, precision=dsea.MIXED) as b:
        for _ in range(100):
            o = b.observables()
            e_gpu.append((o["U"] + o["KE"]) / n)
            b.advance(10)
        o = b.observables()
        e_gpu.append((o["U"] + o["KE"]) / n)
        r_end = b.positions()
        F_end = b.forces()
    _, _, _, obs = oracle.run(pos, vel, box, steps=1000)
    e_ora = (obs[::10, 0] + obs[::10, 2]) / n
    e_gpu = np.array(e_gpu)
    drift_gpu = abs(e_gpu[-10:].mean() - e_gpu[:10].mean())
    drift_ora = abs(e_ora[-10:].mean() - e_ora[:10].mean())
    print(f"drift per atom over 1000 steps: mixed {drift_gpu:.3e}, oracle FP64 {drift_ora:.3e}; "
          f"max |E-E0| mixed {np.abs(e_gpu - e_gpu[0]).max():.3e}")
    # the stated bar, flat: the periodic box's FP64 drift is far below it
    assert drift_gpu <= 1e-4
    # the per-step force gate at the end of the run, where the configuration
    # is furthest from the lattice: the oracle's forces at the GPU's positions
    Fo_end, _, _ = oracle.forces(r_end, box, RC, "cells")
    e_rms, e_max = force_err(F_end, Fo_end)
    print(f"mixed force error after 1000 steps: rms {e_rms:.3e}  max {e_max:.3e} (of rms force)")
    assert e_rms <= 2e-6


def test_smallest_box_and_ragged_units():
    # 3 cells per axis (the minimum) and a 7-cell axis cut by 4-cell units
    pos, box = inputs.fcc_lattice(5, 0.8)            # 8.55 edge: 3 cells
    pos = inputs.jitter(pos, box, 0.1, 3)
    vel = inputs.maxwell_boltzmann(len(pos), 1.2, 4)
    ro, vo, _, _ = oracle.run(pos, vel, box, steps=20)
    with dsea.Box(pos, vel, box, precision=dsea.FP64) as b:
        assert b.info()["cells"] == [3, 3, 3]
        b.advance(20)
        assert np.abs(min_image(b.positions() - ro, box)).max() <= 1e-9
    pos, box = inputs.fcc_lattice(11, 0.8)           # 18.8 edge: 7 cells
    pos = inputs.jitter(pos, box, 0.1, 5)
    vel = inputs.maxwell_boltzmann(len(pos), 1.0, 6)
    ro, _, _, _ = oracle.run(pos, vel, box, steps=20)
    with dsea.Box(pos, vel, box, precision=dsea.FP64, tile_y=4, tile_z=3) as b:
        assert b.info()["cells"] == [7, 7, 7]
        b.advance(20)
        assert np.abs(min_image(b.positions() - ro, box)).max() <= 1e-9


def test_empty_single_atom_and_free_flight():
    box = np.array([9.0, 9.0, 9.0])
    with dsea.Box(np.zeros((0, 3)), None, box) as b:
        b.advance(5)
        assert b.positions().shape == (0, 3)
        assert b.observables() == {"step": 5, "U": 0.0, "W": 0.0, "KE": 0.0}
    pos = np.array([[1.0, 2.0, 3.0], [6.0, 6.0, 6.0]])
    vel = np.array([[0.5, -0.25, 1.0], [0.0, 0.0, 0.0]])
    with dsea.Box(pos, vel, box) as b:
        b.advance(40)
        r = b.positions()
        assert np.allclose(r[0], np.mod(pos[0] + 40 * 0.005 * vel[0], box), atol=1e-13)
        assert np.array_equal(b.velocities(), vel) and np.all(b.forces() == 0)


def test_dimer_across_periodic_boundary():
    box = np.array([9.0, 9.0, 9.0])
    pos = np.array([[0.3, 1.0, 8.8], [8.6, 1.0, 0.1]])
    Fo, Uo, Wo = oracle.forces(pos, box, RC, "brute")
    for prec in (dsea.FP64, dsea.MIXED):
        with dsea.Box(pos, None, box, precision=prec) as b:
            Fg = b.forces()
            tol = 1e-12 if prec == dsea.FP64 else 2e-6
            assert np.abs(Fg - Fo).max() <= tol * np.abs(Fo).max()
            assert b.observables()["U"] == pytest.approx(Uo, rel=10 * tol)


@pytest.mark.parametrize("precision", [dsea.FP64, dsea.MIXED])
def test_full_1m_box_sampled_atoms(precision):
    """1,048,576-atom box (64^3 fcc cells, rho 0.8), 43 slices, in the launch
    form the benchmark times; forces at 256 sampled atoms against the oracle,
    plus Newton's third law over all atoms."""
    spec = inputs.FLUID_1M
    pos, vel, box = spec.state()
    pos = inputs.jitter(pos, box, 0.1, 17)
    rng = np.random.Generator(np.random.PCG64(5))
    idx = np.sort(rng.choice(len(pos), 256, replace=False))
    Fo, _, _ = oracle.forces_subset(pos, box, idx, RC)
    with dsea.Box(pos, vel, box, precision=precision) as b:
        info = b.info()
        assert info["n_slices"] == 43 and info["cells"] == [43, 43, 43]
        Fg = b.forces()
    tol = 1e-12 if precision == dsea.FP64 else 2e-6
    e_rms, e_max = force_err(Fg[idx], Fo)
    print(f"1M box, precision {precision}: force error rms {e_rms:.3e}  max {e_max:.3e} (of rms force)")
    assert e_rms <= tol
    assert np.abs(Fg.sum(0)).max() <= (1e-9 if precision == dsea.FP64 else 1e-3) * rms(Fg) * np.sqrt(len(pos))


def test_1m_box_after_20_mixed_steps():
    """The 1M box after 20 mixed ring steps from the jittered lattice (a
    disordered state): forces at 256 sampled atoms against the oracle at the
    GPU's positions."""
    spec = inputs.FLUID_1M
    pos, vel, box = spec.state()
    pos = inputs.jitter(pos, box, 0.1, 19)
    rng = np.random.Generator(np.random.PCG64(9))
    idx = np.sort(rng.choice(len(pos), 256, replace=False))
    with dsea.Box(pos, vel, box, precision=dsea.MIXED) as b:
        b.advance(20)
        r = b.positions()
        F = b.forces()
    Fo, _, _ = oracle.forces_subset(r, box, idx, RC)
    e_rms, e_max = force_err(F[idx], Fo)
    print(f"1M box after 20 steps: force error rms {e_rms:.3e}  max {e_max:.3e} (of rms force)")
    assert e_rms <= 2e-6


def test_1m_box_energy_drift_over_the_benchmark_run():
    """The benchmark's 1,048,576-atom run as it is timed (fcc start, T* 1.5,
    ten advances of 100 mixed ring steps): the total energy per atom, sampled
    after each advance, drifts by at most the mixed form's bar of 1e-4
    epsilon per atom between the first and the last three samples, and after
    the 1000 steps the forces at 256 sampled atoms are the oracle's at the
    GPU's positions within the per-step gate."""
    spec = inputs.FLUID_1M
    pos, vel, box = spec.state()
    n = len(pos)
    e = []
    with dsea.Box(pos, vel, box, precision=dsea.MIXED) as b:
        o = b.observables()
        e.append((o["U"] + o["KE"]) / n)
        for _ in range(10):
            b.advance(100)
            o = b.observables()
            e.append((o["U"] + o["KE"]) / n)
        assert o["step"] == 1000
        r, F = b.positions(), b.forces()
    e = np.array(e)
    drift = abs(e[-3:].mean() - e[:3].mean())
    print(f"1M box, 1000 mixed steps: drift {drift:.3e} per atom, max |E - E0| {np.abs(e - e[0]).max():.3e}")
    assert drift <= 1e-4
    # from the perfect lattice (zero forces) the velocity-Verlet energy moves by
    # about dt^2 <F^2> / 24 ~ 3e-4 per atom as the lattice melts: the
    # integrator's offset from the true energy, not drift; a sanity bound only
    assert np.abs(e - e[0]).max() <= 1e-3
    rng = np.random.Generator(np.random.PCG64(23))
    idx = np.sort(rng.choice(n, 256, replace=False))
    Fo, _, _ = oracle.forces_subset(r, box, idx, RC)
    e_rms, e_max = force_err(F[idx], Fo)
    print(f"1M box after 1000 steps: force error rms {e_rms:.3e}  max {e_max:.3e} (of rms force)")
    assert e_rms <= 2e-6


def test_full_67m_box_sampled_atoms():
    """67,108,864-atom box (256^3 fcc cells, rho 0.8), 175 slices, mixed form
    as the benchmark runs it: forces at 512 sampled atoms against the oracle
    after one ring step from a jittered lattice, plus Newton's third law."""
    spec = inputs.FLUID_67M
    pos, vel, box = spec.state()
    pos = inputs.jitter(pos, box, 0.1, 23)
    rng = np.random.Generator(np.random.PCG64(6))
    idx = np.sort(rng.choice(len(pos), 512, replace=False))
    with dsea.Box(pos, vel, box, precision=dsea.MIXED) as b:
        info = b.info()
        assert info["n_slices"] == 175 and info["cells"] == [175, 175, 175]
        Fg = b.forces()
        b.advance(1)
        r1 = b.positions()
        F1 = b.forces()
    Fo, _, _ = oracle.forces_subset(pos, box, idx, RC)
    e_rms, e_max = force_err(Fg[idx], Fo)
    print(f"67M box: force error rms {e_rms:.3e}  max {e_max:.3e} (of rms force)")
    assert e_rms <= 2e-6
    assert np.abs(Fg.sum(0)).max() <= 1e-3 * rms(Fg) * np.sqrt(len(pos))
    del Fg
    # one step later: the sampled atoms' forces at the GPU's new positions
    F1o, _, _ = oracle.forces_subset(r1, box, idx, RC)
    e_rms, e_max = force_err(F1[idx], F1o)
    print(f"67M box after one step: force error rms {e_rms:.3e}  max {e_max:.3e} (of rms force)")
    assert e_rms <= 2e-6


@pytest.mark.parametrize("precision", [dsea.FP64, dsea.MIXED])
def test_large_cells_many_chunks_and_windows(precision):
    """Cells of ~39 atoms (wide slices, y/z cells just under 4/3 rc): home
    cells run in two 32-atom chunks and a neighbourhood spans three list
    windows of the mixed form."""
    box = np.array([14.9, 9.99, 9.99])
    g = [np.arange(k) * (L / k) for k, L in zip((13, 9, 9), box)]   # a simple cubic grid, spacing ~1.1
    pos = np.stack(np.meshgrid(*g, indexing="ij"), axis=-1).reshape(-1, 3)
    pos = inputs.jitter(pos, box, 0.05, seed=32)
    n = len(pos)
    vel = inputs.maxwell_boltzmann(n, 1.0, seed=33)
    Fo, Uo, Wo = oracle.forces(pos, box, RC, "cells")
    with dsea.Box(pos, vel, box, n_slices=3, precision=precision) as b:
        inf = b.info()
        per_cell = n / np.prod(inf["cells"])
        assert per_cell > 32, per_cell
        Fg = b.forces()
        e_rms, _ = force_err(Fg, Fo)
        assert e_rms <= (1e-12 if precision == dsea.FP64 else 2e-6), e_rms
        if precision == dsea.FP64:
            ro, _, _, _ = oracle.run(pos, vel, box, steps=30)
            b.advance(30)
            assert np.abs(min_image(b.positions() - ro, box)).max() <= 1e-9



@pytest.mark.parametrize("precision", [dsea.FP64, dsea.MIXED])
@pytest.mark.parametrize("walls", [False, True])
def test_anisotropic_box_with_two_layer_slices(precision, walls):
    """Three different edges and cell counts (6 x 4 x 3 cells of 3.62 x 3.35 x
    3.53) and three slices of two cell layers each, periodic or with mirror
    walls along x: forces against the oracle, then 40 steps.  FP64: positions
    to 1e-9 of the oracle's; mixed: forces at the GPU's own end positions to
    2e-6 of the rms force."""
    box = np.array([21.7, 13.4, 10.6])
    g = [np.arange(k) * (L / k) + 0.25 for k, L in zip((18, 11, 9), box)]   # spacing 1.18-1.22
    pos = np.stack(np.meshgrid(*g, indexing="ij"), axis=-1).reshape(-1, 3)
    pos = inputs.jitter(pos, box, 0.08, seed=41)
    vel = inputs.maxwell_boltzmann(len(pos), 1.2, seed=42)
    Fo, _, _ = oracle.forces(pos, box, RC, "cells", walls=walls)
    tol = 1e-12 if precision == dsea.FP64 else 2e-6
    with dsea.Box(pos, vel, box, n_slices=3, precision=precision, walls=walls) as b:
        inf = b.info()
        assert (inf["n_slices"], inf["cells_per_slice_x"], list(inf["cells"])) == (3, 2, [6, 4, 3])
        e0, _ = force_err(b.forces(), Fo)
        b.advance(40)
        rg, Fg = b.positions(), b.forces()
    print(f"precision {precision} walls {walls}: force error rms {e0:.3e} of rms force")
    assert e0 <= tol
    if precision == dsea.FP64:
        ro, _, _, _ = oracle.run(pos, vel, box, steps=40, walls=walls)
        d = rg - ro
        d[:, 1:] -= box[1:] * np.round(d[:, 1:] / box[1:])
        if not walls:
            d[:, 0] -= box[0] * np.round(d[:, 0] / box[0])
        assert np.abs(d).max() <= 1e-9
    else:
        Fe, _, _ = oracle.forces(rg, box, RC, "cells", walls=walls)
        e1, _ = force_err(Fg, Fe)
        print(f"  after 40 steps, at the GPU's positions: rms {e1:.3e}")
        assert e1 <= 2e-6

def _sparse_gas(n, box, dmin, seed):
    """n atoms uniform in the box, no two closer than dmin (minimum image)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = np.zeros((0, 3))
    while len(pos) < n:
        p = rng.uniform(0.0, 1.0, 3) * box
        if len(pos) == 0 or np.sqrt((min_image(pos - p, box) ** 2).sum(1)).min() >= dmin:
            pos = np.vstack([pos, p])
    return pos


@pytest.mark.parametrize("precision", [dsea.FP64, dsea.MIXED])
@pytest.mark.parametrize("n", [60, 240, 864])
def test_sparse_gas_pairs_at_every_angle(precision, n):
    """Sparse gases (rho 0.016, 0.063 and 0.23): the cells grow to 3.12 (five
    per axis, the most that keeps them within 1.5 rc), so about half an atom,
    two and seven atoms share a cell; pairs reach the cutoff across faces,
    edges and corners in every direction, and the mixed form prunes its lists
    to the neighbours near the box its home atoms span (a lone atom's short
    list is kept whole)."""
    box = np.array([15.6, 15.6, 15.6])
    pos = _sparse_gas(n, box, 0.95, seed=41)
    Fo, Uo, Wo = oracle.forces(pos, box, RC, "brute")
    with dsea.Box(pos, None, box, precision=precision) as b:
        assert b.info()["cells"] == [5, 5, 5]
        Fg = b.forces()
        ob = b.observables()
    tol = 1e-12 if precision == dsea.FP64 else 2e-6
    e_rms, _ = force_err(Fg, Fo)
    assert e_rms <= tol, e_rms
    scale = tol * len(pos) * rms(Fo)                  # U and W are sums of cancelling pair terms
    assert abs(ob["U"] - Uo) <= scale and abs(ob["W"] - Wo) <= scale


@pytest.mark.parametrize("precision", [dsea.FP64, dsea.MIXED])
def test_corner_and_edge_neighbours_near_the_cutoff(precision):
    """Lone atoms near a cell corner with partners in the corner, edge and
    face neighbour cells just inside (2.49) and just outside (2.51) the
    cutoff: the inside pairs interact, the outside ones do not."""
    box = np.array([10.4, 10.4, 10.4])                 # 4 cells of 2.6 per axis
    a = np.array([2.55, 2.55, 2.55])                   # near the corner (2.6, 2.6, 2.6) of cell (0, 0, 0)
    u = [np.array(v, float) / np.linalg.norm(v) for v in ((1, 1, 1), (1, 1, 0), (1, 0, 0))]
    for d, interacting in ((2.49, True), (2.51, False)):
        for k in u:
            pos = np.array([a, a + d * k])
            Fo, Uo, _ = oracle.forces(pos, box, RC, "brute")
            assert (Uo != 0.0) == interacting
            with dsea.Box(pos, None, box, precision=precision) as b:
                Fg = b.forces()
                Ug = b.observables()["U"]
            if interacting:
                tol = 1e-12 if precision == dsea.FP64 else 2e-6
                assert np.abs(Fg - Fo).max() <= tol * np.abs(Fo).max()
                # near the cutoff the shifted pair energy is a small difference
                # of terms of size 4 r^-6: rounding is relative to those
                assert abs(Ug - Uo) <= 10 * tol * 4.0 * d ** -6
            else:
                assert np.all(Fg == 0.0) and Ug == 0.0


@pytest.mark.parametrize("rho", [0.05, 0.1, 0.2, 0.25, 0.3, 0.45, 0.6, 0.75, 0.9])
def test_mixed_force_error_across_densities(rho):
    """The mixed form's per-step force bar across the densities of the batched
    and served workloads (0.05-0.9).  Below rho = 0.77 the cells grow toward
    1.5 rc, so the FP32 coordinates of a neighbourhood grow with them.  Forces
    of a jittered fcc start, then at the GPU's own positions after 100 mixed
    steps at T 2.0, against the oracle at the same positions."""
    pos, box = inputs.fcc_lattice(12, rho)                 # 6,912 atoms
    pos = inputs.jitter(pos, box, 0.1, seed=51)
    vel = inputs.maxwell_boltzmann(len(pos), 2.0, seed=52)
    Fo, _, _ = oracle.forces(pos, box, RC, "cells")
    with dsea.Box(pos, vel, box, precision=dsea.MIXED) as b:
        edge = b.info()["cell_edge"]
        F0 = b.forces()
        b.advance(100)
        rg, Fg = b.positions(), b.forces()
    if rms(Fo) == 0.0:   # rho 0.05: the fcc spacing (3.05) exceeds rc, no pair in range
        assert np.all(F0 == 0.0)
        e0, m0 = 0.0, 0.0
    else:
        e0, m0 = force_err(F0, Fo)
    Fe, _, _ = oracle.forces(rg, box, RC, "cells")
    assert rms(Fe) > 0.0
    e1, m1 = force_err(Fg, Fe)
    print(f"rho {rho}: cell edge {edge[0]:.3f}; force error rms {e0:.3e} (max {m0:.2e}), "
          f"after 100 steps rms {e1:.3e} (max {m1:.2e})")
    assert e0 <= 2e-6 and e1 <= 2e-6
