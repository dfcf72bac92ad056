"""Pins of the oracle's slice thermostat (md_thermo_a/b and md_v3b, Sec. 4.1:
velocity scaling that keeps the temperature constant) and of its spatially
resolved statistics (Sec. 4.2: per-slice results).

Reading pinned here: the synchronised velocities of the atoms of slice j at
step s are scaled by lambda_j(s) = sqrt(T0 / T'_j(s-1)), T'_j(s-1) being the
slice's temperature after the previous step's scaling; lambda = 1 at the
first step.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2507_11289_gb300 import inputs

RC = 2.5


def _gas(n_per_slice, temps, seed=5):
    """Non-interacting atoms (farther apart than rc) in a box cut into
    len(temps) slices of two 3.0-wide cell layers each; slice j at temps[j];
    every atom far from slice boundaries so none changes slice in 60 steps."""
    ns = len(temps)
    box = np.array([6.0 * ns, 80.0, 80.0])
    rng = np.random.Generator(np.random.PCG64(seed))
    pos, vel = [], []
    for j, T in enumerate(temps):
        g = np.arange(n_per_slice)
        p = np.stack([6.0 * j + 3.0 + 0.0 * g, 2.0 + 4.0 * (g % 20), 2.0 + 4.0 * (g // 20)], axis=1)
        v = rng.normal(0.0, 1.0, size=(n_per_slice, 3)) * 0.2
        v *= math.sqrt(T * 3 * n_per_slice / float((v * v).sum()))   # exact slice temperature T
        pos.append(p)
        vel.append(v)
    return np.vstack(pos), np.vstack(vel), box, 2 * ns, 2


def test_nve_limit_is_the_plain_run(melted_4k):
    pos, vel, box = melted_4k
    a = oracle.run(pos, vel, box, steps=20)
    b = oracle.run_nvt(pos, vel, box, steps=20, n_cells_x=4, cells_per_slice=1, temperature=0.0)
    for x, y in zip(a, b[:4]):
        assert np.array_equal(x, y)


def test_ideal_gas_reaches_the_target_in_one_scaling():
    """No forces: KE changes only by the thermostat.  Step 0 measures, step 1
    scales every slice by sqrt(T0 / T_j) exactly, later steps by 1."""
    temps = [2.0, 0.5, 1.2]
    pos, vel, box, ncx, cps = _gas(60, temps)
    T0 = 1.0
    p, v, F, obs, st = oracle.run_nvt(pos, vel, box, steps=40, n_cells_x=ncx, cells_per_slice=cps,
                                      temperature=T0)
    assert np.all(F == 0)
    n = 60
    for j, T in enumerate(temps):
        lam = math.sqrt(T0 / T)
        assert np.allclose(v[j * n:(j + 1) * n], vel[j * n:(j + 1) * n] * lam, rtol=1e-13, atol=1e-15)
        Tj = 2 * st[:, j, 0] / (3 * st[:, j, 1])
        assert Tj[0] == pytest.approx(T, rel=1e-13) and Tj[1] == pytest.approx(T, rel=1e-13)
        assert np.allclose(Tj[2:], T0, rtol=1e-13)
    assert np.all(st[:, :, 1] == n)


def test_liquid_slices_hold_the_target_temperature(melted_4k):
    pos, vel, box = melted_4k
    T0 = 1.1
    _, _, _, _, st = oracle.run_nvt(pos, vel, box, steps=300, n_cells_x=4, cells_per_slice=1,
                                    temperature=T0)
    T = 2 * st[:, :, 0] / (3 * st[:, :, 1])
    late = T[150:].mean(axis=0)
    assert np.allclose(late, T0, rtol=0.01), late
    assert np.all(st[:, :, 1].sum(1) == len(pos))


def test_profiles_sum_to_the_totals(melted_4k):
    pos, vel, box = melted_4k
    pr = oracle.profiles(pos, vel, box, 4, 1)
    F, U, W = oracle.forces(pos, box, RC)
    assert pr[:, 0].sum() == pytest.approx(U, rel=1e-12)
    assert pr[:, 1].sum() == pytest.approx(W, rel=1e-12)
    assert pr[:, 2].sum() == pytest.approx(0.5 * (vel ** 2).sum(), rel=1e-12)
    assert pr[:, 3].sum() == len(pos)


def test_fcc_profiles_are_the_lattice_sums():
    """Perfect fcc (rho 0.8, rc 2.5): every atom carries the lattice sums, so
    U_j / N_j = -5.924190441 and W_j / N_j = -23.283624691 in every slice."""
    pos, box = inputs.fcc_lattice(10, 0.8)
    pr = oracle.profiles(pos, None, box, 4, 1)
    assert np.allclose(pr[:, 0] / pr[:, 3], -5.924190441, rtol=1e-9)
    assert np.allclose(pr[:, 1] / pr[:, 3], -23.283624691, rtol=1e-9)
    assert np.all(pr[:, 3] == 1000) and np.all(pr[:, 2] == 0)
    # with mirror walls the two edge slices lose the pairs across the walls
    pw = oracle.profiles(pos, None, box, 4, 1, walls=True)
    assert pw[0, 0] > pr[0, 0] and pw[3, 0] > pr[3, 0]
    assert np.allclose(pw[1:3, 0], pr[1:3, 0], rtol=1e-12)
