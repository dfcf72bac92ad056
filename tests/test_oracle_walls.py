"""Pins of the oracle's mirror walls along x (Sec. 3 requirement (3) keeps x
non-periodic; Sec. 4.2 places a mirror at the domain boundaries).

The walls are specular: no pair interacts across them, and an atom that the
position update takes past a wall is reflected back with the x components of
its velocity (and of the force it carries into the next velocity update)
reversed.  Pinned here against closed forms (free flight into a wall), brute
force, symmetry and conservation laws.
"""
import numpy as np
import pytest

import oracle
from paper_2507_11289_gb300 import inputs

RC = 2.5


def test_no_pair_across_the_walls():
    box = np.array([9.0, 9.0, 9.0])
    pos = np.array([[0.3, 1.0, 4.0], [8.6, 1.0, 4.0]])   # 0.7 apart through the x boundary
    for method in ("brute", "cells"):
        Fp, Up, _ = oracle.forces(pos, box, RC, method)
        assert np.abs(Fp).max() > 1.0 and Up > 0           # periodic: a close, repulsive pair
        Fw, Uw, Ww = oracle.forces(pos, box, RC, method, walls=True)
        assert np.all(Fw == 0) and Uw == 0 and Ww == 0


def test_pairs_along_y_and_z_still_periodic_between_walls():
    box = np.array([9.0, 9.0, 9.0])
    pos = np.array([[4.0, 0.3, 8.8], [4.0, 8.6, 0.1]])   # separation through the y and z boundaries
    d = np.array([0.0, 0.3 - 8.6 + 9.0, 8.8 - 0.1 - 9.0])
    r = float(np.linalg.norm(d))
    fr, u = oracle.pair(r, RC)
    for method in ("brute", "cells"):
        F, U, _ = oracle.forces(pos, box, RC, method, walls=True)
        assert np.allclose(F[0], d / r * fr, rtol=1e-12, atol=1e-12)
        assert U == pytest.approx(u, rel=1e-13)


@pytest.mark.parametrize("n_i,amp", [(5, 0.15), (10, 0.12)])
def test_bruteforce_equals_cell_list_with_walls(n_i, amp):
    pos, box = inputs.fcc_lattice(n_i, 0.8)
    pos = inputs.jitter(pos, box, amp, seed=40 + n_i)
    Fb, Ub, Wb = oracle.forces(pos, box, RC, "brute", walls=True)
    Fc, Uc, Wc = oracle.forces(pos, box, RC, "cells", walls=True)
    scale = np.sqrt((Fb ** 2).sum(1).mean())
    assert np.abs(Fb - Fc).max() < 1e-12 * scale
    assert Uc == pytest.approx(Ub, rel=1e-12) and Wc == pytest.approx(Wb, rel=1e-12)
    # the walls remove exactly the pairs that met through the x boundary
    Fp, Up, _ = oracle.forces(pos, box, RC, "brute")
    assert Up != Ub


def test_free_flight_into_a_wall_reflects():
    """A lone atom flying at a wall: after the bounce, x(t) = |x0 + vx t| for
    the left wall and 2L - (x0 + vx t) for the right one; vx reverses; y, z
    fly on."""
    box = np.array([12.0, 12.0, 12.0])
    dt, steps = 0.005, 80
    for x0, vx in ((0.3, -1.5), (11.7, 1.5)):
        pos = np.array([[x0, 5.0, 6.0]])
        vel = np.array([[vx, 0.25, -0.5]])
        p, v, F, obs = oracle.run(pos, vel, box, steps=steps, dt=dt, walls=True)
        xt = x0 + vx * steps * dt
        x_expected = abs(xt) if vx < 0 else 2 * box[0] - xt
        assert p[0, 0] == pytest.approx(x_expected, abs=1e-12)
        assert v[0, 0] == -vx and v[0, 1] == 0.25 and v[0, 2] == -0.5
        assert p[0, 1] == pytest.approx(5.0 + 0.25 * steps * dt, abs=1e-12)
        assert 0.0 <= p[0, 0] < box[0]
        assert np.all(F == 0) and np.allclose(obs[:, 2], 0.5 * (vel ** 2).sum())


def test_mirror_symmetric_state_stays_symmetric():
    """Atoms in mirror pairs about the plane x = L/2 (velocities mirrored too)
    stay mirror pairs: the walls treat both halves alike."""
    pos, box = inputs.fcc_lattice(5, 0.8)
    half = pos[pos[:, 0] < box[0] / 2 - 0.3]
    half = inputs.jitter(half, box, 0.1, seed=3)
    half = half[(half[:, 0] > 0.05) & (half[:, 0] < box[0] / 2 - 0.5)]
    vel_h = inputs.maxwell_boltzmann(len(half), 1.2, seed=4)
    mirror = half.copy()
    mirror[:, 0] = box[0] - half[:, 0]
    vel_m = vel_h.copy()
    vel_m[:, 0] = -vel_h[:, 0]
    p, v, F, _ = oracle.run(np.vstack([half, mirror]), np.vstack([vel_h, vel_m]), box, steps=30, walls=True)
    n = len(half)
    assert np.abs(p[:n, 0] - (box[0] - p[n:, 0])).max() < 1e-9
    assert np.abs(p[:n, 1:] - p[n:, 1:]).max() < 1e-9
    assert np.abs(v[:n, 0] + v[n:, 0]).max() < 1e-9


def test_walls_conserve_energy_and_transverse_momentum():
    pos, vel, box = inputs.SMALL_4K.state()
    pos = inputs.jitter(pos, box, 0.05, seed=8)
    p, v, F, obs = oracle.run(pos, vel, box, steps=200, walls=True)
    e = (obs[:, 0] + obs[:, 2]) / len(pos)
    assert np.abs(e - e[0]).max() < 2e-3
    assert np.abs(v[:, 1:].sum(0)).max() < 1e-10          # y and z stay periodic
    assert np.all((p[:, 0] >= 0) & (p[:, 0] < box[0]))
    # the final force is a fresh evaluation between the walls at r_n
    F2, U2, _ = oracle.forces(p, box, RC, "cells", walls=True)
    assert np.array_equal(F2, F) and U2 == obs[-1, 0]


def test_initial_positions_outside_the_walls_are_rejected():
    box = np.array([9.0, 9.0, 9.0])
    with pytest.raises(RuntimeError):
        oracle.run(np.array([[-0.1, 1.0, 1.0]]), np.zeros((1, 3)), box, steps=1, walls=True)
