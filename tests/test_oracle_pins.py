"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own code path: closed forms
computed with exact rationals, textbook fcc lattice sums, brute force against
the cell list, finite differences of the energy, an ODE solver from scipy,
and invariants (Newton's third law, translation, time reversal, energy).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2507_11289_gb300 import inputs

RC = 2.5


def _u_ts(r2: Fraction, rc: Fraction) -> Fraction:
    """Truncated-shifted LJ energy, exact rational arithmetic (Sec. 4)."""
    rc2 = rc * rc
    return 4 * (1 / r2 ** 6 - 1 / r2 ** 3) - 4 * (1 / rc2 ** 6 - 1 / rc2 ** 3)


def _fabs(r2: Fraction) -> Fraction:
    """F_abs of Algorithm 1, exact rational arithmetic."""
    return 24 * (2 / r2 ** 6 - 1 / r2 ** 3) / r2


@pytest.mark.parametrize("r", [0.95, 1.0, 2.0 ** (1 / 6), 1.5, 2.2, 2.4999])
def test_pair_law_closed_form(r):
    f, u = oracle.pair(r, RC)
    r2 = Fraction(r) ** 2
    assert u == pytest.approx(float(_u_ts(r2, Fraction(RC))), rel=1e-14, abs=1e-15)
    assert f == pytest.approx(float(_fabs(r2)) * r, rel=1e-13, abs=1e-14)


def test_pair_law_special_points():
    shift = 4 * (2.5 ** -12 - 2.5 ** -6)           # = -0.016316891136
    assert shift == pytest.approx(-0.016316891136, abs=1e-14)
    f, u = oracle.pair(2.0 ** (1 / 6), RC)          # minimum of the 12-6 well
    assert abs(f) < 1e-13 and u == pytest.approx(-1.0 - shift, abs=1e-14)
    f, u = oracle.pair(1.0, RC)                     # sigma: u = -shift, F = 24
    assert f == pytest.approx(24.0, abs=1e-13) and u == pytest.approx(-shift, abs=1e-15)
    f, u = oracle.pair(RC, RC)                      # inclusive cutoff: force jumps, u -> 0
    assert u == pytest.approx(0.0, abs=1e-15)
    assert f == pytest.approx(-0.0389994775, abs=1e-9)
    f, u = oracle.pair(RC * (1 + 1e-12), RC)
    assert f == 0.0 and u == 0.0


def _dimer_box(r):
    box = np.array([12.0, 11.0, 10.0])
    pos = np.array([[3.0, 4.0, 5.0], [3.0 + r, 4.0, 5.0]])
    return pos, box


@pytest.mark.parametrize("method", ["brute", "cells"])
def test_dimer_forces_and_energy(method):
    for r in (0.97, 1.12, 1.8, 2.49):
        pos, box = _dimer_box(r)
        F, U, W = oracle.forces(pos, box, RC, method)
        fr, u = oracle.pair(r, RC)
        # r_01 = r_0 - r_1 = (-r, 0, 0): a repulsive force pushes atom 0 to -x
        assert F[0, 0] == pytest.approx(-fr, rel=1e-13, abs=1e-14)
        assert F[1, 0] == pytest.approx(fr, rel=1e-13, abs=1e-14)
        assert np.all(F[:, 1:] == 0)
        assert U == pytest.approx(u, rel=1e-13, abs=1e-15)
        assert W == pytest.approx(fr * r, rel=1e-13, abs=1e-14)


@pytest.mark.parametrize("method", ["brute", "cells"])
def test_dimer_across_periodic_boundary(method):
    box = np.array([9.0, 9.0, 9.0])
    pos = np.array([[0.3, 1.0, 8.8], [8.6, 1.0, 0.1]])     # separation (0.7, 0, -0.3) through the walls
    F, U, _ = oracle.forces(pos, box, RC, method)
    d = np.array([0.3 - 8.6 + 9.0, 0.0, 8.8 - 0.1 - 9.0])
    r = float(np.linalg.norm(d))
    fr, u = oracle.pair(r, RC)
    assert np.allclose(F[0], d / r * fr, rtol=1e-12, atol=1e-12)
    assert np.allclose(F[1], -d / r * fr, rtol=1e-12, atol=1e-12)
    assert U == pytest.approx(u, rel=1e-13)


def _fcc_lattice_sums(rho, rc):
    """U/N and W/N of a perfect fcc lattice from the coordination shells."""
    a = (4.0 / rho) ** (1 / 3)
    shells = []
    for line in open(__file__.replace("test_oracle_pins.py", "golden/fcc_shells.txt")):
        if line.strip() and not line.startswith("#"):
            k, c = line.split()
            shells.append((int(k), int(c)))
    u = w = 0.0
    for k, count in shells:
        r2 = Fraction(a * a) * Fraction(k, 2)
        if r2 <= Fraction(rc) ** 2:
            u += 0.5 * count * float(_u_ts(r2, Fraction(rc)))
            w += 0.5 * count * float(r2 * _fabs(r2))
    assert a * math.sqrt(6 / 2) > rc, "shell list must reach past the cutoff"
    return u, w


def test_fcc_lattice_sums():
    pos, box = inputs.fcc_lattice(6, 0.8)
    F, U, W = oracle.forces(pos, box, RC, "cells")
    n = len(pos)
    u_ref, w_ref = _fcc_lattice_sums(0.8, RC)
    assert u_ref == pytest.approx(-5.924190441, abs=1e-9)
    assert w_ref == pytest.approx(-23.283624691, abs=1e-9)
    assert U / n == pytest.approx(u_ref, rel=1e-12)
    assert W / n == pytest.approx(w_ref, rel=1e-12)
    assert np.abs(F).max() < 1e-11        # every site is an inversion centre
    # brute force on a smaller copy (cheaper) gives the same per-atom sums
    pos5, box5 = inputs.fcc_lattice(5, 0.8)
    F5, U5, W5 = oracle.forces(pos5, box5, RC, "brute")
    assert U5 / len(pos5) == pytest.approx(u_ref, rel=1e-12)
    assert W5 / len(pos5) == pytest.approx(w_ref, rel=1e-12)


@pytest.mark.parametrize("n_i,amp", [(5, 0.15), (10, 0.12)])
def test_bruteforce_equals_cell_list(n_i, amp):
    pos, box = inputs.fcc_lattice(n_i, 0.8)
    pos = inputs.jitter(pos, box, amp, seed=11 + n_i)
    Fb, Ub, Wb = oracle.forces(pos, box, RC, "brute")
    Fc, Uc, Wc = oracle.forces(pos, box, RC, "cells")
    frms = np.sqrt((Fb ** 2).sum(1).mean())
    assert np.abs(Fb - Fc).max() <= 1e-12 * frms
    assert Uc == pytest.approx(Ub, rel=1e-12)
    assert Wc == pytest.approx(Wb, rel=1e-12)
    # Newton's third law
    assert np.abs(Fc.sum(0)).max() <= 1e-11 * frms * math.sqrt(len(pos))


def test_subset_matches_full():
    pos, box = inputs.fcc_lattice(6, 0.8)
    pos = inputs.jitter(pos, box, 0.1, seed=5)
    F, U, W = oracle.forces(pos, box, RC, "cells")
    idx = np.array([0, 17, 400, len(pos) - 1])
    Fs, us, ws = oracle.forces_subset(pos, box, idx, RC)
    assert np.array_equal(Fs, F[idx])
    _, u_all, w_all = oracle.forces_subset(pos, box, np.arange(len(pos)), RC)
    assert u_all.sum() == pytest.approx(U, rel=1e-12)
    assert w_all.sum() == pytest.approx(W, rel=1e-12)
    assert np.array_equal(us, u_all[idx]) and np.array_equal(ws, w_all[idx])


def test_force_is_minus_energy_gradient():
    pos, box = inputs.fcc_lattice(5, 0.8)
    pos = inputs.jitter(pos, box, 0.12, seed=3)
    # test atoms with no partner within 1e-4 of the cutoff (U has a kink there)
    d = pos[:, None, :] - pos[None, :, :]
    d -= box * np.round(d / box)
    r = np.sqrt((d ** 2).sum(-1))
    np.fill_diagonal(r, 1.0)
    clear = np.flatnonzero(np.abs(r - RC).min(1) > 1e-4)
    assert len(clear) > 20
    F, _, _ = oracle.forces(pos, box, RC, "brute")
    h = 1e-5
    rng = np.random.Generator(np.random.PCG64(0))
    for i in rng.choice(clear, 6, replace=False):
        for k in range(3):
            p1 = pos.copy(); p1[i, k] += h
            p0 = pos.copy(); p0[i, k] -= h
            dU = (oracle.forces(p1, box, RC, "cells")[1] - oracle.forces(p0, box, RC, "cells")[1]) / (2 * h)
            assert -dU == pytest.approx(F[i, k], abs=2e-6 * max(1.0, abs(F[i, k])))


def test_translation_invariance():
    pos, box = inputs.fcc_lattice(5, 0.8)
    pos = inputs.jitter(pos, box, 0.1, seed=9)
    F0, U0, W0 = oracle.forces(pos, box, RC, "cells")
    moved = np.mod(pos + np.array([3.3, -1.7, 0.41]), box)
    F1, U1, W1 = oracle.forces(moved, box, RC, "cells")
    assert np.abs(F1 - F0).max() < 1e-10
    assert U1 == pytest.approx(U0, rel=1e-12) and W1 == pytest.approx(W0, rel=1e-12)


def test_free_flight():
    box = np.array([20.0, 20.0, 20.0])
    pos = np.array([[1.0, 2.0, 3.0], [10.0, 10.0, 10.0]])    # farther apart than rc
    vel = np.array([[0.5, -0.25, 1.0], [0.0, 0.0, 0.0]])
    p, v, F, obs = oracle.run(pos, vel, box, steps=40, dt=0.005)
    assert np.array_equal(v, vel) and np.all(F == 0)
    assert np.allclose(p[0], np.mod(pos[0] + 40 * 0.005 * vel[0], box), atol=1e-13)
    assert np.all(obs[:, 0] == 0) and np.allclose(obs[:, 2], 0.5 * (vel ** 2).sum())


def test_dimer_trajectory_matches_ode_solver():
    """Velocity Verlet on a head-on dimer against scipy's DOP853 on the same
    ODE; the global error must shrink ~4x when dt halves (second order)."""
    from scipy.integrate import solve_ivp

    r0, vrel, T = 1.3, -1.2, 0.8

    def rhs(t, y):      # relative coordinate, reduced mass 1/2
        fr, _ = oracle.pair(y[0], RC)
        return [y[1], 2.0 * fr]

    ref = solve_ivp(rhs, (0, T), [r0, vrel], method="DOP853", rtol=1e-12, atol=1e-12)
    r_ref = ref.y[0, -1]
    errs = []
    for dt in (0.004, 0.002):
        steps = int(round(T / dt))
        box = np.array([30.0, 30.0, 30.0])
        pos = np.array([[10.0, 10.0, 10.0], [10.0 + r0, 10.0, 10.0]])
        vel = np.array([[-vrel / 2, 0, 0], [vrel / 2, 0, 0]])
        p, v, _, obs = oracle.run(pos, vel, box, steps=steps, dt=dt, method="brute")
        errs.append(abs((p[1, 0] - p[0, 0]) - r_ref))
        e = obs[:, 0] + obs[:, 2]
        assert np.abs(e - e[0]).max() < 0.05
        assert np.allclose(v.sum(0), 0.0, atol=1e-13)
    assert errs[0] < 1e-3
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_nve_run_conserves_momentum_and_energy():
    pos, vel, box = inputs.SMALL_4K.state()
    p, v, F, obs = oracle.run(pos, vel, box, steps=60)
    assert np.abs(v.sum(0)).max() < 1e-10
    e = (obs[:, 0] + obs[:, 2]) / len(pos)
    assert np.abs(e - e[0]).max() < 2e-3
    # the synchronised final force equals a fresh evaluation at r_n
    F2, U2, W2 = oracle.forces(p, box, RC, "cells")
    assert np.array_equal(F2, F) and U2 == obs[-1, 0] and W2 == obs[-1, 1]
    # KE of the start matches the drawn temperature with 3N-3 degrees of freedom
    assert obs[0, 2] == pytest.approx(0.5 * (3 * len(pos) - 3) * 1.5, rel=1e-12)


def test_time_reversibility():
    pos, vel, box = inputs.SMALL_4K.state()
    pos = inputs.jitter(pos, box, 0.05, seed=21)
    p, v, _, _ = oracle.run(pos, vel, box, steps=100)
    p2, v2, _, _ = oracle.run(p, -v, box, steps=100)
    d = p2 - pos
    d -= box * np.round(d / box)
    assert np.abs(d).max() < 1e-9
    assert np.abs(v2 + vel).max() < 1e-9


def test_melted_state_is_liquid_like(melted_4k):
    p, v, box = melted_4k
    F, U, W = oracle.forces(p, box, RC, "cells")
    frms = np.sqrt((F ** 2).sum(1).mean())
    assert 10 < frms < 60          # far from the F = 0 lattice
    assert -6.0 < U / len(p) < -3.0


def test_cell_list_does_not_depend_on_thread_count():
    """The OpenMP force loop gives the same bits with one thread as with all
    cores (per-atom sums, and U, W summed afterwards in atom order)."""
    pos, vel, box = inputs.SMALL_4K.state()
    pos = inputs.jitter(pos, box, 0.15, 77)
    n_all = oracle.set_threads(0)
    try:
        oracle.set_threads(1)
        F1, U1, W1 = oracle.forces(pos, box, RC, "cells")
        oracle.set_threads(n_all)
        Fn, Un, Wn = oracle.forces(pos, box, RC, "cells")
    finally:
        oracle.set_threads(n_all)
    assert np.array_equal(F1, Fn) and U1 == Un and W1 == Wn
