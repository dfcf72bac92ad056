"""Seeded synthetic inputs for the Lennard-Jones workloads.

This module holds no part of the method's arithmetic: it only draws the
initial states that both the CUDA path and the CPU oracle are given.

* fcc start (Sec. 4): N_i lattice cells per edge, four molecules per cell,
  edge b = N_i (4/rho)^(1/3), N = 4 N_i^3.  Cell (ix, iy, iz) in
  lexicographic order with basis (0,0,0), (1/2,1/2,0), (1/2,0,1/2),
  (0,1/2,1/2) times the lattice constant; atom ID = position in that order.
* velocities "according to the temperature" (Sec. 4): Maxwell-Boltzmann,
  N(0, sqrt(T)) per component from numpy's PCG64 with the given seed, mean
  removed, then rescaled so that sum(v^2) = (3N - 3) T exactly.
* workload draws for many-box batches and served job streams: atom counts
  log-uniform, rounded to N = 4 n^3 with n = round((N/4)^(1/3)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

RC = 2.5
DT = 0.005


def fcc_lattice(n_i: int, rho: float):
    """Perfect fcc lattice: positions (N, 3) float64 in [0, b)^3 and box (3,)."""
    if n_i < 1 or not rho > 0:
        raise ValueError("n_i >= 1 and rho > 0 required")
    a = (4.0 / rho) ** (1.0 / 3.0)
    b = n_i * a
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    g = np.arange(n_i, dtype=np.float64)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    pos = ((cells[:, None, :] + basis[None, :, :]) * a).reshape(-1, 3)
    return np.ascontiguousarray(pos), np.array([b, b, b])


def maxwell_boltzmann(n: int, T: float, seed: int):
    """Velocities (n, 3) at temperature T with zero total momentum."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.normal(0.0, math.sqrt(T), size=(n, 3))
    v -= v.mean(axis=0)
    dof = 3 * n - 3
    if dof > 0 and T > 0:
        v *= math.sqrt(dof * T / float((v * v).sum()))
    return np.ascontiguousarray(v)


def jitter(pos, box, amplitude: float, seed: int):
    """Positions displaced by U(-amplitude, amplitude) per component, wrapped
    into the box (a generic, non-lattice configuration)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = np.asarray(pos, dtype=np.float64) + rng.uniform(-amplitude, amplitude, size=np.shape(pos))
    return np.ascontiguousarray(np.mod(p, np.asarray(box)[None, :]))


@dataclass(frozen=True)
class BoxSpec:
    """One periodic cubic LJ box: fcc start, Maxwell-Boltzmann velocities."""
    n_i: int
    rho: float
    T: float
    seed: int
    n_slices: int = 0          # 0: one slice per cell layer along x
    steps: int = 0

    @property
    def n_atoms(self) -> int:
        return 4 * self.n_i ** 3

    @property
    def edge(self) -> float:
        return self.n_i * (4.0 / self.rho) ** (1.0 / 3.0)

    def cells_per_axis(self, rc: float = RC) -> int:
        return int(math.floor(self.edge / rc))

    def slices(self, rc: float = RC) -> int:
        return self.n_slices if self.n_slices > 0 else self.cells_per_axis(rc)

    def state(self):
        """(pos, vel, box) of the initial state."""
        pos, box = fcc_lattice(self.n_i, self.rho)
        vel = maxwell_boltzmann(len(pos), self.T, self.seed)
        return pos, vel, box


# The five workloads: an fcc LJ fluid at rc = 2.5, dt = 0.005.
SMALL_4K = BoxSpec(n_i=10, rho=0.8, T=1.5, seed=1, n_slices=4, steps=100)       # 4,000 atoms
FLUID_1M = BoxSpec(n_i=64, rho=0.8, T=1.5, seed=1, n_slices=0, steps=1000)      # 1,048,576 atoms
FLUID_67M = BoxSpec(n_i=256, rho=0.8, T=1.5, seed=1, n_slices=0, steps=200)     # 67,108,864 atoms


def n_i_for_atoms(n_atoms: float) -> int:
    """fcc cells per edge whose 4 n^3 is nearest to n_atoms."""
    return max(1, int(round((n_atoms / 4.0) ** (1.0 / 3.0))))


def batch_specs(n_boxes: int = 512, seed: int = 2, n_min: float = 500, n_max: float = 50_000,
                rho_range=(0.05, 0.9), T_range=(0.7, 3.0), steps: int = 2000, rc: float = RC):
    """Independent boxes of a many-box batch: N log-uniform in [n_min, n_max],
    rho and T uniform.  Boxes with fewer than 3 cells per axis are grown to
    the smallest n_i that gives 3 cells (the 27-cell stencil needs them)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(n_boxes):
        n_atoms = math.exp(rng.uniform(math.log(n_min), math.log(n_max)))
        rho = float(rng.uniform(*rho_range))
        T = float(rng.uniform(*T_range))
        n_i = n_i_for_atoms(n_atoms)
        while n_i * (4.0 / rho) ** (1.0 / 3.0) < 3 * rc:
            n_i += 1
        out.append(BoxSpec(n_i=n_i, rho=rho, T=T, seed=seed * 1_000_003 + k, steps=steps))
    return out


@dataclass(frozen=True)
class Job:
    arrival_s: float
    spec: BoxSpec


def served_stream(rate_per_s: float = 200.0, duration_s: float = 60.0, seed: int = 3,
                  n_min: float = 1_000, n_max: float = 2_000_000, rho_range=(0.3, 0.9),
                  T_range=(0.8, 2.5), steps_range=(100, 10_000), rc: float = RC):
    """Poisson arrivals of LJ boxes: N and steps log-uniform, rho and T uniform."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    jobs = []
    k = 0
    while True:
        t += float(rng.exponential(1.0 / rate_per_s))
        if t >= duration_s:
            break
        n_atoms = math.exp(rng.uniform(math.log(n_min), math.log(n_max)))
        rho = float(rng.uniform(*rho_range))
        T = float(rng.uniform(*T_range))
        steps = int(round(math.exp(rng.uniform(math.log(steps_range[0]), math.log(steps_range[1])))))
        n_i = n_i_for_atoms(n_atoms)
        while n_i * (4.0 / rho) ** (1.0 / 3.0) < 3 * rc:
            n_i += 1
        jobs.append(Job(arrival_s=t, spec=BoxSpec(n_i=n_i, rho=rho, T=T,
                                                  seed=seed * 1_000_003 + k, steps=steps)))
        k += 1
    return jobs
