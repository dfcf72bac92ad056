"""CPU FP64 oracle for the slice-streamed Lennard-Jones NVE step.

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the library in
``paper_2507_11289_gb300`` never does, and nothing here imports that library.

* ``lj_oracle.c``   -- plain C, FP64: the pair law and the velocity-Verlet
  loop of Algorithm 1 (Sec. 4), an O(N^2) minimum-image force sum, a
  27-cell linked-cell force sum and a sampled-subset force sum; each with a
  periodic x axis or with mirror walls at x = 0 and x = Lx.
* ``schedule.py``   -- the single-worker stage table (Table 1), Eq. 1 and
  the slice dependency rule of the worker ring (Sec. 3.1, 3.3).

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against closed forms, brute force, finite differences, invariants or the
rows of Table 1; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lj_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblj_oracle.so")

ERRORS = {0: "ok", -1: "invalid argument", -2: "fewer than 3 cells along an axis", -3: "out of memory"}


def build(force: bool = False) -> str:
    """Compile lj_oracle.c with gcc into oracle/_build (no FP contraction, so
    the x86 and Arm builds round alike)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
             "-fno-fast-math", "-fopenmp", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def build_variant(out_path: str, defines=()) -> str:
    """Compile lj_oracle.c with extra -D defines into out_path (the mutation
    tests plant deliberate mistakes this way; the oracle itself never does)."""
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math", "-fopenmp", *[f"-D{d}" for d in defines], "-o", out_path, _SRC,
                           "-lm"])
    return out_path


def use_library(path):
    """Point the wrappers at another build of lj_oracle.c (None: the default
    build).  Returns the previously loaded library handle."""
    global _lib
    prev = _lib
    _lib = None if path is None else _configure(ctypes.CDLL(path))
    return prev


def _load():
    global _lib
    if _lib is None:
        _lib = _configure(ctypes.CDLL(build()))
    return _lib


def _configure(lib):
    d, i64, p = ctypes.c_double, ctypes.c_int64, ctypes.c_void_p
    lib.oracle_pair.argtypes = [d, d, p, p]
    lib.oracle_forces_brute.argtypes = [i64, p, p, d, p, p, p]
    lib.oracle_forces_cells.argtypes = [i64, p, p, d, p, p, p]
    lib.oracle_forces_subset.argtypes = [i64, p, p, d, i64, p, p, p, p]
    lib.oracle_run.argtypes = [i64, p, p, p, d, d, i64, ctypes.c_int, p, p]
    c = ctypes.c_int
    lib.oracle_forces_brute_w.argtypes = [i64, p, p, d, c, p, p, p]
    lib.oracle_forces_cells_w.argtypes = [i64, p, p, d, c, p, p, p]
    lib.oracle_forces_subset_w.argtypes = [i64, p, p, d, c, i64, p, p, p, p]
    lib.oracle_run_w.argtypes = [i64, p, p, p, d, d, i64, c, c, p, p]
    lib.oracle_run_ex.argtypes = [i64, p, p, p, d, d, i64, c, c, c, c, d, p, p, p]
    lib.oracle_profiles.argtypes = [i64, p, p, p, d, c, c, c, p]
    lib.oracle_set_threads.argtypes = [c]
    for f in (lib.oracle_pair, lib.oracle_forces_brute, lib.oracle_forces_cells,
              lib.oracle_forces_subset, lib.oracle_run, lib.oracle_forces_brute_w,
              lib.oracle_forces_cells_w, lib.oracle_forces_subset_w, lib.oracle_run_w,
              lib.oracle_run_ex, lib.oracle_profiles):
        f.restype = ctypes.c_int
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(code: int):
    if code != 0:
        raise RuntimeError(f"oracle error {code}: {ERRORS.get(code, 'unknown')}")


def _pos(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1, 3))


def pair(r: float, rc: float = 2.5):
    """(radial force, energy) of one pair at distance r (Algorithm 1, Sec. 4)."""
    f, u = ctypes.c_double(), ctypes.c_double()
    _check(_load().oracle_pair(r, rc, ctypes.byref(f), ctypes.byref(u)))
    return f.value, u.value


def forces(pos, box, rc: float = 2.5, method: str = "cells", walls: bool = False):
    """Forces (N,3), total pair energy U and virial W = sum_{i<j} r_ij.F_ij.

    method: "cells" (27-cell stencil, directed pairs as in Algorithm 1) or
    "brute" (all unordered pairs, minimum image).  walls: mirror walls at
    x = 0 and x = Lx instead of a periodic x axis (no pair across them)."""
    p = _pos(pos)
    b = np.ascontiguousarray(box, dtype=np.float64)
    F = np.zeros_like(p)
    U, W = ctypes.c_double(), ctypes.c_double()
    fn = {"cells": _load().oracle_forces_cells_w, "brute": _load().oracle_forces_brute_w}[method]
    _check(fn(len(p), _ptr(p), _ptr(b), rc, 1 if walls else 0, _ptr(F), ctypes.byref(U), ctypes.byref(W)))
    return F, U.value, W.value


def forces_subset(pos, box, idx, rc: float = 2.5, walls: bool = False):
    """Forces (m,3) and per-atom half pair energy / half virial (m,) of the
    atoms idx only, from a 27-cell list over all atoms."""
    p = _pos(pos)
    b = np.ascontiguousarray(box, dtype=np.float64)
    ix = np.ascontiguousarray(idx, dtype=np.int64)
    F = np.zeros((len(ix), 3))
    u = np.zeros(len(ix))
    w = np.zeros(len(ix))
    _check(_load().oracle_forces_subset_w(len(p), _ptr(p), _ptr(b), rc, 1 if walls else 0, len(ix),
                                          _ptr(ix), _ptr(F), _ptr(u), _ptr(w)))
    return F, u, w


def run(pos, vel, box, steps: int, rc: float = 2.5, dt: float = 0.005, method: str = "cells",
        walls: bool = False):
    """Velocity-Verlet NVE run of Algorithm 1.

    Returns (pos_n, vel_n, F_n, obs) with obs[s] = (U, W, KE) for s = 0..steps.
    Positions come back wrapped into [0, L).  walls: mirror walls at x = 0
    and x = Lx (the initial x must lie in [0, Lx))."""
    p = _pos(pos).copy()
    v = _pos(vel).copy()
    b = np.ascontiguousarray(box, dtype=np.float64)
    F = np.zeros_like(p)
    obs = np.zeros((steps + 1, 3))
    _check(_load().oracle_run_w(len(p), _ptr(p), _ptr(v), _ptr(b), rc, dt, steps,
                                1 if method == "cells" else 0, 1 if walls else 0, _ptr(F), _ptr(obs)))
    return p, v, F, obs


def run_nvt(pos, vel, box, steps: int, n_cells_x: int, cells_per_slice: int, temperature: float,
            rc: float = 2.5, dt: float = 0.005, method: str = "cells", walls: bool = False):
    """Velocity-Verlet run with the slice thermostat (temperature > 0; 0 = NVE).

    Slices: n_cells_x cell layers of width Lx / n_cells_x along x, cells_per_slice
    per slice.  Returns (pos_n, vel_n, F_n, obs, stats) with obs[s] = (U, W, KE)
    and stats[s, j] = (KE_j, N_j) of slice j at step s before that step's scaling."""
    p = _pos(pos).copy()
    v = _pos(vel).copy()
    b = np.ascontiguousarray(box, dtype=np.float64)
    F = np.zeros_like(p)
    obs = np.zeros((steps + 1, 3))
    ns = n_cells_x // cells_per_slice
    stats = np.zeros((steps + 1, ns, 2))
    _check(_load().oracle_run_ex(len(p), _ptr(p), _ptr(v), _ptr(b), rc, dt, steps,
                                 1 if method == "cells" else 0, 1 if walls else 0, n_cells_x,
                                 cells_per_slice, temperature, _ptr(F), _ptr(obs), _ptr(stats)))
    return p, v, F, obs, stats


def profiles(pos, vel, box, n_cells_x: int, cells_per_slice: int, rc: float = 2.5, walls: bool = False):
    """Per-slice (U_j, W_j, KE_j, N_j): half pair energies, half pair virials and
    kinetic energies of the atoms of each slice, and their count."""
    p = _pos(pos)
    v = None if vel is None else _pos(vel)
    b = np.ascontiguousarray(box, dtype=np.float64)
    out = np.zeros((n_cells_x // cells_per_slice, 4))
    _check(_load().oracle_profiles(len(p), _ptr(p), None if v is None else _ptr(v), _ptr(b), rc,
                                   1 if walls else 0, n_cells_x, cells_per_slice, _ptr(out)))
    return out


def set_threads(n: int = 0) -> int:
    """Threads of the OpenMP force loop (0: all cores, the default).  Results
    do not depend on it.  Returns the count now in effect."""
    return int(_load().oracle_set_threads(int(n)))
