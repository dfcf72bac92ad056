"""The allocation-free force call, checked against the regular box path.

dsea_forces_noalloc exists for callers that may not let a library allocate
device memory (hosts that own every byte of GPU memory through their own pool,
or loops that cannot afford cudaMalloc's device synchronisation).  It takes
its scratch from a fixed array inside the library, which every call reuses;
this test makes two calls in a row on different configurations (so a stale
scratch from the first would show in the second) and compares each with the
forces and observables of a box created through the allocating entry points,
at the tolerances the parity tests use.  This file sorts last so that a run
stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2507_11289_gb300 import dsea, inputs

pytestmark = pytest.mark.gpu


def _noalloc(torch, pos, vel, box, precision, stream):
    lib = dsea.load()
    n = len(pos)
    p = torch.as_tensor(pos, dtype=torch.float64, device="cuda").contiguous()
    v = None if vel is None else torch.as_tensor(vel, dtype=torch.float64, device="cuda").contiguous()
    f = torch.full((max(n, 1), 3), float("nan"), dtype=torch.float64, device="cuda")
    o = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    b = (ctypes.c_double * 3)(*[float(x) for x in box])
    rc = lib.dsea_forces_noalloc(p.data_ptr() if n else None, None if v is None else v.data_ptr(), n, b,
                                 2.5, precision, f.data_ptr(), o.data_ptr(), stream.cuda_stream)
    return rc, f.cpu().numpy()[:n], o.cpu().numpy()


def _box_path(pos, vel, box, precision):
    with dsea.Box(pos, vel, box, precision=precision) as bx:
        return bx.forces(), bx.observables()


@pytest.mark.parametrize("precision,tol", [(dsea.FP64, 1e-12), (dsea.MIXED, 2e-6)])
def test_noalloc_matches_box_path_on_two_calls(precision, tol):
    """Three calls in a row: a 4,000-atom box, a larger 6,912-atom box, then a
    smaller 4,000-atom box again (different positions), so the last call runs
    on scratch a larger call has just filled."""
    import torch
    stream = torch.cuda.Stream()
    pos_a, vel_a, box_a = inputs.SMALL_4K.state()
    pos_a = inputs.jitter(pos_a, box_a, 0.12, 31)
    pos_b, box_b = inputs.fcc_lattice(12, 0.7)               # a different size and box
    pos_b = inputs.jitter(pos_b, box_b, 0.1, 32)
    vel_b = inputs.maxwell_boltzmann(len(pos_b), 1.1, 33)
    pos_c = inputs.jitter(inputs.SMALL_4K.state()[0], box_a, 0.08, 34)
    for pos, vel, box in ((pos_a, vel_a, box_a), (pos_b, vel_b, box_b), (pos_c, vel_a, box_a)):
        with torch.cuda.stream(stream):
            rc, F, obs = _noalloc(torch, pos, vel, box, precision, stream)
        assert rc == dsea.OK, dsea.status_string(rc)
        F_ref, o_ref = _box_path(pos, vel, box, precision)
        frms = np.sqrt((F_ref ** 2).sum(1).mean())
        assert np.sqrt(((F - F_ref) ** 2).sum(1).mean()) <= tol * frms
        scale = tol * len(pos) * frms
        assert abs(obs[0] - o_ref["U"]) <= scale and abs(obs[1] - o_ref["W"]) <= scale
        assert obs[2] == pytest.approx(o_ref["KE"], rel=1e-12)


@pytest.mark.parametrize("precision", [dsea.FP64, dsea.MIXED])
def test_noalloc_without_velocities_and_empty(precision):
    """vel = NULL gives KE = 0 with the same forces; an empty box gives zeros."""
    import torch
    stream = torch.cuda.Stream()
    pos, vel, box = inputs.SMALL_4K.state()
    pos = inputs.jitter(pos, box, 0.1, 35)
    with torch.cuda.stream(stream):
        rc, F, obs = _noalloc(torch, pos, vel, box, precision, stream)
        rc0, F0, obs0 = _noalloc(torch, pos, None, box, precision, stream)
    assert rc == dsea.OK and rc0 == dsea.OK
    assert np.array_equal(F, F0)
    assert obs0[0] == obs[0] and obs0[1] == obs[1] and obs0[2] == 0.0
    with torch.cuda.stream(stream):
        rc_e, F_e, obs_e = _noalloc(torch, np.zeros((0, 3)), None, box, precision, stream)
    assert rc_e == dsea.OK and F_e.shape == (0, 3)
    assert list(obs_e) == [0.0, 0.0, 0.0]


def test_noalloc_rejects_boxes_beyond_its_scratch():
    import torch
    pos, box = inputs.fcc_lattice(48, 0.8)                   # 442,368 atoms: over 64 MiB
    lib = dsea.load()
    b = (ctypes.c_double * 3)(*[float(x) for x in box])
    dummy = torch.empty(1, dtype=torch.float64, device="cuda")
    rc = lib.dsea_forces_noalloc(dummy.data_ptr(), None, len(pos), b, 2.5, dsea.FP64,
                                 dummy.data_ptr(), None, 0)
    assert rc == dsea.ERR_SCRATCH_LIMIT
    assert "scratch" in dsea.status_string(rc)
