"""Scenarios run once on the release library and once on the bounds-checked
one (DSEA_VARIANT=checked) by tests/test_gpu_checked.py; each writes every
result array to an .npz file given as the only argument.  They cover the
kernels' index paths: ring and stepwise schedules in both forms, ragged
units, dilute and wide-cell boxes (several list windows, two home-atom
chunks), mirror walls, the slice thermostat, a batch with its autotuner, the
server and the allocation-free force call."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2507_11289_gb300 import dsea, inputs  # noqa: E402


def _box_results(out, name, b):
    out[name + "_r"] = b.positions()
    out[name + "_v"] = b.velocities()
    out[name + "_f"] = b.forces()
    o = b.observables()
    out[name + "_obs"] = np.array([o["step"], o["U"], o["W"], o["KE"]])


def _wide_cells():
    box = np.array([14.9, 9.99, 9.99])
    g = [np.arange(k) * (L / k) for k, L in zip((13, 9, 9), box)]
    pos = np.stack(np.meshgrid(*g, indexing="ij"), axis=-1).reshape(-1, 3)
    pos = inputs.jitter(pos, box, 0.05, seed=32)
    return pos, inputs.maxwell_boltzmann(len(pos), 1.0, seed=33), box


def main(path):
    out = {}
    small = inputs.SMALL_4K.state()
    ragged_pos, ragged_box = inputs.fcc_lattice(11, 0.8)
    ragged = (ragged_pos, inputs.maxwell_boltzmann(len(ragged_pos), 1.5, 5), ragged_box)
    dilute = inputs.batch_specs(n_boxes=1, seed=11, n_min=3000, n_max=3001, rho_range=(0.06, 0.061))[0].state()
    cases = [
        ("small_mixed_ring", small, dict(n_slices=4, precision=dsea.MIXED), 50),
        ("small_fp64_ring", small, dict(n_slices=4, precision=dsea.FP64), 20),
        ("small_mixed_stepwise", small, dict(n_slices=4, precision=dsea.MIXED, schedule=dsea.SCHED_STEPWISE), 10),
        ("small_fp64_stepwise", small, dict(n_slices=4, precision=dsea.FP64, schedule=dsea.SCHED_STEPWISE), 5),
        ("ragged_mixed", ragged, dict(precision=dsea.MIXED), 30),
        ("ragged_fp64", ragged, dict(precision=dsea.FP64), 10),
        ("dilute_mixed", dilute, dict(precision=dsea.MIXED), 30),
        ("wide_mixed", _wide_cells(), dict(n_slices=3, precision=dsea.MIXED), 20),
        ("wide_fp64", _wide_cells(), dict(n_slices=3, precision=dsea.FP64), 10),
        ("walls_mixed", small, dict(n_slices=4, precision=dsea.MIXED, walls=True), 30),
        ("nvt_mixed", small, dict(n_slices=4, precision=dsea.MIXED, temperature=1.2), 30),
        ("nvt_fp64", small, dict(n_slices=4, precision=dsea.FP64, temperature=1.2), 10),
    ]
    for name, (pos, vel, box), kw, steps in cases:
        with dsea.Box(pos, vel, box, **kw) as b:
            _box_results(out, name + "_t0", b)
            b.advance(steps)
            _box_results(out, name, b)
            b.sync()
    # a batch of dilute and dense boxes, its autotuner, then one more advance
    states = [s.state() for s in inputs.batch_specs(n_boxes=5, seed=3, n_max=6000)]
    boxes = [dsea.Box(*st, precision=dsea.MIXED) for st in states]
    try:
        bt = dsea.batch_create([b.h for b in boxes])
        dsea.batch_advance(bt, [12, 7, 0, 12, 3])
        out["batch_shape"] = np.array(dsea.batch_autotune(bt, trial_steps=2))
        dsea.batch_advance(bt, [5, 5, 5, 5, 5])
        dsea.batch_destroy(bt)
        for k, b in enumerate(boxes):
            _box_results(out, f"batch{k}", b)
    finally:
        for b in boxes:
            b.close()
    # the server: three jobs of different lengths in one-to-three-job launches
    srv = dsea.server_create(4 << 30, dsea.make_params(precision=dsea.MIXED), 7, 0)
    try:
        ids = [dsea.server_submit(srv, *states[k], n) for k, n in ((0, 20), (1, 9), (3, 15))]
        dsea.server_drain(srv)
        for q, (jid, k) in enumerate(zip(ids, (0, 1, 3))):
            assert dsea.server_poll(srv, jid) == 2
            r, v, o, _, _ = dsea.server_result(srv, jid, len(states[k][0]))
            out[f"served{q}_r"], out[f"served{q}_v"] = r, v
            out[f"served{q}_obs"] = np.array([o["step"], o["U"], o["W"], o["KE"]])
    finally:
        dsea.server_destroy(srv)
    # the allocation-free force call, both forms
    import ctypes

    import torch
    pos, vel, box = small
    lib = dsea.load()
    stream = torch.cuda.current_stream()
    for prec in (dsea.MIXED, dsea.FP64):
        p = torch.as_tensor(pos, dtype=torch.float64, device="cuda").contiguous()
        v = torch.as_tensor(vel, dtype=torch.float64, device="cuda").contiguous()
        f = torch.zeros((len(pos), 3), dtype=torch.float64, device="cuda")
        o = torch.zeros(3, dtype=torch.float64, device="cuda")
        b3 = (ctypes.c_double * 3)(*[float(x) for x in box])
        rc = lib.dsea_forces_noalloc(p.data_ptr(), v.data_ptr(), len(pos), b3, 2.5, prec, f.data_ptr(),
                                     o.data_ptr(), stream.cuda_stream)
        assert rc == dsea.OK, dsea.status_string(rc)
        out[f"noalloc{prec}_f"] = f.cpu().numpy()
        out[f"noalloc{prec}_obs"] = o.cpu().numpy()
    np.savez(path, **out)
    print(f"{len(out)} arrays, library {os.path.basename(dsea.library_path())}")


if __name__ == "__main__":
    main(sys.argv[1])
