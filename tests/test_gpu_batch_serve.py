"""Many boxes in one persistent launch, the autotuner, and the continuous-
batching server: every box's result is the same alone and in the mix."""
import time

import numpy as np
import pytest

import oracle
from paper_2507_11289_gb300 import dsea, inputs

pytestmark = pytest.mark.gpu


def _boxes(n, seed=2):
    specs = inputs.batch_specs(n_boxes=n, seed=seed, n_max=6000)
    return [s.state() for s in specs]


def _alone(state, steps, precision=dsea.MIXED):
    pos, vel, box = state
    with dsea.Box(pos, vel, box, precision=precision) as b:
        b.advance(steps)
        return b.positions(), b.velocities(), b.observables()


def test_batch_equals_alone_bitwise():
    states = _boxes(6)
    steps = [40, 25, 40, 0, 13, 31]
    ref = [_alone(s, k) for s, k in zip(states, steps)]
    boxes = [dsea.Box(*s, precision=dsea.MIXED) for s in states]
    try:
        bt = dsea.batch_create([b.h for b in boxes])
        # two advances: the second replays the captured graph of the first shape
        dsea.batch_advance(bt, [k // 2 for k in steps])
        dsea.batch_advance(bt, [k - k // 2 for k in steps])
        dsea.batch_destroy(bt)
        for b, (r, v, o), k in zip(boxes, ref, steps):
            assert np.array_equal(b.positions(), r)
            assert np.array_equal(b.velocities(), v)
            assert b.observables() == o and o["step"] == k
    finally:
        for b in boxes:
            b.close()


def test_batch_autotune_keeps_results_and_state():
    """The batch autotuner times its candidates on the batch from snapshots:
    the boxes' steps and states are unchanged by it, every box ends on the
    chosen shape (or the largest that fits it), and the run continues to the
    same bits as each box advanced alone."""
    states = _boxes(5, seed=6)
    ref = [_alone(s, 30) for s in states]
    boxes = [dsea.Box(*s, precision=dsea.MIXED) for s in states]
    try:
        bt = dsea.batch_create([b.h for b in boxes])
        dsea.batch_advance(bt, [10] * 5)
        import torch
        torch.cuda.synchronize()
        m0 = torch.cuda.memory_allocated()
        torch.cuda.reset_peak_memory_stats()
        n_slots = sum(b.info()["cells"][0] * b.info()["cells"][1] * b.info()["cells"][2] * b.info()["cell_capacity"]
                      for b in boxes)
        ty, tz = dsea.batch_autotune(bt, trial_steps=2)
        # the snapshots (at least r and q of every slot) came from the boxes' allocator, torch's here
        assert torch.cuda.max_memory_allocated() - m0 >= n_slots * (24 + 16)
        assert torch.cuda.memory_allocated() == m0
        assert (ty, tz) in {(1, 2), (2, 2), (1, 4), (2, 4), (3, 3), (4, 4)}
        for b in boxes:
            info = b.info()
            assert b.observables()["step"] == 10        # trials left the state untouched
            assert 1 <= info["tile_y"] <= ty and 1 <= info["tile_z"] <= tz
        dsea.batch_advance(bt, [20] * 5)
        dsea.batch_destroy(bt)
        for b, (r, v, o) in zip(boxes, ref):
            assert np.array_equal(b.positions(), r)
            assert np.array_equal(b.velocities(), v)
            assert b.observables() == o
    finally:
        for b in boxes:
            b.close()


def test_batch_fp64_matches_oracle():
    states = _boxes(3, seed=9)
    boxes = [dsea.Box(*s, precision=dsea.FP64) for s in states]
    try:
        bt = dsea.batch_create([b.h for b in boxes])
        dsea.batch_advance(bt, [20, 20, 20])
        dsea.batch_destroy(bt)
        for b, (pos, vel, box) in zip(boxes, states):
            ro, _, _, _ = oracle.run(pos, vel, box, steps=20)
            d = b.positions() - ro
            d -= box * np.round(d / box)
            assert np.abs(d).max() <= 1e-9
    finally:
        for b in boxes:
            b.close()


def test_autotune_keeps_results_and_state():
    pos, vel, box = inputs.SMALL_4K.state()
    r_ref, _, _ = _alone((pos, vel, box), 30)
    with dsea.Box(pos, vel, box, precision=dsea.MIXED) as b:
        b.advance(10)
        chosen = b.autotune(trial_steps=3)
        assert chosen["tile_y"] >= 1 and chosen["tile_z"] >= 1
        assert b.observables()["step"] == 10          # trials left the state untouched
        b.advance(20)
        assert np.array_equal(b.positions(), r_ref)


def test_server_results_same_alone_and_in_mix():
    states = _boxes(5, seed=4)
    steps = [60, 150, 35, 90, 120]
    srv = dsea.server_create(8 << 30, dsea.make_params(precision=dsea.MIXED), 25, 0)
    try:
        # job 0 alone
        j0 = dsea.server_submit(srv, *states[0], steps[0])
        dsea.server_drain(srv)
        alone = dsea.server_result(srv, j0, len(states[0][0]))
        # job 0 again, arriving while the others run
        ids = [dsea.server_submit(srv, *states[k], steps[k]) for k in (1, 2)]
        time.sleep(0.01)
        ids.insert(0, dsea.server_submit(srv, *states[0], steps[0]))
        ids += [dsea.server_submit(srv, *states[k], steps[k]) for k in (3, 4)]
        dsea.server_drain(srv)
        res = {}
        for jid, k in zip(ids, [0, 1, 2, 3, 4]):
            assert dsea.server_poll(srv, jid) == 2
            res[k] = dsea.server_result(srv, jid, len(states[k][0]))
        assert np.array_equal(res[0][0], alone[0]) and np.array_equal(res[0][1], alone[1])
        assert res[0][2] == alone[2]
        for k in range(1, 5):
            r, v, o = _alone(states[k], steps[k])
            assert np.array_equal(res[k][0], r) and o == res[k][2]
            assert res[k][4] >= res[k][3]           # done after arrival
        st = dsea.server_stats(srv)
        assert st["launches"] >= 2 and st["atom_steps"] > 0
    finally:
        dsea.server_destroy(srv)


def test_server_reshapes_units_as_jobs_leave():
    """Two 1,048,576-atom jobs fill the GPU together with 4 x 4-cell units
    (2 x 5,203 units per step against twice the 4,864 resident warp stages);
    once the shorter one has finished, the longer one runs alone at 2 x 4
    (10,406 units).  The server re-chooses the shape at every launch, and a
    shape never changes a result: each job equals its run alone bit for bit."""
    import torch
    pos, box = inputs.fcc_lattice(64, 0.8)
    vels = [inputs.maxwell_boltzmann(len(pos), 1.5, seed) for seed in (21, 22)]
    steps = [60, 20]
    with dsea.Box(pos, vels[0], box, precision=dsea.MIXED) as b:
        info = b.info()
    cells = info["cells"]
    stages = torch.cuda.get_device_properties(0).multi_processor_count * 32

    def units(ty, tz):
        return info["n_slices"] * -(-cells[1] // ty) * -(-cells[2] // tz)

    def rule(n_jobs):
        fill = [s for s in ((4, 4), (3, 3), (2, 4), (2, 2), (1, 4), (1, 2)) if n_jobs * units(*s) >= 2 * stages]
        return fill[0] if fill else (1, 2)

    assert rule(2) != rule(1)                # the test exercises a change of shape
    srv = dsea.server_create(16 << 30, dsea.make_params(precision=dsea.MIXED), 10, 0)
    try:
        ids = [dsea.server_submit(srv, pos, v, box, k) for v, k in zip(vels, steps)]
        dsea.server_drain(srv)
        res = [dsea.server_result(srv, jid, len(pos)) for jid in ids]
    finally:
        dsea.server_destroy(srv)
    for (r, v, o, _, _), vel, k in zip(res, vels, steps):
        ra, va, oa = _alone((pos, vel, box), k)
        assert np.array_equal(r, ra) and np.array_equal(v, va)
        assert o == oa and o["step"] == k


def test_server_isolates_a_failing_job():
    """A job whose atom jumps past a whole slice in its first step fails with
    the migration status; the jobs that shared its launch finish with the
    results they have alone, and the server keeps admitting work.  One-step
    segments end the failing job after the step that reports it."""
    states = _boxes(3, seed=8)
    pos, vel, box = inputs.SMALL_4K.state()
    vel = vel.copy()
    vel[0] = [2000.0, 0.0, 0.0]        # 10 sigma in one step: more than one 4.3-sigma slice
    steps = [12, 9, 7]
    srv = dsea.server_create(8 << 30, dsea.make_params(precision=dsea.MIXED), 1, 0)
    try:
        good = [dsea.server_submit(srv, *states[0], steps[0])]
        bad = dsea.server_submit(srv, pos, vel, box, 5, n_slices=4)
        good += [dsea.server_submit(srv, *states[k], steps[k]) for k in (1, 2)]
        dsea.server_drain(srv)
        assert dsea.server_poll(srv, bad) == dsea.ERR_MIGRATION
        for jid, st, k in zip(good, states, steps):
            assert dsea.server_poll(srv, jid) == 2
            r, v, o, _, _ = dsea.server_result(srv, jid, len(st[0]))
            ra, va, oa = _alone(st, k)
            assert np.array_equal(r, ra) and np.array_equal(v, va) and o == oa
        later = dsea.server_submit(srv, *states[1], 4)
        dsea.server_drain(srv)
        assert dsea.server_poll(srv, later) == 2
    finally:
        dsea.server_destroy(srv)


def test_server_rejects_job_over_budget():
    pos, vel, box = inputs.SMALL_4K.state()
    srv = dsea.server_create(1 << 20, None, 10, 0)          # 1 MiB budget
    try:
        with pytest.raises(dsea.DseaError) as e:
            dsea.server_submit(srv, pos, vel, box, 10)
        assert e.value.code == dsea.ERR_BUDGET
    finally:
        dsea.server_destroy(srv)


def test_torch_allocator_owns_box_memory():
    import torch
    pos, vel, box = inputs.SMALL_4K.state()
    before = torch.cuda.memory_allocated()
    b = dsea.Box(pos, vel, box, precision=dsea.MIXED)
    during = torch.cuda.memory_allocated()
    assert during - before >= b.info()["device_bytes"] * 0.9
    b.close()
    assert torch.cuda.memory_allocated() == before


def test_autotune_choice_does_not_leak_across_densities():
    """The autotuner caches a unit shape per size class.  A sparser box and a
    dense one of about the same edge are different classes (mean atoms per
    cell; below rho 0.77 the cells are also larger), and so are a 17^3-cell
    box and the 43^3-cell 1M-atom box at the same density (total cells):
    tuning the first of each pair leaves the second on its untuned shape.  The
    untuned mixed shape is the launch-filling one: the largest of 4x4, 3x3,
    2x4, 2x2, 1x4, 1x2 home cells whose units per step reach twice the
    resident warp stages (32 per SM), else 1x2.  Run in a fresh process: the
    cache lives as long as the library."""
    import json
    import os
    import subprocess
    import sys
    code = """
import json
import torch
from paper_2507_11289_gb300 import dsea, inputs
cases = (("dilute", 22, 0.55), ("dense", 25, 0.8), ("big", 64, 0.8))
def make(n_i, rho):
    pos, box = inputs.fcc_lattice(n_i, rho)
    return dsea.Box(pos, inputs.maxwell_boltzmann(len(pos), 1.0, 3), box, precision=dsea.MIXED)
out = {"sms": torch.cuda.get_device_properties(0).multi_processor_count}
for name, n_i, rho in cases:
    with make(n_i, rho) as b:
        inf = b.info()
        out[name] = {"cells": inf["cells"], "cap": inf["cell_capacity"], "slices": inf["n_slices"],
                     "untuned": [inf["tile_y"], inf["tile_z"]]}
for name, n_i, rho in cases:
    with make(n_i, rho) as b:
        inf = b.info()
        out[name]["tile"] = [inf["tile_y"], inf["tile_z"]]
        if name != "big":
            p = b.autotune(trial_steps=2)
            out[name]["tuned"] = [p["tile_y"], p["tile_z"]]
print(json.dumps(out))
"""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    out = json.loads(r.stdout.strip().splitlines()[-1])
    d, e, g = out["dilute"], out["dense"], out["big"]
    want = 2 * out["sms"] * 32

    def units(c, ty, tz):
        return c["slices"] * -(-c["cells"][1] // ty) * -(-c["cells"][2] // tz)

    for c in (d, e, g):   # the launch-filling rule, restated
        fill = [s for s in ((4, 4), (3, 3), (2, 4), (2, 2), (1, 4), (1, 2)) if units(c, *s) >= want]
        assert c["untuned"] == list(fill[0] if fill else (1, 2)), out
    assert e["tile"] == e["untuned"], out                          # not the dilute box's choice
    assert g["cap"] == e["cap"] and min(g["cells"][1:]) >= 16 and min(e["cells"][1:]) >= 16
    assert g["tile"] == g["untuned"], out                          # not the 17^3 box's choice


def _force_err(Fg, Fo):
    rms = lambda a: float(np.sqrt((np.asarray(a) ** 2).sum(-1).mean()))
    return rms(Fg - Fo) / rms(Fo)


def test_full_512_box_batch_sampled_boxes():
    """The batch as the benchmark runs it: the 512 boxes (500-50,000 atoms,
    rho 0.05-0.9, T 0.7-3.0), one unit shape from the batch autotuner, one
    graph-replayed launch.  After 20 steps, 8 sampled boxes hold their runs
    alone bit for bit, and their forces are the oracle's at the GPU's
    positions within the mixed form's per-step gate (rms 2e-6 of the rms
    force)."""
    specs = inputs.batch_specs(n_boxes=512, steps=20)
    states = [s.state() for s in specs]
    boxes = [dsea.Box(*st, precision=dsea.MIXED) for st in states]
    try:
        bt = dsea.batch_create([b.h for b in boxes])
        dsea.batch_autotune(bt, trial_steps=2)
        dsea.batch_advance(bt, [20] * len(boxes))
        dsea.batch_destroy(bt)
        rng = np.random.default_rng(5)
        for k in sorted(rng.choice(len(boxes), 8, replace=False)):
            r, v, f = boxes[k].positions(), boxes[k].velocities(), boxes[k].forces()
            ra, va, _ = _alone(states[k], 20)
            assert np.array_equal(r, ra) and np.array_equal(v, va), k
            Fo, _, _ = oracle.forces(r, states[k][2], 2.5, "cells")
            e = _force_err(f, Fo)
            print(f"box {k}: {len(r)} atoms, rho {specs[k].rho:.2f}, force error rms {e:.2e}")
            assert e <= 2e-6, (k, e)
    finally:
        for b in boxes:
            b.close()


def test_served_stream_sampled_jobs_equal_alone():
    """The served stream as the benchmark draws it (Poisson 200 jobs/s, N
    log-uniform 1e3-2e6, rho 0.3-0.9, T 0.8-2.5; 60 GB budget, 100-step
    segments): its first 24 jobs, submitted at their arrival times with their
    step counts capped at 300, run overlapped on the device; 4 sampled jobs
    end bit for bit where they end alone."""
    jobs = inputs.served_stream(rate_per_s=200.0, duration_s=1.0)[:24]
    steps = [min(j.spec.steps, 300) for j in jobs]
    states = [j.spec.state() for j in jobs]
    srv = dsea.server_create(60 << 30, dsea.make_params(precision=dsea.MIXED), 100, 0)
    try:
        t0 = time.perf_counter()
        ids = []
        for j, st, n in zip(jobs, states, steps):
            wait = j.arrival_s - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            ids.append(dsea.server_submit(srv, *st, n))
        dsea.server_drain(srv)
        rng = np.random.default_rng(9)
        for k in sorted(rng.choice(len(jobs), 4, replace=False)):
            assert dsea.server_poll(srv, ids[k]) == 2
            r, v, o, _, _ = dsea.server_result(srv, ids[k], len(states[k][0]))
            ra, va, oa = _alone(states[k], steps[k])
            print(f"job {k}: {len(r)} atoms, {steps[k]} steps")
            assert np.array_equal(r, ra) and np.array_equal(v, va) and o == oa, k
    finally:
        dsea.server_destroy(srv)


def test_server_with_thermostat_jobs_equal_alone():
    """A server whose params set the slice thermostat runs every job under it;
    each job ends bit for bit where it ends alone with the same params."""
    states = _boxes(3, seed=14)
    steps = [30, 12, 21]
    params = dsea.make_params(precision=dsea.MIXED, temperature=1.1)
    srv = dsea.server_create(8 << 30, params, 10, 0)
    try:
        ids = [dsea.server_submit(srv, *st, n) for st, n in zip(states, steps)]
        dsea.server_drain(srv)
        for jid, st, n in zip(ids, states, steps):
            r, v, o, _, _ = dsea.server_result(srv, jid, len(st[0]))
            with dsea.Box(*st, precision=dsea.MIXED, temperature=1.1) as b:
                b.advance(n)
                assert np.array_equal(r, b.positions()) and np.array_equal(v, b.velocities())
                assert o == b.observables()
    finally:
        dsea.server_destroy(srv)


def test_server_policies_order_work_not_results():
    """Three 1,048,576-atom jobs of 1000 steps (100-step segments).  With
    DSEA_SERVE_SHORTEST two of them fill a launch (2^21 atoms), so the third,
    which arrived last, waits until they are done and then runs alone: about
    20 launches.  With DSEA_SERVE_ALL all three run together: 10 to 12 (more
    if the later jobs arrive some segments late).  Either way each job ends
    bit for bit where it ends alone."""
    pos, box = inputs.fcc_lattice(64, 0.8)
    vels = [inputs.maxwell_boltzmann(len(pos), 1.5, seed) for seed in (31, 32, 33)]
    ref = [_alone((pos, v, box), 1000) for v in vels]
    launches = {}
    for policy in (dsea.SERVE_SHORTEST, dsea.SERVE_ALL):
        srv = dsea.server_create(16 << 30, dsea.make_params(precision=dsea.MIXED), 100, 0)
        try:
            dsea.server_set_policy(srv, policy)
            ids = [dsea.server_submit(srv, pos, v, box, 1000) for v in vels]
            dsea.server_drain(srv)
            launches[policy] = dsea.server_stats(srv)["launches"]
            for jid, (r, v, o) in zip(ids, ref):
                rg, vg, og, _, _ = dsea.server_result(srv, jid, len(pos))
                assert np.array_equal(rg, r) and np.array_equal(vg, v) and og == o
        finally:
            dsea.server_destroy(srv)
    print("launches", launches)
    assert launches[dsea.SERVE_SHORTEST] >= 18
    assert launches[dsea.SERVE_ALL] <= 14
    with pytest.raises(dsea.DseaError):
        srv = dsea.server_create(1 << 30, dsea.make_params(precision=dsea.MIXED), 100, 0)
        try:
            dsea.server_set_policy(srv, 7)
        finally:
            dsea.server_destroy(srv)
