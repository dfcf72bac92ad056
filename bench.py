"""Benchmark of the slice-streamed LJ NVE hot path on GB300.

One bench "step" is one dsea_advance of MD_STEPS velocity-Verlet steps over
the whole 1,048,576-atom box (64^3 fcc cells, rho 0.8, T* 1.5, rc 2.5,
dt 0.005, 43 x-slices, ring schedule) -- every part of the hot path runs in
it: force stencil, kick/drift, rebinning and the ring scheduler.  The
default 10 timed steps make the configured 1000 NVE steps.

Printed (rank 0, one JSON line): the mixed FP32/FP64 throughput in
atom-steps/s (value), the plain FP64 form side by side, a many-box batch
and a served stream, the roofline of the dominant kernel, the CPU oracle
baseline, an end-to-end number through the C ABI with host buffers, and the
SM clocks seen during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
  torchrun --nproc-per-node N bench.py --gpus N   (independent replicas)
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "atom-steps/s (LJ NVE, rc=2.5σ) mixed vs plain FP64; served p50/p99 latency"
UNIT = "atom-steps/s"
MD_STEPS = 100                     # MD steps per bench step
PAIRS_PER_ATOM = lambda rho: rho * 4.0 * math.pi / 3.0 * 2.5 ** 3   # directed pairs within rc
FLOPS_PER_PAIR = 27                # FP32 flops counted per directed in-cutoff pair
FP32_LANES = 128                   # FP32 FMA lanes per SM
PROFILE = os.path.join(ROOT, "profiles", "k_ring_mixed_1m.md")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---- distributed plumbing (replicas: no data-path collective) ---------------

def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl"
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))   # each rank's own GPU, before NCCL
        dist.init_process_group(backend=backend)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(x, world, op_name):
    """All-reduce one host number over the ranks (timings and counts only;
    the replicas exchange no simulation data)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=getattr(dist.ReduceOp, op_name))
    return float(t.item())


def max_over_ranks(x, world):
    return _reduce(x, world, "MAX")


def sum_over_ranks(x, world):
    return _reduce(x, world, "SUM")


# ---- clocks during the timed region --------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) != 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[2:]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---- workloads -------------------------------------------------------------------

def flush_l2(buf):
    buf.add_(1.0)      # writes 256 MB > 129 MB L2


def time_box(dsea, torch, spec, precision, steps, warmup, md_steps, flush_buf, stream, walls=False,
             temperature=0.0, profiles=False):
    """Advance one box; returns (seconds over the timed steps, kernel launches,
    per-step event times, info).  walls: mirror walls along x; temperature: the
    slice thermostat's target (0 = NVE); profiles: add the final per-slice
    profiles to info."""
    pos, vel, box = spec.state()
    b = dsea.Box(pos, vel, box, n_slices=spec.n_slices, precision=precision, stream=stream, walls=walls,
                 temperature=temperature)
    try:
        for _ in range(warmup):
            b.advance(md_steps)
        b.sync()
        times = []
        torch.cuda.synchronize()
        for _ in range(steps):
            flush_l2(flush_buf)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.advance(md_steps)
            e1.record(stream)
            times.append((e0, e1))
        b.sync()
        torch.cuda.synchronize()
        per = [a.elapsed_time(c) * 1e-3 for a, c in times]
        launches = steps * math.ceil(md_steps / 4096)
        info = b.info()
        if profiles:
            info["profiles"] = b.profiles()
        return sum(per), launches, per, info
    finally:
        b.close()


def measured_peaks() -> dict:
    """The peaks measured on this GPU model (HBM copy GB/s, bf16 TFLOP/s), if present."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def dataset_run(dsea, torch, stream, n_slices=43, points_per_slice=1 << 23, workers=4, steps=30):
    """The generic slice ring (dsea_dataset_*) with the library's example
    kernel, an explicit FP32 heat-equation step on a periodic rod: HBM-bound,
    8 algorithmic bytes per grid point and step (read and write one value)."""
    m = points_per_slice
    ds = dsea.Dataset(n_slices, m * 4, o_in=1, o_out=0, n_workers=workers, stream=stream)
    try:
        ds.register("heat1d", 0.2)
        rng = np.random.Generator(np.random.PCG64(5))
        for j in range(n_slices):
            ds.write(j, rng.uniform(-1.0, 1.0, m).astype(np.float32))
        ds.run(5)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t0 = time.perf_counter()
        ds.run(steps)
        host_s = time.perf_counter() - t0
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) * 1e-3
    finally:
        ds.close()
    pts = n_slices * m * steps
    gbs = 8.0 * pts / sec / 1e9
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    return {"value": pts / sec, "unit": "grid-point-steps/s", "steps": steps, "seconds": sec,
            "host_enqueue_seconds": host_s,
            "achieved_gbs": gbs, "hbm_peak_gbs": hbm, "frac_of_measured_hbm": gbs / hbm if hbm else None,
            "workload": f"generic slice ring: {n_slices} slices x {m} FP32 points, {workers} workers, "
                        "explicit heat-equation step per slice (O_in = 1)"}


def e2e_run(dsea, torch, spec, precision, steps, md_steps, stream):
    """End to end through the C ABI: host pos/vel in (pinned), create + bin
    on the device, advance, read positions and velocities back to pinned host
    arrays."""
    pos, vel, box = spec.state()

    def pinned(shape):   # page-locked host array (NumPy view of a pinned tensor)
        t = torch.empty(shape, dtype=torch.float64, pin_memory=True)
        return t, t.numpy()

    keep = []
    for a in (pos, vel, pos, vel):
        keep.append(pinned(a.shape))
    pos_h, vel_h, out_r, out_v = (k[1] for k in keep)
    pos_h[...] = pos
    vel_h[...] = vel

    def one():
        b = dsea.Box(pos_h, vel_h, box, n_slices=spec.n_slices, precision=precision, stream=stream)
        b.advance(md_steps)
        dsea.read_positions(b.h, out_r)
        dsea.read_velocities(b.h, out_v)
        b.close()

    one()                      # warm-up: the allocator's cache and the kernels' first launch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    n = len(pos_h)
    return {"value": n * md_steps * steps / dt, "unit": UNIT,
            "h2d_bytes_per_step": int(pos_h.nbytes + vel_h.nbytes),
            "d2h_bytes_per_step": int(out_r.nbytes + out_v.nbytes)}


def batch_run(dsea, torch, n_boxes, md_steps, stream, tile=None):
    """Many independent boxes (N log-uniform 500-50,000, rho 0.05-0.9,
    T 0.7-3.0) advanced together in one graph-captured persistent launch.
    tile: a fixed (tile_y, tile_z) for every box instead of the batch
    autotuner's choice (for profiling, where the autotuner's timings are
    distorted)."""
    from paper_2507_11289_gb300 import inputs
    specs = inputs.batch_specs(n_boxes=n_boxes, steps=md_steps)
    boxes = []
    try:
        for s in specs:
            pos, vel, box = s.state()
            kw = dict(tile_y=tile[0], tile_z=tile[1]) if tile else {}
            boxes.append(dsea.Box(pos, vel, box, precision=dsea.MIXED, stream=stream, **kw))
        bt = dsea.batch_create([b.h for b in boxes])
        n_atoms = sum(b.n_atoms for b in boxes)
        # one unit shape for the whole batch, timed on the batch itself (the
        # boxes fill the GPU together: a lone box's choice is smaller)
        t0 = time.perf_counter()
        shape = tuple(tile) if tile else dsea.batch_autotune(bt, trial_steps=3)
        t_tune = time.perf_counter() - t0
        dsea.batch_advance(bt, [10] * len(boxes))          # warm-up, graph capture
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dsea.batch_advance(bt, [md_steps] * len(boxes))
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) * 1e-3
        for b in boxes:
            b.sync()
        dsea.batch_destroy(bt)
        return {"value": n_atoms * md_steps / sec, "unit": UNIT, "boxes": len(boxes),
                "atoms": n_atoms, "md_steps": md_steps, "seconds": sec,
                "autotune_seconds": t_tune, "unit_shape": list(shape),
                "workload": f"{len(boxes)} fcc LJ boxes, N log-uniform 500-50,000, rho U(0.05,0.9), "
                            f"T U(0.7,3.0), mixed, one graph-replayed persistent launch"}
    finally:
        for b in boxes:
            b.close()


def _union_length(intervals):
    """Total length of the union of [a, b) intervals (time with a job in the system)."""
    total, end = 0.0, -math.inf
    for a, b in sorted(intervals):
        if b <= end:
            continue
        total += b - max(a, end)
        end = b
    return total


def serve_run(dsea, torch, rate, duration, budget_gb, seed=3, segment=100, why_window=None,
              policy="shortest"):
    """Poisson job stream into the continuous-batching server; latency from
    arrival (submit) to completion on the server clock.  Every job's state is
    generated before the arrival window opens, so submissions keep to the
    Poisson arrival times (host memory: the window's jobs, a few GB)."""
    from paper_2507_11289_gb300 import inputs
    jobs = inputs.served_stream(rate_per_s=rate, duration_s=duration, seed=seed)
    states = [job.spec.state() for job in jobs]
    srv = dsea.server_create(int(budget_gb * 2 ** 30),
                             dsea.make_params(precision=dsea.MIXED), segment, 0)
    dsea.server_set_policy(srv, {"shortest": dsea.SERVE_SHORTEST, "all": dsea.SERVE_ALL}[policy])
    ids = []
    late = []
    try:
        t0 = time.perf_counter()
        offered = 0.0
        for job, (pos, vel, box) in zip(jobs, states):
            while time.perf_counter() - t0 < job.arrival_s:
                time.sleep(0.0002)
            late.append(time.perf_counter() - t0 - job.arrival_s)
            ids.append((dsea.server_submit(srv, pos, vel, box, job.spec.steps), job.spec.n_atoms))
            offered += job.spec.n_atoms * job.spec.steps
        submit_s = time.perf_counter() - t0
        dsea.server_drain(srv)
        wall = time.perf_counter() - t0
        lat, spans = [], []
        for jid, n in ids:
            _, _, _, ta, td = dsea.server_result(srv, jid, n)
            lat.append(td - ta)
            spans.append((ta, td))
        st = dsea.server_stats(srv)
    finally:
        dsea.server_destroy(srv)
    lat = np.array(lat)
    occupied = _union_length(spans)
    out = {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
           "mean_s": float(lat.mean()), "max_s": float(lat.max()), "policy": policy,
           "jobs": len(ids), "rate_per_s": rate, "arrival_window_s": duration,
           "achieved_arrival_rate_per_s": len(ids) / max(submit_s, 1e-9),
           "max_submit_lateness_s": float(max(late)) if late else 0.0,
           "atom_steps_per_s": st["atom_steps"] / wall,
           "occupied_atom_steps_per_s": st["atom_steps"] / max(occupied, 1e-9),
           "busy_atom_steps_per_s": st["atom_steps"] / max(st["busy_seconds"], 1e-9),
           "offered_atom_steps_per_s": offered / duration, "drain_s": wall - submit_s,
           "launches": st["launches"], "budget_gb": budget_gb,
           "workload": "Poisson arrivals; fcc LJ boxes N log-uniform 1e3-2e6, rho U(0.3,0.9), "
                       "T U(0.8,2.5), steps log-uniform 100-10,000; mixed"}
    if why_window:
        out["window_note"] = why_window
    return out


def device_peaks(dsea, torch, stream):
    """The roofline denominators: the FP32 and FP64 FMA rates measured by the
    library's probe on this GPU, beside the FP32 rate derived from the
    device's SM count and maximum SM clock (both queried, not assumed)."""
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sms = props.multi_processor_count
    max_mhz = None
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(torch.cuda.current_device()),
                              "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=20).stdout.strip()
        max_mhz = float(out.splitlines()[0])
    except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
        pass
    derived = sms * FP32_LANES * 2 * max_mhz * 1e6 / 1e12 if max_mhz else None
    return {"fp32_measured": dsea.probe_peak(dsea.PROBE_FP32, stream),
            "fp32x2_measured": dsea.probe_peak(dsea.PROBE_FP32X2, stream),
            "fp64_measured": dsea.probe_peak(dsea.PROBE_FP64, stream),
            "fp32_derived": derived, "sms": sms, "sm_max_mhz": max_mhz}


def cpu_model():
    """The host CPU's model name and logical core count."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                name = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.TimeoutExpired):
        pass
    if not name:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    name = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return name or "unknown", os.cpu_count()


def profile_traffic_per_atom_step():
    """DRAM bytes per atom-step of the ring kernel from the committed ncu
    summary (null if absent)."""
    try:
        for line in open(PROFILE):
            if line.startswith("traffic_bytes_per_atom_step:"):
                return float(line.split(":")[1])
    except OSError:
        pass
    return None


def cpu_baseline(spec, sample_steps, threads=0):
    """The CPU oracle as it stands (plain C, its force loop shared among
    `threads` OpenMP threads, 0 = all cores) on a bounded sample:
    `sample_steps` velocity-Verlet steps of the same box."""
    import oracle
    pos, vel, box = spec.state()
    oracle.build()
    n_all = oracle.set_threads(0)
    used = oracle.set_threads(threads if threads > 0 else n_all)
    try:
        t0 = time.perf_counter()
        oracle.run(pos, vel, box, steps=sample_steps)
        dt = time.perf_counter() - t0
    finally:
        oracle.set_threads(n_all)
    model, logical = cpu_model()
    # the oracle run does sample_steps + 1 force evaluations (closing pass included)
    return {"value": len(pos) * sample_steps / dt, "unit": UNIT, "cores": used, "kind": "oracle",
            "cpu": model, "host_logical_cores": logical,
            "sample": f"{sample_steps} velocity-Verlet steps of the {len(pos):,}-atom box "
                      f"({dt:.1f} s, {used} thread{'s' if used != 1 else ''}, cell-list oracle)"}


def reference_arm(args, rank, world):
    if rank != 0:
        return
    from paper_2507_11289_gb300 import inputs
    spec = inputs.FLUID_1M
    per = []
    n = spec.n_atoms
    import oracle
    oracle.build()
    cores = oracle.set_threads(0)
    model, _ = cpu_model()
    pos, vel, box = spec.state()
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.run(pos, vel, box, steps=args.ref_md_steps)
        if k >= args.warmup:
            per.append(time.perf_counter() - t0)
    total = sum(per)
    value = n * args.ref_md_steps * len(per) / total
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / len(per), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"LJ fluid {n:,} atoms (64^3 fcc), rho 0.8, T 1.5, rc 2.5, "
                                   f"dt 0.005; each step = {args.ref_md_steps} velocity-Verlet "
                                   f"steps of the CPU FP64 oracle (bounded sample)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": model,
                             "sample": f"{args.ref_md_steps} oracle steps per bench step, "
                                       f"{len(per)} timed steps, {cores} OpenMP threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def build_parser() -> argparse.ArgumentParser:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--md-steps", type=int, default=MD_STEPS)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--ref-md-steps", type=int, default=10)
    ap.add_argument("--cpu-sample-steps", type=int, default=8)
    ap.add_argument("--cpu-sample-steps-all", type=int, default=40,
                    help="oracle steps of the all-cores CPU baseline")
    ap.add_argument("--big-n-i", type=int, default=256,
                    help="fcc cells per axis of the large-box leg (default 256: the 67,108,864-atom box)")
    ap.add_argument("--big-md-steps", type=int, default=200,
                    help="MD steps of the large-box leg's advance (default 200)")
    ap.add_argument("--batch-boxes", type=int, default=512)
    ap.add_argument("--batch-md-steps", type=int, default=2000)
    ap.add_argument("--batch-tile", default="",
                    help="fixed unit shape 'Y,Z' for every batch box instead of the batch autotuner's "
                         "(for profiling)")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-window", type=float, default=1.0,
                    help="arrival window of the configured stream (s); 60 s would take about half an "
                         "hour to drain on one GPU")
    ap.add_argument("--serve-window-sustainable", type=float, default=8.0)
    ap.add_argument("--serve-rate-sustainable", type=float, default=2.5,
                    help="arrival rate of the second served run (about 0.7 utilisation)")
    ap.add_argument("--serve-budget-gb", type=float, default=60.0)
    ap.add_argument("--serve-policy", default="shortest", choices=["shortest", "all"],
                    help="which resident jobs each server launch advances")
    ap.add_argument("--skip", default="",
                    help="comma list of legs to skip: fp64,walls,nvt,67m,batch,serve,dataset,cpu,e2e")
    ap.add_argument("--walls-steps", type=int, default=3, help="timed steps of the mirror-wall leg")
    ap.add_argument("--nvt-steps", type=int, default=3, help="timed steps of the thermostat leg")
    return ap


def main():
    ap = build_parser()
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world = dist_setup(args.gpus)
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    skip = set(filter(None, args.skip.split(",")))

    import torch
    from paper_2507_11289_gb300 import dsea, inputs
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dsea.load()
    stream = torch.cuda.current_stream()
    flush_buf = torch.zeros(64 * 2 ** 20, dtype=torch.float32, device="cuda")   # 256 MB

    spec = inputs.FLUID_1M
    # headline: mixed, ring schedule
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        sec, launches, per, info = time_box(dsea, torch, spec, dsea.MIXED, args.steps, args.warmup,
                                            args.md_steps, flush_buf, stream)
    barrier(world)
    torch.cuda.synchronize()
    sec_max = max_over_ranks(sec, world)
    atom_steps = spec.n_atoms * args.md_steps * args.steps
    value = sum_over_ranks(atom_steps, world) / sec_max
    launch_s = sum(per) / len(per)        # one ring launch per bench step
    flops_per_atom_step = PAIRS_PER_ATOM(spec.rho) * FLOPS_PER_PAIR
    achieved = spec.n_atoms * args.md_steps * flops_per_atom_step / launch_s / 1e12
    tpa = profile_traffic_per_atom_step()
    peaks = device_peaks(dsea, torch, stream)
    fp32_peak = peaks["fp32_measured"]
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak,
                "traffic": None if tpa is None else tpa * spec.n_atoms * args.md_steps,
                "kernel": "k_ring_mixed (warp-level ring, mixed form)",
                "counted": f"{FLOPS_PER_PAIR} flops x {PAIRS_PER_ATOM(spec.rho):.2f} directed "
                           f"in-cutoff pairs per atom-step",
                "peak_note": (f"FP32 peak measured on this GPU by dsea_probe_peak (scalar FMA chains on all "
                              f"{peaks['sms']} SMs): {fp32_peak:.1f} TFLOP/s; derived from the queried SM "
                              f"count and maximum SM clock ({peaks['sms']} x 128 lanes x 2 x "
                              f"{peaks['sm_max_mhz']} MHz): "
                              + (f"{peaks['fp32_derived']:.1f}" if peaks["fp32_derived"] else "n/a")
                              + f" TFLOP/s; packed FP32x2 FMAs measured at {peaks['fp32x2_measured']:.1f}"),
                "frac_of_derived": achieved / peaks["fp32_derived"] if peaks["fp32_derived"] else None,
                "peaks": peaks}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sec_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64",
            "data": "synthetic",
            "config": {"workload": "LJ fluid 1,048,576 atoms (64^3 fcc), rho 0.8, T 1.5, rc 2.5, "
                                   "dt 0.005, 43 x-slices, ring schedule, mixed FP32 pair math / "
                                   "FP64 state",
                       "md_steps_per_step": args.md_steps, "l2": "flushed between timed steps",
                       "parallelism": f"replicas x{world}", "unit_shape": [info["tile_y"], info["tile_z"]],
                       "cell_capacity": info["cell_capacity"]},
            "gpu_launches": launches, "roofline": roofline}
    if "fp64" not in skip:
        sec64, _, _, _ = time_box(dsea, torch, spec, dsea.FP64, args.fp64_steps, 3, args.md_steps,
                                  flush_buf, stream)
        sec64 = max_over_ranks(sec64, world)
        v64 = sum_over_ranks(spec.n_atoms * args.md_steps * args.fp64_steps, world) / sec64
        ach64 = v64 * flops_per_atom_step / 1e12
        fp64_peak = peaks["fp64_measured"]
        line["fp64"] = {"value": v64, "unit": UNIT, "steps": args.fp64_steps,
                        "ms_per_step": 1e3 * sec64 / args.fp64_steps, "mixed_over_fp64": value / v64,
                        "roofline": {"bound": "fp64", "achieved": ach64, "peak": fp64_peak,
                                     "unit": "TFLOP/s", "frac": ach64 / fp64_peak,
                                     "peak_note": "FP64 FMA rate measured on this GPU by dsea_probe_peak"}}
    if "walls" not in skip:
        sec_w, _, _, _ = time_box(dsea, torch, spec, dsea.MIXED, args.walls_steps, 3, args.md_steps,
                                  flush_buf, stream, walls=True)
        sec_w = max_over_ranks(sec_w, world)
        v_w = sum_over_ranks(spec.n_atoms * args.md_steps * args.walls_steps, world) / sec_w
        line["walls"] = {"value": v_w, "unit": UNIT, "steps": args.walls_steps,
                         "ms_per_step": 1e3 * sec_w / args.walls_steps,
                         "workload": "the headline box with mirror walls at x = 0 and x = Lx "
                                     "(DSEA_BOUNDARY_MIRROR), mixed, ring schedule"}
    if "nvt" not in skip:
        T0 = spec.T
        sec_t, _, _, info_t = time_box(dsea, torch, spec, dsea.MIXED, args.nvt_steps, 3, args.md_steps,
                                       flush_buf, stream, temperature=T0, profiles=True)
        sec_t = max_over_ranks(sec_t, world)
        v_t = sum_over_ranks(spec.n_atoms * args.md_steps * args.nvt_steps, world) / sec_t
        pr = info_t["profiles"]
        t_slice = 2.0 * pr["KE"] / (3.0 * np.maximum(pr["N"], 1))
        line["nvt"] = {"value": v_t, "unit": UNIT, "steps": args.nvt_steps,
                       "ms_per_step": 1e3 * sec_t / args.nvt_steps, "target_T": T0,
                       "slice_T_mean": float(t_slice.mean()), "slice_T_min": float(t_slice.min()),
                       "slice_T_max": float(t_slice.max()),
                       "workload": "the headline box under the slice thermostat (NVT, T0 = 1.5), "
                                   "mixed, ring schedule; slice temperatures from dsea_read_profiles "
                                   "after the run"}
    if "67m" not in skip:
        big = dataclasses.replace(inputs.FLUID_67M, n_i=args.big_n_i, steps=args.big_md_steps)
        sec_b, _, _, info_b = time_box(dsea, torch, big, dsea.MIXED, 1, 3, big.steps, flush_buf, stream)
        sec_b = max_over_ranks(sec_b, world)
        v_b = sum_over_ranks(big.n_atoms * big.steps, world) / sec_b
        ach_b = big.n_atoms * big.steps * PAIRS_PER_ATOM(big.rho) * FLOPS_PER_PAIR / sec_b / 1e12
        key = "box_67m" if big == inputs.FLUID_67M else "box_large"
        line[key] = {"value": v_b, "unit": UNIT, "md_steps": big.steps, "seconds": sec_b,
                     "roofline_frac": ach_b / fp32_peak, "achieved_tflops": ach_b,
                     "workload": f"LJ fluid {big.n_atoms:,} atoms ({big.n_i}^3 fcc), rho 0.8, T 1.5, "
                                 f"{info_b['n_slices']} x-slices, mixed, ring schedule, one "
                                 f"{big.steps}-step advance",
                     "unit_shape": [info_b["tile_y"], info_b["tile_z"]],
                     "device_bytes": info_b["device_bytes"]}
    if "batch" not in skip:
        tile = tuple(int(x) for x in args.batch_tile.split(",")) if args.batch_tile else None
        line["batch"] = batch_run(dsea, torch, args.batch_boxes, args.batch_md_steps, stream, tile)
    if "serve" not in skip:
        why = None
        if args.serve_window < 60.0:
            why = (f"arrival window {args.serve_window:g} s instead of 60 s: the stream offers about "
                   f"1.1e11 atom-steps/s (200 jobs/s x E[N steps] 5.6e8), some 30 times what one GPU "
                   f"advances, so the 60 s stream would take about half an hour to drain; the shorter "
                   f"window keeps the arrival process (rate, size and step draws) and the queueing it causes")
        line["served"] = serve_run(dsea, torch, args.serve_rate, args.serve_window, args.serve_budget_gb,
                                   why_window=why, policy=args.serve_policy)
        line["served_sustainable"] = serve_run(dsea, torch, args.serve_rate_sustainable,
                                               args.serve_window_sustainable, args.serve_budget_gb,
                                               policy=args.serve_policy)
    if "dataset" not in skip:
        line["dataset_heat1d"] = dataset_run(dsea, torch, stream)
    if "e2e" not in skip:
        line["e2e"] = e2e_run(dsea, torch, spec, dsea.MIXED, 3, args.md_steps, stream)
    if rank == 0 and world == 1 and "cpu" not in skip:
        line["cpu_baseline"] = cpu_baseline(spec, args.cpu_sample_steps_all, threads=0)
        line["cpu_baseline_1core"] = cpu_baseline(spec, args.cpu_sample_steps, threads=1)
    line["clocks"] = clk.summary()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
