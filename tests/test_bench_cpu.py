"""Host-side checks of bench.py that need no GPU: the roofline's DRAM traffic
comes from the committed ncu summary, and the large-box leg defaults to the
67,108,864-atom workload."""
import dataclasses

import bench
from paper_2507_11289_gb300 import inputs


def test_profile_traffic_is_read_and_plausible():
    t = bench.profile_traffic_per_atom_step()
    assert t is not None
    # at least the 112 B of state read and written per atom-step, and not wildly above it
    assert 112.0 <= t <= 400.0


def test_large_box_leg_defaults_to_the_67m_workload():
    args = bench.build_parser().parse_args([])
    big = dataclasses.replace(inputs.FLUID_67M, n_i=args.big_n_i, steps=args.big_md_steps)
    assert big == inputs.FLUID_67M and big.n_atoms == 67_108_864 and big.steps == 200
    args = bench.build_parser().parse_args(["--big-n-i", "128", "--big-md-steps", "10"])
    small = dataclasses.replace(inputs.FLUID_67M, n_i=args.big_n_i, steps=args.big_md_steps)
    assert small != inputs.FLUID_67M and small.n_atoms == 8_388_608


def test_warmup_below_three_is_refused(monkeypatch):
    import sys

    import pytest
    monkeypatch.setattr(sys, "argv", ["bench.py", "--warmup", "2"])
    with pytest.raises(SystemExit) as e:
        bench.main()          # refused before any device work
    assert e.value.code == 2
