"""Pins of the schedule oracle: Table 1 row by row, Eq. 1, and the ring's
slice dependency rule."""
import os

import pytest

from oracle import schedule

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_one_worker.txt")


def _parse_cell(cell: str, n: int):
    cell = cell.strip()
    if cell == "-":
        return ()
    out = []
    for tok in cell.split(","):
        tok = tok.strip()
        out.append(n + int(tok[1:] or 0) if tok.startswith("N") else int(tok))
    return tuple(out)


def _golden_rows(n):
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        cols = line.split("|")
        stage = _parse_cell(cols[0], n)[0]
        rows[stage] = tuple(_parse_cell(c, n) for c in cols[1:])
    return rows


def _as_cols(row):
    stage, store, receive, worker, partial, send = row
    one = lambda x: () if x is None else (x,)
    return stage, (store, one(receive), one(worker), partial, one(send))


@pytest.mark.parametrize("n_s", [6, 8, 13, 40])
def test_table1_rows(n_s):
    rows = dict(_as_cols(r) for r in schedule.one_worker_table(n_s))
    golden = _golden_rows(n_s)
    assert len(rows) == n_s + 3              # N_S + 3 stages per super-cycle
    for stage, cols in golden.items():
        assert rows[stage] == cols, f"stage {stage}"
    # rows between 5 and N_S follow the pattern of stage 5 shifted by one
    for k in range(6, n_s):
        store, recv, work, partial, send = rows[k]
        assert store == (k - 3, k - 2, k - 1) and recv == (k,) and work == (k - 2,)
        assert partial == (k - 2, k - 1) and send == (k - 3,)


def test_table1_lag_gives_eq1():
    # at stage 4 slice 4 is received while slice 1 is sent: four slices in
    # flight per worker, so N_S / 4 processes can work at once (Eq. 1)
    rows = schedule.one_worker_table(16)
    st4 = rows[3]
    assert st4[2] == 4 and st4[5] == 1
    assert schedule.n_max(16) == 16 / 4
    assert schedule.n_max(596, n_wgpu=1) == 149      # Sec. 4.3: 149 GPUs
    assert schedule.n_max(277, n_wgpu=2) == pytest.approx(277 / 6)


def test_ring_dependencies():
    assert schedule.ring_dependencies(5, 0, 10) == []
    assert schedule.ring_dependencies(0, 3, 10) == [(0, 2), (1, 2), (2, 2), (8, 2), (9, 2)]
    assert schedule.ring_dependencies(1, 1, 3) == [(0, 0), (1, 0), (2, 0)]
    # every unit reads its own slice and both neighbours of the previous level
    for j in range(7):
        deps = schedule.ring_dependencies(j, 4, 7)
        assert {(j - 1) % 7, j, (j + 1) % 7} <= {d[0] for d in deps}
