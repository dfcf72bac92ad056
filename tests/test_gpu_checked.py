"""The bounds-checked build (DSEA_VARIANT=checked, -DDSEA_CHECKED=1) stands in
for a memory checker: every computed global index and shared-memory list
position is tested before use, and one out of range fails the box with
DSEA_ERR_BOUNDS instead of touching memory.  The scenarios of
checked_scenarios.py run on it without such an error and give the release
build's results bit for bit (the checks change no arithmetic).  Each build
runs in its own process: a process loads one library."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _run(tmp_path, checked):
    env = dict(os.environ)
    env.pop("DSEA_VARIANT", None)
    if checked:
        env["DSEA_VARIANT"] = "checked"
    out = tmp_path / ("checked.npz" if checked else "release.npz")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_scenarios.py"), str(out)], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-4000:]
    return np.load(out), r.stdout


def test_checked_build_meets_no_bad_index_and_changes_no_bit(tmp_path):
    rel, out_rel = _run(tmp_path, False)
    chk, out_chk = _run(tmp_path, True)
    assert "libdsea.so" in out_rel and "libdsea_checked.so" in out_chk
    assert set(rel.files) == set(chk.files) and len(rel.files) > 100
    for k in rel.files:
        if k == "batch_shape":   # timed, so either build may pick another shape (results do not change)
            continue
        assert np.array_equal(rel[k], chk[k]), k
