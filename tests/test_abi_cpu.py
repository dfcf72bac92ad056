"""CPU checks of the C ABI: the library builds and loads, exports every call
include/dsea.h declares, and its host-side schedule logic obeys the ring's
dependency rule (no GPU is touched)."""
import os
import re

import numpy as np
import pytest

from oracle import schedule
from paper_2507_11289_gb300 import dsea

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "dsea.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dsea_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_call():
    lib = dsea.load()
    names = _declared()
    assert len(names) >= 25
    for name in names:
        assert hasattr(lib, name), name
    # and the binding wraps exactly those calls
    assert set(dsea._SIGS) == set(names)


def test_checked_variant_builds_and_exports_the_same_calls():
    """The bounds-checked build (-DDSEA_CHECKED=1) is the same ABI."""
    import ctypes

    from paper_2507_11289_gb300 import build
    lib = ctypes.CDLL(build.build(checked=True))
    for name in _declared():
        assert hasattr(lib, name), name
    fn = lib.dsea_status_string
    fn.restype, fn.argtypes = ctypes.c_char_p, [ctypes.c_int]
    assert fn(dsea.ERR_BOUNDS) == b"index out of range (checked build)"


def test_status_strings_and_version():
    assert dsea.version() == "0.1.0"
    for code in range(-13, 1):
        s = dsea.status_string(code)
        assert s and s != "unknown status"
    assert dsea.status_string(-99) == "unknown status"


@pytest.mark.parametrize("n_s,ups,steps,start", [(3, 1, 6, 0), (4, 2, 5, 3), (7, 3, 6, 0), (43, 2, 4, 11)])
def test_ring_order_is_topological(n_s, ups, steps, start):
    sl, st = dsea.ring_order(n_s, ups, steps, start)
    assert len(sl) == n_s * ups * steps
    seen = {}
    for k, (j, s) in enumerate(zip(sl.tolist(), st.tolist())):
        seen.setdefault((j, s), []).append(k)
    # every (slice, step) unit appears ups times, steps in order
    assert all(len(v) == ups for v in seen.values()) and len(seen) == n_s * steps
    assert np.all(np.diff(st) >= 0)
    for (j, s), ks in seen.items():
        for dep in schedule.ring_dependencies(j, s, n_s):
            assert max(seen[dep]) < min(ks), f"unit {(j, s)} dispatched before its dependency {dep}"


def test_ring_order_time_skew():
    # each level starts two slices after the previous one (time-skewed cyclic order)
    n_s = 10
    sl, st = dsea.ring_order(n_s, 1, 4, 0)
    firsts = [int(sl[st == s][0]) for s in range(4)]
    assert firsts == [0, 2, 4, 6]
    # so a unit of level s waits only on the first five slices of level s-1
    order = list(zip(sl.tolist(), st.tolist()))
    pos = {u: k for k, u in enumerate(order)}
    lag = [pos[(sl[k], st[k])] - max(pos[d] for d in schedule.ring_dependencies(sl[k], st[k], n_s))
           for k in range(n_s, len(order))]
    assert min(lag) >= 1 and max(lag) <= n_s


def test_invalid_arguments_without_gpu():
    with pytest.raises(dsea.DseaError) as e:
        dsea.ring_order(2, 1, 1)            # fewer than three slices
    assert e.value.code == dsea.ERR_INVALID_ARG


def test_mirror_walls_reject_atoms_outside_without_gpu():
    """Box validation runs before any device call: with mirror walls every x
    must lie in [0, Lx); an unknown boundary code is rejected too."""
    box = [9.0, 9.0, 9.0]

    def create(desc):
        h = dsea.ctypes.c_void_p()
        return dsea.load().dsea_box_create(dsea.ctypes.byref(desc), None, None, dsea.ctypes.byref(h))

    for x in (-0.1, 9.0):
        d, keep = dsea._desc([[x, 1.0, 1.0]], None, box, 0, walls=True)
        assert create(d) == dsea.ERR_INVALID_ARG
    d, keep = dsea._desc([[1.0, 1.0, 1.0]], None, box, 0)
    d.boundary_x = 7
    assert create(d) == dsea.ERR_INVALID_ARG


@pytest.mark.parametrize("n,o_in,o_out,workers,steps", [(7, 1, 0, 1, 5), (9, 1, 1, 3, 7), (5, 2, 0, 2, 4),
                                                         (43, 1, 1, 4, 6)])
def test_dataset_plan_is_a_valid_time_skewed_ring(n, o_in, o_out, workers, steps):
    """The generic ring's dispatch order (Sec. 3.1): every step sweeps each
    slice once, on worker s mod K; every unit's dependencies (slices j-R..j+R,
    R = O_in + O_out, of the previous step; Sec. 3.3's rule for O_in = O_out =
    1 is oracle.schedule.ring_dependencies) come earlier; and each step starts
    R slices further, so its first unit needs only the first 2R+1 of the
    previous step."""
    from oracle import schedule
    sl, st, wk = dsea.dataset_plan(n, o_in, o_out, workers, steps, start_step=3)
    R = o_in + o_out
    pos = {(int(a), int(b)): k for k, (a, b) in enumerate(zip(sl, st))}
    assert len(pos) == n * steps
    for k, (j, s, w) in enumerate(zip(sl.tolist(), st.tolist(), wk.tolist())):
        assert w == s % workers
        if s == 3:
            continue
        deps = [((j + d) % n, s - 1) for d in range(-R, R + 1)]
        if o_in == 1 and o_out == 1:
            assert sorted(deps) == sorted((int(a), int(b)) for a, b in schedule.ring_dependencies(j, s, n))
        assert max(pos[x] for x in deps) < k
    for s in range(4, 3 + steps):
        first = pos[(int(sl[(s - 3) * n]), s)]
        need = max(pos[((int(sl[(s - 3) * n]) + d) % n, s - 1)] for d in range(-R, R + 1))
        assert need - (s - 4) * n <= 2 * R


def test_dataset_plan_rejects_overlapping_views():
    with pytest.raises(dsea.DseaError) as e:
        dsea.dataset_plan(4, 1, 1, 1, 1)     # 2 (O_in + O_out) + 1 = 5 views of 4 slices
    assert e.value.code == dsea.ERR_INVALID_ARG
