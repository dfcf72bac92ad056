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


def test_status_strings_and_version():
    assert dsea.version() == "0.1.0"
    for code in range(-10, 1):
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
