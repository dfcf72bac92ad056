"""The generic slice ring (dsea_dataset_*, Sec. 3.1/3.3) on the GPU: the
library's example slice kernel (an explicit FP32 heat-equation step on a
periodic rod) streamed over the slices in the time-skewed order equals a
plain NumPy evaluation of the same update bit for bit, whatever the number of
workers, the run split and the output radius."""
import ctypes

import numpy as np
import pytest

from paper_2507_11289_gb300 import dsea

pytestmark = pytest.mark.gpu


def heat_reference(u0, a, steps):
    """The same update in float32, every operation rounded (NumPy never fuses)."""
    u = u0.astype(np.float32)
    a, two = np.float32(a), np.float32(2.0)
    for _ in range(steps):
        ul, ur = np.roll(u, 1), np.roll(u, -1)
        u = u + a * ((ul - two * u) + ur)
    return u


def rod(n_slices, m, seed=11):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-1.0, 1.0, n_slices * m).astype(np.float32)


@pytest.mark.parametrize("workers,m", [(1, 1000), (2, 1000), (3, 1000), (2, 1001)])
def test_heat_ring_equals_numpy_bitwise(workers, m):
    """m = 1000: the kernel's four-point path; m = 1001: its one-point path."""
    n, a = 7, 0.23
    u0 = rod(n, m)
    with dsea.Dataset(n, m * 4, o_in=1, o_out=0, n_workers=workers) as ds:
        ds.register("heat1d", a)
        for j in range(n):
            ds.write(j, u0[j * m:(j + 1) * m])
        ds.run(20)
        ds.run(17)
        assert ds.step == 37
        got = np.concatenate([ds.read(j) for j in range(n)])
    assert np.array_equal(got, heat_reference(u0, a, 37))


def test_output_radius_one_through_a_python_kernel():
    """O_out = 1 (views of both neighbours' outputs, R = 2): a kernel that
    writes only its own output view gives the same rod."""
    n, m, a = 9, 512, 0.2
    u0 = rod(n, m, seed=12)
    lib = dsea.load()
    coef = ctypes.c_float(a)
    calls = []

    @dsea.SLICE_FN
    def kernel(user, j, step, inp, out, nbytes, stream):
        calls.append((j, step))
        own = ctypes.c_void_p(out + ctypes.sizeof(ctypes.c_void_p))   # out[O_out] = out[1]
        return lib.dsea_example_heat1d(ctypes.addressof(coef), j, step, inp, own, nbytes, stream)

    with dsea.Dataset(n, m * 4, o_in=1, o_out=1, n_workers=3) as ds:
        ds.register(kernel)
        for j in range(n):
            ds.write(j, u0[j * m:(j + 1) * m])
        ds.run(11)
        got = np.concatenate([ds.read(j) for j in range(n)])
    assert np.array_equal(got, heat_reference(u0, a, 11))
    sl, st, _ = dsea.dataset_plan(n, 1, 1, 3, 11)
    assert calls == list(zip(sl.tolist(), st.tolist()))      # launched in the planned order


def test_kernel_error_stops_the_run():
    n, m = 5, 64

    @dsea.SLICE_FN
    def failing(user, j, step, inp, out, nbytes, stream):
        return dsea.ERR_INVALID_ARG if j == 3 else 0

    with dsea.Dataset(n, m * 4, o_in=1, o_out=0, n_workers=2) as ds:
        ds.register(failing)
        with pytest.raises(dsea.DseaError) as e:
            ds.run(2)
        assert e.value.code == dsea.ERR_INVALID_ARG
    with dsea.Dataset(n, m * 4) as ds:                    # no kernel registered
        with pytest.raises(dsea.DseaError) as e:
            ds.run(1)
        assert e.value.code == dsea.ERR_STATE
