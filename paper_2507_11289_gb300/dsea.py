"""Thin Python binding of the C ABI in include/dsea.h (ctypes).

Every function here has the name of the C call it wraps (without the
``dsea_`` prefix) and only marshals arguments: all of the method's work runs
in the CUDA kernels of libdsea.so.  PyTorch provides the CUDA stream and, by
default, the device memory (its caching allocator, passed in through the
ABI's allocator callbacks).  Importing this module does not touch the GPU;
the first call loads libdsea.so and raises if it is missing or cannot be
built -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

OK = 0
ERR_INVALID_ARG = -1
ERR_OOM = -2
ERR_CUDA = -3
ERR_TIMEOUT = -4
ERR_CAPACITY = -5
ERR_MIGRATION = -6
ERR_BUDGET = -7
ERR_STATE = -8
ERR_NOT_FOUND = -9
ERR_NO_DEVICE = -10
ERR_SCRATCH_LIMIT = -11
ERR_BOUNDS = -12           # checked build only: a kernel met an index out of range
ERR_RANGE = -13            # a thermostat kinetic energy beyond its fixed-point range

FP64 = 0
MIXED = 1
KERNEL_LJ_TS = 1
SCHED_RING = 0
BOUNDARY_PERIODIC = 0
BOUNDARY_MIRROR = 1
SCHED_STEPWISE = 1
DEBUG_WITHHOLD_SLICE = 1
DEBUG_WAIT_LIMIT_NS = 2
PROBE_FP32 = 0
PROBE_FP32X2 = 1
PROBE_FP64 = 2

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("rc", ctypes.c_double), ("dt", ctypes.c_double), ("precision", ctypes.c_int),
                ("schedule", ctypes.c_int), ("tile_y", ctypes.c_int), ("tile_z", ctypes.c_int),
                ("cell_capacity", ctypes.c_int), ("ctas", ctypes.c_int), ("temperature", ctypes.c_double)]


class BoxDesc(ctypes.Structure):
    _fields_ = [("n_slices", ctypes.c_int), ("box", ctypes.c_double * 3), ("n_atoms", ctypes.c_int64),
                ("pos", ctypes.c_void_p), ("vel", ctypes.c_void_p), ("boundary_x", ctypes.c_int)]


class Observables(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("U", ctypes.c_double), ("W", ctypes.c_double),
                ("KE", ctypes.c_double)]


class BoxInfo(ctypes.Structure):
    _fields_ = [("n_slices", ctypes.c_int), ("cells_per_slice_x", ctypes.c_int),
                ("cells", ctypes.c_int * 3), ("tile_y", ctypes.c_int), ("tile_z", ctypes.c_int),
                ("units_per_step", ctypes.c_int), ("cell_capacity", ctypes.c_int),
                ("precision", ctypes.c_int), ("schedule", ctypes.c_int), ("n_atoms", ctypes.c_int64),
                ("step", ctypes.c_int64), ("device_bytes", ctypes.c_size_t),
                ("cell_edge", ctypes.c_double * 3), ("boundary_x", ctypes.c_int)]


class DseaError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} ({code})")


# name -> (restype, argtypes) of every exported entry point
_P, _I, _I64, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
_SIGS = {
    "dsea_version": (ctypes.c_char_p, []),
    "dsea_status_string": (ctypes.c_char_p, [_I]),
    "dsea_box_create": (_I, [ctypes.POINTER(BoxDesc), _P, _P, ctypes.POINTER(_P)]),
    "dsea_register_kernel": (_I, [_P, _I, _I, _I, ctypes.POINTER(Params)]),
    "dsea_advance": (_I, [_P, _I64]),
    "dsea_sync": (_I, [_P]),
    "dsea_read_positions": (_I, [_P, _P, _I64]),
    "dsea_read_velocities": (_I, [_P, _P, _I64]),
    "dsea_read_forces": (_I, [_P, _P, _I64]),
    "dsea_read_observables": (_I, [_P, ctypes.POINTER(Observables)]),
    "dsea_read_profiles": (_I, [_P, _P, _P, _P, _P, _I]),
    "dsea_box_get_info": (_I, [_P, ctypes.POINTER(BoxInfo)]),
    "dsea_box_destroy": (_I, [_P]),
    "dsea_batch_create": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(_P)]),
    "dsea_batch_advance": (_I, [_P, ctypes.POINTER(_I64)]),
    "dsea_batch_destroy": (_I, [_P]),
    "dsea_autotune": (_I, [_P, _I, ctypes.POINTER(Params)]),
    "dsea_batch_autotune": (_I, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "dsea_server_create": (_I, [ctypes.c_size_t, ctypes.POINTER(Params), _I, _P, ctypes.POINTER(_P)]),
    "dsea_server_set_policy": (_I, [_P, _I]),
    "dsea_server_submit": (_I, [_P, ctypes.POINTER(BoxDesc), _I64, ctypes.POINTER(ctypes.c_uint64)]),
    "dsea_server_poll": (_I, [_P, ctypes.c_uint64, ctypes.POINTER(_I)]),
    "dsea_server_result": (_I, [_P, ctypes.c_uint64, _P, _P, ctypes.POINTER(Observables),
                                ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "dsea_server_drain": (_I, [_P]),
    "dsea_server_clock": (_D, [_P]),
    "dsea_server_stats": (_I, [_P, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_I)]),
    "dsea_server_destroy": (_I, [_P]),
    "dsea_debug_set": (_I, [_P, _I, _I64]),
    "dsea_forces_noalloc": (_I, [_P, _P, _I64, _P, _D, _I, _P, _P, _P]),
    "dsea_ring_order": (_I, [_I, _I, _I64, _I64, _P, _P]),
    "dsea_dataset_create": (_I, [_I, ctypes.c_size_t, _I, _I, _I, _P, _P, ctypes.POINTER(_P)]),
    "dsea_dataset_write_slice": (_I, [_P, _I, _P, ctypes.c_size_t]),
    "dsea_dataset_read_slice": (_I, [_P, _I, _P, ctypes.c_size_t]),
    "dsea_dataset_register": (_I, [_P, _P, _P]),
    "dsea_dataset_run": (_I, [_P, _I64]),
    "dsea_dataset_step": (_I64, [_P]),
    "dsea_dataset_destroy": (_I, [_P]),
    "dsea_dataset_plan": (_I, [_I, _I, _I, _I, _I64, _I64, _P, _P, _P]),
    "dsea_example_heat1d": (_I, [_P, _I, _I64, _P, _P, ctypes.c_size_t, _P]),
    "dsea_probe_peak": (_I, [_I, _P, ctypes.POINTER(_D)]),
}

_lib = None
_lock = threading.Lock()


def checked_variant() -> bool:
    """Whether the process loads the bounds-checked library: environment
    variable DSEA_VARIANT=checked, read when the library is first loaded."""
    return os.environ.get("DSEA_VARIANT", "") == "checked"


def library_path() -> str:
    name = "libdsea_checked.so" if checked_variant() else "libdsea.so"
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", name)


def load(build: bool = True):
    """Load libdsea.so (building it in-tree first if stale and nvcc exists);
    libdsea_checked.so instead under DSEA_VARIANT=checked."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if build:
                from . import build as _build
                try:
                    path = _build.build(checked=checked_variant())
                except RuntimeError:
                    if not os.path.exists(path):
                        raise
            if not os.path.exists(path):
                raise RuntimeError(f"libdsea.so not found at {path}; build it with "
                                   "`python -m paper_2507_11289_gb300.build`")
            lib = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(code: int, where: str):
    if code != OK:
        raise DseaError(code, where)


def status_string(code: int) -> str:
    return load().dsea_status_string(code).decode()


def version() -> str:
    return load().dsea_version().decode()


def _f64(a, n=None) -> np.ndarray:
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1, 3))
    if n is not None and len(arr) != n:
        raise ValueError("array length does not match the atom count")
    return arr


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class TorchAllocator:
    """The ABI's allocator callbacks backed by PyTorch's caching allocator."""

    def __init__(self, stream=None):
        import torch
        self._torch = torch
        self.device = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._alloc = ALLOC_FN(self._do_alloc)
        self._free = FREE_FN(self._do_free)
        self.struct = Allocator(self._alloc, self._free, None)

    def _do_alloc(self, nbytes, ctx):
        try:
            return self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
        except Exception:          # out of memory: the library reports DSEA_ERR_OOM
            return None

    def _do_free(self, ptr, ctx):
        if ptr:
            self._torch.cuda.caching_allocator_delete(ptr)


def make_params(rc=2.5, dt=0.005, precision=FP64, schedule=SCHED_RING, tile_y=0, tile_z=0,
                cell_capacity=0, ctas=0, temperature=0.0) -> Params:
    """temperature > 0: NVT with the slice thermostat at that kT/epsilon."""
    return Params(rc, dt, precision, schedule, tile_y, tile_z, cell_capacity, ctas, float(temperature))


def _desc(pos, vel, box, n_slices, walls=False):
    p = _f64(pos)
    v = None if vel is None else _f64(vel, len(p))
    d = BoxDesc(int(n_slices), (ctypes.c_double * 3)(*[float(x) for x in box]), len(p),
                p.ctypes.data, None if v is None else v.ctypes.data,
                BOUNDARY_MIRROR if walls else BOUNDARY_PERIODIC)
    return d, (p, v)


# ---- box lifecycle --------------------------------------------------------

def box_create(pos, vel, box, n_slices: int = 0, stream=None, allocator="torch", walls=False):
    """dsea_box_create.  allocator: "torch" (caching allocator), None (cudaMalloc)
    or a TorchAllocator.  walls: mirror walls at x = 0 and x = Lx instead of a
    periodic x axis.  Returns an opaque handle (keep it for every call)."""
    lib = load()
    d, keep = _desc(pos, vel, box, n_slices, walls)
    sh = _stream_handle(stream)
    alloc = None
    if allocator == "torch":
        import torch
        alloc = TorchAllocator(torch.cuda.ExternalStream(sh) if sh else torch.cuda.default_stream())
    elif isinstance(allocator, TorchAllocator):
        alloc = allocator
    h = ctypes.c_void_p()
    _check(lib.dsea_box_create(ctypes.byref(d), ctypes.byref(alloc.struct) if alloc else None,
                               sh, ctypes.byref(h)), "dsea_box_create")
    return Handle(h.value, len(keep[0]), alloc)


class Handle:
    """An opaque box handle plus what must stay alive with it."""

    def __init__(self, ptr, n_atoms, alloc):
        self.ptr = ptr
        self.n_atoms = n_atoms
        self._alloc = alloc

    def __int__(self):
        return self.ptr


def register_kernel(h: Handle, params: Params | None = None, kind: int = KERNEL_LJ_TS, o_in: int = 1,
                    o_out: int = 1):
    _check(load().dsea_register_kernel(h.ptr, kind, o_in, o_out,
                                       ctypes.byref(params) if params is not None else None),
           "dsea_register_kernel")


def advance(h: Handle, n_steps: int):
    _check(load().dsea_advance(h.ptr, int(n_steps)), "dsea_advance")


def sync(h: Handle):
    _check(load().dsea_sync(h.ptr), "dsea_sync")


def _read(fn_name, h: Handle, out=None):
    out = np.empty((h.n_atoms, 3)) if out is None else out
    if out.dtype != np.float64 or not out.flags.c_contiguous or out.shape != (h.n_atoms, 3):
        raise ValueError("out must be a C-contiguous float64 (n, 3) array")
    _check(getattr(load(), fn_name)(h.ptr, out.ctypes.data, h.n_atoms), fn_name)
    return out


def read_positions(h: Handle, out=None):
    return _read("dsea_read_positions", h, out)


def read_velocities(h: Handle, out=None):
    return _read("dsea_read_velocities", h, out)


def read_forces(h: Handle, out=None):
    return _read("dsea_read_forces", h, out)


def read_observables(h: Handle) -> dict:
    o = Observables()
    _check(load().dsea_read_observables(h.ptr, ctypes.byref(o)), "dsea_read_observables")
    return {"step": o.step, "U": o.U, "W": o.W, "KE": o.KE}


def read_profiles(h: Handle, n_slices: int) -> dict:
    """dsea_read_profiles: per-slice U, W, KE (half pair energies, half pair
    virials, kinetic energies of each slice's atoms) and atom counts N."""
    U, W, KE = (np.zeros(n_slices) for _ in range(3))
    N = np.zeros(n_slices, dtype=np.int64)
    _check(load().dsea_read_profiles(h.ptr, U.ctypes.data, W.ctypes.data, KE.ctypes.data, N.ctypes.data,
                                     int(n_slices)), "dsea_read_profiles")
    return {"U": U, "W": W, "KE": KE, "N": N}


def box_get_info(h: Handle) -> dict:
    i = BoxInfo()
    _check(load().dsea_box_get_info(h.ptr, ctypes.byref(i)), "dsea_box_get_info")
    return {f: (list(getattr(i, f)) if f in ("cells", "cell_edge") else getattr(i, f))
            for f, _ in BoxInfo._fields_}


def box_destroy(h: Handle):
    if h.ptr:
        _check(load().dsea_box_destroy(h.ptr), "dsea_box_destroy")
        h.ptr = None


def debug_set(h: Handle, key: int, value: int):
    _check(load().dsea_debug_set(h.ptr, key, int(value)), "dsea_debug_set")


def autotune(h: Handle, trial_steps: int = 5) -> dict:
    p = Params()
    _check(load().dsea_autotune(h.ptr, int(trial_steps), ctypes.byref(p)), "dsea_autotune")
    return {f: getattr(p, f) for f, _ in Params._fields_}


# ---- batches --------------------------------------------------------------

def batch_create(handles):
    arr = (ctypes.c_void_p * len(handles))(*[h.ptr for h in handles])
    b = ctypes.c_void_p()
    _check(load().dsea_batch_create(arr, len(handles), ctypes.byref(b)), "dsea_batch_create")
    return b.value


def batch_advance(batch, steps):
    s = (ctypes.c_int64 * len(steps))(*[int(x) for x in steps])
    _check(load().dsea_batch_advance(batch, s), "dsea_batch_advance")


def batch_autotune(batch, trial_steps: int = 3) -> tuple[int, int]:
    """One unit shape for every box of the batch, timed on the batch itself;
    returns (tile_y, tile_z)."""
    ty, tz = ctypes.c_int(0), ctypes.c_int(0)
    _check(load().dsea_batch_autotune(batch, int(trial_steps), ctypes.byref(ty), ctypes.byref(tz)),
           "dsea_batch_autotune")
    return ty.value, tz.value


def batch_destroy(batch):
    _check(load().dsea_batch_destroy(batch), "dsea_batch_destroy")


# ---- serving --------------------------------------------------------------

def server_create(mem_budget_bytes: int, params: Params | None = None, segment_steps: int = 100,
                  stream=0):
    s = ctypes.c_void_p()
    _check(load().dsea_server_create(int(mem_budget_bytes),
                                     ctypes.byref(params) if params is not None else None,
                                     int(segment_steps), stream, ctypes.byref(s)),
           "dsea_server_create")
    return s.value


SERVE_ALL = 0         # every resident job in every launch
SERVE_SHORTEST = 1    # least remaining work first, aged, filling the GPU (the default)


def server_set_policy(srv, policy: int):
    _check(load().dsea_server_set_policy(srv, int(policy)), "dsea_server_set_policy")


def server_submit(srv, pos, vel, box, steps: int, n_slices: int = 0, walls=False) -> int:
    d, keep = _desc(pos, vel, box, n_slices, walls)
    jid = ctypes.c_uint64()
    _check(load().dsea_server_submit(srv, ctypes.byref(d), int(steps), ctypes.byref(jid)),
           "dsea_server_submit")
    del keep
    return jid.value


def server_poll(srv, job_id: int) -> int:
    st = ctypes.c_int()
    _check(load().dsea_server_poll(srv, job_id, ctypes.byref(st)), "dsea_server_poll")
    return st.value


def server_result(srv, job_id: int, n_atoms: int):
    pos = np.empty((n_atoms, 3))
    vel = np.empty((n_atoms, 3))
    o = Observables()
    ta, td = ctypes.c_double(), ctypes.c_double()
    _check(load().dsea_server_result(srv, job_id, pos.ctypes.data, vel.ctypes.data, ctypes.byref(o),
                                     ctypes.byref(ta), ctypes.byref(td)), "dsea_server_result")
    return pos, vel, {"step": o.step, "U": o.U, "W": o.W, "KE": o.KE}, ta.value, td.value


def server_drain(srv):
    _check(load().dsea_server_drain(srv), "dsea_server_drain")


def server_clock(srv) -> float:
    return load().dsea_server_clock(srv)


def server_stats(srv) -> dict:
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    _check(load().dsea_server_stats(srv, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "dsea_server_stats")
    return {"atom_steps": a.value, "busy_seconds": b.value, "launches": c.value}


def server_destroy(srv):
    _check(load().dsea_server_destroy(srv), "dsea_server_destroy")


# ---- schedule introspection ------------------------------------------------

def ring_order(n_slices: int, units_per_slice: int, n_steps: int, start_step: int = 0):
    n = n_slices * units_per_slice * n_steps
    sl = np.empty(n, dtype=np.int32)
    st = np.empty(n, dtype=np.int32)
    _check(load().dsea_ring_order(n_slices, units_per_slice, n_steps, start_step, sl.ctypes.data,
                                  st.ctypes.data), "dsea_ring_order")
    return sl, st


class Box:
    """Convenience owner of one box handle (same calls as above)."""

    def __init__(self, pos, vel, box, n_slices=0, precision=FP64, schedule=SCHED_RING, rc=2.5,
                 dt=0.005, tile_y=0, tile_z=0, cell_capacity=0, ctas=0, stream=None,
                 allocator="torch", walls=False, temperature=0.0):
        self.h = box_create(pos, vel, box, n_slices, stream, allocator, walls)
        try:
            register_kernel(self.h, make_params(rc, dt, precision, schedule, tile_y, tile_z,
                                                cell_capacity, ctas, temperature))
        except Exception:
            box_destroy(self.h)
            raise
        self.n_atoms = self.h.n_atoms

    def advance(self, n):
        advance(self.h, n)

    def sync(self):
        sync(self.h)

    def positions(self):
        return read_positions(self.h)

    def velocities(self):
        return read_velocities(self.h)

    def forces(self):
        return read_forces(self.h)

    def observables(self):
        return read_observables(self.h)

    def profiles(self):
        return read_profiles(self.h, self.info()["n_slices"])

    def info(self):
        return box_get_info(self.h)

    def debug_set(self, key, value):
        debug_set(self.h, key, value)

    def autotune(self, trial_steps=5):
        return autotune(self.h, trial_steps)

    def close(self):
        box_destroy(self.h)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---- the generic slice ring ------------------------------------------------

SLICE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                            ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


def dataset_plan(n_slices: int, o_in: int, o_out: int, n_workers: int, n_steps: int, start_step: int = 0):
    """dsea_dataset_plan: (slice, step, worker) of every unit in dispatch order."""
    n = n_slices * n_steps
    sl = np.empty(n, dtype=np.int32)
    st = np.empty(n, dtype=np.int64)
    wk = np.empty(n, dtype=np.int32)
    _check(load().dsea_dataset_plan(n_slices, o_in, o_out, n_workers, n_steps, start_step, sl.ctypes.data,
                                    st.ctypes.data, wk.ctypes.data), "dsea_dataset_plan")
    return sl, st, wk


class Dataset:
    """A sliced dataset streamed through a registered slice kernel (dsea_dataset_*).

    kernel: "heat1d" (the library's example; user = the coefficient a) or a
    ctypes function pointer of type SLICE_FN / an address."""

    def __init__(self, n_slices, slice_bytes, o_in=1, o_out=0, n_workers=2, stream=None):
        self.n_slices, self.slice_bytes = int(n_slices), int(slice_bytes)
        h = ctypes.c_void_p()
        _check(load().dsea_dataset_create(self.n_slices, self.slice_bytes, int(o_in), int(o_out),
                                          int(n_workers), None, _stream_handle(stream), ctypes.byref(h)),
               "dsea_dataset_create")
        self.h = h.value
        self._keep = None

    def register(self, kernel, user=None):
        if kernel == "heat1d":
            self._keep = (ctypes.c_float(float(user)),)
            fn = ctypes.cast(load().dsea_example_heat1d, ctypes.c_void_p).value
            up = ctypes.addressof(self._keep[0])
        else:
            self._keep = (kernel, user)
            fn = ctypes.cast(kernel, ctypes.c_void_p).value
            up = user
        _check(load().dsea_dataset_register(self.h, fn, up), "dsea_dataset_register")

    def write(self, slice_index, data: np.ndarray):
        a = np.ascontiguousarray(data)
        _check(load().dsea_dataset_write_slice(self.h, int(slice_index), a.ctypes.data, a.nbytes),
               "dsea_dataset_write_slice")

    def read(self, slice_index, dtype=np.float32) -> np.ndarray:
        out = np.empty(self.slice_bytes // np.dtype(dtype).itemsize, dtype=dtype)
        _check(load().dsea_dataset_read_slice(self.h, int(slice_index), out.ctypes.data, out.nbytes),
               "dsea_dataset_read_slice")
        return out

    def run(self, n_steps):
        _check(load().dsea_dataset_run(self.h, int(n_steps)), "dsea_dataset_run")

    @property
    def step(self):
        return load().dsea_dataset_step(self.h)

    def close(self):
        if self.h:
            load().dsea_dataset_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def probe_peak(kind: int = PROBE_FP32, stream=None) -> float:
    """dsea_probe_peak: the measured FMA rate of this GPU in TFLOP/s."""
    out = ctypes.c_double()
    _check(load().dsea_probe_peak(int(kind), _stream_handle(stream), ctypes.byref(out)), "dsea_probe_peak")
    return out.value
