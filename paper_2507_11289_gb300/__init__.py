"""GB300-native slice-streamed Lennard-Jones NVE molecular dynamics.

The data-parallel hot path of the paper's molecular-dynamics case study
(DSEAmd, Sec. 4): a cell-list short-range force stencil over each x-slice and
its two neighbours, fused with the velocity-Verlet update and the rebinning
of atoms that cross cell or slice boundaries, with (slice, step) units
streamed in a time-skewed cyclic order through a ring of persistent on-chip
stages.  The work runs in hand-written CUDA kernels for sm_103a behind the C
ABI of include/dsea.h; ``dsea`` is its thin Python binding and ``inputs``
draws the seeded synthetic workloads.

Submodules are imported lazily; nothing here touches the GPU at import time.
"""
__all__ = ["dsea", "inputs", "build"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
