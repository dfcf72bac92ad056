import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def melted_4k():
    """The 4,000-atom fcc start (rho 0.8, T 1.5) melted by 300 oracle steps:
    a liquid-like configuration produced by the oracle alone."""
    import oracle
    from paper_2507_11289_gb300 import inputs
    pos, vel, box = inputs.SMALL_4K.state()
    p, v, _, _ = oracle.run(pos, vel, box, steps=300)
    return p, v, box
