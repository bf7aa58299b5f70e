import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the compiled library")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def small_setup():
    """Fine 4^4 Wilson-clover lattice -> coarse 2^4, Nv = 4 (n = 8). Built by the oracle."""
    from oracle import multigrid
    from synthetic import draws
    from synthetic.gauge import su3_links
    dims = (4, 4, 4, 4)
    key = (900, 0)
    U = su3_links(key, dims).numpy()
    nv = 4
    starts = draws.test_vector_starts(key, 256, nv)
    D, P, s, h, tv = multigrid.build(U, dims, nv, m0=-0.4, csw=1.0, starts=starts)
    return {"dims": dims, "cdims": (2, 2, 2, 2), "U": U, "D": D, "P": P, "self": s, "hop": h,
            "nv": nv, "m0": -0.4, "csw": 1.0, "key": key, "tv": tv}


@pytest.fixture(scope="session")
def ragged_setup():
    """Fine 8x4x6x4 lattice -> coarse 4x2x3x2, Nv = 4: non-cubic, mixed extents."""
    from oracle import multigrid
    from synthetic import draws
    from synthetic.gauge import su3_links
    dims = (8, 4, 6, 4)
    key = (901, 0)
    U = su3_links(key, dims).numpy()
    nv = 4
    V = int(np.prod(dims))
    starts = draws.test_vector_starts(key, V, nv)
    D, P, s, h, tv = multigrid.build(U, dims, nv, m0=-0.3, csw=1.0, starts=starts)
    return {"dims": dims, "cdims": (4, 2, 3, 2), "U": U, "D": D, "P": P, "self": s, "hop": h,
            "nv": nv, "m0": -0.3, "csw": 1.0, "key": key}
