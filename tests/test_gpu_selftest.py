"""Failure detection without a GPU fault: a grid barrier of the refinement
engine that can never be released (it waits for one block more than the grid
has) gives up after its time limit, the blocks leave the kernel, the failure
is reported as MAP_E_TIMEOUT, and the device keeps working."""
import time

import numpy as np
import pytest

import oracle as O
from paper_2510_12196_gb300 import gpumap as G
from paper_2510_12196_gb300 import inputs as I

from gpu_helpers import make_ctx, oracle_params

pytestmark = pytest.mark.gpu


def test_grid_barrier_wait_expires_and_is_reported():
    t0 = time.perf_counter()
    st = G.map_selftest_barrier_timeout()
    dt = time.perf_counter() - t0
    assert st == 5, G.map_last_error(None)  # MAP_E_TIMEOUT: the wait ran out and was reported
    assert 0.5 < dt < 60.0
    # the context and the device stay usable
    g = I.rgg2d(3000, I.rgg_radius(3000, 12), 3, wmax=10)
    ctx = make_ctx(g, (4, 8), (1, 10))
    try:
        pi = np.zeros(g.n, np.int32)
        J = G.map_run(ctx, pi)
    finally:
        G.map_destroy(ctx)
    opi, oJ, _ = O.map_run(g, (4, 8), (1, 10), 0.03, oracle_params())
    assert J == oJ and np.array_equal(pi, opi)
