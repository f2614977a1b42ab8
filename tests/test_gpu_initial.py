"""GPU parity of the breadth-first initial mapping on coarsest graphs too large
for the one-CTA kernel (more than 12,288 vertices): components labelled by
their smallest id, one layered search from all roots, a sort by (component,
layer position).  The result must equal the oracle's FIFO search exactly:
many components, isolated vertices, hubs, deep searches, shuffled ids and
vertex weights."""
import numpy as np
import pytest

import oracle as O
from paper_2510_12196_gb300 import gpumap as G
from paper_2510_12196_gb300 import inputs as I

from gpu_helpers import make_ctx

pytestmark = pytest.mark.gpu


def _initial_only(g, hier=(2, 2), dist=(1, 10)):
    """map_initial on the input graph itself (coarsening stops at once)."""
    k = O.num_pes(hier)
    ctx = make_ctx(g, hier, dist, coarsest_factor=1 << 30)
    try:
        assert G.map_coarsen(ctx) == 1
        G.map_initial(ctx)
        pi = G.map_get_mapping(ctx, 0)
    finally:
        G.map_destroy(ctx)
    assert np.array_equal(pi, O.initial(g, k))
    return pi


def _components(n, sizes, seed):
    """Random trees of the given sizes plus a few extra edges, ids shuffled."""
    rng = np.random.default_rng(seed)
    us, vs, base = [], [], 0
    for s in sizes:
        for i in range(1, s):
            us.append(base + i)
            vs.append(base + int(rng.integers(0, i)))
        for _ in range(s // 3):
            a, b = rng.integers(0, s, 2)
            if a != b:
                us.append(base + int(a))
                vs.append(base + int(b))
        base += s
    perm = rng.permutation(n)
    u, v = perm[np.array(us)], perm[np.array(vs)]
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    pairs = np.unique(np.stack([lo, hi], 1), axis=0)
    return I.csr_from_pairs(n, pairs[:, 0], pairs[:, 1], name="components")


@pytest.mark.parametrize("case", ["rgg", "rgg_shuffled", "rmat", "er_sparse", "components", "weights"])
def test_large_initial_mapping(case):
    if case == "rgg":
        g = I.rgg2d(1 << 15, I.rgg_radius(1 << 15, 8), 3, wmax=10)
    elif case == "rgg_shuffled":
        g = I.rgg2d(1 << 15, I.rgg_radius(1 << 15, 8), 4, wmax=10, shuffled=True)
    elif case == "rmat":  # hubs and many isolated vertices
        g = I.rmat(15, 8, 0.57, 0.19, 0.19, 6)
    elif case == "er_sparse":  # a giant component and many small ones
        g = I.erdos_renyi(20000, 1.2 / 20000, 7, wmax=5)
    elif case == "components":
        sizes = [1] * 500 + [2] * 300 + [7] * 200 + [300] * 20 + [9000]
        g = _components(sum(sizes), sizes, 8)
    else:
        g = I.erdos_renyi(16000, 3.0 / 16000, 9, wmax=7, vwmax=6)
    _initial_only(g, hier=(4, 8, 4), dist=(1, 10, 100))


def test_large_initial_deep_search():
    """A shuffled path of 14,000 vertices: 14,000 search levels."""
    n = 14000
    perm = I.random_permutation(n, 11)
    u, v = perm[:-1], perm[1:]
    g = I.csr_from_pairs(n, np.minimum(u, v), np.maximum(u, v), name="path")
    _initial_only(g, hier=(2, 4), dist=(1, 10))


def test_map_run_large_coarsest():
    """Whole pipelines whose coarsest graph is mapped by the multi-CTA search:
    R-MAT 2^15 and an RGG 2^16 refined on the input graph directly."""
    from gpu_helpers import map_run_compare
    map_run_compare(I.rmat(15, 16, 0.57, 0.19, 0.19, 12), (4, 4), (1, 10), coarsest_factor=1 << 30)
    map_run_compare(I.rgg2d(1 << 16, I.rgg_radius(1 << 16, 12), 13, wmax=10), (4, 8, 8), (1, 10, 100),
                    coarsest_factor=1 << 30)
