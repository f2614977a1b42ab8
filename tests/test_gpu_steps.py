"""GPU parity of the single steps (objective J, block weights, Alg. 4 label
propagation, weak / strong rebalancing, Alg. 6) against the CPU oracle.
Everything is integer, so the bar is bit-exact equality."""
import numpy as np
import pytest

import oracle as O
from paper_2510_12196_gb300 import gpumap as G
from paper_2510_12196_gb300 import inputs as I

from gpu_helpers import TOPOS, graph_zoo, make_ctx, oracle_params

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("ti", range(len(TOPOS)))
def test_objective_and_block_weights(ti):
    hier, dist = TOPOS[ti]
    k = O.num_pes(hier)
    for gi, g in enumerate(graph_zoo()):
        ctx = make_ctx(g, hier, dist)
        try:
            for s in range(3):
                pi = I.random_mapping(g.n, k, 100 * gi + s)
                G.map_set_mapping(ctx, 0, pi)
                J, mx = G.map_objective(ctx, 0)
                Jo, mxo, Wo = O.objective(g, hier, dist, pi)
                assert (J, mx) == (Jo, mxo), (g.name, s)
                assert np.array_equal(G.map_block_weights(ctx, 0), Wo)
                assert np.array_equal(G.map_get_mapping(ctx, 0), pi)
        finally:
            G.map_destroy(ctx)


@pytest.mark.parametrize("ti", [0, 1, 2, 4, 5])
def test_lp_step_parity(ti):
    hier, dist = TOPOS[ti]
    k = O.num_pes(hier)
    for gi, g in enumerate(graph_zoo()):
        ctx = make_ctx(g, hier, dist)
        try:
            # a mapping with locality (ids in chunks) plus noise, and a few locks
            pi = ((np.arange(g.n) * k) // g.n).astype(np.int32)
            noise = I.random_mapping(g.n, k, gi)
            flip = I.splitmix64(7 + gi, np.arange(g.n, dtype=np.uint64)) % np.uint64(5) == 0
            pi[flip] = noise[flip]
            lock = (I.splitmix64(9 + gi, np.arange(g.n, dtype=np.uint64)) % np.uint64(7) == 0).astype(np.uint8)
            G.map_set_mapping(ctx, 0, pi)
            G.map_set_lock(ctx, 0, lock)
            opi, olock = pi.copy(), lock.copy()
            for step in range(3):
                mv = G.map_lp_step(ctx, 0)
                opi, olock, pp, gn, inx, omv, cnt = O.lp_step(g, hier, dist, opi, olock)
                gpp, gg, ginx, gmv = G.map_get_lp_state(ctx, 0)
                assert np.array_equal(ginx, inx), (g.name, step, "X")
                assert np.array_equal(gpp, pp), (g.name, step, "P'")
                assert np.array_equal(gg, gn), (g.name, step, "gain")
                assert np.array_equal(gmv, omv), (g.name, step, "moved")
                assert mv == cnt
                assert np.array_equal(G.map_get_mapping(ctx, 0), opi), (g.name, step, "P")
        finally:
            G.map_destroy(ctx)


@pytest.mark.parametrize("strong", [False, True])
@pytest.mark.parametrize("ti", [0, 1, 2, 5])
def test_rebalance_parity(strong, ti):
    hier, dist = TOPOS[ti]
    k = O.num_pes(hier)
    for gi, g in enumerate(graph_zoo()):
        ctx = make_ctx(g, hier, dist)
        try:
            cv = int(g.vw.sum())
            L = O.lmax(cv, k, 0.03)
            # skewed mapping: a third of the PEs take most vertices
            raw = I.random_mapping(g.n, 3 * k, 31 + gi)
            pi = np.minimum(raw, k - 1).astype(np.int32)
            opi = pi.copy()
            G.map_set_mapping(ctx, 0, pi)
            for t in range(1, 4):
                mv = G.map_rebalance_step(ctx, 0, strong, t)
                opi, dest, omv, cnt = O.rebalance(g, hier, dist, L, strong, opi, seed=0x5EED0000, level=0, t=t)
                assert mv == cnt, (g.name, t)
                assert np.array_equal(G.map_get_mapping(ctx, 0), opi), (g.name, t)
        finally:
            G.map_destroy(ctx)


def _refine_compare(g, hier, dist, pi0, rounds, level=0, eps=0.03, **cfg):
    k = O.num_pes(hier)
    L = O.lmax(int(g.vw.sum()), k, eps)
    ctx = make_ctx(g, hier, dist, eps=eps, **cfg)
    try:
        G.map_set_mapping(ctx, 0, pi0)
        J, mx, it = G.map_refine(ctx, 0, rounds)
        kinds, Js, Ws, cnt = G.map_get_refine_trace(ctx)
        opi, oJ, omx, oit, okinds, oJs, oWs = O.refine(g, hier, dist, L, pi0, rounds=rounds,
                                                        params=oracle_params(**cfg))
        assert it == oit
        assert np.array_equal(kinds, okinds)
        assert np.array_equal(Js, oJs)
        assert np.array_equal(Ws, oWs)
        assert (J, mx) == (oJ, omx)
        assert np.array_equal(G.map_get_mapping(ctx, 0), opi)
        assert G.map_objective(ctx, 0) == (oJ, omx)
    finally:
        G.map_destroy(ctx)
    return oJ


def test_refine_grid64_ten_rounds():
    """64x64 grid, 4:8 / 1:10, eps 0.03, random initial mapping, 10 rounds."""
    w = I.workload_grid64()
    _refine_compare(w.graph, w.topo.hier, w.topo.dist, w.pi0, 10)


@pytest.mark.parametrize("gi", range(7))
def test_refine_alg6_zoo(gi):
    g = graph_zoo()[gi]
    for hier, dist in (TOPOS[0], TOPOS[1], TOPOS[5]):
        k = O.num_pes(hier)
        _refine_compare(g, hier, dist, I.random_mapping(g.n, k, gi), -1)


def test_refine_rgg_alg6():
    g = I.rgg2d(1 << 14, I.rgg_radius(1 << 14, 12), 2, wmax=10)
    _refine_compare(g, (4, 8, 8), (1, 10, 100), I.random_mapping(g.n, 256, 1), -1)
    # patience / phi variants and a tight imbalance
    _refine_compare(g, (4, 8, 8), (1, 10, 100), I.random_mapping(g.n, 256, 2), -1, eps=0.0, patience=5,
                    weak_max=1, sigma_gap=7)
