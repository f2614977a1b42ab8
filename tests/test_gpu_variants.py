"""GPU parity of the refinement variants of Section 4.2 with the CPU oracle:
the relaxed negative-gain label-propagation filter and rebalancing with the
J objective (single steps on every kernel path, and whole runs through the
graph, stream and fused-engine paths)."""
import numpy as np
import pytest

import oracle as O
from paper_2510_12196_gb300 import gpumap as G
from paper_2510_12196_gb300 import inputs as I

from gpu_helpers import TOPOS, graph_zoo, make_ctx, map_run_compare

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("relax", [(1, 4), (3, 4), (2, 1)])
@pytest.mark.parametrize("ti", [0, 1, 5])
def test_lp_step_relaxed_parity(relax, ti):
    hier, dist = TOPOS[ti]
    k = O.num_pes(hier)
    for gi, g in enumerate(graph_zoo()):
        ctx = make_ctx(g, hier, dist, lp_relax_num=relax[0], lp_relax_den=relax[1])
        try:
            pi = ((np.arange(g.n) * k) // g.n).astype(np.int32)
            noise = I.random_mapping(g.n, k, gi)
            flip = I.splitmix64(17 + gi, np.arange(g.n, dtype=np.uint64)) % np.uint64(4) == 0
            pi[flip] = noise[flip]
            lock = np.zeros(g.n, np.uint8)
            G.map_set_mapping(ctx, 0, pi)
            G.map_set_lock(ctx, 0, lock)
            opi, olock = pi.copy(), lock.copy()
            for step in range(3):
                mv = G.map_lp_step(ctx, 0)
                opi, olock, pp, gn, inx, omv, cnt = O.lp_step(g, hier, dist, opi, olock, relax=relax)
                gpp, gg, ginx, gmv = G.map_get_lp_state(ctx, 0)
                assert np.array_equal(ginx, inx), (g.name, step, "X")
                assert np.array_equal(gpp, pp), (g.name, step, "P'")
                assert np.array_equal(gg, gn), (g.name, step, "gain")
                assert np.array_equal(gmv, omv), (g.name, step, "moved")
                assert mv == cnt
                assert np.array_equal(G.map_get_mapping(ctx, 0), opi), (g.name, step, "P")
        finally:
            G.map_destroy(ctx)


@pytest.mark.parametrize("mode", ["graph", "stream", "engine_only"])
def test_map_run_relaxed_parity(mode):
    g = I.rgg2d(1 << 15, I.rgg_radius(1 << 15, 12), 6, wmax=10)
    over = dict(lp_relax_num=3, lp_relax_den=4)
    if mode == "stream":
        over.update(launch_mode=1, engine_max_n=-1, grid_engine_max_n=-1)
    elif mode == "engine_only":
        over.update(engine_max_n=1 << 15)
    map_run_compare(g, (4, 8, 8), (1, 10, 100), **over)


def test_map_run_relaxed_rmat_hubs():
    # hubs exercise the CTA-per-vertex gain kernel's own-block connectivity
    map_run_compare(I.rmat(13, 16, 0.57, 0.19, 0.19, 5), (4, 16), (1, 10), lp_relax_num=1, lp_relax_den=2)


def test_relax_config_validation():
    g = I.grid2d(8, 8)
    for bad in [dict(lp_relax_num=-1), dict(lp_relax_den=0)]:
        with pytest.raises(G.MapError):
            make_ctx(g, (2, 2), (1, 10), **bad)


@pytest.mark.parametrize("strong", [False, True])
@pytest.mark.parametrize("ti", [0, 1, 2, 5])
def test_rebalance_j_objective_parity(strong, ti):
    hier, dist = TOPOS[ti]
    k = O.num_pes(hier)
    for gi, g in enumerate(graph_zoo()):
        ctx = make_ctx(g, hier, dist, reb_objective=1)
        try:
            L = O.lmax(int(g.vw.sum()), k, 0.03)
            raw = I.random_mapping(g.n, 3 * k, 57 + gi)
            pi = np.minimum(raw, k - 1).astype(np.int32)
            opi = pi.copy()
            G.map_set_mapping(ctx, 0, pi)
            for t in range(1, 4):
                mv = G.map_rebalance_step(ctx, 0, strong, t)
                opi, dest, omv, cnt = O.rebalance(g, hier, dist, L, strong, opi, seed=0x5EED0000, level=0, t=t,
                                                  objective=1)
                assert mv == cnt, (g.name, t)
                assert np.array_equal(G.map_get_mapping(ctx, 0), opi), (g.name, t)
        finally:
            G.map_destroy(ctx)


@pytest.mark.parametrize("mode", ["graph", "stream", "engine_only"])
def test_map_run_j_rebalancing_parity(mode):
    g = I.rgg2d(1 << 15, I.rgg_radius(1 << 15, 12), 8, wmax=10)
    over = dict(reb_objective=1)
    if mode == "stream":
        over.update(launch_mode=1, engine_max_n=-1, grid_engine_max_n=-1)
    elif mode == "engine_only":
        over.update(engine_max_n=1 << 15)
    map_run_compare(g, (4, 8, 8), (1, 10, 100), **over)


def test_map_run_both_variants_rmat():
    map_run_compare(I.rmat(13, 16, 0.57, 0.19, 0.19, 7), (4, 16), (1, 10), reb_objective=1, lp_relax_num=1,
                    lp_relax_den=4)


def test_reb_objective_validation():
    with pytest.raises(G.MapError):
        make_ctx(I.grid2d(8, 8), (2, 2), (1, 10), reb_objective=2)


def test_batch_with_variant_jobs():
    """A batch whose jobs mix the plain refinement and the variants runs the
    variant build of the engine; every job equals its own Alg. 6 run."""
    cases = []
    for i, n in enumerate((3000, 7000, 12000, 2000)):
        g = I.rgg2d(n, I.rgg_radius(n, 10.0), 0x5EED2000 + i, wmax=10)
        hier = ((4, 8), (4, 8, 8))[i % 2]
        dist = (1, 10, 100)[:len(hier)]
        over = [dict(), dict(reb_objective=1), dict(lp_relax_num=3, lp_relax_den=4),
                dict(reb_objective=1, lp_relax_num=1, lp_relax_den=4)][i]
        cases.append((g, hier, dist, I.random_mapping(n, int(np.prod(hier)), i), over))
    ctxs = []
    try:
        for g, hier, dist, pi0, over in cases:
            c = make_ctx(g, hier, dist, **over)
            G.map_set_mapping(c, 0, pi0)
            ctxs.append(c)
        b = G.map_batch_create(ctxs, G.map_batch_opts_default(rounds=-1))
        try:
            G.map_batch_launch(b)
            J, mw, it = G.map_batch_results(b, len(ctxs))
            sched = G.map_batch_schedule(b)
        finally:
            G.map_batch_destroy(b)
        assert sched[1] == 512
        for j, (g, hier, dist, pi0, over) in enumerate(cases):
            L = O.lmax(int(g.vw.sum()), int(np.prod(hier)), 0.03)
            from gpu_helpers import oracle_params
            opi, oJ, omx, oit, _, _, _ = O.refine(g, hier, dist, L, pi0, rounds=-1, params=oracle_params(**over))
            assert (J[j], mw[j], it[j]) == (oJ, omx, oit), j
            assert np.array_equal(G.map_get_mapping(ctxs[j], 0), opi), j
    finally:
        for c in ctxs:
            G.map_destroy(c)
