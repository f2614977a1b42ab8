"""GPU parity of the two-hop matching coarsener (Section 4.2, "Matching")
against the CPU oracle: every level's M and coarse graph, and the full
pipeline with matching in place of label-propagation clustering.  All
integer, so the bar is bit-exact equality."""
import numpy as np
import pytest

import oracle as O
from paper_2510_12196_gb300 import gpumap as G
from paper_2510_12196_gb300 import inputs as I

from gpu_helpers import make_ctx, oracle_params

pytestmark = pytest.mark.gpu


def _bipartite_twins(a=2, b=50):
    """K_{a,b}: the b vertices share the neighbour set {0..a-1} (twins)."""
    src = np.repeat(np.arange(a), b)
    dst = np.tile(np.arange(a, a + b), a)
    return I.csr_from_pairs(a + b, src, dst, name=f"K{a},{b}")


def _star(n=300):
    return I.csr_from_pairs(n, np.zeros(n - 1, np.int64), np.arange(1, n), name=f"star{n}")


def _oracle_chain(g, k, lmax, prm, max_levels=64):
    out = []
    cur = g
    while len(out) + 1 < max_levels and cur.n >= prm.coarsest_factor * k:
        M, nc, _, _ = O.match(cur, lmax, prm, level=len(out))
        if nc * prm.stall_den > prm.stall_num * cur.n:
            break
        xc, ac, wc, vc = O.contract(cur, M, nc)
        out.append((cur, M))
        cur = I.Graph(nc, xc, ac, wc, vc)
    out.append((cur, None))
    return out


def _check_levels(g, hier, dist, eps=0.03, seed=0x5EED0000, **over):
    k = O.num_pes(hier)
    prm = oracle_params(seed, coarsener=1, **over)
    lmax = O.lmax(int(g.vw.sum()), k, eps)
    chain = _oracle_chain(g, k, lmax, prm)
    ctx = make_ctx(g, hier, dist, eps=eps, seed=seed, coarsener=1, **over)
    try:
        nl = G.map_coarsen(ctx)
        assert nl == len(chain)
        for lvl, (og, oM) in enumerate(chain):
            xadj, adj, w, vw, M = G.map_get_level_graph(ctx, lvl, with_M=oM is not None)
            assert np.array_equal(xadj, og.xadj), lvl
            assert np.array_equal(adj, og.adj), lvl
            assert np.array_equal(w, og.adjw), lvl
            assert np.array_equal(vw, og.vw), lvl
            if oM is not None:
                assert np.array_equal(M, oM), lvl
    finally:
        G.map_destroy(ctx)
    return chain


@pytest.mark.parametrize("case", ["rgg", "rmat", "er_weights", "star", "twins", "grid"])
def test_match_levels(case):
    if case == "rgg":
        chain = _check_levels(I.rgg2d(1 << 15, I.rgg_radius(1 << 15, 12), 7, wmax=10), (4, 8, 8), (1, 10, 100))
        assert len(chain) >= 3
    elif case == "rmat":   # hubs, leaves and isolated vertices: every two-hop stage
        _check_levels(I.rmat(13, 8, 0.57, 0.19, 0.19, 9), (4, 8), (1, 10))
    elif case == "er_weights":   # vertex weights 1..5, many PEs: L_max binds on coarse levels
        _check_levels(I.erdos_renyi(2000, 0.004, 4, wmax=7, vwmax=5), (2, 4, 16), (1, 10, 100), coarsest_factor=2)
    elif case == "star":
        _check_levels(_star(300), (2, 2), (1, 10), coarsest_factor=1)
    elif case == "twins":
        _check_levels(_bipartite_twins(2, 50), (2, 2), (1, 10), coarsest_factor=1)
    else:
        _check_levels(I.grid3d(24, 16, 8), (4, 16), (1, 10), match_rounds=3)


def test_match_rounds_zero_and_one():
    g = I.rmat(12, 8, 0.57, 0.19, 0.19, 4)
    _check_levels(g, (4, 4), (1, 10), match_rounds=0)
    _check_levels(g, (4, 4), (1, 10), match_rounds=1)


def _map_run_compare(g, hier, dist, eps=0.03, seed=0x5EED0000, **over):
    ctx = make_ctx(g, hier, dist, eps=eps, seed=seed, coarsener=1, **over)
    try:
        pi = np.zeros(g.n, np.int32)
        J = G.map_run(ctx, pi)
        st = G.map_stats(ctx)
    finally:
        G.map_destroy(ctx)
    fields = {f[0] for f in O.Params._fields_}
    prm = oracle_params(seed, coarsener=1, **{k: v for k, v in over.items() if k in fields})
    opi, oJ, ost = O.map_run(g, hier, dist, eps, prm)
    assert st.levels == ost.levels
    assert [st.n[i] for i in range(st.levels)] == [ost.n[i] for i in range(ost.levels)]
    assert [st.iters[i] for i in range(st.levels)] == [ost.iters[i] for i in range(ost.levels)]
    assert [st.J[i] for i in range(st.levels)] == [ost.J[i] for i in range(ost.levels)]
    assert J == oJ
    assert np.array_equal(pi, opi)
    return J


@pytest.mark.parametrize("case", ["rgg15", "rmat13", "grid3d", "stream"])
def test_map_run_matching_parity(case):
    if case == "rgg15":
        _map_run_compare(I.rgg2d(1 << 15, I.rgg_radius(1 << 15, 12), 3, wmax=10), (4, 8, 8), (1, 10, 100))
    elif case == "rmat13":
        _map_run_compare(I.rmat(13, 16, 0.57, 0.19, 0.19, 5), (4, 16), (1, 10))
    elif case == "grid3d":
        _map_run_compare(I.grid3d(32, 32, 16), (4, 16, 8), (1, 10, 100))
    else:   # stream launches, no fused engine
        _map_run_compare(I.rgg2d(1 << 14, I.rgg_radius(1 << 14, 12), 4, wmax=10, shuffled=True), (4, 8, 6),
                         (1, 10, 100), launch_mode=1, engine_max_n=-1, grid_engine_max_n=-1)


def test_map_run_matching_rgg_2_20():
    """RGG 2^20 with the matching coarsener, bit-identical to the oracle."""
    w = I.workload_rgg(20)
    _map_run_compare(w.graph, w.topo.hier, w.topo.dist, w.topo.eps, seed=w.seed)


def test_coarsener_config_validation():
    g = I.grid2d(8, 8)
    for bad in [dict(coarsener=2), dict(coarsener=-1), dict(coarsener=1, match_rounds=-1)]:
        with pytest.raises(G.MapError):
            make_ctx(g, (2, 2), (1, 10), **bad)


def test_matching_graph_reuse_across_runs():
    """Repeated runs replay the cached per-level matching graphs; every run
    gives the oracle's result, in graph and in stream launch mode alike."""
    g = I.rmat(13, 8, 0.57, 0.19, 0.19, 2)
    hier, dist = (4, 8), (1, 10)
    opi, oJ, _ = O.map_run(g, hier, dist, 0.03, oracle_params(coarsener=1))
    for mode in (0, 1):
        ctx = make_ctx(g, hier, dist, coarsener=1, launch_mode=mode)
        try:
            for _ in range(3):
                pi = np.zeros(g.n, np.int32)
                l0 = G.map_launch_count()
                assert G.map_run(ctx, pi) == oJ
                assert np.array_equal(pi, opi)
                assert G.map_launch_count() > l0
        finally:
            G.map_destroy(ctx)
