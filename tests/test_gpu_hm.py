"""GPU parity of hierarchical multisection (GPU-HM: Eq. 2, Alg. 2, Alg. 3)
with the CPU oracle: the final mapping, J, the partitioner calls per level
and Eq. 2's eps' bit for bit; independence of the worker count; empty
subgraphs, a_i = 1, isolated vertices and the full-size RGG workload."""
import numpy as np
import pytest

import oracle as O
from paper_2510_12196_gb300 import gpumap as G
from paper_2510_12196_gb300 import inputs as I

from gpu_helpers import make_ctx, oracle_params

pytestmark = pytest.mark.gpu


def _hm_compare(g, hier, dist, eps=0.03, seed=0x5EED0000, workers=0, **over):
    ctx = make_ctx(g, hier, dist, eps=eps, seed=seed, **over)
    try:
        pi = np.zeros(g.n, np.int32)
        J = G.map_run_hm(ctx, pi, workers=workers)
        st = G.map_hm_stats(ctx)
        Jd, _ = G.map_objective(ctx, 0)
        assert np.array_equal(G.map_get_mapping(ctx, 0), pi)
    finally:
        G.map_destroy(ctx)
    fields = {f[0] for f in O.Params._fields_}
    opi, oJ, ost = O.hm_run(g, hier, dist, eps, oracle_params(seed, **{k: v for k, v in over.items() if k in fields}))
    l = len(hier)
    assert [st.calls[i] for i in range(l)] == [ost.calls[i] for i in range(l)]
    assert [st.first_eps[i] for i in range(l)] == [ost.first_eps[i] for i in range(l)]
    assert J == oJ == Jd
    assert np.array_equal(pi, opi)
    return J, st


@pytest.mark.parametrize("case", ["rgg14", "grid3d", "rmat12", "er_weights"])
def test_hm_parity(case):
    if case == "rgg14":
        _hm_compare(I.rgg2d(1 << 14, I.rgg_radius(1 << 14, 12), 3, wmax=10), (4, 8, 8), (1, 10, 100))
    elif case == "grid3d":
        _hm_compare(I.grid3d(24, 16, 16), (4, 16, 8), (1, 10, 100))
    elif case == "rmat12":   # hubs and isolated vertices
        _hm_compare(I.rmat(12, 8, 0.57, 0.19, 0.19, 4), (1, 4, 2), (1, 10, 100))
    else:
        _hm_compare(I.erdos_renyi(3000, 0.003, 6, wmax=9, vwmax=5), (2, 3, 4, 2), (1, 5, 20, 100))


def test_hm_workers_do_not_change_the_result():
    g = I.rgg2d(1 << 13, I.rgg_radius(1 << 13, 12), 9, wmax=10)
    J1, st1 = _hm_compare(g, (4, 8), (1, 10), workers=1)
    J8, st8 = _hm_compare(g, (4, 8), (1, 10), workers=8)
    assert J1 == J8 and st1.workers == 1 and st8.workers == 8


def test_hm_empty_subgraphs_and_matching_coarsener():
    # 16 vertices on 32 PEs: some level-1 subgraphs are empty
    _hm_compare(I.grid2d(4, 4), (4, 8), (1, 10))
    # the partitioner may coarsen by matching as well
    _hm_compare(I.rgg2d(1 << 12, I.rgg_radius(1 << 12, 12), 5, wmax=10), (4, 4), (1, 10), coarsener=1)


def test_hm_rgg_2_20_full_size():
    """RGG 2^20, mean degree 12, weights 1..10, 4:8:8 / 1:10:100, eps 0.03."""
    w = I.workload_rgg(20)
    J, st = _hm_compare(w.graph, w.topo.hier, w.topo.dist, w.topo.eps, seed=w.seed)
    assert [st.calls[i] for i in range(3)] == [64, 8, 1]


def test_hm_invalid_workers():
    g = I.grid2d(8, 8)
    ctx = make_ctx(g, (2, 2), (1, 10))
    try:
        with pytest.raises(G.MapError):
            G.map_run_hm(ctx, workers=-1)
    finally:
        G.map_destroy(ctx)


@pytest.mark.parametrize("case", ["rgg15", "rmat13", "grid3d_match", "stream"])
def test_map_run_hm_initial_parity(case):
    """The integrated pipeline with the hierarchical-multisection initial
    mapping of the coarsest graph, bit-identical to the oracle."""
    from gpu_helpers import map_run_compare
    if case == "rgg15":
        map_run_compare(I.rgg2d(1 << 15, I.rgg_radius(1 << 15, 12), 3, wmax=10), (4, 8, 8), (1, 10, 100), initial=1)
    elif case == "rmat13":
        map_run_compare(I.rmat(13, 16, 0.57, 0.19, 0.19, 5), (4, 16), (1, 10), initial=1)
    elif case == "grid3d_match":
        map_run_compare(I.grid3d(32, 32, 16), (4, 16, 8), (1, 10, 100), initial=1, coarsener=1)
    else:
        map_run_compare(I.rgg2d(1 << 14, I.rgg_radius(1 << 14, 12), 4, wmax=10, shuffled=True), (4, 8, 6),
                        (1, 10, 100), initial=1, launch_mode=1, engine_max_n=-1, grid_engine_max_n=-1)


def test_map_run_hm_initial_rgg_2_20():
    from gpu_helpers import map_run_compare
    w = I.workload_rgg(20)
    map_run_compare(w.graph, w.topo.hier, w.topo.dist, w.topo.eps, seed=w.seed, initial=1)
