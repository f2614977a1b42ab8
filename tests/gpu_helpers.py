"""Shared helpers of the GPU parity tests: build a context from a seeded graph
and compare the CUDA library with the CPU oracle on the same inputs."""
import numpy as np

import oracle as O
from paper_2510_12196_gb300 import gpumap as G
from paper_2510_12196_gb300 import inputs as I


def make_ctx(g, hier, dist, eps=0.03, seed=0x5EED0000, **cfg_over):
    cfg = G.map_config_default(seed)
    for k, v in cfg_over.items():
        setattr(cfg, k, v)
    return G.map_create(g.xadj, g.adj if g.m_dir else None, g.adjw if g.m_dir else None, g.vw, g.n,
                        hier, dist, eps, cfg)


def oracle_params(seed=0x5EED0000, **over):
    p = O.default_params(seed)
    for k, v in over.items():
        setattr(p, k, v)
    return p


def graph_zoo():
    """Small graphs covering the degree classes and structure of the paper's
    workload families, plus degenerate cases."""
    zoo = [
        I.grid2d(16, 12),
        I.grid3d(6, 5, 4),
        I.rgg2d(3000, I.rgg_radius(3000, 12), 11, wmax=10),
        I.erdos_renyi(60, 0.7, 5, wmax=9, vwmax=4),      # degrees ~40: CTA-per-vertex path
        I.rmat(11, 8, 0.57, 0.19, 0.19, 3),               # hubs + isolated vertices
        I.erdos_renyi(40, 0.05, 8, wmax=3, vwmax=5),      # sparse, isolated vertices
    ]
    # a star: one vertex of degree 299 plus leaves
    n = 300
    zoo.append(I.csr_from_pairs(n, np.zeros(n - 1, np.int64), np.arange(1, n), name="star300"))
    return zoo


TOPOS = [((4, 8), (1, 10)), ((4, 8, 6), (1, 10, 100)), ((2, 3), (3, 7)), ((3,), (5,)),
         ((1, 4, 2), (2, 9, 40)), ((2, 4, 16, 8), (1, 10, 100, 1000))]


def g_graph_from_level(xadj, adj, w, vw):
    return I.Graph(len(vw), xadj, adj, w, vw)


def map_run_compare(g, hier, dist, eps=0.03, seed=0x5EED0000, **over):
    """map_run on the GPU against the oracle's pipeline with the same
    settings: levels, per-level n, iterations, J and the final mapping."""
    ctx = make_ctx(g, hier, dist, eps=eps, seed=seed, **over)
    try:
        pi = np.zeros(g.n, np.int32)
        J = G.map_run(ctx, pi)
        st = G.map_stats(ctx)
    finally:
        G.map_destroy(ctx)
    fields = {f[0] for f in O.Params._fields_}  # execution settings do not reach the oracle
    opi, oJ, ost = O.map_run(g, hier, dist, eps, oracle_params(seed, **{k: v for k, v in over.items() if k in fields}))
    assert st.levels == ost.levels
    assert [st.n[i] for i in range(st.levels)] == [ost.n[i] for i in range(ost.levels)]
    assert [st.iters[i] for i in range(st.levels)] == [ost.iters[i] for i in range(ost.levels)]
    assert [st.J[i] for i in range(st.levels)] == [ost.J[i] for i in range(ost.levels)]
    for i in range(st.levels):  # the per-level split of the iterations into LP, weak and strong steps
        assert st.lp_iters[i] + st.weak_iters[i] + st.strong_iters[i] == min(st.iters[i], 4096), i
    assert J == oJ
    assert np.array_equal(pi, opi)
    return J
