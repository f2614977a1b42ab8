"""The seeded input generators: sizes and structure of the workload recipes."""
import numpy as np

from paper_2510_12196_gb300 import inputs as I


def test_grid64_shape():
    w = I.workload_grid64()
    g = w.graph
    I.check_graph(g)
    assert (g.n, g.m, g.m_dir) == (4096, 8064, 16128)
    assert w.topo.k == 32 and w.pi0.min() >= 0 and w.pi0.max() < 32
    assert np.array_equal(w.pi0, I.random_mapping(4096, 32, w.seed))


def test_grid3d_and_rgg_structure():
    g = I.grid3d(8, 4, 2)
    I.check_graph(g)
    assert g.m == 7 * 4 * 2 + 8 * 3 * 2 + 8 * 4 * 1
    r = I.rgg2d(5000, I.rgg_radius(5000, 12), 9, wmax=10)
    I.check_graph(r)
    assert 10 < r.m_dir / r.n < 13
    assert r.adjw.min() >= 1 and r.adjw.max() <= 10
    # geometric locality of the cell ordering: most edges join nearby ids
    src = np.repeat(np.arange(r.n), r.degrees())
    assert np.median(np.abs(src - r.adj)) < 200
    s = I.rgg2d(5000, I.rgg_radius(5000, 12), 9, wmax=10, shuffled=True)
    I.check_graph(s)
    assert s.m == r.m


def test_generators_deterministic():
    a = I.rgg2d(3000, 0.03, 4, wmax=10)
    b = I.rgg2d(3000, 0.03, 4, wmax=10)
    assert np.array_equal(a.adj, b.adj) and np.array_equal(a.adjw, b.adjw)


def test_rmat_small():
    g = I.rmat(12, 16, 0.57, 0.19, 0.19, 77)
    I.check_graph(g)
    deg = g.degrees()
    assert deg.max() > 20 * max(1, np.median(deg))  # power-law skew
    assert (deg == 0).sum() > 0


def test_batch_and_serve_recipes():
    ws = I.workload_batch(count=6, lo_log2=8, hi_log2=10)
    for w in ws:
        I.check_graph(w.graph)
        assert 2**8 <= w.graph.n <= 2**10
        assert w.topo.hier in ((4, 8), (4, 8, 8), (2, 4, 16, 8))
        assert w.topo.dist == (1, 10, 100, 1000)[:w.topo.levels]
    for i in range(6):
        w = I.serve_request(i, max_log2_grid=12, max_log2_rgg=13)
        I.check_graph(w.graph)
        assert w.topo.k in (32, 256, 512, 1024)
    t = I.poisson_arrivals(1000, 0.005, 1)
    assert np.all(np.diff(t) > 0) and 0.004 < t[-1] / 1000 < 0.006


def test_degree_mix_classes():
    g = I.degree_mix()
    deg = np.diff(g.xadj)
    assert g.n == 1600 and list(deg[1596:]) == list(I.DEGREE_MIX_EXACT)
    assert ((deg[:400] > 32) & (deg[:400] <= 255)).all() and (deg[400:406] > 255).all()
    assert (deg[406:1596] <= 32).all()
    I.check_graph(g)
    h = I.degree_mix()
    assert np.array_equal(g.adj, h.adj) and np.array_equal(g.adjw, h.adjw) and np.array_equal(g.vw, h.vw)
