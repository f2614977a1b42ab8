"""Pins of the oracle's two-hop matching coarsener (Section 4.2, "Matching"):
hand-computed outcomes on small graphs for each stage, the exp*2 rating
against plain heavy-edge choice, the 75% rule, validity (an involution
within the weight bound, pairs numbered by their smallest member) and the
contraction invariant J(G_c, P) = J(G, P o M)."""
import numpy as np
import pytest

import oracle as O
from paper_2510_12196_gb300 import inputs as I


def _g(n, pairs, w=None, vw=None):
    u = np.array([a for a, b in pairs], np.int64)
    v = np.array([b for a, b in pairs], np.int64)
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    return I.csr_from_pairs(n, lo, hi, None if w is None else np.array(w, np.int64),
                            vw=None if vw is None else np.array(vw, np.int32))


def _valid(g, mate, M, nc, lmax):
    n = g.n
    for v in range(n):
        if mate[v] >= 0:
            u = mate[v]
            assert u != v and mate[u] == v
            assert int(g.vw[v]) + int(g.vw[u]) <= lmax
            assert M[v] == M[u]
    reps = sorted({min(v, mate[v]) if mate[v] >= 0 else v for v in range(n)})
    assert nc == len(reps) == n - int(np.sum(mate >= 0)) // 2
    for v in range(n):
        rep = min(v, mate[v]) if mate[v] >= 0 else v
        assert M[v] == reps.index(rep)


def test_path_heavy_edge_then_no_two_hop_partner():
    # 0 -1- 1 -5- 2 -1- 3: 1 and 2 prefer each other; 0 and 3 have only matched
    # neighbours, are leaves of different neighbours and relatives of different
    # matchmakers: they stay single
    g = _g(4, [(0, 1), (1, 2), (2, 3)], w=[1, 5, 1])
    M, nc, mate, st = O.match(g, 100)
    assert list(mate) == [-1, 2, 1, -1]
    assert nc == 3 and list(M) == [0, 1, 1, 2]
    assert list(st[:5]) == [2, 0, 0, 0, 0]


def test_rating_divides_by_vertex_weights():
    # v0 -4- v1 (weight 4), v0 -3- v2 (weight 1): 16/4 < 9/1, so v0 prefers v2
    # although the edge to v1 is heavier; v2's only neighbour is v0
    g = _g(3, [(0, 1), (0, 2)], w=[4, 3], vw=[1, 4, 1])
    M, nc, mate, st = O.match(g, 100)
    assert mate[0] == 2 and mate[2] == 0 and mate[1] == -1


def test_weight_bound_excludes_partners():
    g = _g(2, [(0, 1)], w=[7], vw=[5, 6])
    M, nc, mate, _ = O.match(g, 10)
    assert list(mate) == [-1, -1] and nc == 2
    M, nc, mate, _ = O.match(g, 11)
    assert list(mate) == [1, 0] and nc == 1


def test_star_leaves_pair_in_id_order():
    # centre 0 with leaves 1..7: the heavy-edge rounds match 0 with one leaf,
    # then the remaining six leaves (one group, neighbour 0) pair in id order
    g = _g(8, [(0, i) for i in range(1, 8)])
    M, nc, mate, st = O.match(g, 100)
    partner = mate[0]
    assert 1 <= partner <= 7
    rest = [i for i in range(1, 8) if i != partner]
    for a, b in zip(rest[0::2], rest[1::2]):
        assert mate[a] == b and mate[b] == a
    assert st[0] == 2 and st[1] == 6 and nc == 4


def test_twins_pair_when_heavy_edges_leave_them():
    # K_{6,2}: left 0..5, right 6, 7.  Heavy-edge rounds match two left vertices
    # with 6 and 7 (50% matched); the other four left vertices are twins
    # (neighbour set {6, 7}) and pair by (hash, id): all in one group, so in id order
    g = _g(8, [(a, b) for a in range(6) for b in (6, 7)])
    M, nc, mate, st = O.match(g, 100)
    assert mate[6] in range(6) and mate[7] in range(6)
    left = [a for a in range(6) if a not in (mate[6], mate[7])]
    assert len(left) == 4
    for a, b in zip(left[0::2], left[1::2]):
        assert mate[a] == b
    assert st[0] == 4 and st[2] == 4 and st[1] == 0 and nc == 4


def test_relatives_share_their_matchmaker():
    # on a power-law graph the heavy-edge rounds leave many vertices; every
    # pair that is not adjacent (and not two isolated vertices) has a common
    # neighbour: a leaf pair or twin pair shares one, a relative pair shares
    # its matchmaker
    g = I.rmat(9, 6, 0.57, 0.19, 0.19, 11)
    lmax = O.lmax(int(g.vw.sum()), 16, 0.03)
    M, nc, mate, st = O.match(g, lmax)
    _valid(g, mate, M, nc, lmax)
    assert st[3] > 0  # the stage ran and matched pairs
    deg = np.diff(g.xadj)
    nb = [set(g.adj[g.xadj[v]:g.xadj[v + 1]].tolist()) for v in range(g.n)]
    # pairs that are neither adjacent nor leaves/twins must share a neighbour
    for v in range(g.n):
        u = mate[v]
        if u < 0 or u < v or u in nb[v]:
            continue
        if deg[v] == 0 and deg[u] == 0:
            continue  # isolated pairing
        assert nb[v] & nb[u], (v, u)


def test_isolated_vertices_pair_in_id_order():
    g = _g(7, [], vw=[3, 3, 5, 1, 1, 2, 9])
    M, nc, mate, st = O.match(g, 6)
    # (0,1): 6 <= 6; (2,3): 6; (4,5): 3; 6 alone
    assert list(mate) == [1, 0, 3, 2, 5, 4, -1]
    assert st[4] == 6 and nc == 4


def test_more_than_75_percent_skips_two_hop():
    g = I.grid2d(8, 8)  # a perfect matching of heavy edges exists on a grid
    M, nc, mate, st = O.match(g, 100)
    _valid(g, mate, M, nc, 100)
    if 4 * st[0] > 3 * g.n:
        assert list(st[1:5]) == [0, 0, 0, 0]


@pytest.mark.parametrize("gi", range(4))
def test_matching_valid_and_contraction_preserves_J(gi):
    graphs = [I.rgg2d(2000, I.rgg_radius(2000, 10), 7, wmax=10), I.grid3d(10, 8, 6),
              I.rmat(10, 8, 0.57, 0.19, 0.19, 4), I.erdos_renyi(300, 0.03, 9, wmax=5, vwmax=4)]
    g = graphs[gi]
    hier, dist = (4, 4), (1, 10)
    lmax = O.lmax(int(g.vw.sum()), 16, 0.03)
    M, nc, mate, st = O.match(g, lmax, level=gi)
    _valid(g, mate, M, nc, lmax)
    xc, ac, wc, vc = O.contract(g, M, nc)
    gc = I.Graph(nc, xc, ac, wc, vc)
    assert int(vc.sum()) == int(g.vw.sum())
    pc = I.random_mapping(nc, 16, 5 + gi)
    assert O.objective(gc, hier, dist, pc)[0] == O.objective(g, hier, dist, pc[M])[0]


def test_map_run_with_matching_halves_levels():
    g = I.grid3d(24, 24, 12)
    prm = O.default_params()
    prm.coarsener = 1
    pi, J, st = O.map_run(g, (4, 8), (1, 10), 0.03, prm)
    k = 32
    L = O.lmax(g.n, k, 0.03)
    assert st.levels >= 3
    for i in range(1, st.levels):
        assert st.n[i] >= st.n[i - 1] // 2  # a matching at most halves a level
    Jo, mx, _ = O.objective(g, (4, 8), (1, 10), pi)
    assert Jo == J and mx <= L


def test_gpu_parity_graphs_reach_every_stage():
    """The graphs of the GPU matching parity tests (R-MAT with hubs, a star,
    K_{2,50}) between them match vertices in every stage: heavy edges, leaves,
    twins, relatives and isolated pairs."""
    seen = np.zeros(6, np.int64)
    star = I.csr_from_pairs(300, np.zeros(299, np.int64), np.arange(1, 300))
    k250 = I.csr_from_pairs(52, np.repeat(np.arange(2), 50), np.tile(np.arange(2, 52), 2))
    for g, k in [(I.rmat(13, 8, 0.57, 0.19, 0.19, 9), 32), (star, 4), (k250, 4)]:
        lmax = O.lmax(int(g.vw.sum()), k, 0.03)
        _, _, _, st = O.match(g, lmax, level=0)
        seen += st
    assert (seen[:5] > 0).all(), seen
