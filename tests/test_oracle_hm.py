"""Pins of the oracle's hierarchical multisection (GPU-HM: Eq. 2, Alg. 2,
Alg. 3): the adaptive imbalance against the balance guarantee it is built
for, the subgraph build against an independent induced-subgraph
construction, and the recursion (PE digits, per-block subproblems) against
the already pinned multilevel pipeline on independently built subgraphs."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2510_12196_gb300 import inputs as I


def _induced(g, part, b):
    """Induced subgraph of block b built from an edge list (not Alg. 2):
    members renumbered in ascending id, each row sorted."""
    members = np.flatnonzero(part == b)
    new = -np.ones(g.n, np.int64)
    new[members] = np.arange(len(members))
    src = np.repeat(np.arange(g.n), np.diff(g.xadj))
    keep = (part[src] == b) & (part[g.adj] == b)
    u, v, w = new[src[keep]], new[g.adj[keep]], g.adjw[keep]
    order = np.lexsort((v, u))
    u, v, w = u[order], v[order], w[order]
    xadj = np.zeros(len(members) + 1, np.int64)
    np.add.at(xadj, u + 1, 1)
    xadj = np.cumsum(xadj)
    return I.Graph(len(members), xadj, v.astype(np.int32), w.astype(np.int32),
                   g.vw[members].astype(np.int32)), members


# --- Eq. 2 ------------------------------------------------------------------

@pytest.mark.parametrize("hier", [(4, 8, 8), (2, 3), (4, 16, 8), (2, 4, 16, 8), (5,)])
@pytest.mark.parametrize("eps", [0.0, 0.03, 0.1])
@pytest.mark.parametrize("skew", [1.0, 0.9, 1.07])
def test_adaptive_eps_composes_to_eps(hier, eps, skew):
    """If every partition hands a block (1+eps') c(V')/a_i, the blocks at the
    bottom weigh exactly (1+eps) c(V)/k: the guarantee Eq. 2 is built for.
    When an upper level misses its target by `skew`, the levels below absorb
    it and the bottom still lands on (1+eps) c(V)/k."""
    k = math.prod(hier)
    cV = 10 ** 12
    w, kp = float(cV), k
    for d in range(len(hier), 0, -1):
        e = O.adaptive_eps(eps, cV, int(round(w)), k, kp, d)
        w = (1 + e) * w / hier[d - 1]
        kp //= hier[d - 1]
        if d == len(hier) and d > 1:
            w *= skew
    assert w == pytest.approx((1 + eps) * cV / k, rel=1e-8)


def test_adaptive_eps_special_cases():
    # top level: c(V') = c(V), k' = k
    for l in (1, 2, 3, 4):
        assert O.adaptive_eps(0.03, 5000, 5000, 256, 256, l) == pytest.approx(1.03 ** (1 / l) - 1, rel=1e-12)
    # a block at exactly its share, one level left: eps' = eps
    assert O.adaptive_eps(0.05, 1024, 32, 256, 8, 1) == pytest.approx(0.05, rel=1e-12)
    # a heavier-than-share block gets less room, a lighter one more
    assert O.adaptive_eps(0.03, 1000, 300, 16, 4, 2) < O.adaptive_eps(0.03, 1000, 250, 16, 4, 2) \
        < O.adaptive_eps(0.03, 1000, 200, 16, 4, 2)


# --- Alg. 2 -----------------------------------------------------------------

def _zoo():
    return [I.grid2d(12, 9), I.rgg2d(800, I.rgg_radius(800, 10), 5, wmax=10),
            I.erdos_renyi(120, 0.08, 3, wmax=5, vwmax=4), I.rmat(9, 8, 0.57, 0.19, 0.19, 2)]


@pytest.mark.parametrize("gi", range(4))
def test_build_subgraph_is_the_induced_subgraph(gi):
    g = _zoo()[gi]
    for a in (1, 3, 7):
        part = (I.splitmix64(40 + gi, np.arange(g.n, dtype=np.uint64)) % np.uint64(a)).astype(np.int32)
        tot_m = 0
        for b in range(a):
            (ns, xs, as_, ws, vs), M, m_, w_ = O.build_subgraph(g, part, b)
            ref, members = _induced(g, part, b)
            assert ns == ref.n
            assert np.array_equal(xs, ref.xadj) and np.array_equal(as_, ref.adj) and np.array_equal(ws, ref.adjw)
            assert np.array_equal(vs, ref.vw)
            assert m_ == len(as_) and w_ == int(g.vw[members].sum())
            assert np.array_equal(M[members], np.arange(ns)) and (M[part != b] == -1).all()
            tot_m += m_
        # every CSR entry is either inside one block or cut
        src = np.repeat(np.arange(g.n), np.diff(g.xadj))
        assert tot_m + int(np.sum(part[src] != part[g.adj])) == g.m_dir


# --- Alg. 3 -----------------------------------------------------------------

def _clamp(e):
    return min(max(e, 0.0), 0.999999)


def test_single_level_is_one_partition():
    g = I.rgg2d(3000, I.rgg_radius(3000, 12), 8, wmax=10)
    pi, J, st = O.hm_run(g, (16,), (7,), 0.03)
    e = _clamp(O.adaptive_eps(0.03, int(g.vw.sum()), int(g.vw.sum()), 16, 16, 1))
    ref, Jc, _ = O.map_run(g, (16,), (1,), e)
    assert np.array_equal(pi, ref)
    assert J == 7 * Jc
    assert list(st.calls[:1]) == [1]


@pytest.mark.parametrize("hier", [(4, 3), (2, 2, 4)])
def test_recursion_against_independent_subgraphs(hier):
    """Digit i of every PE id is the partition of that vertex's level-i
    subgraph, built here from an edge list and partitioned by the pinned
    pipeline on the one-level hierarchy a_i with distance 1 and Eq. 2's eps'."""
    g = I.rgg2d(2500, I.rgg_radius(2500, 12), 13, wmax=10)
    l = len(hier)
    k = math.prod(hier)
    cV = int(g.vw.sum())
    pi, J, st = O.hm_run(g, hier, (1, 10, 100)[:l], 0.03)
    # walk the recursion: (graph, original ids, level i, PE base)
    expect = -np.ones(g.n, np.int64)
    stack = [(g, np.arange(g.n), l, 0)]
    calls = [0] * l
    while stack:
        sg, orig, i, base = stack.pop()
        if sg.n == 0:
            continue
        a = hier[i - 1]
        kp = math.prod(hier[:i])
        e = _clamp(O.adaptive_eps(0.03, cV, int(sg.vw.sum()), k, kp, i))
        part, _, _ = O.map_run(sg, (a,), (1,), e)
        calls[i - 1] += 1
        if i == 1:
            expect[orig] = base + part
            continue
        for b in range(a):
            sub, members = _induced(sg, part, b)
            stack.append((sub, orig[members], i - 1, base + b * (kp // a)))
    assert np.array_equal(pi, expect)
    assert list(st.calls[:l]) == calls
    Jo, _, _ = O.objective(g, hier, (1, 10, 100)[:l], pi)
    assert J == Jo


def test_balanced_and_every_pe_used():
    g = I.rgg2d(1 << 12, I.rgg_radius(1 << 12, 12), 21, wmax=10)
    hier = (4, 8, 4)
    pi, J, _ = O.hm_run(g, hier, (1, 10, 100), 0.03)
    k = math.prod(hier)
    W = np.bincount(pi, weights=g.vw, minlength=k)
    assert W.max() <= O.lmax(int(g.vw.sum()), k, 0.03)
    assert (W > 0).all()


def test_map_run_hm_initial_composes():
    """With the hierarchical-multisection initial mapping, the pipeline is the
    clustering chain, hm_run on the coarsest graph, then Alg. 6 on every level
    after projection: recomposed here from the separately pinned pieces."""
    g = I.rgg2d(1 << 13, I.rgg_radius(1 << 13, 12), 17, wmax=10)
    hier, dist = (4, 8), (1, 10)
    k = math.prod(hier)
    prm = O.default_params()
    prm.initial = 1
    pi, J, st = O.map_run(g, hier, dist, 0.03, prm)
    L = O.lmax(int(g.vw.sum()), k, 0.03)
    chain, cur = [], g
    while len(chain) + 1 < prm.max_levels and cur.n >= prm.coarsest_factor * k:
        wcap = max(L // prm.cluster_cap_div, int(cur.vw.max()))
        M, nc = O.cluster(cur, wcap, prm, level=len(chain))
        if nc * prm.stall_den > prm.stall_num * cur.n:
            break
        chain.append((cur, M))
        xc, ac, wc, vc = O.contract(cur, M, nc)
        cur = I.Graph(nc, xc, ac, wc, vc)
    assert len(chain) + 1 == st.levels >= 2
    p0 = O.default_params()
    p, _, _ = O.hm_run(cur, hier, dist, 0.03, p0)
    p, Jl, _, _, _, _, _ = O.refine(cur, hier, dist, L, p, params=prm, level=len(chain))
    for lvl in range(len(chain) - 1, -1, -1):
        fg, M = chain[lvl]
        p = O.project(M, p)
        p, Jl, _, _, _, _, _ = O.refine(fg, hier, dist, L, p, params=prm, level=lvl)
    assert np.array_equal(p, pi) and Jl == J
    # and it differs from the breadth-first start
    assert not np.array_equal(O.map_run(g, hier, dist, 0.03)[0], pi)
