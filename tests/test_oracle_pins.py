"""Pins for the CPU oracle: each check ties it to something other than itself.

* the published SplitMix64 reference sequence (tests/golden);
* the hierarchy distance rebuilt from an explicit PE tree (Section 2 wording);
* J recomputed in the dense matrix form of Section 2 (sum_ij C_ij D_P(i)P(j));
* closed forms: D = 1:...:1 gives J = 2 * edge-cut (Section 5.3), l = 1
  gives 2 d_1 * cut; printed L_max examples;
* Eq. 1 through the identity J(P[v->q]) = J(P) - 2 G_q(v), every v, q;
* Alg. 4 selections and afterburner decisions recomputed from objective
  differences on brute-force states;
* invariants of rebalancing (conserved weight, heavy rule, excess removal,
  strong never overloads a destination), of Alg. 6 (best feasible state,
  patience rule) and of contraction (dense S^T C S, J preserved);
* exhaustive enumeration of all mappings on tiny instances;
* breadth-first order of the initial mapping against networkx.
"""
import itertools
import os

import numpy as np
import pytest

import oracle as O
from paper_2510_12196_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")

TOPOS = [((4, 8), (1, 10)), ((4, 8, 6), (1, 10, 100)), ((2, 3), (3, 7)), ((3,), (5,)),
         ((2, 2, 2), (1, 10, 100)), ((1, 4), (2, 9)), ((2, 3, 2), (0, 4, 50))]


# ----------------------------------------------------------------------------
# independent brute-force helpers
# ----------------------------------------------------------------------------

def dmat_from_tree(hier, dist):
    """Distance matrix built from an explicit PE tree: PE p has coordinates
    (pe-in-processor, processor-in-node, node-in-rack, ...), enumerated with
    the first coordinate varying fastest; the cost of two different PEs is
    d_i for the highest coordinate i in which they differ."""
    coords = [tuple(reversed(t)) for t in itertools.product(*[range(a) for a in reversed(hier)])]
    k = len(coords)
    D = np.zeros((k, k), np.int64)
    for p in range(k):
        for q in range(k):
            diff = [i for i in range(len(hier)) if coords[p][i] != coords[q][i]]
            D[p, q] = dist[max(diff)] if diff else 0
    return D


def dense(g):
    C = np.zeros((g.n, g.n), np.int64)
    src = np.repeat(np.arange(g.n), g.degrees())
    C[src, g.adj] = g.adjw
    return C


def J_dense(C, D, pi):
    pi = np.asarray(pi)
    return int((C * D[np.ix_(pi, pi)]).sum())


def edge_cut(g, pi):
    src = np.repeat(np.arange(g.n), g.degrees())
    return int(g.adjw[pi[src] != pi[g.adj]].sum()) // 2


def small_graphs(count=12, nmax=10, seed0=100):
    out = []
    for s in range(count):
        n = 3 + s % (nmax - 2)
        out.append(I.erdos_renyi(n, 0.45, seed0 + s, wmax=5, vwmax=3))
    return out


def rand_pi(n, k, seed):
    return I.random_mapping(n, k, seed)


# ----------------------------------------------------------------------------
# hash, distance, L_max, J
# ----------------------------------------------------------------------------

def test_hash_reference_sequence():
    vals = [int(x) for x in open(os.path.join(GOLD, "splitmix64_seed1234567.txt")) if x.strip() and x[0] != "#"]
    gamma = 0x9E3779B97F4A7C15
    got = [O.hash64((1234567 + n * gamma) % 2**64, 0) for n in range(len(vals))]
    assert got == vals


@pytest.mark.parametrize("hier,dist", TOPOS)
def test_dist_matches_pe_tree(hier, dist):
    D = dmat_from_tree(hier, dist)
    k = O.num_pes(hier)
    assert k == D.shape[0]
    for p in range(k):
        for q in range(k):
            assert O.dist(hier, dist, p, q) == D[p, q]


def test_dist_paper_wording():
    # 4:8 with 1:10: PEs 0..3 share a processor (d_1), 4..7 another one.
    assert O.dist((4, 8), (1, 10), 0, 3) == 1
    assert O.dist((4, 8), (1, 10), 0, 4) == 10
    assert O.dist((4, 8), (1, 10), 5, 5) == 0
    # 4:8:8 with 1:10:100: PEs 0 and 31 share a node, 0 and 32 do not.
    assert O.dist((4, 8, 8), (1, 10, 100), 0, 31) == 10
    assert O.dist((4, 8, 8), (1, 10, 100), 0, 32) == 100


def test_lmax_values():
    # ceil(1.03 * c(V) / k) for the 64x64 grid (k = 32), RGG 2^20 (k = 256)
    # and R-MAT scale 22 (k = 512) with unit vertex weights.
    assert O.lmax(4096, 32, 0.03) == 132
    assert O.lmax(1 << 20, 256, 0.03) == 4219
    assert O.lmax(1 << 22, 512, 0.03) == 8438
    from fractions import Fraction
    rng = np.random.default_rng(5)
    for _ in range(200):
        cv = int(rng.integers(1, 10**9))
        k = int(rng.integers(1, 5000))
        eps_ppm = int(rng.integers(0, 999999))
        exact = Fraction(10**6 + eps_ppm, 10**6) * Fraction(cv, k)
        want = -((-exact.numerator) // exact.denominator)
        assert O.lmax(cv, k, eps_ppm / 1e6) == want


@pytest.mark.parametrize("hier,dist", TOPOS)
def test_objective_dense_form(hier, dist):
    D = dmat_from_tree(hier, dist)
    k = D.shape[0]
    for i, g in enumerate(small_graphs()):
        C = dense(g)
        pi = rand_pi(g.n, k, 7 + i)
        J, mx, W = O.objective(g, hier, dist, pi)
        assert J == J_dense(C, D, pi)
        assert np.array_equal(W, np.bincount(pi, weights=g.vw, minlength=k).astype(np.int64))
        assert mx == W.max()


def test_objective_special_cases():
    for i, g in enumerate(small_graphs(seed0=300)):
        pi = rand_pi(g.n, 8, i)
        cut = edge_cut(g, pi)
        # D = 1:1:1 turns the mapping objective into twice the edge-cut.
        assert O.objective(g, (2, 2, 2), (1, 1, 1), pi)[0] == 2 * cut
        # a one-level hierarchy with distance d_1: J = 2 d_1 cut.
        assert O.objective(g, (8,), (7,), pi)[0] == 14 * cut
    # all vertices on one PE: J = 0
    g = I.grid2d(8, 8)
    assert O.objective(g, (4, 8), (1, 10), np.zeros(g.n, np.int32))[0] == 0


@pytest.mark.parametrize("hier,dist", TOPOS[:5])
def test_gain_identity(hier, dist):
    """Eq. 1 gains match objective differences: J(P[v->q]) - J(P) = -2 G_q(v)."""
    D = dmat_from_tree(hier, dist)
    k = D.shape[0]
    for i, g in enumerate(small_graphs(6, seed0=500)):
        C = dense(g)
        pi = rand_pi(g.n, k, 11 + i)
        J0 = J_dense(C, D, pi)
        for v in range(g.n):
            for q in range(k):
                p2 = pi.copy()
                p2[v] = q
                assert J_dense(C, D, p2) - J0 == -2 * O.gain(g, hier, dist, pi, v, q)


# ----------------------------------------------------------------------------
# Alg. 4
# ----------------------------------------------------------------------------

def _bf_gain(C, D, pi, v, q):
    p2 = pi.copy()
    p2[v] = q
    return (J_dense(C, D, pi) - J_dense(C, D, p2)) // 2


@pytest.mark.parametrize("hier,dist", [((4, 8), (1, 10)), ((2, 2, 2), (1, 10, 100)), ((2, 3), (3, 7))])
def test_lp_step_bruteforce(hier, dist):
    D = dmat_from_tree(hier, dist)
    k = D.shape[0]
    for i, g in enumerate(small_graphs(10, seed0=700)):
        C = dense(g)
        pi = rand_pi(g.n, k, 3 + i)
        lock = (I.splitmix64(i, np.arange(g.n, dtype=np.uint64)) % np.uint64(4) == 0).astype(np.uint8)
        npi, nlock, pp, gn, inx, mv, cnt = O.lp_step(g, hier, dist, pi, lock)
        # step 1: best neighbouring block by objective difference
        for v in range(g.n):
            nb = sorted({int(pi[u]) for u in np.nonzero(C[v])[0]} - {int(pi[v])})
            if lock[v] or not nb:
                assert not inx[v] and pp[v] == pi[v] and gn[v] == 0
                continue
            gains = [(_bf_gain(C, D, pi, v, q), -q) for q in nb]
            bg, bq = max(gains)
            if bg >= 0:
                assert inx[v] and pp[v] == -bq and gn[v] == bg
            else:
                assert not inx[v] and pp[v] == pi[v]
        # step 2: recomputed gain on the state where neighbours earlier in
        # the ord order (higher gain, then lower id) are already moved.
        for v in range(g.n):
            if not inx[v]:
                assert not mv[v]
                continue
            st = pi.copy()
            for u in np.nonzero(C[v])[0]:
                if inx[u] and (gn[u] > gn[v] or (gn[u] == gn[v] and u < v)):
                    st[u] = pp[u]
            assert bool(mv[v]) == (_bf_gain(C, D, st, v, pp[v]) >= 0)
        # step 3
        assert np.array_equal(npi, np.where(mv == 1, pp, pi))
        assert np.array_equal(nlock, mv)
        assert cnt == int(mv.sum())


@pytest.mark.parametrize("relax", [(1, 4), (3, 4), (2, 1)])
def test_lp_step_relaxed_filter_bruteforce(relax):
    """Jet's relaxed filter: v enters X when its best gain G >= 0 or
    -G < floor(c conn(v, P(v))), c = num/den, conn(v, P(v)) read here off the
    dense weight matrix; the afterburner and the apply are unchanged.  Unit
    distances keep gains on the scale of connectivities, so the relaxation
    has something to admit."""
    hier, dist = (4, 8), (1, 1)
    D = dmat_from_tree(hier, dist)
    k = D.shape[0]
    num, den = relax
    neg_in = 0
    for i, g in enumerate(small_graphs(12, seed0=910)):
        C = dense(g)
        # a mapping with locality, so that own-block connectivity is common
        pi = ((np.arange(g.n) * 4) // g.n).astype(np.int32)
        flip = rand_pi(g.n, k, 50 + i)
        pi = np.where(np.arange(g.n) % 3 == 0, flip, pi).astype(np.int32)
        lock = np.zeros(g.n, np.uint8)
        npi, nlock, pp, gn, inx, mv, cnt = O.lp_step(g, hier, dist, pi, lock, relax=relax)
        for v in range(g.n):
            nb = sorted({int(pi[u]) for u in np.nonzero(C[v])[0]} - {int(pi[v])})
            if not nb:
                assert not inx[v]
                continue
            bg, bq = max((_bf_gain(C, D, pi, v, q), -q) for q in nb)
            own = int(sum(C[v, u] for u in range(g.n) if pi[u] == pi[v] and u != v))
            admit = bg >= 0 or -bg < (num * own) // den
            assert bool(inx[v]) == admit
            if admit:
                assert pp[v] == -bq and gn[v] == bg
                neg_in += bg < 0
        for v in range(g.n):
            if not inx[v]:
                assert not mv[v]
                continue
            st = pi.copy()
            for u in np.nonzero(C[v])[0]:
                if inx[u] and (gn[u] > gn[v] or (gn[u] == gn[v] and u < v)):
                    st[u] = pp[u]
            assert bool(mv[v]) == (_bf_gain(C, D, st, v, pp[v]) >= 0)
        assert np.array_equal(npi, np.where(mv == 1, pp, pi))
    if 4 * num >= 3 * den:
        assert neg_in > 0  # the relaxation admitted negative moves somewhere


def test_lp_independent_moves_exact_delta():
    """When the moved vertices are pairwise non-adjacent, J drops by exactly
    twice the sum of their Eq. 1 gains."""
    hits = 0
    for s in range(200):
        g = I.erdos_renyi(10, 0.25, 900 + s, wmax=4)
        pi = rand_pi(g.n, 8, s)
        J0 = O.objective(g, (2, 4), (1, 10), pi)[0]
        npi, _, pp, gn, inx, mv, cnt = O.lp_step(g, (2, 4), (1, 10), pi, np.zeros(g.n, np.uint8))
        movers = np.nonzero(mv)[0]
        C = dense(g)
        if cnt == 0 or C[np.ix_(movers, movers)].any():
            continue
        hits += 1
        assert O.objective(g, (2, 4), (1, 10), npi)[0] == J0 - 2 * int(gn[movers].sum())
    assert hits >= 10


# ----------------------------------------------------------------------------
# rebalancing
# ----------------------------------------------------------------------------

def _conn(C, pi, v, k):
    return np.bincount(pi, weights=C[v], minlength=k).astype(np.int64)


def _check_rebalance(g, hier, dist, pi, strong, seed=1, level=0, t=1, gap=100):
    k = O.num_pes(hier)
    cv = int(g.vw.sum())
    L = O.lmax(cv, k, 0.03)
    C = dense(g)
    W = np.bincount(pi, weights=g.vw, minlength=k).astype(np.int64)
    npi, dest, mv, cnt = O.rebalance(g, hier, dist, L, strong, pi, sigma_gap=gap, seed=seed, level=level, t=t)
    W2 = np.bincount(npi, weights=g.vw, minlength=k).astype(np.int64)
    assert W2.sum() == W.sum() == cv
    assert cnt == int(mv.sum())
    assert np.array_equal(npi != pi, mv.astype(bool))
    sigma = L if strong else max(-(-cv // k), L - gap)
    for v in np.nonzero(mv)[0]:
        A = pi[v]
        assert W[A] > L, "only vertices of overloaded blocks move"
        assert 2 * k * g.vw[v] <= 3 * (k * W[A] - cv), "heavy vertex moved"
        assert npi[v] != A
        if not strong:
            assert W[npi[v]] <= sigma
            conn = _conn(C, pi, v, k)
            cand = [b for b in range(k) if b != A and conn[b] > 0 and W[b] <= sigma]
            if cand:  # edge-cut best destination, lowest id on ties
                best = max(cand, key=lambda b: (conn[b], -b))
                assert npi[v] == best
    if strong:
        for b in range(k):
            if W[b] <= L:
                assert W2[b] <= L, "strong rebalancing overloaded a destination"
    else:
        # every overloaded block sheds at least min(excess, movable weight)
        for A in range(k):
            if W[A] <= L:
                continue
            members = np.nonzero(pi == A)[0]
            light = [v for v in members if 2 * k * g.vw[v] <= 3 * (k * W[A] - cv)]
            movable = sum(int(g.vw[v]) for v in light)
            out = int(g.vw[members][mv[members] == 1].sum())
            if any((W <= sigma)):
                assert out >= min(W[A] - L, movable)
    return npi, W, W2, L


@pytest.mark.parametrize("strong", [False, True])
def test_rebalance_invariants(strong):
    done = 0
    for s in range(40):
        g = I.erdos_renyi(40, 0.12, 1100 + s, wmax=5, vwmax=4)
        k = 8
        # skewed mapping: overload the first blocks
        pi = (I.splitmix64(s, np.arange(g.n, dtype=np.uint64)) % np.uint64(13)).astype(np.int64)
        pi = np.minimum(pi, k - 1).astype(np.int32)
        npi, W, W2, L = _check_rebalance(g, (2, 4), (1, 10), pi, strong, seed=s, gap=2)
        done += int((W > L).any())
    assert done > 20


def test_rebalance_grid_reduces_overload():
    w = I.workload_grid64()
    g, t = w.graph, w.topo
    pi = w.pi0
    for strong in (False, True):
        npi, W, W2, L = _check_rebalance(g, t.hier, t.dist, pi, strong)
        assert (W > L).sum() > 0
        assert np.maximum(W2 - L, 0).sum() < np.maximum(W - L, 0).sum()
    npi, W, W2, L = _check_rebalance(g, t.hier, t.dist, pi, True)
    assert W2.max() <= max(L, W.max())


def _loss_bucket(g):
    if g > 0:
        return 0
    if g == 0:
        return 1
    return 2 + int(np.floor(np.log2(-g)))


def test_rebalance_j_objective_bruteforce():
    """Rebalancing adapted to J (Section 4.2): every eligible vertex of an
    overloaded block gets the neighbouring destination below sigma of largest
    J gain (dense objective difference, lowest id on ties), its bucket is
    taken of that gain (of the drawn block's gain when no neighbour
    qualifies), and each block moves the prefix of its eligible vertices in
    (bucket, id) order that covers its excess."""
    hier, dist = (2, 4), (1, 10)
    D = dmat_from_tree(hier, dist)
    k = D.shape[0]
    checked = 0
    for s in range(30):
        g = I.erdos_renyi(36, 0.13, 1500 + s, wmax=5, vwmax=4)
        C = dense(g)
        pi = (I.splitmix64(70 + s, np.arange(g.n, dtype=np.uint64)) % np.uint64(13)).astype(np.int64)
        pi = np.minimum(pi, k - 1).astype(np.int32)
        cv = int(g.vw.sum())
        L = O.lmax(cv, k, 0.03)
        gap = 2
        W = np.bincount(pi, weights=g.vw, minlength=k).astype(np.int64)
        sigma = max(-(-cv // k), L - gap)
        npi, dest, mv, cnt = O.rebalance(g, hier, dist, L, False, pi, sigma_gap=gap, seed=s, objective=1)
        order = {}
        for v in range(g.n):
            A = int(pi[v])
            if W[A] <= L or 2 * k * int(g.vw[v]) > 3 * (k * int(W[A]) - cv):
                assert not mv[v]
                continue
            cand = sorted({int(pi[u]) for u in np.nonzero(C[v])[0]} - {A})
            cand = [b for b in cand if W[b] <= sigma]
            if cand:
                gb, nb = max((_bf_gain(C, D, pi, v, b), -b) for b in cand)
                b = -nb
            else:
                U = np.nonzero(W <= sigma)[0]
                if len(U) == 0:
                    continue
                # the drawn block: U[h(level 0, t 1, v) mod |U|]
                h = O.hash64(s, (3 << 60) | (1 << 32) | v)
                b = int(U[h % len(U)])
                gb = _bf_gain(C, D, pi, v, b)
            if mv[v]:
                assert dest[v] == b
            order.setdefault(A, []).append((_loss_bucket(gb), v))
        for A, lst in order.items():
            pre = 0
            for _, v in sorted(lst):
                assert bool(mv[v]) == (pre < W[A] - L)
                pre += int(g.vw[v])
            checked += 1
        assert np.array_equal(npi, np.where(mv == 1, dest, pi))
    assert checked > 20


# ----------------------------------------------------------------------------
# Alg. 6
# ----------------------------------------------------------------------------

def _check_trace(g, hier, dist, L, pi0, kinds, Js, Ws, best_J, best_W, it, rounds, patience=12):
    J0, W0, _ = O.objective(g, hier, dist, pi0)
    prev_w = W0
    weak_run = 0
    for t in range(it):
        if prev_w <= L:
            assert kinds[t] == 0
            weak_run = 0
        elif weak_run < 2:
            assert kinds[t] == 1
            weak_run += 1
        else:
            assert kinds[t] == 2
            weak_run = 0
        prev_w = Ws[t]
    # best state: the feasible state of lowest J if any feasible one was seen,
    # else the state of lowest max block weight (earliest on ties)
    states = [(J0, W0)] + list(zip(Js.tolist(), Ws.tolist()))
    feas = [j for j, w in states if w <= L]
    if feas:
        assert best_W <= L and best_J == min(feas)
    else:
        assert best_W == min(w for _, w in states)
    if rounds >= 0:
        assert it == rounds
    else:
        # patience rule: no reset event in the last `patience` iterations
        bj, bw = J0, W0
        i = 0
        for t in range(it):
            j, w = Js[t], Ws[t]
            i += 1
            if w <= L:
                if bw > L:
                    bj, bw, i = j, w, 0
                else:
                    reset = 1000 * j < 999 * bj
                    if j < bj:
                        bj, bw = j, w
                    if reset:
                        i = 0
            elif w < bw:
                bj, bw, i = j, w, 0
            if t < it - 1:
                assert i < patience
        assert i == patience


def test_refine_fixed_rounds_grid64():
    w = I.workload_grid64()
    g, t = w.graph, w.topo
    L = O.lmax(g.n, t.k, t.eps)
    pi, J, mx, it, kinds, Js, Ws = O.refine(g, t.hier, t.dist, L, w.pi0, rounds=10)
    assert it == 10 and len(kinds) == 10
    _check_trace(g, t.hier, t.dist, L, w.pi0, kinds, Js, Ws, J, mx, it, 10)
    assert O.objective(g, t.hier, t.dist, pi)[:2] == (J, mx)


@pytest.mark.parametrize("seed", range(6))
def test_refine_alg6_state_machine(seed):
    g = I.rgg2d(2000, I.rgg_radius(2000, 8), 40 + seed, wmax=10)
    hier, dist = (4, 8), (1, 10)
    k = 32
    L = O.lmax(int(g.vw.sum()), k, 0.03)
    pi0 = rand_pi(g.n, k, seed)
    pi, J, mx, it, kinds, Js, Ws = O.refine(g, hier, dist, L, pi0, rounds=-1)
    _check_trace(g, hier, dist, L, pi0, kinds, Js, Ws, J, mx, it, -1)
    assert O.objective(g, hier, dist, pi)[:2] == (J, mx)


def _all_mappings(n, k):
    return np.array(list(itertools.product(range(k), repeat=n)), dtype=np.int64)


@pytest.mark.parametrize("hier,dist", [((2, 2), (1, 10)), ((4,), (3,)), ((2, 2), (2, 5))])
def test_refine_not_better_than_exhaustive_optimum(hier, dist):
    D = dmat_from_tree(hier, dist)
    k = D.shape[0]
    checked = 0
    for s in range(10):
        g = I.erdos_renyi(8, 0.5, 1300 + s, wmax=6)
        L = O.lmax(int(g.vw.sum()), k, 0.03)
        maps = _all_mappings(g.n, k)
        src = np.repeat(np.arange(g.n), g.degrees())
        Jall = (D[maps[:, src], maps[:, g.adj]] * g.adjw).sum(axis=1)
        Wall = np.stack([(g.vw * (maps == b)).sum(axis=1) for b in range(k)], axis=1)
        feas = Wall.max(axis=1) <= L
        opt = Jall[feas].min()
        pi0 = np.arange(g.n, dtype=np.int32) % k  # balanced start
        assert (np.bincount(pi0, weights=g.vw, minlength=k) <= L).all()
        pi, J, mx, it, *_ = O.refine(g, hier, dist, L, pi0, rounds=-1)
        assert mx <= L and J >= opt
        assert J <= O.objective(g, hier, dist, pi0)[0]
        checked += 1
    assert checked == 10


# ----------------------------------------------------------------------------
# coarsening: clustering, contraction, projection, initial mapping
# ----------------------------------------------------------------------------

def _check_contraction(g, M, nc):
    xc, ac, wc, vc = O.contract(g, M, nc)
    gc = I.Graph(nc, xc, ac, wc, vc)
    I.check_graph(gc)  # symmetric, sorted, no self-loops, no duplicates
    # dense S^T C S with the diagonal removed
    C = dense(g)
    S = np.zeros((g.n, nc), np.int64)
    S[np.arange(g.n), M] = 1
    Cc = S.T @ C @ S
    np.fill_diagonal(Cc, 0)
    assert np.array_equal(dense(gc), Cc)
    assert np.array_equal(vc, S.T @ g.vw)
    intra = int(C[M[:, None] == M[None, :]].sum())
    assert int(wc.sum()) == int(g.adjw.sum()) - intra
    return gc


def test_contraction_dense_and_objective():
    for s in range(10):
        g = I.erdos_renyi(30, 0.2, 1500 + s, wmax=7, vwmax=3)
        nc = 5 + s % 7
        M = (I.splitmix64(s, np.arange(g.n, dtype=np.uint64)) % np.uint64(nc)).astype(np.int32)
        M[:nc] = np.arange(nc)  # surjective
        gc = _check_contraction(g, M, nc)
        for hier, dist in TOPOS[:3]:
            k = O.num_pes(hier)
            pc = rand_pi(nc, k, s)
            # J(G_c, P) = J(G, P o M): self-loops carry distance 0
            assert O.objective(gc, hier, dist, pc)[0] == O.objective(g, hier, dist, pc[M])[0]
            assert np.array_equal(O.project(M, pc), pc[M])


@pytest.mark.parametrize("wcap", [3, 10, 50])
def test_cluster_invariants(wcap):
    for s in range(6):
        g = I.erdos_renyi(60, 0.06, 1700 + s, wmax=5, vwmax=2)
        M, nc = O.cluster(g, wcap, O.default_params(seed=s))
        assert M.min() == 0 and M.max() == nc - 1 and len(np.unique(M)) == nc
        Wc = np.bincount(M, weights=g.vw, minlength=nc)
        assert Wc.max() <= max(wcap, g.vw.max())
        # isolated vertices: chunks of id-consecutive isolated vertices
        iso = np.nonzero(g.degrees() == 0)[0]
        s_pre = np.concatenate([[0], np.cumsum(g.vw[iso])[:-1]])
        first, last = s_pre // wcap, (s_pre + g.vw[iso] - 1) // wcap
        for a in range(len(iso)):
            for b in range(a + 1, len(iso)):
                same_chunk = first[a] == last[a] and first[b] == last[b] and first[a] == first[b]
                assert (M[iso[a]] == M[iso[b]]) == bool(same_chunk)
            # isolated vertices never share a cluster with connected ones
            assert not np.any(M[g.degrees() > 0] == M[iso[a]])
        _check_contraction(g, M, nc)
        M2, nc2 = O.cluster(g, wcap, O.default_params(seed=s))
        assert nc2 == nc and np.array_equal(M, M2)


def test_cluster_merges_on_rgg():
    g = I.rgg2d(4096, I.rgg_radius(4096, 12), 3, wmax=10)
    M, nc = O.cluster(g, 64)
    assert nc < g.n // 4
    assert np.bincount(M, weights=g.vw).max() <= 64


def test_initial_mapping_bfs():
    nx = pytest.importorskip("networkx")
    for s in range(4):
        g = I.erdos_renyi(50, 0.04, 1900 + s, vwmax=3)
        k = 6
        pi = O.initial(g, k)
        G = nx.Graph()
        G.add_nodes_from(range(g.n))
        for v in range(g.n):
            for u in g.adj[g.xadj[v]:g.xadj[v + 1]]:
                G.add_edge(v, int(u))
        order, seen = [], set()
        for s0 in range(g.n):
            if s0 in seen:
                continue
            comp = [s0] + [b for _, b in nx.bfs_edges(G, s0, sort_neighbors=sorted)]
            order += comp
            seen.update(comp)
        cv = int(g.vw.sum())
        pre = np.concatenate([[0], np.cumsum(g.vw[order])[:-1]])
        assert np.array_equal(pi[order], (pre * k) // cv)
        assert pi.min() >= 0 and pi.max() < k


# ----------------------------------------------------------------------------
# whole pipeline
# ----------------------------------------------------------------------------

def test_map_run_small_rgg_invariants():
    w = I.workload_rgg(14)
    g, t = w.graph, w.topo
    pi, J, st = O.map_run(g, t.hier, t.dist, t.eps)
    J2, mx, _ = O.objective(g, t.hier, t.dist, pi)
    L = O.lmax(g.n, t.k, t.eps)
    assert J == J2 and mx <= L
    ns = [st.n[i] for i in range(st.levels)]
    assert ns[0] == g.n and all(10 * b <= 9 * a for a, b in zip(ns, ns[1:]))
    assert all(a >= 8 * t.k for a in ns[:-1])
    # refinement never loses to the projected initial mapping of the same run
    assert st.J[0] <= st.J[1] * 10


def test_map_run_grid_and_unit_distances():
    g = I.grid2d(96, 96)
    pi, J, st = O.map_run(g, (4, 8), (1, 1), 0.03)
    cut = edge_cut(g, pi)
    assert J == 2 * cut  # D = 1:1 is graph partitioning
    assert O.objective(g, (4, 8), (1, 1), pi)[1] <= O.lmax(g.n, 32, 0.03)
