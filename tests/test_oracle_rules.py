"""Pins of the oracle's decision rules for clustering and rebalancing.

Each rule is restated here from its written reading, in a different form
from the oracle (dense connectivity matrices R = C @ onehot(labels), whole
candidate sets ranked by Python tuples, interval lookups by searchsorted),
and the oracle's complete output is compared with it element by element on
many small seeded graphs with ties and contention:

* label-propagation clustering (the task's coarsening alternative to the
  paper's matching, Section 4.2): per sub-round, the target of every active
  vertex is the argmax over its own and its neighbouring clusters of the
  edge weight into them, ties to the smaller tie-hash, then the smaller
  label; a request exists iff the target is another cluster that fits the
  cap at the sub-round's start; the admitted requests of a target are the
  longest prefix in (hash >> 32, id) order whose weight fits; isolated
  vertices are chunked in id order; clusters are numbered by ascending label.
* weak and strong rebalancing (Alg. 5 and the strong variant of Section 4.2
  "Rebalancing"): eligibility, destinations (edge-cut gain or Eq. 1 gain,
  lowest id on ties, the drawn fallback block), log2 loss buckets, the
  per-source prefix selection in (bucket, id) order, and for the strong
  variant the per-destination acceptance in (bucket, id) order under L_max
  and the water-filling of the rejected movers over the residual room of
  the non-overloaded blocks.

Coverage counters assert that the seeded cases really exercise ties,
contested admission, rejected strong movers that are re-placed, and cases
where id order and (bucket, id) order would accept different movers.
"""
import numpy as np
import pytest

import oracle as O
from paper_2510_12196_gb300 import inputs as I

MASK64 = (1 << 64) - 1


def _h(seed, x):
    return int(I.splitmix64(seed, np.uint64(x & MASK64)))


def h_active(seed, level, v):
    return _h(seed, (1 << 60) | (level << 32) | v)


def h_tie(seed, level, t):
    return _h(seed, (2 << 60) | (level << 32) | t)


def h_rebalance(seed, level, t, v):
    return _h(seed, (3 << 60) | (level << 52) | ((t & 0xFFFFF) << 32) | v)


def dense(g):
    A = np.zeros((g.n, g.n), np.int64)
    src = np.repeat(np.arange(g.n), g.degrees())
    A[src, g.adj] = g.adjw
    return A


def onehot(labels, width):
    X = np.zeros((labels.size, width), np.int64)
    X[np.arange(labels.size), labels] = 1
    return X


# ----------------------------------------------------------------------------
# clustering, restated
# ----------------------------------------------------------------------------

def cluster_restated(g, wcap, seed, level, iters, stats=None):
    n = g.n
    A = dense(g)
    deg = g.degrees()
    vw = g.vw.astype(np.int64)
    label = np.arange(n, dtype=np.int64)
    for it in range(iters):
        moved = 0
        for r in (0, 1):
            start = label.copy()
            Wstart = np.bincount(start, weights=vw, minlength=n).astype(np.int64)
            R = A @ onehot(start, n)  # R[v, t]: edge weight from v into cluster t
            requests = {}
            for v in range(n):
                if deg[v] == 0 or ((h_active(seed, level, v) >> it) & 1) != r:
                    continue
                cands = set(np.nonzero(R[v])[0].tolist()) | {int(start[v])}
                ranked = sorted(cands, key=lambda t: (-int(R[v, t]), h_tie(seed, level, t), t))
                if stats is not None and len(ranked) > 1 and R[v, ranked[0]] == R[v, ranked[1]]:
                    stats["ties"] += 1
                t = ranked[0]
                if t != start[v] and Wstart[t] + vw[v] <= wcap:
                    requests.setdefault(t, []).append((h_active(seed, level, v) >> 32, v))
            for t, lst in requests.items():
                lst.sort()
                room = wcap - Wstart[t]
                ws = np.array([vw[v] for _, v in lst])
                fits = np.cumsum(ws) <= room
                # the admitted set is a prefix of the ordered requests
                assert np.all(fits[:int(fits.sum())])
                if stats is not None and not fits.all():
                    stats["contested"] += 1
                    if sorted(v for _, v in lst) != [v for _, v in lst]:
                        stats["hash_order_differs"] += 1
                for (hv, v), ok in zip(lst, fits):
                    if ok:
                        label[v] = t
                        moved += 1
        if moved * 100 < n:
            break
    # isolated vertices: id-order chunks of weight <= wcap, labelled n + chunk
    s = 0
    for v in range(n):
        if deg[v] != 0:
            continue
        first, last = s // wcap, (s + vw[v] - 1) // wcap
        if first == last:
            label[v] = n + first
        s += int(vw[v])
    uniq = np.unique(label)
    return np.searchsorted(uniq, label).astype(np.int32), int(uniq.size)


def _cluster_cases():
    cases = []
    for s in range(14):
        # unit weights: many equal ratings, so the tie-hash decides
        cases.append((I.erdos_renyi(24 + s, 0.15, 4100 + s, wmax=1, vwmax=1), 3 + s % 4))
    for s in range(10):
        cases.append((I.erdos_renyi(30, 0.12, 4200 + s, wmax=4, vwmax=3), 5 + 2 * (s % 3)))
    for s in range(4):
        cases.append((I.grid2d(6 + s, 5), 4 + s))
    cases.append((I.erdos_renyi(40, 0.05, 4300, wmax=2, vwmax=2), 6))
    return cases


@pytest.mark.parametrize("iters", [1, 2, 5])
def test_cluster_rule_restated(iters):
    stats = {"ties": 0, "contested": 0, "hash_order_differs": 0}
    for i, (g, wcap) in enumerate(_cluster_cases()):
        seed, level = 0x5EED0000 + i, i % 3
        prm = O.default_params(seed)
        prm.cluster_iters = iters
        M, nc = O.cluster(g, wcap, prm, level=level)
        M2, nc2 = cluster_restated(g, wcap, seed, level, iters, stats)
        assert nc == nc2, f"case {i}: {nc} clusters vs restated {nc2}"
        assert np.array_equal(M, M2), f"case {i}: cluster labels differ"
    # the cases exercise the tie-hash and the hashed admission order
    assert stats["ties"] > 50
    assert stats["contested"] > 10
    assert stats["hash_order_differs"] > 5


def test_cluster_rule_isolated_and_heavy():
    """Isolated vertices chunked by weight (a straddling vertex stays alone)
    next to connected vertices heavier than the cap, which never request."""
    n = 18
    u = np.array([0, 1, 2, 3, 4, 5, 6, 10], np.int64)
    v = np.array([1, 2, 3, 4, 5, 6, 10, 11], np.int64)
    vw = np.array([1, 2, 9, 1, 1, 3, 2, 1, 4, 3, 1, 2, 5, 5, 1, 2, 6, 1], np.int32)
    g = I.csr_from_pairs(n, u, v, np.ones(u.size, np.int32), vw=vw)
    for wcap in (4, 6, 9):
        M, nc = O.cluster(g, wcap, O.default_params(7))
        M2, nc2 = cluster_restated(g, wcap, 7, 0, 5)
        assert nc == nc2 and np.array_equal(M, M2)


# ----------------------------------------------------------------------------
# rebalancing, restated
# ----------------------------------------------------------------------------

def _loss_bucket(x):
    if x > 0:
        return 0
    if x == 0:
        return 1
    return 2 + (int(-x).bit_length() - 1)


def rebalance_restated(g, hier, dist, L, strong, pi, gap, seed, level, t, objective=0, stats=None):
    """One weak / strong step.  Returns (new pi, moved flags)."""
    n = g.n
    k = int(np.prod(hier))
    Dm = _dmat(hier, dist)
    vw = g.vw.astype(np.int64)
    A = dense(g)
    W = np.bincount(pi, weights=vw, minlength=k).astype(np.int64)
    cV = int(vw.sum())
    if strong:
        sigma = L
    else:
        sigma = max(-(-cV // k), L - gap)
    U = np.nonzero(W <= sigma)[0]
    conn = A @ onehot(pi, k)  # conn[v, b]
    # Eq. 1 gain of every (v, q): sum_b conn(v, b) (D(P(v), b) - D(q, b))
    G = (conn * Dm[pi]).sum(1)[:, None] - conn @ Dm.T
    dest = pi.copy()
    bucket = {}
    for v in range(n):
        a = int(pi[v])
        if W[a] <= L or 2 * k * vw[v] > 3 * (k * W[a] - cV):
            continue
        nb = [b for b in np.nonzero(conn[v])[0].tolist() if b != a and W[b] <= sigma]
        if nb:
            score = (lambda b: G[v, b]) if objective == 1 else (lambda b: conn[v, b] - conn[v, a])
            b = min(nb, key=lambda x: (-int(score(x)), x))
            gain = int(score(b))
        elif U.size:
            b = int(U[h_rebalance(seed, level, t, v) % U.size])
            gain = int(G[v, b]) if objective == 1 else -int(conn[v, a])
        else:
            continue
        dest[v] = b
        bucket[v] = _loss_bucket(gain)
    sel = np.zeros(n, bool)
    for a in range(k):
        members = sorted((bucket[v], v) for v in bucket if pi[v] == a)
        before = 0
        for _, v in members:
            sel[v] = before < W[a] - L
            before += int(vw[v])
    moved = np.zeros(n, bool)
    if not strong:
        moved = sel.copy()
    else:
        acc = np.zeros(n, bool)
        accepted = np.zeros(k, np.int64)
        for b in range(k):
            group = sorted((bucket[v], v) for v in np.nonzero(sel)[0] if dest[v] == b)
            incl = np.cumsum([vw[v] for _, v in group]) if group else np.zeros(0)
            for (_, v), x in zip(group, incl):
                if W[b] + x <= L:
                    acc[v] = True
                    accepted[b] += vw[v]
            if stats is not None and group:
                by_id = sorted(v for _, v in group)
                inc_id = np.cumsum([vw[v] for v in by_id])
                if {v for v, x in zip(by_id, inc_id) if W[b] + x <= L} != {v for (_, v) in group if acc[v]}:
                    stats["order_matters"] += 1
        room = np.where(W <= L, np.maximum(0, L - W - accepted), 0)
        ends = np.cumsum(room)
        starts = ends - room
        s = 0
        for v in np.nonzero(sel & ~acc)[0]:
            if stats is not None:
                stats["rejected"] += 1
            # the block whose room interval contains s (empty rooms skipped)
            b = int(np.searchsorted(ends, s, side="right"))
            if b < k and room[b] > 0 and starts[b] <= s and s + vw[v] <= ends[b]:
                dest[v] = b
                acc[v] = True
                if stats is not None:
                    stats["replaced"] += 1
            s += int(vw[v])
        moved = sel & acc
    out = pi.copy()
    out[moved] = dest[moved]
    return out, moved


def _dmat(hier, dist):
    k = int(np.prod(hier))
    P = np.cumprod([1] + list(hier))
    p = np.arange(k)
    D = np.zeros((k, k), np.int64)
    for i in range(len(hier)):
        # p and q differ at level i or above iff floor(p / P_i) != floor(q / P_i)
        differ = (p[:, None] // P[i]) != (p[None, :] // P[i])
        D[differ] = dist[i]
    return D


def _skewed_mapping(n, k, s, spread):
    pi = (I.splitmix64(s, np.arange(n, dtype=np.uint64)) % np.uint64(spread)).astype(np.int64)
    return np.minimum(pi, k - 1).astype(np.int32)


@pytest.mark.parametrize("objective", [0, 1])
@pytest.mark.parametrize("strong", [False, True])
def test_rebalance_rule_restated(strong, objective):
    stats = {"order_matters": 0, "rejected": 0, "replaced": 0}
    hiers = [((2, 4), (1, 10)), ((4, 2), (1, 5)), ((2, 2, 2), (1, 10, 100))]
    cases = 0
    for s in range(60):
        hier, dist = hiers[s % len(hiers)]
        k = int(np.prod(hier))
        g = I.erdos_renyi(30 + s % 17, 0.1 + 0.05 * (s % 3), 5100 + s, wmax=1 + s % 4, vwmax=1 + s % 5)
        pi = _skewed_mapping(g.n, k, 900 + s, k + 2 + s % 7)
        cV = int(g.vw.sum())
        L = O.lmax(cV, k, 0.03)
        gap = s % 4
        level, t = s % 3, 1 + s % 5
        npi, dest, mv, cnt = O.rebalance(g, hier, dist, L, strong, pi, sigma_gap=gap, seed=s, level=level, t=t,
                                         objective=objective)
        rpi, rmv = rebalance_restated(g, hier, dist, L, strong, pi, gap, s, level, t, objective, stats)
        assert np.array_equal(mv.astype(bool), rmv), f"case {s}: moved sets differ"
        assert np.array_equal(npi, rpi), f"case {s}: destinations differ"
        assert cnt == int(rmv.sum())
        cases += int(rmv.any())
    assert cases > 30
    if strong:
        assert stats["rejected"] > 20
        assert stats["replaced"] > 10
        assert stats["order_matters"] > 3


def test_rebalance_strong_hand_case():
    """Hand-built strong step: block 0 holds 8 unit vertices with L_max = 3,
    so it must shed 5; blocks 1..3 are empty.  Vertices 0..3 are tied to
    block 1 (their best destination), 4..7 have no neighbour outside block 0
    except vertex 7, which is tied to block 2.  Acceptance into block 1 is
    the (bucket, id) prefix under L_max, the rejected movers are water-filled
    over the residual rooms of blocks 1, 2, 3 in id order."""
    n = 12
    # vertices 8..11 sit in blocks 1, 1, 2, 3 and anchor the destinations
    u = np.array([0, 1, 2, 3, 3, 7, 0, 1, 2, 4], np.int64)
    v = np.array([8, 8, 9, 9, 8, 10, 1, 2, 3, 5], np.int64)
    w = np.array([1, 2, 3, 1, 4, 2, 1, 1, 1, 1], np.int32)
    g = I.csr_from_pairs(n, u, v, w)
    pi = np.array([0] * 8 + [1, 1, 2, 3], np.int32)
    hier, dist = (2, 2), (1, 10)
    k = 4
    L = 3
    npi, dest, mv, cnt = O.rebalance(g, hier, dist, L, True, pi, sigma_gap=0, seed=3)
    rpi, rmv = rebalance_restated(g, hier, dist, L, True, pi, 0, 3, 0, 1)
    assert np.array_equal(npi, rpi) and np.array_equal(mv.astype(bool), rmv)
    W2 = np.bincount(npi, minlength=k)
    assert W2[1:].max() <= L
    assert W2[0] < 8
