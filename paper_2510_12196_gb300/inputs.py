"""Seeded synthetic inputs: task graphs (CSR), hierarchies and initial mappings.

This module only *builds inputs*. It holds none of the mapping method's
arithmetic (no distance, objective, gain, clustering or balance rule), so that
both the CPU oracle tests and the CUDA path can be fed from it without sharing
any code of the method itself.

Randomness is counter-based: every draw is SplitMix64 (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014) applied to
``seed XOR counter``, so a value depends only on (seed, counter) and not on the
order in which values are drawn.

Graph shapes follow the paper's workload families (Table 1 and the instance
description of Section 5): mesh-like task graphs (2D / 3D grids), random
geometric graphs in the unit square, and a power-law (R-MAT) stand-in for the
irregular instances.  The paper's public suites are not available, so these
seeded graphs stand in for them.

CSR convention used everywhere: ``xadj`` int64[n+1], ``adj`` int32[m_dir],
``adjw`` int32[m_dir], ``vw`` int32[n]; every undirected edge is stored in
both rows with the same weight; each row is sorted strictly ascending; no
self-loops.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import os

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_U64 = np.uint64


def splitmix64(seed: int, counter) -> np.ndarray:
    """SplitMix64 output for state ``seed ^ counter`` (vectorised, uint64)."""
    with np.errstate(over="ignore"):
        z = np.asarray(counter, dtype=np.uint64) ^ _U64(seed & 0xFFFFFFFFFFFFFFFF)
        z = z + _GAMMA
        z = (z ^ (z >> _U64(30))) * _M1
        z = (z ^ (z >> _U64(27))) * _M2
        return z ^ (z >> _U64(31))


def uniform01(seed: int, counter) -> np.ndarray:
    """Doubles uniform in [0, 1) with 53 random bits."""
    return (splitmix64(seed, counter) >> _U64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclasses.dataclass
class Graph:
    n: int
    xadj: np.ndarray  # int64 [n+1]
    adj: np.ndarray   # int32 [m_dir]
    adjw: np.ndarray  # int32 [m_dir]
    vw: np.ndarray    # int32 [n]
    name: str = ""

    @property
    def m_dir(self) -> int:
        return int(self.xadj[-1])

    @property
    def m(self) -> int:
        return self.m_dir // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.xadj)


@dataclasses.dataclass
class Topology:
    hier: Tuple[int, ...]   # a_1 : ... : a_l (a_1 = PEs per processor)
    dist: Tuple[int, ...]   # d_1 : ... : d_l
    eps: float = 0.03

    @property
    def k(self) -> int:
        return int(np.prod(self.hier))

    @property
    def levels(self) -> int:
        return len(self.hier)


@dataclasses.dataclass
class Workload:
    graph: Graph
    topo: Topology
    seed: int
    pi0: Optional[np.ndarray] = None   # initial mapping (fixed-round configs only)
    rounds: int = -1                   # -1: full multilevel run with the Alg. 6 stopping rule
    multilevel: bool = True
    name: str = ""


# ----------------------------------------------------------------------------
# CSR assembly
# ----------------------------------------------------------------------------

def csr_from_pairs(n: int, u: np.ndarray, v: np.ndarray, w: Optional[np.ndarray] = None,
                   vw: Optional[np.ndarray] = None, name: str = "") -> Graph:
    """Symmetric CSR from unique undirected pairs ``u < v`` (weights per pair)."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    assert u.shape == v.shape
    if u.size:
        assert np.all(u < v), "pairs must satisfy u < v"
    src = np.concatenate([u, v])
    dst = np.concatenate([v, u])
    if w is None:
        key = np.sort(src * n + dst)
        src = key // n
        dst = key - src * n
        ww = np.ones(key.size, dtype=np.int32)
    else:
        w = np.asarray(w, dtype=np.int64)
        ww2 = np.concatenate([w, w])
        order = np.argsort(src * n + dst, kind="stable")
        src = src[order]
        dst = dst[order]
        ww = ww2[order].astype(np.int32)
    counts = np.bincount(src, minlength=n) if n else np.zeros(0, np.int64)
    xadj = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=xadj[1:])
    if vw is None:
        vw = np.ones(n, dtype=np.int32)
    return Graph(n=n, xadj=xadj, adj=dst.astype(np.int32), adjw=ww, vw=np.asarray(vw, dtype=np.int32), name=name)


def relabel(g: Graph, perm: np.ndarray, name: str = "") -> Graph:
    """Graph with vertex ``v`` renamed ``perm[v]`` (rows re-sorted)."""
    perm = np.asarray(perm, dtype=np.int64)
    src = np.repeat(np.arange(g.n, dtype=np.int64), g.degrees())
    dst = g.adj.astype(np.int64)
    keep = src < dst
    nu, nv = perm[src[keep]], perm[dst[keep]]
    lo, hi = np.minimum(nu, nv), np.maximum(nu, nv)
    vw = np.empty(g.n, dtype=np.int32)
    vw[perm] = g.vw
    return csr_from_pairs(g.n, lo, hi, g.adjw[keep], vw=vw, name=name or g.name)


def random_permutation(n: int, seed: int) -> np.ndarray:
    return np.argsort(splitmix64(seed, np.arange(n, dtype=np.uint64)), kind="stable")


# ----------------------------------------------------------------------------
# Graph families
# ----------------------------------------------------------------------------

def grid2d(nx: int, ny: int) -> Graph:
    """4-neighbour grid, vertex id = y*nx + x, unit weights."""
    ids = np.arange(nx * ny, dtype=np.int64).reshape(ny, nx)
    hu, hv = ids[:, :-1].ravel(), ids[:, 1:].ravel()
    vu, vv = ids[:-1, :].ravel(), ids[1:, :].ravel()
    return csr_from_pairs(nx * ny, np.concatenate([hu, vu]), np.concatenate([hv, vv]),
                          name=f"grid2d_{nx}x{ny}")


def grid3d(nx: int, ny: int, nz: int) -> Graph:
    """6-neighbour grid, vertex id = (z*ny + y)*nx + x, unit weights."""
    ids = np.arange(nx * ny * nz, dtype=np.int64).reshape(nz, ny, nx)
    us, vs = [], []
    for sl_a, sl_b in (((slice(None), slice(None), slice(None, -1)), (slice(None), slice(None), slice(1, None))),
                       ((slice(None), slice(None, -1), slice(None)), (slice(None), slice(1, None), slice(None))),
                       ((slice(None, -1), slice(None), slice(None)), (slice(1, None), slice(None), slice(None)))):
        us.append(ids[sl_a].ravel())
        vs.append(ids[sl_b].ravel())
    return csr_from_pairs(nx * ny * nz, np.concatenate(us), np.concatenate(vs),
                          name=f"grid3d_{nx}x{ny}x{nz}")


def rgg2d(n: int, radius: float, seed: int, wmax: int = 10, shuffled: bool = False) -> Graph:
    """Random geometric graph: n points uniform in [0,1)^2, edge iff dist^2 < r^2.

    Vertex ids are assigned in order of the r-cell (row-major), ties by draw
    index.  Edge weight = 1 + (SplitMix64(seed ^ 0x57, lo*2^32 + hi) mod wmax)
    for the pair (lo, hi) of final ids; wmax = 1 gives unit weights.
    """
    idx = np.arange(n, dtype=np.uint64)
    x = uniform01(seed, 2 * idx)
    y = uniform01(seed, 2 * idx + _U64(1))
    G = max(1, int(math.floor(1.0 / radius)))
    cx = np.minimum((x * G).astype(np.int64), G - 1)
    cy = np.minimum((y * G).astype(np.int64), G - 1)
    cell = cy * G + cx
    order = np.argsort(cell, kind="stable")
    x, y, cell, cx, cy = x[order], y[order], cell[order], cx[order], cy[order]
    start = np.searchsorted(cell, np.arange(G * G + 1, dtype=np.int64))
    cnt_cell = np.diff(start)
    r2 = radius * radius
    us, vs = [], []
    pts = np.arange(n, dtype=np.int64)
    for dx, dy in ((0, 0), (1, 0), (-1, 1), (0, 1), (1, 1)):
        ncx, ncy = cx + dx, cy + dy
        ok = (ncx >= 0) & (ncx < G) & (ncy < G)
        src = pts[ok]
        ncell = (ncy * G + ncx)[ok]
        cnt = cnt_cell[ncell]
        tot = int(cnt.sum())
        if tot == 0:
            continue
        rep_src = np.repeat(src, cnt)
        base = np.repeat(start[ncell], cnt)
        off = np.arange(tot, dtype=np.int64) - np.repeat(np.cumsum(cnt) - cnt, cnt)
        dst = base + off
        if dx == 0 and dy == 0:
            keep = dst > rep_src
            rep_src, dst = rep_src[keep], dst[keep]
        ddx = x[rep_src] - x[dst]
        ddy = y[rep_src] - y[dst]
        close = ddx * ddx + ddy * ddy < r2
        us.append(rep_src[close])
        vs.append(dst[close])
    u = np.concatenate(us) if us else np.zeros(0, np.int64)
    v = np.concatenate(vs) if vs else np.zeros(0, np.int64)
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    if shuffled:
        perm = random_permutation(n, seed ^ 0x5A5A)
        lo, hi = perm[lo], perm[hi]
        lo, hi = np.minimum(lo, hi), np.maximum(lo, hi)
    if wmax > 1:
        key = (lo.astype(np.uint64) << _U64(32)) | hi.astype(np.uint64)
        w = (splitmix64(seed ^ 0x57, key) % _U64(wmax)).astype(np.int64) + 1
    else:
        w = None
    return csr_from_pairs(n, lo, hi, w, name=f"rgg2d_n{n}")


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int,
         relabel_seed: Optional[int] = None, chunk: int = 1 << 22) -> Graph:
    """R-MAT graph (Chakrabarti, Zhan & Faloutsos 2004), symmetrised.

    edge_factor * 2^scale samples; at each of ``scale`` bit levels a quadrant is
    chosen with probabilities (a, b, c, 1-a-b-c) from uniform draw number
    ``sample*scale + level``.  Self-loops and duplicates are dropped, then the
    vertices are relabelled by a seeded random permutation.  Unit weights.
    """
    n = 1 << scale
    total = edge_factor * n
    ab, abc = a + b, a + b + c

    def block(s0):
        s = np.arange(s0, min(total, s0 + chunk), dtype=np.uint64)
        u = np.zeros(s.size, dtype=np.int64)
        v = np.zeros(s.size, dtype=np.int64)
        for lvl in range(scale):
            r = uniform01(seed, s * _U64(scale) + _U64(lvl))
            bu = (r >= ab).astype(np.int64)
            bv = ((r >= a) & (r < ab)) | (r >= abc)
            u = (u << 1) | bu
            v = (v << 1) | bv.astype(np.int64)
        keep = u != v
        lo = np.minimum(u[keep], v[keep])
        hi = np.maximum(u[keep], v[keep])
        return lo * n + hi

    # chunks are independent (counter-based draws): numpy releases the GIL,
    # so threads shorten the generation of the large graphs
    starts = list(range(0, total, chunk))
    if len(starts) > 1:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(max_workers=min(len(starts), os.cpu_count() or 1)) as ex:
            keys = list(ex.map(block, starts))
    else:
        keys = [block(s0) for s0 in starts]
    key = np.sort(np.concatenate(keys))  # sorted distinct keys (a sort is faster than a hash here)
    if key.size:
        key = key[np.concatenate(([True], key[1:] != key[:-1]))]
    lo, hi = key // n, key % n
    perm = random_permutation(n, seed ^ 0xA11CE if relabel_seed is None else relabel_seed)
    lo, hi = perm[lo], perm[hi]
    return csr_from_pairs(n, np.minimum(lo, hi), np.maximum(lo, hi), name=f"rmat_s{scale}_ef{edge_factor}")


def erdos_renyi(n: int, p: float, seed: int, wmax: int = 1, vwmax: int = 1) -> Graph:
    """Small G(n, p) graphs for tests (pair (i<j) kept iff draw < p)."""
    iu, ju = np.triu_indices(n, 1)
    if iu.size == 0:
        return csr_from_pairs(n, iu, ju, vw=np.ones(n, np.int32), name=f"er_n{n}")
    keyp = iu.astype(np.uint64) * _U64(n) + ju.astype(np.uint64)
    keep = uniform01(seed, keyp) < p
    u, v = iu[keep], ju[keep]
    w = None
    if wmax > 1:
        w = (splitmix64(seed ^ 0x77, keyp[keep]) % _U64(wmax)).astype(np.int64) + 1
    vw = (splitmix64(seed ^ 0x99, np.arange(n, dtype=np.uint64)) % _U64(vwmax)).astype(np.int32) + 1
    return csr_from_pairs(n, u, v, w, vw=vw, name=f"er_n{n}")


DEGREE_MIX_EXACT = (32, 33, 255, 256)


def degree_mix(seed: int = 21) -> Graph:
    """A 1,600-vertex graph whose degrees straddle the bounds of the
    per-vertex paths (32 and 255): a dense core 0..399 (degrees ~160), six
    hubs 400..405 (degrees 300..700), a sparse rest 406..1595 (degrees ~7)
    and the vertices 1596..1599 of degree exactly 32, 33, 255 and 256.  Edge
    weights 1..9, vertex weights 1..4 (numpy's PCG64 stream of `seed`)."""
    rng = np.random.default_rng(seed)
    n, core, hub0, sparse0, exact0 = 1600, 400, 400, 406, 1596
    pairs = []
    iu, ju = np.triu_indices(core, 1)
    keep = rng.random(iu.size) < 0.4
    pairs.append(np.stack([iu[keep], ju[keep]], 1))
    for h in range(hub0, sparse0):
        deg = int(rng.integers(300, 701))
        nb = rng.choice(np.setdiff1d(np.arange(exact0), [h]), size=deg, replace=False)
        pairs.append(np.stack([np.full(deg, h), nb], 1))
    ns = exact0 - sparse0
    iu, ju = np.triu_indices(ns, 1)
    keep = rng.random(iu.size) < 0.004
    pairs.append(np.stack([iu[keep] + sparse0, ju[keep] + sparse0], 1))
    for i, deg in enumerate(DEGREE_MIX_EXACT):
        nb = rng.choice(np.arange(sparse0, exact0), size=deg, replace=False)
        pairs.append(np.stack([np.full(deg, exact0 + i), nb], 1))
    p = np.concatenate(pairs).astype(np.int64)
    p = np.unique(np.stack([p.min(1), p.max(1)], 1), axis=0)
    w = rng.integers(1, 10, size=len(p))
    vw = rng.integers(1, 5, size=n).astype(np.int32)
    return csr_from_pairs(n, p[:, 0], p[:, 1], w, vw, name="degree_mix")


def random_mapping(n: int, k: int, seed: int) -> np.ndarray:
    """Pi_0(v) = SplitMix64(seed ^ v) mod k."""
    return (splitmix64(seed, np.arange(n, dtype=np.uint64)) % _U64(k)).astype(np.int32)


# ----------------------------------------------------------------------------
# The workload recipes (sizes and distributions of the paper's instance mix)
# ----------------------------------------------------------------------------

SEED_BASE = 0x5EED0000
SEED_ITEM = 0x5EED1000


def workload_grid64() -> Workload:
    """2D 64x64 grid, hierarchy 4:8 (k=32), distances 1:10, eps 0.03,
    random initial mapping, 10 fixed refinement rounds, no coarsening."""
    seed = SEED_BASE + 1
    g = grid2d(64, 64)
    topo = Topology((4, 8), (1, 10), 0.03)
    return Workload(g, topo, seed, pi0=random_mapping(g.n, topo.k, seed), rounds=10,
                    multilevel=False, name="grid2d_64x64_h4:8_d1:10_r10")


def rgg_radius(n: int, mean_degree: float) -> float:
    return math.sqrt(mean_degree / (math.pi * n))


def workload_rgg(log2n: int = 20, shuffled: bool = False) -> Workload:
    """RGG, mean degree ~12, weights 1..10, hierarchy 4:8:8 (k=256),
    distances 1:10:100, eps 0.03, full multilevel."""
    seed = SEED_BASE + 2
    n = 1 << log2n
    g = rgg2d(n, rgg_radius(n, 12.0), seed, wmax=10, shuffled=shuffled)
    topo = Topology((4, 8, 8), (1, 10, 100), 0.03)
    return Workload(g, topo, seed, name=f"rgg2d_n2^{log2n}_deg12_h4:8:8_d1:10:100")


def workload_rmat(scale: int = 22) -> Workload:
    """R-MAT scale 22, edge factor 16, (.57,.19,.19,.05), unit weights,
    hierarchy 4:16:8 (k=512), distances 1:10:100, eps 0.03, full multilevel."""
    seed = SEED_BASE + 3
    g = rmat(scale, 16, 0.57, 0.19, 0.19, seed)
    topo = Topology((4, 16, 8), (1, 10, 100), 0.03)
    return Workload(g, topo, seed, name=f"rmat_s{scale}_ef16_h4:16:8_d1:10:100")


_BATCH_HIERS = ((4, 8), (4, 8, 8), (2, 4, 16, 8))
_BATCH_DISTS = (1, 10, 100, 1000)


def workload_batch(count: int = 64, lo_log2: int = 12, hi_log2: int = 18) -> List[Workload]:
    """Batch of RGGs, n log-uniform in [2^lo, 2^hi], mean degree 10, weights
    1..10, hierarchies drawn from {4:8, 4:8:8, 2:4:16:8}, distances the prefix
    of 1:10:100:1000, eps 0.03; 10 fixed rounds from Pi_0 = h(v) mod k."""
    out = []
    for i in range(count):
        seed = SEED_ITEM + i
        u = float(uniform01(seed, np.uint64(0xB0)))
        n = int(round(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * u)))
        hier = _BATCH_HIERS[int(splitmix64(seed, np.uint64(0xB1)) % _U64(len(_BATCH_HIERS)))]
        topo = Topology(hier, _BATCH_DISTS[:len(hier)], 0.03)
        g = rgg2d(n, rgg_radius(n, 10.0), seed, wmax=10)
        out.append(Workload(g, topo, seed, pi0=random_mapping(n, topo.k, seed), rounds=10,
                            multilevel=False, name=f"batch{i}_rgg_n{n}"))
    return out


_SERVE_HIERS = ((4, 8), (4, 8, 8), (4, 16, 8), (4, 16, 16))


def serve_request(i: int, max_log2_grid: int = 21, max_log2_rgg: int = 20) -> Workload:
    """Request i of the serving stream: 50% 3D 6-neighbour grids with 2^j cells
    (j uniform in 10..21), 50% RGGs with n log-uniform in 2^12..2^20 (mean
    degree 12); hierarchy from {4:8, 4:8:8, 4:16:8, 4:16:16}, distances the
    prefix of 1:10:100, eps 0.03; full multilevel."""
    seed = SEED_ITEM + 0x10000 + i
    kind = int(splitmix64(seed, np.uint64(0xC0)) & _U64(1))
    hier = _SERVE_HIERS[int(splitmix64(seed, np.uint64(0xC1)) % _U64(len(_SERVE_HIERS)))]
    topo = Topology(hier, (1, 10, 100)[:len(hier)], 0.03)
    if kind == 0:
        j = 10 + int(splitmix64(seed, np.uint64(0xC2)) % _U64(max_log2_grid - 10 + 1))
        dims = (1 << -(-j // 3), 1 << -(-(j - 1) // 3), 1 << (j // 3))
        g = grid3d(*dims)
    else:
        u = float(uniform01(seed, np.uint64(0xC3)))
        n = int(round(2.0 ** (12 + (max_log2_rgg - 12) * u)))
        g = rgg2d(n, rgg_radius(n, 12.0), seed, wmax=10)
    return Workload(g, topo, seed, name=f"serve{i}_{g.name}")


def poisson_arrivals(count: int, mean_gap_s: float, seed: int) -> np.ndarray:
    """Arrival times (s) with exponential inter-arrival gaps of the given mean."""
    u = uniform01(seed, np.arange(count, dtype=np.uint64))
    return np.cumsum(-mean_gap_s * np.log1p(-u))


def check_graph(g: Graph) -> None:
    """Structural checks of the CSR convention (used by tests)."""
    assert g.xadj.dtype == np.int64 and g.adj.dtype == np.int32
    assert g.xadj[0] == 0 and np.all(np.diff(g.xadj) >= 0)
    deg = g.degrees()
    src = np.repeat(np.arange(g.n, dtype=np.int64), deg)
    assert np.all(g.adj >= 0) and np.all(g.adj < g.n)
    assert not np.any(src == g.adj), "self-loop"
    if g.m_dir:
        key = src * g.n + g.adj
        assert np.all(np.diff(key) > 0), "rows must be strictly ascending"
        rkey = g.adj.astype(np.int64) * g.n + src
        order = np.argsort(rkey)
        assert np.array_equal(rkey[order], key), "not symmetric"
        assert np.array_equal(g.adjw[order], g.adjw), "asymmetric weights"
    assert np.all(g.adjw >= 1) and np.all(g.vw >= 1)
