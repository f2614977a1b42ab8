"""Batched refinement (one persistent launch over many contexts) against the
CPU oracle: every job of the batch must equal Alg. 6 run on that graph alone,
for every schedule the autotuner can pick, on graph replays, on degree-skewed
jobs (rows above 128 entries rated by whole CTAs), and on the full 64-graph
batch workload (RGGs of 2^12..2^18 vertices, 10 fixed rounds)."""
import numpy as np
import pytest

import oracle as O
from paper_2510_12196_gb300 import gpumap as G
from paper_2510_12196_gb300 import inputs as I

from gpu_helpers import make_ctx, oracle_params

pytestmark = pytest.mark.gpu


def _jobs(sizes, seed0=0x5EED1000):
    hiers = ((4, 8), (4, 8, 8), (2, 4, 16, 8))
    out = []
    for i, n in enumerate(sizes):
        seed = seed0 + i
        hier = hiers[i % len(hiers)]
        dist = (1, 10, 100, 1000)[:len(hier)]
        g = I.rgg2d(n, I.rgg_radius(n, 10.0), seed, wmax=10)
        k = int(np.prod(hier))
        out.append((g, hier, dist, I.random_mapping(n, k, seed)))
    return out


def _oracle(jobs, rounds):
    res = []
    for g, hier, dist, pi0 in jobs:
        L = O.lmax(int(g.vw.sum()), int(np.prod(hier)), 0.03)
        opi, oJ, omx, oit, okinds, _, _ = O.refine(g, hier, dist, L, pi0, rounds=rounds, params=oracle_params())
        res.append((opi, oJ, omx, oit, okinds))
    return res


def _make(jobs):
    ctxs = []
    for g, hier, dist, pi0 in jobs:
        c = make_ctx(g, hier, dist)
        G.map_set_mapping(c, 0, pi0)
        ctxs.append(c)
    return ctxs


def _reset(ctxs, jobs):
    for c, (_, _, _, pi0) in zip(ctxs, jobs):
        G.map_set_mapping(c, 0, pi0)


def _run_batch(ctxs, **opts):
    b = G.map_batch_create(ctxs, G.map_batch_opts_default(**opts))
    try:
        G.map_batch_launch(b)
        J, mw, it = G.map_batch_results(b, len(ctxs))
        sched = G.map_batch_schedule(b)
    finally:
        G.map_batch_destroy(b)
    return J, mw, it, sched


def _check(ctxs, J, mw, it, ref):
    for i, (c, (opi, oJ, omx, oit, okinds)) in enumerate(zip(ctxs, ref)):
        assert (J[i], mw[i], it[i]) == (oJ, omx, oit), i
        assert np.array_equal(G.map_get_mapping(c, 0), opi), i
        kinds, _, _, cnt = G.map_get_refine_trace(c)
        assert cnt == oit and np.array_equal(kinds, okinds), i


SIZES = [700, 4096, 1500, 20000, 9000, 300, 40000, 2500, 6000, 12000, 1024, 33000]


def test_batch_fixed_rounds_matches_oracle():
    jobs = _jobs(SIZES)
    ref = _oracle(jobs, 10)
    ctxs = _make(jobs)
    try:
        J, mw, it, sched = _run_batch(ctxs, rounds=10)
        _check(ctxs, J, mw, it, ref)
        assert sched[0] in (1, 2, 4, 8, 16) and sched[1] in (256, 512) and sched[2] >= 1
    finally:
        for c in ctxs:
            G.map_destroy(c)


def test_batch_schedules_and_replay_agree():
    """Results do not depend on CTAs per job, staging capacity or replays."""
    jobs = _jobs(SIZES[:8], seed0=0x5EED1100)
    ref = _oracle(jobs, 10)
    ctxs = _make(jobs)
    try:
        for cl, te in ((1, 512), (4, 256), (16, 512), (2, 256)):
            _reset(ctxs, jobs)
            J, mw, it, sched = _run_batch(ctxs, rounds=10, autotune=0, cluster=cl, tile_entries=te)
            assert sched[:2] == (cl, te)
            _check(ctxs, J, mw, it, ref)
        # one batch object launched twice (the second launch replays the graph)
        _reset(ctxs, jobs)
        b = G.map_batch_create(ctxs, G.map_batch_opts_default(rounds=10, autotune=0))
        try:
            G.map_batch_launch(b)
            G.map_batch_results(b, len(ctxs))
            _reset(ctxs, jobs)
            G.map_batch_launch(b)
            J, mw, it = G.map_batch_results(b, len(ctxs))
            _check(ctxs, J, mw, it, ref)
        finally:
            G.map_batch_destroy(b)
    finally:
        for c in ctxs:
            G.map_destroy(c)


def test_batch_alg6_termination_and_single_path():
    """rounds = -1 (Alg. 6 termination) in the batch equals map_refine alone."""
    jobs = _jobs([3000, 800, 15000, 5000], seed0=0x5EED1200)
    ref = _oracle(jobs, -1)
    ctxs = _make(jobs)
    try:
        J, mw, it, _ = _run_batch(ctxs, rounds=-1)
        _check(ctxs, J, mw, it, ref)
        for c, (g, hier, dist, pi0), (opi, oJ, omx, oit, _) in zip(ctxs, jobs, ref):
            G.map_set_mapping(c, 0, pi0)
            assert G.map_refine(c, 0, -1) == (oJ, omx, oit)
            assert np.array_equal(G.map_get_mapping(c, 0), opi)
    finally:
        for c in ctxs:
            G.map_destroy(c)


def test_batch_coarse_level_jobs():
    """A batch over a coarse level of each context (after map_coarsen and a
    projected mapping) refines that level like map_refine does."""
    jobs = _jobs([30000, 20000], seed0=0x5EED1300)
    ctxs = [make_ctx(g, h, d) for g, h, d, _ in jobs]
    try:
        singles = []
        for c, (g, h, d, _) in zip(ctxs, jobs):
            assert G.map_coarsen(c) >= 2
            xadj, adj, w, vw, _ = G.map_get_level_graph(c, 1)
            pc = I.random_mapping(len(vw), int(np.prod(h)), 9)
            cg = I.Graph(len(vw), xadj, adj, w, vw)
            L = O.lmax(int(g.vw.sum()), int(np.prod(h)), 0.03)
            opi, oJ, omx, oit, _, _, _ = O.refine(cg, h, d, L, pc, rounds=10, params=oracle_params(), level=1)
            singles.append((pc, opi, oJ, omx, oit))
            G.map_set_mapping(c, 1, pc)
        J, mw, it, _ = _run_batch(ctxs, rounds=10, level=1)
        for i, (c, (pc, opi, oJ, omx, oit)) in enumerate(zip(ctxs, singles)):
            assert (J[i], mw[i], it[i]) == (oJ, omx, oit)
            assert np.array_equal(G.map_get_mapping(c, 1), opi)
    finally:
        for c in ctxs:
            G.map_destroy(c)


def test_batch_refuses_after_coarsening():
    """A coarsening (map_coarsen, or map_run, which coarsens) may move a job's
    level buffers, which the batch's descriptors and graph point into: the
    next launch is refused with MAP_E_STATE instead of replaying on them."""
    jobs = _jobs([5000, 7000], seed0=0x5EED1500)
    ctxs = _make(jobs)
    try:
        for c, (_, _, _, p0) in zip(ctxs, jobs):
            G.map_set_mapping(c, 0, p0)
        b = G.map_batch_create(ctxs, G.map_batch_opts_default(rounds=3, autotune=0))
        try:
            G.map_batch_launch(b)
            G.map_batch_results(b, len(ctxs))
            G.map_coarsen(ctxs[1])
            with pytest.raises(G.MapError) as e:
                G.map_batch_launch(b)
            assert e.value.status == 6
        finally:
            G.map_batch_destroy(b)
        # a batch built afterwards runs
        b = G.map_batch_create(ctxs, G.map_batch_opts_default(rounds=3, autotune=0))
        G.map_batch_launch(b)
        G.map_batch_results(b, len(ctxs))
        G.map_batch_destroy(b)
    finally:
        for c in ctxs:
            G.map_destroy(c)


def test_batch_errors():
    jobs = _jobs([500, 600], seed0=0x5EED1400)
    ctxs = _make(jobs)
    star = I.csr_from_pairs(300, np.zeros(299, np.int64), np.arange(1, 300), name="star300")
    # a row of degree 299 with 2^14 PE codes in binary groups: its table (conn
    # per code plus the level group sums) does not fit in shared memory
    cs = make_ctx(star, (2,) * 14, tuple(range(1, 15)))
    try:
        with pytest.raises(G.MapError) as e:
            G.map_batch_create([ctxs[0], ctxs[0]])
        assert e.value.status == 1
        with pytest.raises(G.MapError) as e:
            G.map_batch_create(ctxs, G.map_batch_opts_default(level=3))
        assert e.value.status == 6
        with pytest.raises(G.MapError) as e:
            G.map_batch_create([ctxs[1], cs])  # degree 299, 2^14 binary codes
        assert e.value.status == 1
        with pytest.raises(G.MapError) as e:
            G.map_batch_create(ctxs, G.map_batch_opts_default(rounds=0))
        assert e.value.status == 1
        with pytest.raises(G.MapError) as e:
            G.map_batch_create(ctxs, G.map_batch_opts_default(autotune=0, cluster=3))
        assert e.value.status == 1
    finally:
        for c in ctxs + [cs]:
            G.map_destroy(c)


def test_batch_workload_64_rggs_full_size():
    """The 64-graph batch workload (n log-uniform in 2^12..2^18, mean degree
    10, hierarchies from {4:8, 4:8:8, 2:4:16:8}, 10 fixed rounds from
    h(v) mod k): every job bit-identical to the oracle."""
    ws = I.workload_batch()
    jobs = [(w.graph, w.topo.hier, w.topo.dist, w.pi0) for w in ws]
    ctxs = [make_ctx(g, h, d, seed=w.seed) for (g, h, d, _), w in zip(jobs, ws)]
    try:
        _reset(ctxs, jobs)
        ref = []  # each job with its own seed (the hash streams of Alg. 5)
        for (g, hier, dist, pi0), w in zip(jobs, ws):
            L = O.lmax(int(g.vw.sum()), int(np.prod(hier)), 0.03)
            opi, oJ, omx, oit, okinds, _, _ = O.refine(g, hier, dist, L, pi0, rounds=10,
                                                       params=oracle_params(w.seed))
            ref.append((opi, oJ, omx, oit, okinds))
        J, mw, it, _ = _run_batch(ctxs, rounds=10)
        _check(ctxs, J, mw, it, ref)
    finally:
        for c in ctxs:
            G.map_destroy(c)


def _skewed_jobs(seed0=0x5EED1600):
    """Degree-skewed jobs: R-MAT graphs (hubs of hundreds to thousands of
    entries, isolated vertices), a star, the degree-mix graph and a dense
    Erdos-Renyi graph, under hierarchies of two to four levels."""
    graphs = [I.rmat(10, 8, 0.57, 0.19, 0.19, seed0), I.rmat(12, 16, 0.57, 0.19, 0.19, seed0 + 1),
              I.csr_from_pairs(300, np.zeros(299, np.int64), np.arange(1, 300), name="star300"),
              I.degree_mix(), I.erdos_renyi(400, 0.5, seed0 + 2, wmax=9, vwmax=4),
              I.rmat(13, 16, 0.57, 0.19, 0.19, seed0 + 3), I.rgg2d(5000, I.rgg_radius(5000, 10.0), seed0 + 4, wmax=10)]
    hiers = ((4, 8), (4, 8, 8), (2, 4, 16, 8), (4, 16, 8))
    out = []
    for i, g in enumerate(graphs):
        hier = hiers[i % len(hiers)]
        dist = (1, 10, 100, 1000)[:len(hier)]
        out.append((g, hier, dist, I.random_mapping(g.n, int(np.prod(hier)), seed0 + 16 + i)))
    return out


@pytest.mark.parametrize("rounds", [10, -1])
def test_batch_degree_skewed_jobs(rounds):
    """Rows of more than 128 entries are rated by whole CTAs inside the
    engine (connectivity tables over the PE codes): every job of a batch of
    power-law, star and dense graphs equals the oracle, whichever number of
    CTAs per job and staging capacity runs it."""
    jobs = _skewed_jobs()
    assert max(int(np.diff(g.xadj).max()) for g, _, _, _ in jobs) > 1000
    ref = _oracle(jobs, rounds)
    ctxs = _make(jobs)
    try:
        for opts in ({}, dict(autotune=0, cluster=1, tile_entries=512), dict(autotune=0, cluster=16, tile_entries=256)):
            _reset(ctxs, jobs)
            J, mw, it, _ = _run_batch(ctxs, rounds=rounds, **opts)
            _check(ctxs, J, mw, it, ref)
    finally:
        for c in ctxs:
            G.map_destroy(c)


def test_batch_degree_skewed_variants():
    """The same with the refinement variants (relaxed Alg. 4 filter, Eq. 1
    gains in rebalancing), which the CTA-per-row decisions also take."""
    jobs = _skewed_jobs(seed0=0x5EED1700)[:5]
    ref = []
    for g, hier, dist, pi0 in jobs:
        L = O.lmax(int(g.vw.sum()), int(np.prod(hier)), 0.03)
        prm = oracle_params(lp_relax_num=3, lp_relax_den=4, reb_objective=1)
        opi, oJ, omx, oit, okinds, _, _ = O.refine(g, hier, dist, L, pi0, rounds=12, params=prm)
        ref.append((opi, oJ, omx, oit, okinds))
    ctxs = []
    for g, hier, dist, pi0 in jobs:
        c = make_ctx(g, hier, dist, lp_relax_num=3, lp_relax_den=4, reb_objective=1)
        G.map_set_mapping(c, 0, pi0)
        ctxs.append(c)
    try:
        J, mw, it, _ = _run_batch(ctxs, rounds=12)
        _check(ctxs, J, mw, it, ref)
    finally:
        for c in ctxs:
            G.map_destroy(c)


@pytest.mark.parametrize("engine", ["cluster", "grid"])
def test_engine_power_law_level(engine):
    """map_refine of an R-MAT scale-16 level (65,536 vertices, hubs of
    thousands of entries) in the fused engine: on one cluster, or over all
    SMs (the default for levels above 32,768 vertices); Alg. 6 termination."""
    g = I.rmat(16, 16, 0.57, 0.19, 0.19, 0x5EED1800)
    hier, dist = (4, 16, 8), (1, 10, 100)
    pi0 = I.random_mapping(g.n, 512, 0x5EED1801)
    L = O.lmax(int(g.vw.sum()), 512, 0.03)
    opi, oJ, omx, oit, okinds, _, _ = O.refine(g, hier, dist, L, pi0, rounds=-1, params=oracle_params())
    over = dict(engine_max_n=1 << 17, grid_engine_max_n=-1) if engine == "cluster" else {}
    c = make_ctx(g, hier, dist, **over)
    try:
        G.map_set_mapping(c, 0, pi0)
        assert G.map_refine(c, 0, -1) == (oJ, omx, oit)
        assert np.array_equal(G.map_get_mapping(c, 0), opi)
        kinds, _, _, cnt = G.map_get_refine_trace(c)
        assert cnt == oit and np.array_equal(kinds, okinds)
    finally:
        G.map_destroy(c)
