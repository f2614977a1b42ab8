"""The mapping server on the GPU: jobs of the serving mix (3D grids and RGGs,
hierarchies up to 4:16:16) and degree-skewed jobs give the same J and mapping
when they run alone and when they overlap with others under memory admission,
with their small levels batched across requests or not; the admission
estimate bounds what each job's context really held."""
import numpy as np
import pytest

import oracle as O
from paper_2510_12196_gb300 import gpumap as G
from paper_2510_12196_gb300 import inputs as I

from gpu_helpers import oracle_params

pytestmark = pytest.mark.gpu


def _mix():
    """Ten jobs of the serving mix at test sizes."""
    out = []
    hiers = ((4, 8), (4, 8, 8), (4, 16, 8), (4, 16, 16))
    for i in range(10):
        h = hiers[i % 4]
        d = (1, 10, 100)[:len(h)]
        if i % 2 == 0:
            j = 10 + (i % 7)
            dims = (1 << -(-j // 3), 1 << -(-(j - 1) // 3), 1 << (j // 3))
            g = I.grid3d(*dims)
        else:
            n = [5000, 20000, 70000, 3000, 130000][i // 2]
            g = I.rgg2d(n, I.rgg_radius(n, 12.0), 0x5EED2000 + i, wmax=10)
        out.append((g, h, d))
    return out


def _alone(g, h, d):
    cfg = G.map_config_default()
    ctx = G.map_create(g.xadj, g.adj, g.adjw, g.vw, g.n, h, d, 0.03, cfg)
    try:
        pi = np.zeros(g.n, np.int32)
        J = G.map_run(ctx, pi)
    finally:
        G.map_destroy(ctx)
    return J, pi


def test_served_results_equal_alone_and_oracle():
    jobs = _mix()
    alone = [_alone(*j) for j in jobs]
    for (g, h, d), (J, pi) in list(zip(jobs, alone))[:3]:
        opi, oJ, _ = O.map_run(g, h, d, 0.03, oracle_params())
        assert J == oJ and np.array_equal(pi, opi)
    ests = [G.map_job_estimate_bytes(g.n, g.m_dir, h) for g, h, _ in jobs]
    # a budget that holds about three average jobs: admission has to queue
    budget = int(3 * np.mean(ests))
    srv = G.MapServer(slots=4, lookahead=4, mem_budget=budget)
    try:
        tickets = [srv.submit(g, h, d, user=i) for i, (g, h, d) in enumerate(jobs)]
        res = [srv.wait(t) for t in tickets]
        st = srv.stats()
    finally:
        srv.close()
    for i, ((r, pi), (J, opi)) in enumerate(zip(res, alone)):
        assert r.status == 0, r.error
        assert r.user == i or (r.user is None and i == 0)
        assert r.J == J and np.array_equal(pi, opi), i
        assert r.device_bytes_peak <= r.device_bytes_est, (i, r.device_bytes_peak, r.device_bytes_est)
        assert r.t_submit_ms <= r.t_start_ms <= r.t_done_ms
    assert st.completed == len(jobs) and st.failed == 0
    assert st.peak_running >= 2  # jobs did overlap
    # a job larger than the whole budget runs alone; otherwise the budget holds
    assert st.peak_bytes_in_flight <= max(budget, max(ests))


def test_served_job_errors_do_not_stop_the_loop():
    g = I.grid2d(16, 16)
    bad = I.Graph(g.n, g.xadj.copy(), g.adj.copy(), g.adjw.copy(), g.vw.copy())
    bad.adjw[3] += 1  # asymmetric: map_create rejects it
    srv = G.MapServer(slots=2)
    try:
        t_bad = srv.submit(bad, (4, 8), (1, 10))
        t_ok = srv.submit(g, (4, 8), (1, 10))
        rb, _ = srv.wait(t_bad)
        ro, pi = srv.wait(t_ok)
        st = srv.stats()
    finally:
        srv.close()
    assert rb.status == 1 and rb.error
    J, opi = _alone(g, (4, 8), (1, 10))
    assert ro.status == 0 and ro.J == J and np.array_equal(pi, opi)
    assert st.failed == 1 and st.completed == 1


def test_estimate_bounds_full_size_jobs():
    """The admission estimate is an upper bound of the device memory of the
    largest serving jobs (3D grid 2^21, RGG 2^20) and of an R-MAT graph."""
    cases = [(I.grid3d(128, 128, 128), (4, 16, 16), (1, 10, 100)),
             (I.workload_rgg(20).graph, (4, 16, 8), (1, 10, 100)),
             (I.rmat(16, 16, 0.57, 0.19, 0.19, 5), (4, 16, 8), (1, 10, 100))]
    for g, h, d in cases:
        ctx = G.map_create(g.xadj, g.adj, g.adjw, g.vw, g.n, h, d, 0.03, G.map_config_default())
        try:
            G.map_run(ctx)
            peak = G.map_stats(ctx).device_bytes_peak
        finally:
            G.map_destroy(ctx)
        est = G.map_job_estimate_bytes(g.n, g.m_dir, h)
        assert peak <= est, (g.n, peak, est)


def _small_mix():
    """Twenty small jobs (every level refined by the fused engine): 3D grids,
    RGGs and R-MAT graphs (rows of hundreds of entries)."""
    out = []
    hiers = ((4, 8), (4, 8, 8), (4, 16, 8), (4, 16, 16))
    for i in range(20):
        h = hiers[i % 4]
        d = (1, 10, 100)[:len(h)]
        if i % 3 == 0:
            g = I.grid3d(8 << (i % 2), 8, 8 << (i % 3 == 0))
        elif i % 3 == 1:
            n = 2000 + 1500 * i
            g = I.rgg2d(n, I.rgg_radius(n, 12.0), 0x5EED2100 + i, wmax=10)
        else:
            g = I.rmat(10 + i % 4, 8, 0.57, 0.19, 0.19, 0x5EED2200 + i)
        out.append((g, h, d))
    return out


@pytest.mark.parametrize("lanes,whole_gpu", [(1, 0), (2, 0), (-1, 1)])
def test_batched_small_levels_equal_alone(lanes, whole_gpu):
    """Small levels of concurrent jobs refined in shared engine launches
    (one or two batcher lanes), or each job on its own (lanes -1, whole-GPU
    engine allowed): every result equals the job alone, which equals the
    oracle on the degree-skewed jobs."""
    jobs = _small_mix()
    alone = [_alone(*j) for j in jobs]
    for k in (2, 5):  # R-MAT jobs against the oracle
        (g, h, d), (J, pi) = jobs[k], alone[k]
        opi, oJ, _ = O.map_run(g, h, d, 0.03, oracle_params())
        assert J == oJ and np.array_equal(pi, opi)
    srv = G.MapServer(slots=8, lookahead=8, batch_lanes=lanes, whole_gpu_levels=whole_gpu)
    try:
        tickets = [srv.submit(g, h, d, user=i) for i, (g, h, d) in enumerate(jobs)]
        res = [srv.wait(t) for t in tickets]
        st = srv.stats()
    finally:
        srv.close()
    for i, ((r, pi), (J, opi)) in enumerate(zip(res, alone)):
        assert r.status == 0, r.error
        assert r.J == J and np.array_equal(pi, opi), i
    assert st.completed == len(jobs) and st.failed == 0
    if lanes > 0:
        # every job's levels went through the batcher; with one lane and
        # eight jobs in flight, refinements of several requests shared a launch
        assert st.engine_jobs >= len(jobs) and st.engine_launches >= 1
        if lanes == 1:
            assert st.engine_launches < st.engine_jobs and st.peak_batch >= 2
    else:
        assert st.engine_launches == 0 and st.engine_jobs == 0
