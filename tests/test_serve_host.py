"""Host logic of the mapping server (request loop, memory admission,
lookahead, starvation guard, results, cancellation), run on the CPU with a
job runner that stands in for the GPU pipeline: each job blocks until the
test releases it, so the admission decisions are observed deterministically."""
import threading
import time

import numpy as np
import pytest

from paper_2510_12196_gb300 import gpumap as G
from paper_2510_12196_gb300 import inputs as I

HIER, DIST = (4, 8), (1, 10)


def _graph(n):
    """A path on n vertices (only its size matters to the stand-in runner)."""
    return I.csr_from_pairs(n, np.arange(n - 1), np.arange(1, n))


class Harness:
    def __init__(self, **opts):
        self.lock = threading.Lock()
        self.release = {}
        self.started = []
        self.running = 0
        self.max_running = 0
        self.srv = G.MapServer(runner=self._run, **opts)

    def _run(self, job, stream, user, res):
        idx = int(job.contents.user or 0)
        with self.lock:
            self.started.append(idx)
            self.running += 1
            self.max_running = max(self.max_running, self.running)
            ev = self.release.setdefault(idx, threading.Event())
        ev.wait(20)
        with self.lock:
            self.running -= 1
        res.contents.J = 1000 + idx
        res.contents.levels = 1
        return 0

    def submit(self, idx, n):
        with self.lock:
            self.release.setdefault(idx, threading.Event())
        return self.srv.submit(_graph(n), HIER, DIST, user=idx)

    def let_go(self, idx):
        with self.lock:
            ev = self.release.setdefault(idx, threading.Event())
        ev.set()

    def wait_started(self, count, timeout=10):
        t0 = time.time()
        while time.time() - t0 < timeout:
            with self.lock:
                if len(self.started) >= count:
                    return list(self.started)
            time.sleep(0.005)
        with self.lock:
            return list(self.started)

    def close(self):
        for ev in list(self.release.values()):
            ev.set()
        self.srv.close()


def _est(n):
    return G.map_job_estimate_bytes(n, 2 * (n - 1), HIER)


def test_estimate_grows_with_size():
    assert _est(1000) < _est(2000) < _est(100000)
    assert G.map_job_estimate_bytes(10, 18, (4, 16, 16)) > G.map_job_estimate_bytes(10, 18, (4, 8))
    assert G.map_job_estimate_bytes(-1, 0, HIER) == -1


def test_memory_budget_limits_concurrency():
    n = 50000
    h = Harness(slots=6, lookahead=8, mem_budget=int(_est(n) * 2.5))
    try:
        tickets = [h.submit(i, n) for i in range(6)]
        assert h.wait_started(2) == [0, 1]
        time.sleep(0.1)
        assert len(h.started) == 2  # a third would exceed the budget
        h.let_go(0)
        assert h.wait_started(3) == [0, 1, 2]
        for i in range(1, 6):
            h.let_go(i)
        res = [h.srv.wait(t)[0] for t in tickets]
        assert [r.J for r in res] == [1000 + i for i in range(6)]
        assert all(r.status == 0 and r.t_submit_ms <= r.t_start_ms <= r.t_done_ms for r in res)
        st = h.srv.stats()
        assert st.peak_running == 2 and h.max_running == 2
        assert st.peak_bytes_in_flight <= st.mem_budget
        assert (st.submitted, st.completed, st.failed, st.queued, st.running) == (6, 6, 0, 0, 0)
    finally:
        h.close()


def test_slots_limit_concurrency():
    h = Harness(slots=3, mem_budget=1 << 50)
    try:
        tickets = [h.submit(i, 1000) for i in range(7)]
        assert h.wait_started(3) == [0, 1, 2]
        time.sleep(0.1)
        assert len(h.started) == 3
        for i in range(7):
            h.let_go(i)
        for t in tickets:
            h.srv.wait(t)
        assert h.max_running == 3
    finally:
        h.close()


def test_oversized_job_runs_alone():
    small, big = 1000, 400000
    h = Harness(slots=4, mem_budget=int(_est(big) * 0.5))
    try:
        t0 = h.submit(0, small)
        assert h.wait_started(1) == [0]
        t1 = h.submit(1, big)   # larger than the whole budget: waits until nothing runs
        t2 = h.submit(2, small)
        time.sleep(0.1)
        assert h.started == [0, 2]  # the small one overtakes (lookahead)
        h.let_go(0)
        time.sleep(0.1)
        assert h.started == [0, 2]
        h.let_go(2)
        assert h.wait_started(3) == [0, 2, 1]
        time.sleep(0.05)
        assert h.max_running == 2
        h.let_go(1)
        for t in (t0, t1, t2):
            assert h.srv.wait(t)[0].status == 0
    finally:
        h.close()


def test_strict_order_with_lookahead_one():
    small, big = 1000, 200000
    h = Harness(slots=4, lookahead=1, mem_budget=int(_est(big) * 1.5))
    try:
        ts = [h.submit(0, big)]
        assert h.wait_started(1) == [0]
        ts.append(h.submit(1, big))    # does not fit next to job 0
        ts.append(h.submit(2, small))  # would fit, but may not overtake
        time.sleep(0.1)
        assert h.started == [0]
        h.let_go(0)
        assert h.wait_started(3) == [0, 1, 2]
        for i in (1, 2):
            h.let_go(i)
        for t in ts:
            h.srv.wait(t)
    finally:
        h.close()


def test_starvation_guard():
    """After 4 x lookahead overtakes, the oldest job is admitted first."""
    small, big = 1000, 200000
    h = Harness(slots=2, lookahead=2, mem_budget=int(_est(big) * 1.5))
    try:
        ts = [h.submit(0, big)]
        assert h.wait_started(1) == [0]
        ts.append(h.submit(1, big))  # head of the queue, does not fit beside job 0
        nxt = 2
        for k in range(8):           # 8 = 4 x lookahead small jobs overtake it, one at a time
            ts.append(h.submit(nxt, small))
            assert h.wait_started(2 + k)[-1] == nxt
            h.let_go(nxt)
            h.srv.wait(ts[-1])
            nxt += 1
        ts.append(h.submit(nxt, small))  # now it must wait behind job 1
        time.sleep(0.1)
        assert h.started[-1] == nxt - 1
        h.let_go(0)
        assert h.wait_started(11)[-2:] == [1, nxt]
        h.let_go(1)
        h.let_go(nxt)
        for t in (ts[0], ts[1], ts[-1]):
            h.srv.wait(t)
    finally:
        h.close()


def test_wait_timeout_poll_and_cancel():
    h = Harness(slots=1, mem_budget=1 << 50)
    try:
        t0 = h.submit(0, 1000)
        t1 = h.submit(1, 1000)
        assert h.wait_started(1) == [0]
        assert not h.srv.poll(t0)
        with pytest.raises(G.MapError) as e:
            h.srv.wait(t0, timeout_ms=30)
        assert e.value.status == 5
        h.let_go(0)
        r, _ = h.srv.wait(t0)
        assert r.J == 1000
        with pytest.raises(G.MapError):
            h.srv.wait(t0)  # already collected
        assert h.wait_started(2) == [0, 1]
        t2 = h.submit(2, 1000)  # queued behind job 1: cancelled by close()
        h.let_go(1)
        h.srv.wait(t1)
        # job 2 starts after job 1 finished; block it and destroy with one queued
        assert h.wait_started(3) == [0, 1, 2]
        h.submit(3, 1000)
    finally:
        h.close()


def test_invalid_options_and_jobs():
    with pytest.raises(G.MapError):
        G.MapServer(slots=-1)
    # batcher lanes in -1..16 (0: the default), whole_gpu_levels 0 or 1
    for bad_opts in (dict(batch_lanes=-2), dict(batch_lanes=17), dict(whole_gpu_levels=2),
                     dict(whole_gpu_levels=-1)):
        with pytest.raises(G.MapError) as e:
            G.MapServer(runner=lambda *a: 0, **bad_opts)
        assert e.value.status == 1, bad_opts
    h = Harness(slots=1)
    try:
        bad = I.Graph(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32),
                      np.zeros(0, np.int32))
        with pytest.raises(G.MapError) as e:
            h.srv.submit(bad, HIER, DIST)
        assert e.value.status == 1
    finally:
        h.close()


def test_runner_servers_have_no_level_batcher():
    """With a stand-in runner there is no GPU pipeline, so no level batcher
    runs (its counters stay zero), whatever batch_lanes asks for."""
    h = Harness(slots=2, batch_lanes=4)
    try:
        t = h.submit(0, 100)
        h.let_go(0)
        r, _ = h.srv.wait(t)
        assert r.status == 0
        st = h.srv.stats()
        assert (st.engine_launches, st.engine_jobs, st.peak_batch) == (0, 0, 0)
    finally:
        h.close()
