"""Device-memory exhaustion, injected on the host.

The context's allocator callback (map_config.alloc / free) is a counting
wrapper around torch's caching allocator that returns NULL once a given
number of allocations has been served.  Whichever call then needs memory
(map_create, or the coarsening inside map_run) must fail with MAP_E_OOM and
leave nothing allocated once the context is destroyed, and a fresh context
must still map bit-exactly like the oracle.  No GPU fault is involved: the
failure is a NULL returned by host code before any kernel sees the pointer.
"""
import numpy as np
import pytest

import oracle as O
from paper_2510_12196_gb300 import gpumap as G
from paper_2510_12196_gb300 import inputs as I

from gpu_helpers import oracle_params

pytestmark = pytest.mark.gpu

MAP_E_OOM = 2


class FailingAllocator:
    """Serves `limit` allocations through torch's caching allocator, then
    returns NULL; tracks the live blocks."""

    def __init__(self, limit=None):
        import torch
        self.dev = torch.cuda.current_device()
        self.limit = limit
        self.calls = 0
        self.live = set()

        def _alloc(nbytes, user, stream):
            self.calls += 1
            if self.limit is not None and self.calls > self.limit:
                return None
            try:
                p = torch.cuda.caching_allocator_alloc(int(nbytes), self.dev, stream)
            except Exception:
                return None
            self.live.add(p)
            return p

        def _free(ptr, nbytes, user, stream):
            self.live.discard(ptr)
            torch.cuda.caching_allocator_delete(ptr)

        self.fns = (G.ALLOC_FN(_alloc), G.FREE_FN(_free))

    def config(self, seed):
        cfg = G.map_config_default(seed)
        cfg.alloc, cfg.free = self.fns
        return cfg


def _attempt(g, hier, dist, seed, limit):
    """map_create + map_run under the limit: ('create' | 'run' | 'ok', ctx
    state checks done, allocator)."""
    fa = FailingAllocator(limit)
    try:
        ctx = G.map_create(g.xadj, g.adj, g.adjw, g.vw, g.n, hier, dist, 0.03, fa.config(seed))
    except G.MapError as e:
        assert e.status == MAP_E_OOM, e
        assert not fa.live, "a failed map_create left device memory allocated"
        return "create", fa, None
    try:
        pi = np.zeros(g.n, np.int32)
        try:
            J = G.map_run(ctx, pi)
            where, res = "ok", (J, pi)
        except G.MapError as e:
            assert e.status == MAP_E_OOM, e
            assert "NULL" in G.map_last_error(ctx)
            where, res = "run", None
    finally:
        G.map_destroy(ctx)
    assert not fa.live, "map_destroy left device memory allocated"
    return where, fa, res


def test_oom_from_allocator_callback():
    g = I.rgg2d(1 << 14, I.rgg_radius(1 << 14, 12), 0x5EED0AA0, wmax=10)
    hier, dist = (4, 8, 8), (1, 10, 100)
    seed = 0x5EED0AA0
    # unlimited: how many allocations a create + map takes
    where, fa, (J, pi) = _attempt(g, hier, dist, seed, None)
    assert where == "ok"
    total = fa.calls
    where, fa0, _ = _attempt(g, hier, dist, seed, 0)
    assert where == "create"
    seen = set()
    for limit in sorted({0, 1, 2, total // 4, total // 2, (3 * total) // 4, total - 1}):
        where, _, _ = _attempt(g, hier, dist, seed, limit)
        assert where in ("create", "run"), (limit, where)
        seen.add(where)
    assert seen == {"create", "run"}
    # the device stays usable: a fresh context (default allocator) maps exactly as the oracle
    ctx = G.map_create(g.xadj, g.adj, g.adjw, g.vw, g.n, hier, dist, 0.03, G.map_config_default(seed))
    try:
        pi2 = np.zeros(g.n, np.int32)
        J2 = G.map_run(ctx, pi2)
    finally:
        G.map_destroy(ctx)
    opi, oJ, _ = O.map_run(g, hier, dist, 0.03, oracle_params(seed))
    assert J == J2 == oJ and np.array_equal(pi, opi) and np.array_equal(pi2, opi)
