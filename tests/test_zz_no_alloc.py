"""The allocation-free objective entry point against the context-based one.

map_objective_noalloc serves callers that cannot or must not allocate device
memory (the CUDA allocation calls may synchronise the whole device; some
callers live under a fixed memory budget of their own pool).  It must return
exactly what map_objective returns, and what the CPU oracle computes, also
when called twice in a row: the second call reuses the shared scratch array
and must not see the first call's block weights or J.  This file is
collected last on purpose.
"""
import numpy as np
import pytest

import oracle as O
from paper_2510_12196_gb300 import gpumap as G
from paper_2510_12196_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _context_objective(g, hier, dist, pi):
    ctx = G.map_create(g.xadj, g.adj, g.adjw, g.vw, g.n, hier, dist, 0.03)
    try:
        G.map_set_mapping(ctx, 0, pi)
        return G.map_objective(ctx, 0)
    finally:
        G.map_destroy(ctx)


@pytest.mark.parametrize("hier,dist", [((4, 8, 8), (1, 10, 100)), ((4, 8, 6), (1, 10, 100)), ((4, 16, 16, 16), (1, 10, 100, 1000))])
def test_noalloc_objective_matches_map_objective_twice(hier, dist):
    import torch
    g = I.rgg2d(1 << 15, I.rgg_radius(1 << 15, 12), 77, wmax=10)
    k = int(np.prod(hier))
    dev = [torch.from_numpy(a).cuda() for a in (g.xadj, g.adj, g.adjw, g.vw)]
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    # two different mappings in a row: the second call must not inherit the
    # first one's block weights or objective from the shared scratch
    pis = [I.random_mapping(g.n, k, 1), ((np.arange(g.n) * k) // g.n).astype(np.int32)]
    for pi in pis:
        want = _context_objective(g, hier, dist, pi)
        oJ, omx, _ = O.objective(g, hier, dist, pi)
        assert want == (oJ, omx)
        pi_d = torch.from_numpy(pi).cuda()
        G.map_objective_noalloc(*dev, g.n, pi_d, hier, dist, out)
        torch.cuda.synchronize()
        assert tuple(int(x) for x in out.cpu()) == want


def test_noalloc_unit_weights_and_size_limit():
    import torch
    g = I.grid2d(40, 30)
    pi = I.random_mapping(g.n, 32, 3)
    want = _context_objective(g, (4, 8), (1, 10), pi)
    dx, da, dv = (torch.from_numpy(a).cuda() for a in (g.xadj, g.adj, g.vw))
    out = torch.full((2,), -1, dtype=torch.int64, device="cuda")
    G.map_objective_noalloc(dx, da, None, dv, g.n, torch.from_numpy(pi).cuda(), (4, 8), (1, 10), out)
    torch.cuda.synchronize()
    assert tuple(int(x) for x in out.cpu()) == want
    with pytest.raises(G.MapError) as ei:
        G.map_objective_noalloc(dx, da, None, dv, g.n, torch.from_numpy(pi).cuda(), (256, 256), (1, 10), out)
    assert ei.value.status == 1 and "16384" in str(ei.value)
