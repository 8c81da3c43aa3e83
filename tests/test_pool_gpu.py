"""The library's default memory pool keeps what gp_graph_free gives back (so a
graph of the same size uploads again without new mappings) until gp_pool_trim
returns it to the driver."""
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu


def test_pool_keeps_freed_memory_until_trimmed():
    import torch

    import paper_2010_16012_gb300 as gp

    assert torch.cuda.is_available()
    g = gg.rmat(20, 16, seed=1)
    gp.pool_trim(0)  # start from a pool that holds nothing beyond what is in use
    r0, u0 = gp.pool_usage()
    G = gp.Graph.from_graphgen(g, copy=True)  # the arrays are copied into library-owned memory
    torch.cuda.synchronize()
    r1, u1 = gp.pool_usage()
    held = u1 - u0
    assert held >= 4 * g.m, (held, g.m)  # at least the copied CSR indices
    G.free()
    torch.cuda.synchronize()
    r2, u2 = gp.pool_usage()
    assert u2 == u0  # everything the graph held is back in the pool ...
    assert r2 >= r0 + held * 9 // 10  # ... and the pool still reserves it
    gp.pool_trim(0)
    r3, u3 = gp.pool_usage()
    assert u3 == u0
    assert r3 <= r2 - held * 9 // 10, (r2, r3, held)  # returned to the driver
    # the pool is still usable after a trim
    G = gp.Graph.from_graphgen(g, copy=True)
    x, st = gp.pagerank(G, gp.PULL, 0.85, iters=2)
    assert st["iters_done"] == 2 and bool(torch.isfinite(x).all())
    G.free()
    with pytest.raises(gp.GpError):
        gp.pool_trim(-1)
