"""Triangle counting (gp_triangles, the push/pull NodeIterator) against the
oracle: per-vertex counts bit-exact (integers) for push (fetch-and-add), pull
(owner-only writes) and AUTO, over graphs with no triangles, complete graphs,
wheels, hubs above every chunk threshold and power-law graphs."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gp():
    import torch

    import paper_2010_16012_gb300 as gp

    assert torch.cuda.is_available()
    gp.load()
    return gp


def wheel(r):
    rim = np.arange(1, r + 1)
    return gg.from_edges(r + 1, np.concatenate([np.zeros(r, int), rim]), np.concatenate([rim, np.roll(rim, -1)]),
                         symmetrize=True)


def complete_sym(k):
    u, v = np.triu_indices(k, 1)
    return gg.from_edges(k, u, v, symmetrize=True)


ZOO = [
    lambda: complete_sym(12),
    lambda: wheel(50),
    lambda: wheel(3000),
    lambda: gg.star(2000),
    lambda: gg.binary_tree(500),
    lambda: gg.random_small(60, 0.3, seed=3, directed=False),
    lambda: gg.rmat(12, 16, seed=4),
    lambda: gg.rmat(14, 16, seed=5),
    lambda: gg.from_edges(5, np.array([], dtype=np.int64), np.array([], dtype=np.int64), symmetrize=True),
]


@pytest.mark.parametrize("gi", range(len(ZOO)))
@pytest.mark.parametrize("mode", ["push", "pull", "auto"])
def test_triangles_match_oracle(gp, gi, mode):
    g = ZOO[gi]()
    G = gp.Graph.from_graphgen(g)
    ref, rtot = oracle.OracleGraph.from_graph(g).triangles(oracle.PULL, nthreads=oracle.max_threads())
    tc, total, st = gp.triangles(G, {"push": gp.PUSH, "pull": gp.PULL, "auto": gp.AUTO}[mode])
    assert np.array_equal(tc.cpu().numpy(), ref), g.name
    assert total == rtot == st["triangles"]
    assert st["mode_used"] == (gp.PUSH if mode == "push" else gp.PULL)


@pytest.mark.parametrize("opts", [dict(push_light_max=8, chunk_edges=128), dict(push_light_max=64, chunk_edges=512),
                                  dict(push_light_max=1, chunk_edges=32)])
def test_triangles_chunk_boundaries(gp, opts):
    g = gg.rmat(13, 16, seed=6)
    G = gp.Graph.from_graphgen(g)
    G.set_options(**opts)
    ref, _ = oracle.OracleGraph.from_graph(g).triangles(oracle.PULL, nthreads=oracle.max_threads())
    for mode in (gp.PUSH, gp.PULL):
        tc, _, _ = gp.triangles(G, mode)
        assert np.array_equal(tc.cpu().numpy(), ref), (opts, mode)


def test_triangles_host_output_and_errors(gp):
    g = wheel(20)
    G = gp.Graph.from_graphgen(g)
    out = np.zeros(g.n, dtype=np.int64)
    _, total, _ = gp.triangles(G, gp.PULL, out=out)
    assert out[0] == 20 and (out[1:] == 2).all() and total == 20
    d = gp.Graph.from_graphgen(gg.rmat(8, 8, seed=7, symmetrize=False))
    with pytest.raises(gp.GpError):
        gp.triangles(d, gp.PULL)
    with pytest.raises(gp.GpError):
        gp.triangles(G, 9)
