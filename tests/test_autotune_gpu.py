"""gp_autotune picks options from its candidate sets by timing them, leaves them on
the graph, and the results afterwards still match the oracle."""
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


def test_autotune_and_cache(gp, tmp_path):
    g = gg.rmat(13, 16, seed=3)
    G = gp.Graph.from_graphgen(g)
    srcs = gg.pick_vertices(g, 4, seed=9)
    path = str(tmp_path / "tune.json")
    r = gp.autotune(G, gp.TUNE_ALL, sources=srcs, cache=path)
    o = r["options"]
    assert not r["cached"] and r["evaluated"] >= 10
    assert o["pull_light_max"] in (8, 16, 32) and o["chunk_edges"] in (128, 256, 512)
    assert o["pull_hot_slots"] in (0, 8192, 16384, 20480, 24576) and o["push_light_max"] in (8, 16, 32, 64)
    assert o["pr_auto_mode"] in (gp.PUSH, gp.PULL) and o["bfs_alpha"] in (4, 8, 14, 24, 48)
    assert o["bfs_light_max"] in (8, 16, 32, 64, 128) and o["bfs_groups"] in (0, 1, 2, 4, 8, 32)
    assert gp.options_dict(G.options()) == o
    # results with the tuned options
    O = oracle.OracleGraph.from_graph(g)
    ref, _, _, _ = O.pagerank(oracle.PULL, 0.85, iters=15)
    for mode in (gp.PULL, gp.PUSH, gp.AUTO):
        x, st = gp.pagerank(G, mode, 0.85, 15)
        assert np.abs(x.cpu().numpy() - ref).max() <= 1e-6
        if mode == gp.AUTO:
            assert st["mode_used"] == o["pr_auto_mode"]
    lref, _ = O.bfs(int(srcs[0]))
    lv, _, _ = gp.bfs(G, int(srcs[0]), gp.AUTO)
    assert np.array_equal(lv.cpu().numpy(), lref)
    lvs, _, _ = gp.bfs_multi(G, srcs, gp.AUTO)  # the tuned group count
    for i, s in enumerate(srcs):
        assert np.array_equal(lvs[i].cpu().numpy(), O.bfs(int(s))[0])
    # a second graph handle of the same graph takes the cached options without timing
    G2 = gp.Graph.from_graphgen(g)
    r2 = gp.autotune(G2, gp.TUNE_ALL, sources=srcs, cache=path)
    assert r2["cached"] and r2["options"] == o and gp.options_dict(G2.options()) == o
