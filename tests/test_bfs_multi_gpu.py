"""Several searches per launch (gp_bfs_multi) against the CPU oracle: each
search's levels bit for bit, its parents by rule, its summary against the
levels; every group count, sources repeated, the asynchronous form, bad input."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from helpers import check_parents_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gp():
    import torch

    import paper_2010_16012_gb300 as gp

    assert torch.cuda.is_available()
    gp.load()
    return gp


def check_all(g, O, sources, levels, parents, summary=None):
    dout = np.diff(g.csr_off)
    for i, s in enumerate(sources):
        ref, _ = O.bfs(int(s))
        lv = levels[i].cpu().numpy()
        assert np.array_equal(lv, ref), (g.name, i, int(s), np.nonzero(lv != ref)[0][:10])
        if parents is not None:
            assert check_parents_np(g.csr_off, g.csr_idx, int(s), lv, parents[i].cpu().numpy()) == 0
        if summary is not None:
            reached = lv >= 0
            assert summary[i]["reached"] == int(reached.sum())
            assert summary[i]["levels"] == int(lv.max()) + 1
            assert summary[i]["edges_reached"] == int(dout[reached].sum())


GRAPHS = [
    lambda: gg.path(70),
    lambda: gg.star(100),
    lambda: gg.random_small(50, 0.05, seed=2),
    lambda: gg.rmat(9, 8, seed=3, symmetrize=False),
    lambda: gg.erdos_renyi(3000, 9000, seed=4),
    lambda: gg.rmat(12, 16, seed=1),
]


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_multi_matches_oracle(gp, gi, mode):
    g = GRAPHS[gi]()
    G = gp.Graph.from_graphgen(g, validate=True)
    O = oracle.OracleGraph.from_graph(g)
    rng = np.random.default_rng(gi)
    sources = rng.integers(0, g.n, size=11).astype(np.int32)
    sources[3] = sources[7]  # a repeated source
    for groups in (0, 1, 3, 11, 40):
        levels, parents, summary = gp.bfs_multi(G, sources, mode, groups=groups)
        check_all(g, O, sources, levels, parents, summary)
    G.free()


def test_multi_small_options(gp):
    """Chunked hubs and the bottom-up hub pass inside groups of few blocks."""
    g = gg.rmat(12, 16, seed=5)
    G = gp.Graph.from_graphgen(g)
    G.set_options(push_light_max=0, pull_light_max=0, bfs_light_max=0, chunk_edges=32)
    O = oracle.OracleGraph.from_graph(g)
    sources = gg.pick_vertices(g, 9, seed=1)
    levels, parents, summary = gp.bfs_multi(G, sources, gp.AUTO, groups=9)
    check_all(g, O, sources, levels, parents, summary)
    G.free()


def test_multi_star_hub_sources(gp):
    """Every search from the hub or a leaf of a large star (the hub in-list
    spans many chunks), several groups at once."""
    g = gg.star(20000)
    G = gp.Graph.from_graphgen(g)
    G.set_options(chunk_edges=32)
    O = oracle.OracleGraph.from_graph(g)
    sources = np.array([0, 1, 19999, 0, 5], dtype=np.int32)
    for mode in (gp.PUSH, gp.PULL, gp.AUTO):
        levels, parents, summary = gp.bfs_multi(G, sources, mode, groups=5)
        check_all(g, O, sources, levels, parents, summary)
    G.free()


def test_multi_deep_graph(gp):
    """Searches far deeper than GP_BFS_MAX_LEVELS in several groups."""
    g = gg.path(2000)
    G = gp.Graph.from_graphgen(g)
    O = oracle.OracleGraph.from_graph(g)
    sources = np.array([0, 1999, 1000, 3], dtype=np.int32)
    levels, parents, summary = gp.bfs_multi(G, sources, gp.AUTO, groups=2)
    check_all(g, O, sources, levels, parents, summary)
    G.free()


def test_multi_async_and_equals_single(gp):
    """Two asynchronous calls in a row (no summary, no parents) and the
    single-search entry point give the same levels."""
    import torch

    g = gg.rmat(13, 16, seed=2)
    G = gp.Graph.from_graphgen(g)
    O = oracle.OracleGraph.from_graph(g)
    s1 = gg.pick_vertices(g, 6, seed=3)
    s2 = gg.pick_vertices(g, 13, seed=4)
    l1, p1, _ = gp.bfs_multi(G, s1, gp.AUTO, want_parent=False, want_summary=False)
    l2, _, _ = gp.bfs_multi(G, s2, gp.AUTO, groups=2, want_summary=False)
    torch.cuda.synchronize()
    assert p1 is None
    check_all(g, O, s1, l1, None)
    check_all(g, O, s2, l2, None)
    for i, s in enumerate(s2[:3]):
        lv, _, _ = gp.bfs(G, int(s), gp.AUTO)
        assert torch.equal(lv, l2[i])
    G.free()


def test_multi_rejects_bad_input(gp):
    import torch

    g = gg.rmat(8, 8, seed=1)
    G = gp.Graph.from_graphgen(g)
    with pytest.raises(gp.GpError) as e:
        gp.bfs_multi(G, np.array([0, g.n], dtype=np.int32))
    assert e.value.status == gp.ERR_INVALID
    with pytest.raises(gp.GpError) as e:
        gp.bfs_multi(G, np.array([0, -1], dtype=np.int32))
    assert e.value.status == gp.ERR_INVALID
    host = [torch.empty(g.n, dtype=torch.int32)]  # host memory: rejected, nothing launched
    with pytest.raises(gp.GpError) as e:
        gp.bfs_multi(G, np.array([0], dtype=np.int32), levels=host, want_parent=False)
    assert e.value.status == gp.ERR_INVALID
    with pytest.raises(gp.GpError) as e:
        gp.bfs_multi(G, np.array([0], dtype=np.int32), groups=-1)
    assert e.value.status == gp.ERR_INVALID
    levels, parents, summary = gp.bfs_multi(G, np.zeros(0, dtype=np.int32))
    assert levels == [] and summary == []
    # the graph stays usable
    O = oracle.OracleGraph.from_graph(g)
    lv, pa, sm = gp.bfs_multi(G, np.array([3], dtype=np.int32))
    check_all(g, O, [3], lv, pa, sm)
    G.free()


def test_multi_groups_option(gp):
    """groups 0 takes the graph's bfs_groups option; changing the option frees
    the multi-search workspace, which the next call sizes for the new count;
    results never depend on it.  Out-of-range values are rejected."""
    g = gg.rmat(12, 16, seed=6)
    G = gp.Graph.from_graphgen(g)
    O = oracle.OracleGraph.from_graph(g)
    sources = gg.pick_vertices(g, 13, seed=5)
    assert G.options().bfs_groups == 0  # the library's choice
    for k in (32, 1, 5, 0, 2):
        G.set_options(bfs_groups=k)
        levels, parents, summary = gp.bfs_multi(G, sources, gp.AUTO)
        check_all(g, O, sources, levels, parents, summary)
        # an explicit count still wins over the option
        levels, parents, summary = gp.bfs_multi(G, sources[:4], gp.PULL, groups=3)
        check_all(g, O, sources[:4], levels, parents, summary)
    for bad in (-1, 33):
        with pytest.raises(gp.GpError) as e:
            G.set_options(bfs_groups=bad)
        assert e.value.status == gp.ERR_INVALID
    assert G.options().bfs_groups == 2
    G.free()
