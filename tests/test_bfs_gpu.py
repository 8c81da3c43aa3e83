"""BFS parity: CUDA top-down / bottom-up / switching BFS (through the C ABI)
against the CPU oracle.  Levels must match bit for bit; parents are not unique,
so each GPU parent is checked by rule (edge exists, one level up)."""
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


def to_np(t):
    return t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)


def check(g, O, src, level, parent):
    ref, _ = O.bfs(src)
    lv = to_np(level)
    assert np.array_equal(lv, ref), (g.name, src, np.nonzero(lv != ref)[0][:10])
    if parent is not None:
        assert check_parents_np(g.csr_off, g.csr_idx, src, lv, to_np(parent)) == 0


ZOO = [
    lambda: gg.path(70),
    lambda: gg.binary_tree(300),
    lambda: gg.star(100),
    lambda: gg.cycle(65),
    lambda: gg.complete(9),
    lambda: gg.empty(3),
    lambda: gg.random_small(50, 0.05, seed=2),
    lambda: gg.rmat(9, 8, seed=3, symmetrize=False),
    lambda: gg.erdos_renyi(3000, 9000, seed=4),
    lambda: gg.rmat(12, 16, seed=1),
]
OPTS = [None, {"push_light_max": 0, "pull_light_max": 0, "bfs_light_max": 0, "chunk_edges": 32},
        {"push_light_max": 3, "chunk_edges": 32},  # BFS bins of their own (limit 32), push's at 3
        {"bfs_light_max": 3, "chunk_edges": 32},   # BFS bins at 3, push's at their default
        {"bfs_light_max": 1 << 20}]                # every frontier vertex in tiles
MODES = [0, 1, 2]


@pytest.mark.parametrize("gi", range(len(ZOO)))
@pytest.mark.parametrize("oi", range(len(OPTS)))
def test_zoo_all_modes(gp, gi, oi):
    g = ZOO[gi]()
    G = gp.Graph.from_graphgen(g, validate=True)
    if OPTS[oi]:
        G.set_options(**OPTS[oi])
    O = oracle.OracleGraph.from_graph(g)
    srcs = sorted({0, g.n - 1, g.n // 2})
    for src in srcs:
        for mode in MODES:
            lv, pa, st = gp.bfs(G, src, mode)
            check(g, O, src, lv, pa)
            assert st["reached"] == int((to_np(lv) >= 0).sum())


@pytest.mark.parametrize("seed", range(6))
def test_forced_direction_sequences(gp, seed):
    """Levels do not depend on the direction chosen at each level."""
    rng = np.random.default_rng(seed)
    g = gg.rmat(11, 8, seed=seed, symmetrize=seed % 2 == 0)
    G = gp.Graph.from_graphgen(g)
    O = oracle.OracleGraph.from_graph(g)
    src = int(gg.pick_vertices(g, 1, seed=seed)[0])
    for dirs in ([0], [1], [0, 1], [1, 0], [0, 0, 1, 1, 0], rng.integers(0, 2, size=20).tolist()):
        lv, pa, st = gp.bfs(G, src, dirs=dirs)
        check(g, O, src, lv, pa)
        L = st["levels"]
        assert st["direction"] == [dirs[min(i, len(dirs) - 1)] for i in range(L)]


def test_topdown_examines_every_reached_out_edge(gp):
    """Top-down scans each reached vertex's out-edges exactly once (Section 4.3: O(m) work)."""
    g = gg.rmat(12, 16, seed=2)
    G = gp.Graph.from_graphgen(g)
    lv, _, st = gp.bfs(G, 0, gp.PUSH)
    reached = to_np(lv) >= 0
    assert st["edges_examined"] == int(g.out_degree()[reached].sum()) == st["edges_reached"]
    _, _, st2 = gp.bfs(G, 0, gp.PULL)
    assert st2["reached"] == st["reached"]


def test_auto_switches_on_rmat(gp):
    g = gg.rmat(14, 16, seed=1)
    G = gp.Graph.from_graphgen(g)
    O = oracle.OracleGraph.from_graph(g)
    lv, pa, st = gp.bfs(G, 0, gp.AUTO)
    check(g, O, 0, lv, pa)
    assert 1 in st["direction"] and 0 in st["direction"]
    assert st["switches"] >= 1


def test_isolated_source_and_no_parent(gp):
    g = gg.rmat(10, 4, seed=5)
    iso = int(np.nonzero((g.out_degree() == 0) & (g.in_degree() == 0))[0][0])
    G = gp.Graph.from_graphgen(g)
    for mode in MODES:
        lv, pa, st = gp.bfs(G, iso, mode, want_parent=False)
        lvn = to_np(lv)
        assert pa is None and lvn[iso] == 0 and (lvn >= 0).sum() == 1 and st["levels"] == 1


def test_host_outputs(gp):
    g = gg.rmat(11, 8, seed=6)
    G = gp.Graph.from_graphgen(g)
    O = oracle.OracleGraph.from_graph(g)
    lv = np.empty(g.n, dtype=np.int32)
    pa = np.empty(g.n, dtype=np.int32)
    gp.bfs(G, 3, gp.AUTO, level=lv, parent=pa)
    check(g, O, 3, lv, pa)


def test_invalid_source(gp):
    G = gp.Graph.from_graphgen(gg.path(5))
    for src in (-1, 5):
        with pytest.raises(gp.GpError) as e:
            gp.bfs(G, src)
        assert e.value.status == gp.ERR_INVALID
    with pytest.raises(gp.GpError):
        gp.bfs(G, 0, dirs=[0, 2])


def test_async_searches_back_to_back(gp):
    """Searches enqueued without statistics return before they run; eight of
    them back to back on one stream, each into its own buffers, then a
    synchronous one."""
    import torch

    g = gg.rmat(12, 16, seed=5, symmetrize=False)
    G = gp.Graph.from_graphgen(g)
    O = oracle.OracleGraph.from_graph(g)
    srcs = gg.pick_vertices(g, 8, seed=6)
    lv = [torch.empty(g.n, dtype=torch.int32, device="cuda") for _ in srcs]
    pa = [torch.empty(g.n, dtype=torch.int32, device="cuda") for _ in srcs]
    modes = [gp.AUTO, gp.PUSH, gp.PULL, gp.AUTO] * 2
    for s, l, p, mode in zip(srcs, lv, pa, modes):
        _, _, st = gp.bfs(G, int(s), mode, level=l, parent=p, want_stats=False)
        assert st is None
    torch.cuda.synchronize()
    for s, l, p in zip(srcs, lv, pa):
        check(g, O, int(s), l, p)
    level, parent, st = gp.bfs(G, int(srcs[0]), gp.AUTO)
    check(g, O, int(srcs[0]), level, parent)
    assert st["reached"] == int((to_np(level) >= 0).sum())


def test_candidate_bitmap_after_top_down_levels(gp):
    """Bottom-up levels after top-down ones meet vertices that top-down claimed
    and vertices without in-edges (directed graph with sources-only vertices):
    every direction sequence gives the oracle's levels."""
    src_v = np.array([0, 0, 1, 2, 3, 5, 6, 6, 7, 9, 9, 10, 11], dtype=np.int64)
    dst_v = np.array([1, 2, 3, 4, 4, 6, 7, 8, 8, 10, 3, 11, 12], dtype=np.int64)
    g = gg.from_edges(40, np.concatenate([src_v, [20, 21]]), np.concatenate([dst_v, [0, 0]]))
    G = gp.Graph.from_graphgen(g)
    O = oracle.OracleGraph.from_graph(g)
    for src in (0, 20, 9, 5):
        for dirs in ([0, 1], [1, 0], [0, 0, 1], [1, 1, 0, 1], [0, 1, 0, 1, 0]):
            level, parent, _ = gp.bfs(G, src, dirs=dirs)
            check(g, O, src, level, parent)


def test_level_times_reported(gp):
    """Per-level device times: one positive entry per level, summing (with the
    start-up) to no more than the call's event time."""
    g = gg.rmat(13, 16, seed=8)
    G = gp.Graph.from_graphgen(g)
    src = int(gg.pick_vertices(g, 1, seed=9)[0])
    _, _, st = gp.bfs(G, src, gp.AUTO)
    assert len(st["level_us"]) == st["levels"] > 1
    assert all(t > 0 for t in st["level_us"]) and st["init_us"] > 0
    assert st["init_us"] + sum(st["level_us"]) <= st["ms"] * 1e3 * 1.05 + 5.0


def _grid(r, c):
    v = np.arange(r * c, dtype=np.int32).reshape(r, c)
    u = np.concatenate([v[:, :-1].ravel(), v[:-1, :].ravel()])
    w = np.concatenate([v[:, 1:].ravel(), v[1:, :].ravel()])
    return gg.from_edges(r * c, u, w, symmetrize=True, name=f"grid{r}x{c}")


DEEP = [lambda: gg.path(2000), lambda: gg.path(1500, directed=True), lambda: _grid(60, 60),
        lambda: gg.cycle(1200)]


@pytest.mark.parametrize("gi", range(len(DEEP)))
def test_deeper_than_the_level_statistics(gp, gi):
    """Searches of more than GP_BFS_MAX_LEVELS levels (paths of 1500-2000
    vertices, a 60x60 grid of depth 118 from a corner and 60 from the centre, a
    directed 1200-cycle): every mode and a forced direction sequence longer
    than the statistics arrays, levels bit-exact, parents valid, and the level
    count beyond the statistics reported."""
    g = DEEP[gi]()
    G = gp.Graph.from_graphgen(g, validate=True)
    O = oracle.OracleGraph.from_graph(g)
    srcs = [0, g.n // 2 + (30 if gi == 2 else 0)]
    rng = np.random.default_rng(gi)
    for src in srcs:
        ref, _ = O.bfs(src)
        depth = int(ref.max()) + 1
        for mode in MODES:
            lv, pa, st = gp.bfs(G, src, mode)
            check(g, O, src, lv, pa)
            assert st["levels"] == depth, (mode, st["levels"], depth)
            assert st["reached"] == int((ref >= 0).sum())
        dirs = rng.integers(0, 2, size=depth + 40).astype(np.int8)
        lv, pa, st = gp.bfs(G, src, dirs=dirs)
        check(g, O, src, lv, pa)
        k = min(depth, gp.BFS_MAX_LEVELS)
        assert list(st["direction"][:k]) == list(dirs[:k])
        # the oracle's level-synchronous search with the same sequence
        ref2, _, used = O.bfs_levelsync(src, dirs=dirs)
        assert np.array_equal(to_np(lv), ref2)


def test_forced_directions_beyond_512_levels_are_used(gp):
    """On a 1500-vertex path from vertex 0, levels 600-1499 forced to bottom-up
    scan in-edges, top-down ones out-edges: the edges examined tell which
    direction each level beyond the statistics took."""
    g = gg.path(1500)
    G = gp.Graph.from_graphgen(g)
    O = oracle.OracleGraph.from_graph(g)
    depth = 1500
    td = np.zeros(depth, dtype=np.int8)
    mixed = td.copy()
    mixed[600:] = 1
    _, _, s_td = gp.bfs(G, 0, dirs=td)
    lv, pa, s_mx = gp.bfs(G, 0, dirs=mixed)
    check(g, O, 0, lv, pa)
    # a top-down level of a path examines its frontier's 1-2 out-edges; a
    # bottom-up level examines the in-edges of every unvisited vertex until a hit
    assert s_mx["edges_examined"] > s_td["edges_examined"] + 100000, (s_mx["edges_examined"], s_td["edges_examined"])


@pytest.mark.parametrize("src", [1, 32, 33, 64, 65, 200, 256, 257, 4095, 5000])
@pytest.mark.parametrize("chunk", [256, 32])
def test_bottom_up_hub(gp, src, chunk):
    """Star with 5000 leaves from leaf `src`, bottom-up: the centre is a hub
    candidate whose one frontier in-neighbour sits at position src - 1 of its
    in-list.  Within the first 64 in-edges (the lane's probe) the centre's own
    lane finds it and the level examines every other leaf's single in-edge plus
    the centre's first src; further out the lane gives up after 64 and the
    centre's in-edge chunks are scanned across the grid, which examines each
    edge at most once more."""
    g = gg.star(5000)
    G = gp.Graph.from_graphgen(g)
    G.set_options(chunk_edges=chunk)
    O = oracle.OracleGraph.from_graph(g)
    lv, pa, st = gp.bfs(G, src, dirs=[1])
    check(g, O, src, lv, pa)
    assert int(to_np(pa)[0]) == src
    if src <= 64:
        assert st["examined"][0] == (5000 - 1) + src
    else:
        assert (5000 - 1) + 64 + (src - 1) % chunk < st["examined"][0] <= (5000 - 1) + 64 + 5000


def test_bottom_up_hubs_on_rmat(gp):
    """Forced bottom-up from R-MAT sources (every hub scans its whole in-list at
    the first levels, so the chunk pass runs) with several chunk sizes and pull
    light limits: levels bit-exact and parents valid."""
    g = gg.rmat(14, 16, seed=6)
    G = gp.Graph.from_graphgen(g)
    O = oracle.OracleGraph.from_graph(g)
    srcs = gg.pick_vertices(g, 3, seed=7)
    for opts in ({}, {"chunk_edges": 32}, {"pull_light_max": 200}, {"pull_light_max": 0, "chunk_edges": 64}):
        if opts:
            G.set_options(**opts)
        for src in srcs:
            for dirs in ([1], [1, 1, 0], [0, 1]):
                lv, pa, _ = gp.bfs(G, int(src), dirs=dirs)
                check(g, O, int(src), lv, pa)


def test_bfs_light_limit_changes_between_searches(gp):
    """The top-down bins follow bfs_light_max from one search to the next
    (workspaces re-sized for the new chunk count), for single and grouped
    searches; out-of-range values are rejected and leave the options as they were."""
    g = gg.rmat(12, 16, seed=6)
    G = gp.Graph.from_graphgen(g)
    O = oracle.OracleGraph.from_graph(g)
    srcs = gg.pick_vertices(g, 5, seed=3)
    for lim in (32, 1, 0, 1 << 20, 8):
        G.set_options(bfs_light_max=lim)
        for s in srcs[:2]:
            lv, pa, _ = gp.bfs(G, int(s), gp.PUSH)
            check(g, O, int(s), lv, pa)
        levels, parents, _ = gp.bfs_multi(G, srcs, gp.AUTO, groups=3)
        for i, s in enumerate(srcs):
            check(g, O, int(s), levels[i], parents[i])
    before = gp.options_dict(G.options())
    for bad in (-1, (1 << 20) + 1):
        with pytest.raises(gp.GpError) as e:
            G.set_options(bfs_light_max=bad)
        assert e.value.status == gp.ERR_INVALID
    assert gp.options_dict(G.options()) == before
    G.free()
