"""Betweenness centrality (gp_bc, Brandes with push/pull steps) against the
oracle's sequential Brandes.

Both sides compute in FP64; path counts are integer sums (exact below 2^53),
the dependencies sums of positive terms in a different order, so the results
agree to a relative 1e-9 (well above the ~1e-15 x depth rounding of either)."""
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


def grid(r, c):
    v = np.arange(r * c).reshape(r, c)
    u = np.concatenate([v[:, :-1].ravel(), v[:-1, :].ravel()])
    w = np.concatenate([v[:, 1:].ravel(), v[1:, :].ravel()])
    return gg.from_edges(r * c, u, w, symmetrize=True, name=f"grid{r}x{c}")


def bipartite(a, b):
    u, v = np.meshgrid(np.arange(a), a + np.arange(b), indexing="ij")
    return gg.from_edges(a + b, u.ravel(), v.ravel(), symmetrize=True, name=f"K{a},{b}")


def multi_edges():
    rng = np.random.default_rng(11)
    src = rng.integers(0, 300, size=3000)
    dst = rng.integers(0, 300, size=3000)
    return gg.from_edges(300, src, dst, drop_self=False, dedup=False, name="multi")


ZOO = [
    lambda: gg.rmat(10, 8, seed=1),
    lambda: gg.rmat(11, 16, seed=2, symmetrize=False),
    lambda: gg.star(3000),
    lambda: gg.path(300),
    lambda: gg.path(200, directed=True),
    lambda: gg.erdos_renyi(4000, 20000, seed=5),
    lambda: grid(40, 40),
    lambda: bipartite(3, 1500),
    lambda: multi_edges(),
    lambda: gg.binary_tree(1000),
    lambda: gg.empty(50),
]

MODES = ["push", "pull", "auto"]


def close(x, ref):
    x = np.asarray(x, dtype=np.float64)
    scale = max(1.0, float(np.abs(ref).max()) if ref.size else 1.0)
    err = np.abs(x - ref)
    assert np.all(err <= 1e-9 * np.maximum(np.abs(ref), 1e-3 * scale)), (err.max(), scale)


def sources_for(g, count, seed):
    if g.n <= count:
        return np.arange(g.n, dtype=np.int32)
    return np.random.default_rng(seed).choice(g.n, size=count, replace=False).astype(np.int32)


@pytest.mark.parametrize("gi", range(len(ZOO)))
@pytest.mark.parametrize("mode", MODES)
def test_bc_matches_oracle(gp, gi, mode):
    g = ZOO[gi]()
    G = gp.Graph.from_graphgen(g)
    O = oracle.OracleGraph.from_graph(g)
    src = sources_for(g, 256, seed=gi)
    m = {"push": gp.PUSH, "pull": gp.PULL, "auto": gp.AUTO}[mode]
    x, st = gp.bc(G, src, m)
    ref = O.bc(src)
    close(x.cpu().numpy(), ref)
    assert st["sources"] == len(src)
    if mode == "push":
        assert st["pulls"] == 0
    if mode == "pull":
        assert st["pushes"] == 0


def test_bc_step_record(gp):
    g = gg.rmat(12, 16, seed=3, symmetrize=False)
    G = gp.Graph.from_graphgen(g)
    O = oracle.OracleGraph.from_graph(g)
    s = int(gg.pick_vertices(g, 1, seed=4)[0])
    lv, _ = O.bfs(s)
    L = int(lv.max())
    _, st = gp.bc(G, [s], gp.AUTO)
    assert st["steps"] == 2 * L + 1 and st["levels"] == L + 1
    assert st["phase"] == [0] * (L + 1) + [1] * L
    assert st["level"] == list(range(L + 1)) + list(range(L, 0, -1))
    sizes = np.bincount(lv[lv >= 0], minlength=L + 1)
    assert st["frontier"][: L + 1] == list(sizes)
    assert st["frontier"][L + 1:] == list(sizes[L:0:-1])
    assert st["reached"] == int((lv >= 0).sum())
    # forward push examines the frontier's out-edges, forward pull the unvisited vertices' in-edges
    outdeg = g.out_degree()
    for i in range(L + 1):
        if st["direction"][i] == gp.PUSH:
            assert st["examined"][i] == int(outdeg[lv == i].sum())
    assert sum(st["examined"]) == st["edges_examined"]


def test_bc_forced_directions(gp):
    g = gg.rmat(11, 8, seed=6, symmetrize=False)
    G = gp.Graph.from_graphgen(g)
    O = oracle.OracleGraph.from_graph(g)
    src = sources_for(g, 64, seed=7)
    ref = O.bc(src)
    rng = np.random.default_rng(8)
    for dirs in ([0, 1], [1, 0, 0, 1], list(rng.integers(0, 2, size=40))):
        x, st = gp.bc(G, src, gp.AUTO, dirs=dirs)
        close(x.cpu().numpy(), ref)
        k = min(len(dirs), st["steps"])
        assert st["direction"][:k] == [int(d) for d in dirs[:k]]


def test_bc_more_sources_than_a_launch(gp):
    g = gg.erdos_renyi(5000, 15000, seed=9)
    G = gp.Graph.from_graphgen(g)
    src = np.arange(g.n, dtype=np.int32)  # exact centrality: every vertex a source
    x, st = gp.bc(G, src, gp.AUTO)
    close(x.cpu().numpy(), oracle.OracleGraph.from_graph(g).bc(src))
    assert st["sources"] == g.n


def test_bc_repeated_sources_device_inputs_and_host_output(gp):
    import torch

    g = gg.rmat(10, 16, seed=10)
    G = gp.Graph.from_graphgen(g)
    O = oracle.OracleGraph.from_graph(g)
    src = np.array([3, 3, 17, 900, 3], dtype=np.int32)
    ref = O.bc(src)
    out = np.full(g.n, np.nan)
    gp.bc(G, src, gp.AUTO, out=out)
    close(out, ref)
    x, st = gp.bc(G, torch.from_numpy(src).cuda(), gp.PULL, want_stats=False)  # enqueued only
    torch.cuda.synchronize()
    close(x.cpu().numpy(), ref)
    x, st = gp.bc(G, [], gp.AUTO)
    assert not x.cpu().numpy().any() and st["sources"] == 0


def test_bc_closed_forms(gp):
    n = 64
    G = gp.Graph.from_graphgen(gg.path(n))
    x, _ = gp.bc(G, np.arange(n, dtype=np.int32), gp.AUTO)
    assert np.array_equal(x.cpu().numpy(), [2.0 * i * (n - 1 - i) for i in range(n)])
    k = 2000
    G = gp.Graph.from_graphgen(gg.star(k))
    for mode in (gp.PUSH, gp.PULL):
        x, _ = gp.bc(G, np.arange(k + 1, dtype=np.int32), mode)
        h = x.cpu().numpy()
        assert h[0] == k * (k - 1) and not h[1:].any()


def test_bc_bad_input(gp):
    import torch

    G = gp.Graph.from_graphgen(gg.rmat(8, 8, seed=12))
    for kw in (dict(sources=[G.n]), dict(sources=[-1]), dict(mode=7), dict(dirs=[0, 2])):
        args = dict(sources=[0, 1], mode=gp.AUTO)
        args.update(kw)
        with pytest.raises(gp.GpError):
            gp.bc(G, **args)
    with pytest.raises(gp.GpError):  # checked by the kernel for device sources
        gp.bc(G, torch.tensor([0, G.n + 5], dtype=torch.int32, device="cuda"), gp.AUTO)
    x, _ = gp.bc(G, [0, 1], gp.AUTO)  # the graph stays usable
    close(x.cpu().numpy(), oracle.OracleGraph.from_graph(gg.rmat(8, 8, seed=12)).bc([0, 1]))


def test_bc_async_error_reported_by_next_call(gp):
    import torch

    g = gg.rmat(9, 8, seed=13)
    G = gp.Graph.from_graphgen(g)
    out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    bad = torch.tensor([1, g.n + 3], dtype=torch.int32, device="cuda")
    gp.bc(G, bad, gp.AUTO, out=out, want_stats=False)  # enqueued: the kernel finds the bad source
    with pytest.raises(gp.GpError, match="previous asynchronous"):
        gp.bc(G, [0], gp.AUTO)
    x, _ = gp.bc(G, [0, 1], gp.AUTO)  # and the graph works afterwards
    close(x.cpu().numpy(), oracle.OracleGraph.from_graph(g).bc([0, 1]))
