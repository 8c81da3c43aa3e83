"""Batched personalised PageRank and multi-source BFS (one persistent launch
over several graphs, replayed from a CUDA graph) against the CPU oracle and
against the one-at-a-time entry points: every PPR vector within max-abs 1e-6 /
L1 1e-5 of the oracle at its own sweep count, every BFS level bit-exact."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

MAX_ABS, L1 = 1e-6, 1e-5


@pytest.fixture(scope="module")
def gp():
    import torch

    import paper_2010_16012_gb300 as gp

    assert torch.cuda.is_available()
    gp.load()
    return gp


def uneven_graphs():
    return [gg.rmat(9, 16, seed=41), gg.rmat(11, 8, seed=42, symmetrize=False),
            gg.rmat(12, 16, seed=43).with_weights(44), gg.star(300), gg.path(77)]


def seeds_for(g, k, seed):
    s = gg.pick_vertices(g, min(k, int((g.out_degree() > 0).sum())), seed=seed)
    return np.resize(s, k).astype(np.int32)


@pytest.mark.parametrize("k", [32, 256])
@pytest.mark.parametrize("start", [1, 0])
def test_ppr_batched_matches_oracle(gp, k, start):
    """Both start vectors: each seed's one-hot vector (the default) and 1/n; the
    oracle runs from the same start."""
    graphs = uneven_graphs()
    G = [gp.Graph.from_graphgen(g) for g in graphs]
    B = gp.Batch(G, k_ppr=k)
    B.set_options(ppr_start=start)
    seeds = np.stack([seeds_for(g, k, 50 + i) for i, g in enumerate(graphs)])
    outs, done, st = B.ppr(seeds, damping=0.85, iters=500, tol=1e-6)
    assert st["sweeps"] == done.max() and done.min() >= 1
    rng = np.random.default_rng(0)
    for i, g in enumerate(graphs):
        X = outs[i].cpu().numpy()
        O = oracle.OracleGraph.from_graph(g)
        for j in sorted(set(rng.choice(k, size=min(k, 12), replace=False).tolist()) | {0, k - 1}):
            e = np.zeros(g.n)
            e[seeds[i, j]] = 1.0
            x0 = e if start else None
            ref, kk, r, _ = O.pagerank(oracle.PULL, 0.85, iters=int(done[i, j]), personalization=e, x0=x0)
            err = np.abs(X[:, j].astype(np.float64) - ref)
            assert err.max() <= MAX_ABS and err.sum() <= L1, (i, j, err.max(), err.sum())
            # it stopped at the first sweep where the change fell below tol, up to the
            # rounding of FP32 iterates: each sweep rounds every y_v by half an ulp,
            # so an iterate carries up to 2^-24 * sum(y) / (1 - d) ~ 4e-7 of L1 error
            # (values sum to at most 1), and the difference of two iterates twice that
            # (reached on a star, whose alternating mode decays slowest)
            rho = 8e-7
            kd = int(done[i, j])
            assert r < 1e-6 + rho, (i, j, kd, r)
            if kd > 1:
                _, _, r_prev, _ = O.pagerank(oracle.PULL, 0.85, iters=kd - 1, personalization=e, x0=x0)
                assert r_prev >= 1e-6 - rho, (i, j, kd, r_prev)
    B.free()


@pytest.mark.parametrize("pack", [1, 16, 128])
def test_ppr_batched_packed_columns(gp, pack):
    """Columns a job leaves to packed jobs (ppr_pack: 1, the default 16, and
    128, which hands every column still iterating after the first sweep to
    packed jobs) finish as the oracle does: each sampled vector within the
    tolerance at its own sweep count, stopped at the oracle's first sweep under
    tol (up to FP32 rounding: a packed job splits a column's sums over more
    edge groups than its slice did, so its stop sweep can move within that
    rounding window, as any change of the summation order can)."""
    graphs = uneven_graphs() + [gg.rmat(13, 16, seed=46)]
    G = [gp.Graph.from_graphgen(g) for g in graphs]
    k = 128
    B = gp.Batch(G, k_ppr=k)
    seeds = np.stack([seeds_for(g, k, 210 + i) for i, g in enumerate(graphs)])
    B.set_options(ppr_pack=0)
    _, _, st0 = B.ppr(seeds, iters=500, tol=1e-6)
    assert st0["packed"] == 0
    B.set_options(ppr_pack=pack)
    assert B.options()["ppr_pack"] == pack
    outs, done, st = B.ppr(seeds, iters=500, tol=1e-6)
    assert st["packed"] > 0 and st["sweeps"] == done.max()
    rng = np.random.default_rng(pack)
    rho = 8e-7
    for i, g in enumerate(graphs):
        O = oracle.OracleGraph.from_graph(g)
        X = outs[i].cpu().numpy()
        # the slowest columns (those most likely packed) and a few others
        slow = np.argsort(done[i])[-6:].tolist()
        for j in sorted(set(slow) | {0, k - 1, int(rng.integers(k))}):
            e = np.zeros(g.n)
            e[seeds[i, j]] = 1.0
            kd = int(done[i, j])
            ref, _, r, _ = O.pagerank(oracle.PULL, 0.85, iters=kd, personalization=e, x0=e)
            err = np.abs(X[:, j].astype(np.float64) - ref)
            assert err.max() <= MAX_ABS and err.sum() <= L1, (pack, i, j, err.max(), err.sum())
            assert r < 1e-6 + rho, (pack, i, j, kd, r)
            if kd > 1:
                _, _, r_prev, _ = O.pagerank(oracle.PULL, 0.85, iters=kd - 1, personalization=e, x0=e)
                assert r_prev >= 1e-6 - rho, (pack, i, j, kd, r_prev)
    # the cap holds for packed columns too
    B.set_options(ppr_pack=128)
    _, done_c, st_c = B.ppr(seeds, iters=3, tol=1e-6)
    assert done_c.max() <= 3 and st_c["sweeps"] <= 3
    B.free()


@pytest.mark.parametrize("k", [64, 128])
def test_ppr_batched_matches_serial(gp, k):
    import torch

    graphs = [gg.rmat(10, 16, seed=61), gg.rmat(8, 16, seed=62)]
    G = [gp.Graph.from_graphgen(g) for g in graphs]
    B = gp.Batch(G, k_ppr=k)
    seeds = np.stack([seeds_for(g, k, 70 + i) for i, g in enumerate(graphs)])
    outs, done, _ = B.ppr(seeds, iters=500, tol=1e-6)
    for i, g in enumerate(graphs):
        for j in (0, 7, k - 1):
            e = torch.zeros(g.n, device="cuda")
            e[int(seeds[i, j])] = 1.0
            x, st = gp.pagerank(G[i], gp.PULL, 0.85, int(done[i, j]), 0.0, personalization=e, x0=e)
            err = (outs[i][:, j] - x).abs()
            assert float(err.max()) <= MAX_ABS, (i, j)


def test_ppr_batched_replay_with_new_seeds(gp):
    graphs = [gg.rmat(9, 8, seed=81), gg.rmat(10, 8, seed=82)]
    G = [gp.Graph.from_graphgen(g) for g in graphs]
    B = gp.Batch(G, k_ppr=32)
    for rep in range(3):
        seeds = np.stack([seeds_for(g, 32, 90 + 10 * rep + i) for i, g in enumerate(graphs)])
        outs, done, _ = B.ppr(seeds, iters=300, tol=1e-6)
        for i, g in enumerate(graphs):
            O = oracle.OracleGraph.from_graph(g)
            j = rep * 5
            e = np.zeros(g.n)
            e[seeds[i, j]] = 1.0
            ref, _, _, _ = O.pagerank(oracle.PULL, 0.85, iters=int(done[i, j]), personalization=e, x0=e)
            assert np.abs(outs[i][:, j].cpu().numpy() - ref).max() <= MAX_ABS


@pytest.mark.parametrize("nsrc", [64, 5])
def test_msbfs_batched_matches_oracle(gp, nsrc):
    graphs = uneven_graphs() + [gg.erdos_renyi(2000, 6000, seed=91), gg.empty(3)]
    G = [gp.Graph.from_graphgen(g) for g in graphs]
    B = gp.Batch(G, k_ppr=32)
    srcs = []
    for i, g in enumerate(graphs):
        s = gg.pick_vertices(g, nsrc, seed=100 + i, min_out_degree=0)
        srcs.append(np.resize(s, nsrc))
    srcs = np.stack(srcs).astype(np.int32)
    outs, st = B.msbfs(srcs)
    for i, g in enumerate(graphs):
        L = outs[i].cpu().numpy()
        O = oracle.OracleGraph.from_graph(g)
        for j in range(nsrc):
            ref, _ = O.bfs(int(srcs[i, j]))
            assert np.array_equal(L[:, j], ref), (i, j)
        assert (L[:, nsrc:] == -1).all()
    # replay through the captured graph with other sources
    outs2, _ = B.msbfs(srcs[:, ::-1].copy())
    for i, g in enumerate(graphs):
        O = oracle.OracleGraph.from_graph(g)
        ref, _ = O.bfs(int(srcs[i, -1]))
        assert np.array_equal(outs2[i].cpu().numpy()[:, 0], ref)


def test_batched_rejects_bad_input(gp):
    G = [gp.Graph.from_graphgen(gg.path(10))]
    with pytest.raises(gp.GpError):
        gp.Batch(G, k_ppr=48)
    B = gp.Batch(G, k_ppr=32)
    with pytest.raises(gp.GpError):
        B.ppr(np.full((1, 32), 10, dtype=np.int32))
    with pytest.raises(gp.GpError):
        B.msbfs(np.full((1, 3), -1, dtype=np.int32))


BATCH_OPTS = [{"big_in_degree": 8, "chunk_edges": 32, "l2_budget_mb": 1},  # many chunks, 32-column jobs
              {"big_in_degree": 0, "chunk_edges": 64},                   # every vertex chunked
              {"big_in_degree": 100000, "l2_budget_mb": 4096},           # nothing chunked, widest slices
              {"msbfs_alpha": 1e-6},                                     # BFS stays top-down
              {"msbfs_alpha": 1e6, "msbfs_beta": 1e-6}]                  # BFS bottom-up from level 1 on


@pytest.mark.parametrize("oi", range(len(BATCH_OPTS)))
def test_batch_options_do_not_change_results(gp, oi):
    """Every batch option value gives the oracle's results: PPR vectors within
    the tolerance at their sweep counts (whatever the column slices and chunk
    layout), BFS levels bit-exact (whatever mix of top-down and bottom-up)."""
    graphs = uneven_graphs() + [gg.rmat(13, 16, seed=45)]
    G = [gp.Graph.from_graphgen(g) for g in graphs]
    k = 128
    B = gp.Batch(G, k_ppr=k)
    B.set_options(**BATCH_OPTS[oi])
    assert {kk: B.options()[kk] for kk in BATCH_OPTS[oi]} == pytest.approx(BATCH_OPTS[oi])
    seeds = np.stack([seeds_for(g, k, 150 + i) for i, g in enumerate(graphs)])
    outs, done, st = B.ppr(seeds, iters=500, tol=1e-6)
    # a graph's slice is the widest of 128, 64, 32 columns whose two iterates fit the budget
    budget = B.options()["l2_budget_mb"] << 20

    def width(n):
        return next((w for w in (128, 64) if w <= k and 2 * n * w * 4 <= budget), 32)

    assert st["jobs"] == sum(k // width(g.n) for g in graphs)
    rng = np.random.default_rng(oi)
    for i, g in enumerate(graphs):
        O = oracle.OracleGraph.from_graph(g)
        X = outs[i].cpu().numpy()
        for j in sorted({0, 31, 32, 63, 64, k - 1, int(rng.integers(k))}):
            e = np.zeros(g.n)
            e[seeds[i, j]] = 1.0
            ref, _, _, _ = O.pagerank(oracle.PULL, 0.85, iters=int(done[i, j]), personalization=e, x0=e)
            err = np.abs(X[:, j].astype(np.float64) - ref)
            assert err.max() <= MAX_ABS and err.sum() <= L1, (oi, i, j, err.max(), err.sum())
    srcs = np.stack([np.resize(gg.pick_vertices(g, 64, seed=170 + i, min_out_degree=0), 64)
                     for i, g in enumerate(graphs)]).astype(np.int32)
    louts, _ = B.msbfs(srcs)
    for i, g in enumerate(graphs):
        O = oracle.OracleGraph.from_graph(g)
        L = louts[i].cpu().numpy()
        for j in (0, 17, 63):
            ref, _ = O.bfs(int(srcs[i, j]))
            assert np.array_equal(L[:, j], ref), (oi, i, j)
    B.free()


def test_batch_option_validation(gp):
    B = gp.Batch([gp.Graph.from_graphgen(gg.path(10))], k_ppr=32)
    for bad in ({"chunk_edges": 8}, {"l2_budget_mb": 0}, {"msbfs_alpha": 0.0}, {"big_in_degree": -1}, {"ppr_start": 2},
                {"ppr_pack": -1}, {"ppr_pack": 129}):
        with pytest.raises(gp.GpError):
            B.set_options(**bad)


def test_batch_autotune(gp):
    """The tuner installs one of its candidates per axis and the results stay
    the oracle's."""
    graphs = uneven_graphs()
    G = [gp.Graph.from_graphgen(g) for g in graphs]
    k = 64
    B = gp.Batch(G, k_ppr=k)
    seeds = np.stack([seeds_for(g, k, 200 + i) for i, g in enumerate(graphs)])
    srcs = np.stack([np.resize(gg.pick_vertices(g, 64, seed=210 + i, min_out_degree=0), 64)
                     for i, g in enumerate(graphs)]).astype(np.int32)
    r = B.autotune(seeds, srcs, ppr_sweeps=4)
    o = r["options"]
    assert r["trials"] == 5 + 3 + 5 + 6 + 3 and r["ppr_ms"] > 0 and r["msbfs_ms"] > 0
    assert o["big_in_degree"] in (8, 16, 32, 64, 128) and o["chunk_edges"] in (64, 128, 256)
    assert o["l2_budget_mb"] in (48, 64, 96, 128, 192) and o["msbfs_alpha"] in (2, 4, 8, 16, 32, 64)
    assert o["msbfs_beta"] in (8, 24, 64) and B.options() == o
    outs, done, _ = B.ppr(seeds, iters=500, tol=1e-6)
    louts, _ = B.msbfs(srcs)
    for i, g in enumerate(graphs):
        O = oracle.OracleGraph.from_graph(g)
        for j in (0, k - 1):
            e = np.zeros(g.n)
            e[seeds[i, j]] = 1.0
            ref, _, _, _ = O.pagerank(oracle.PULL, 0.85, iters=int(done[i, j]), personalization=e, x0=e)
            assert np.abs(outs[i][:, j].cpu().numpy() - ref).max() <= MAX_ABS
            lref, _ = O.bfs(int(srcs[i, j]))
            assert np.array_equal(louts[i].cpu().numpy()[:, j], lref)
