"""Delta-Stepping SSSP (gp_sssp, through the C ABI) against the FP64 Dijkstra
oracle.  Integer-valued weights keep every path sum exact in FP32, so distances
must match bit for bit; the predecessor must be the smallest vertex with a
tight edge into the vertex (unique whatever the order of relaxations).  Every
mode, bucket widths from Dijkstra-like to Bellman-Ford-like, forced per-
iteration direction sequences, hubs above every chunk threshold, unweighted
graphs (= BFS levels) and non-integer weights (within FP32 rounding)."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from helpers import check_sssp_certificate, parse_sssp_cases, smallest_tight_pred

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gp():
    import torch

    import paper_2010_16012_gb300 as gp

    assert torch.cuda.is_available()
    gp.load()
    return gp


def np_(t):
    return t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)


def check(g, O, src, dist, pred):
    ref, _ = O.sssp(src)
    d = np_(dist)
    assert np.array_equal(d.astype(np.float64), ref), (g.name, src, np.nonzero(d.astype(np.float64) != ref)[0][:8])
    if pred is not None:
        want = smallest_tight_pred(g.csr_off, g.csr_idx, g.csr_w, src, d)
        assert np.array_equal(np_(pred).astype(np.int64), want), (g.name, src)


def weighted(g, seed, hi=64):
    return gg.with_int_weights(g, seed=seed, lo=1, hi=hi)


ZOO = [
    lambda: weighted(gg.path(50), 1),
    lambda: weighted(gg.star(300), 2),
    lambda: weighted(gg.star(5000), 3),
    lambda: weighted(gg.binary_tree(200), 4),
    lambda: weighted(gg.rmat(10, 8, seed=5, symmetrize=False), 6),
    lambda: weighted(gg.rmat(12, 16, seed=7), 8, hi=255),
    lambda: weighted(gg.erdos_renyi(3000, 12000, seed=9), 10),
    lambda: gg.with_int_weights(gg.rmat(11, 8, seed=11), seed=12, lo=0, hi=3),  # zero weights
]


@pytest.mark.parametrize("gi", range(len(ZOO)))
@pytest.mark.parametrize("mode", ["push", "pull", "auto"])
def test_sssp_matches_oracle(gp, gi, mode):
    g = ZOO[gi]()
    G = gp.Graph.from_graphgen(g)
    O = oracle.OracleGraph.from_graph(g)
    m = {"push": gp.PUSH, "pull": gp.PULL, "auto": gp.AUTO}[mode]
    for src in gg.pick_vertices(g, 3, seed=40 + gi):
        for delta in (1.0, 16.0, 1e7):
            dist, pred, st = gp.sssp(G, int(src), delta, m)
            check(g, O, int(src), dist, pred)
            assert st["pushes"] + st["pulls"] == st["iterations"] >= st["epochs"] >= 1
            assert st["reached"] == int(np.isfinite(np_(dist)).sum())
            if mode == "push":
                assert st["pulls"] == 0
            if mode == "pull":
                assert st["pushes"] == 0


def test_sssp_forced_direction_sequences(gp):
    g = weighted(gg.rmat(11, 16, seed=13, symmetrize=False), 14)
    G = gp.Graph.from_graphgen(g)
    O = oracle.OracleGraph.from_graph(g)
    rng = np.random.default_rng(15)
    src = int(gg.pick_vertices(g, 1, seed=16)[0])
    for dirs in ([0, 1], [1, 0], [0, 0, 1, 1], list(rng.integers(0, 2, size=64)), list(rng.integers(0, 2, size=7))):
        dist, pred, st = gp.sssp(G, src, 8.0, gp.AUTO, dirs=dirs)
        check(g, O, src, dist, pred)
        L = min(len(st["direction"]), len(dirs))
        assert st["direction"][:L] == [int(x) for x in dirs[:L]]


def test_sssp_worked_example(gp):
    n, s, d, w, cases = parse_sssp_cases()
    order = np.lexsort((np.array(d), np.array(s)))
    base = gg.from_edges(n, np.array(s), np.array(d), dedup=False)
    wc = np.array(w, dtype=np.float32)[order]
    g = gg.Graph("golden", n, base.csr_off, base.csr_idx, base.csc_off, base.csc_idx, False, wc,
                 np.ascontiguousarray(wc[gg._transpose_perm(base)]))
    G = gp.Graph.from_graphgen(g)
    for src, dist, pred in cases:
        for mode in (gp.PUSH, gp.PULL, gp.AUTO):
            got, p, _ = gp.sssp(G, src, 2.0, mode)
            assert np.array_equal(np_(got), np.array(dist, dtype=np.float32))
            assert list(np_(p)) == pred


def test_sssp_unweighted_is_bfs(gp):
    g = gg.rmat(11, 8, seed=17, symmetrize=False)
    G = gp.Graph.from_graphgen(g)
    O = oracle.OracleGraph.from_graph(g)
    for src in gg.pick_vertices(g, 3, seed=18):
        dist, _, _ = gp.sssp(G, int(src), 1.0, gp.AUTO, want_pred=False)
        lv, _ = O.bfs(int(src))
        d = np_(dist)
        assert np.array_equal(np.where(np.isfinite(d), d, -1).astype(np.int64), lv.astype(np.int64))


def test_sssp_float_weights(gp):
    """Non-integer weights: each sum is rounded in FP32 as it is formed, so the
    distances agree with the FP64 oracle to FP32 rounding along the path, and
    the certificate holds exactly on the FP32 sums."""
    g = gg.rmat(11, 16, seed=19).with_weights(20, normalize=False)
    G = gp.Graph.from_graphgen(g)
    O = oracle.OracleGraph.from_graph(g)
    for src in gg.pick_vertices(g, 2, seed=21):
        dist, pred, _ = gp.sssp(G, int(src), 0.25, gp.AUTO)
        ref, _ = O.sssp(int(src))
        d = np_(dist).astype(np.float64)
        fin = np.isfinite(ref)
        assert np.array_equal(np.isfinite(d), fin)
        assert np.all(np.abs(d[fin] - ref[fin]) <= 1e-5 * np.maximum(ref[fin], 1e-3))
        assert check_sssp_certificate(g.csr_off, g.csr_idx, g.csr_w, int(src), np_(dist), np_(pred)) == 0


def test_sssp_host_buffers_and_unreachable(gp):
    g = weighted(gg.from_edges(6, np.array([0, 1, 3]), np.array([1, 2, 4])), 22)
    G = gp.Graph.from_graphgen(g)
    O = oracle.OracleGraph.from_graph(g)
    dist = np.zeros(6, dtype=np.float32)
    pred = np.zeros(6, dtype=np.int32)
    gp.sssp(G, 0, 4.0, gp.AUTO, dist=dist, pred=pred)
    check(g, O, 0, dist, pred)
    assert np.isinf(dist[3:]).all() and (pred[3:] == -1).all()


def test_sssp_rejects_bad_input(gp):
    g = weighted(gg.path(10), 23)
    G = gp.Graph.from_graphgen(g)
    for args in ((-1, 1.0, gp.AUTO), (10, 1.0, gp.AUTO), (0, 0.0, gp.AUTO), (0, float("nan"), gp.AUTO),
                 (0, float("inf"), gp.AUTO), (0, 1.0, 7)):
        with pytest.raises(gp.GpError):
            gp.sssp(G, *args)
    with pytest.raises(gp.GpError):
        gp.sssp(G, 0, 1.0, gp.AUTO, dirs=[0, 2])
    neg = g.csr_w.copy()
    neg[3] = -1.0
    gn = gg.Graph("neg", g.n, g.csr_off, g.csr_idx, g.csc_off, g.csc_idx, False, neg,
                  np.ascontiguousarray(neg[gg._transpose_perm(g)]))
    with pytest.raises(gp.GpError):
        gp.sssp(gp.Graph.from_graphgen(gn), 0, 1.0, gp.AUTO)
