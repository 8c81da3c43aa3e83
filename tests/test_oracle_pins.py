"""Pins for the CPU oracle: each check compares it with something other than
itself -- hand-derived worked examples, closed forms, invariants, a dense linear
solve (LU, numpy) and brute-force shortest paths (Floyd-Warshall)."""
import math

import numpy as np
import pytest

import graphgen as gg
import oracle
from helpers import (check_levels_by_edges, check_parents, check_parents_np, dense_pagerank, dense_transition,
                     check_sssp_certificate, edge_sources, floyd_warshall_dist, floyd_warshall_levels,
                     parse_bfs_case, parse_pagerank_cases, parse_sssp_cases, smallest_tight_pred)

VARIANTS = [oracle.PUSH, oracle.PULL]


def og(g, weighted=True):
    return oracle.OracleGraph.from_graph(g, weighted=weighted)


# ----------------------------------------------------------------- worked examples

@pytest.mark.parametrize("case", parse_pagerank_cases(), ids=lambda c: c["name"])
@pytest.mark.parametrize("variant", VARIANTS)
def test_pagerank_worked_example(case, variant):
    """Section 3.1 / Algorithm 1 on hand-derived sweeps (tests/golden)."""
    w = None if case["w"] is None else np.array([float(x) for x in case["w"]], dtype=np.float32)
    G = oracle.OracleGraph(case["n"], case["src"], case["dst"], w)
    d = float(case["d"])
    for k, key, rkey in ((1, "sweep1", "res1"), (2, "sweep2", "res2")):
        x, done, r, _ = G.pagerank(variant, d, iters=k, tol=0.0)
        assert done == k
        np.testing.assert_allclose(x, [float(f) for f in case[key]], rtol=0, atol=1e-15)
        assert abs(r - float(case[rkey])) < 1e-15
    x, done, r, conv = G.pagerank(variant, d, iters=10000, tol=1e-15)
    assert conv
    np.testing.assert_allclose(x, [float(f) for f in case["fixed"]], rtol=0, atol=1e-13)


def test_bfs_worked_example():
    """Section 3.3 / Algorithm 3 on a hand-derived directed example (tests/golden)."""
    c = parse_bfs_case()
    G = oracle.OracleGraph(c["n"], c["src_e"], c["dst_e"])
    level, parent = G.bfs(c["src"])
    assert level.tolist() == c["level"]
    assert parent.tolist() == c["parent"]
    for dirs in ([0], [1], [0, 1], [1, 0], [1, 1, 0, 0, 1]):
        lv, pa, _ = G.bfs_levelsync(c["src"], dirs)
        assert lv.tolist() == c["level"]
        assert check_parents(c["n"], c["src_e"], c["dst_e"], c["src"], lv, pa) == []


# ----------------------------------------------------------------- closed forms

@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n", [2, 3, 7, 16])
def test_complete_graph_uniform(variant, n):
    """K_n: x = 1/n is the fixed point and every sweep from x0 = 1/n stays there."""
    G = og(gg.complete(n))
    for k in (1, 2, 5):
        x, _, r, _ = G.pagerank(variant, 0.85, iters=k)
        np.testing.assert_allclose(x, 1.0 / n, rtol=1e-14, atol=0)
        assert r < 1e-14


@pytest.mark.parametrize("variant", VARIANTS)
def test_directed_cycle_and_regular(variant):
    """Directed n-cycle and a 3-regular circulant: uniform ranks at every sweep."""
    G = og(gg.cycle(11))
    x, _, _, _ = G.pagerank(variant, 0.85, iters=7)
    np.testing.assert_allclose(x, 1 / 11, rtol=1e-14)
    n = 10
    s = np.repeat(np.arange(n), 3)
    t = (s + np.tile([1, 3, 7], n)) % n
    G = og(gg.from_edges(n, s, t))
    x, _, _, _ = G.pagerank(variant, 0.85, iters=9)
    np.testing.assert_allclose(x, 1 / n, rtol=1e-14)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("k", [1, 2, 5, 40])
def test_star_closed_form(variant, k):
    """Undirected star S_k: x_c = (1-d)(1+dk)/(n(1-d^2)), x_l = (1-d)(1+d/k)/(n(1-d^2))."""
    d, n = 0.85, k + 1
    G = og(gg.star(k))
    # the FP64 rounding floor of the L1 residual on this graph is ~6e-15
    x, _, _, conv = G.pagerank(variant, d, iters=100000, tol=1e-13)
    assert conv
    xc = (1 - d) * (1 + d * k) / (n * (1 - d * d))
    xl = (1 - d) * (1 + d / k) / (n * (1 - d * d))
    np.testing.assert_allclose(x[0], xc, rtol=1e-12)
    np.testing.assert_allclose(x[1:], xl, rtol=1e-12)


# ----------------------------------------------------------------- dense linear solve

@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("variant", VARIANTS)
def test_dense_solve(seed, variant):
    """Random directed graphs, n <= 12, with dangling vertices and self-loops:
    the iterated fixed point equals (I - d P)^-1 (1-d) s solved by LU."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 13))
    mask = rng.random((n, n)) < 0.3
    u, v = np.nonzero(mask)
    d = float(rng.uniform(0.5, 0.95))
    weighted = seed % 3 == 0
    w = None
    if weighted:  # P_vu = w_uv with every source's out-weights summing to at most one
        w = rng.uniform(0.05, 1.0, size=len(u))
        w = (w / np.bincount(u, weights=w, minlength=n)[u] * rng.uniform(0.5, 1.0)).astype(np.float32)
    s = rng.random(n)
    s /= s.sum()
    G = oracle.OracleGraph(n, u, v, w)
    x, _, _, conv = G.pagerank(variant, d, iters=100000, tol=1e-14, personalization=s)
    assert conv
    ref = dense_pagerank(n, u, v, d, s=s, w=w)
    np.testing.assert_allclose(x, ref, rtol=0, atol=1e-12)


# ----------------------------------------------------------------- invariants

@pytest.mark.parametrize("variant", VARIANTS)
def test_mass_and_isolated(variant):
    """sum(y) = (1-d) + d * sum_{deg_out(u) > 0} x_u after one sweep; isolated
    vertices hold exactly (1-d)/n."""
    g = gg.rmat(8, 8, seed=3, symmetrize=False)
    G = og(g)
    d = 0.85
    rng = np.random.default_rng(0)
    x0 = rng.random(g.n)
    x0 /= x0.sum()
    y, _, _, _ = G.pagerank(variant, d, iters=1, x0=x0)
    live = g.out_degree() > 0
    assert abs(y.sum() - ((1 - d) + d * x0[live].sum())) < 1e-13
    iso = (g.out_degree() == 0) & (g.in_degree() == 0)
    assert iso.any()
    np.testing.assert_array_equal(y[iso], (1 - d) / g.n)


@pytest.mark.parametrize("seed", range(6))
def test_push_equals_pull(seed):
    """The two sweep forms compute the same iterate (to rounding)."""
    g = gg.rmat(9 + seed % 3, 8, seed=seed, symmetrize=seed % 2 == 0)
    if seed % 3 == 0:
        g = g.with_weights(seed + 100)
    G = og(g)
    a, _, _, _ = G.pagerank(oracle.PUSH, 0.85, iters=25)
    b, _, _, _ = G.pagerank(oracle.PULL, 0.85, iters=25)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)


def test_pull_threads_identical():
    """The threaded pull sums each vertex in the same order: bitwise equal."""
    g = gg.rmat(11, 8, seed=4)
    G = og(g)
    a, _, _, _ = G.pagerank(oracle.PULL, 0.85, iters=10, nthreads=1)
    b, _, _, _ = G.pagerank(oracle.PULL, 0.85, iters=10, nthreads=4)
    assert np.array_equal(a, b)


def test_adjoint_threads_identical():
    """The threaded adjoint sums each lambda_u in the same order: bitwise equal."""
    g = gg.rmat(11, 8, seed=5, symmetrize=False).with_weights(6)
    G = og(g)
    x, _, _, _ = G.pagerank(oracle.PULL, 0.85, iters=50)
    gvec = np.random.default_rng(7).normal(size=g.n)
    a = G.pagerank_adjoint(x, gvec, 0.85, iters=40, nthreads=1)
    b = G.pagerank_adjoint(x, gvec, 0.85, iters=40, nthreads=4)
    for u, v in zip(a[:3], b[:3]):
        assert np.array_equal(u, v)


def test_convergence_contract():
    """tol stops at the first sweep with residual < tol; tol = 0 runs `iters` sweeps."""
    G = og(gg.rmat(9, 8, seed=2))
    x, k, r, conv = G.pagerank(oracle.PULL, 0.85, iters=500, tol=1e-9)
    assert conv and r < 1e-9
    _, k1, r1, _ = G.pagerank(oracle.PULL, 0.85, iters=k - 1, tol=0.0)
    assert r1 >= 1e-9
    _, k2, _, conv2 = G.pagerank(oracle.PULL, 0.85, iters=5, tol=1e-9)
    assert k2 == 5 and not conv2


# ----------------------------------------------------------------- personalised PR

def test_ppr_linearity():
    """The mean of the n one-hot personalised vectors equals global PageRank."""
    g = gg.rmat(5, 4, seed=9, symmetrize=False)
    G = og(g)
    n = g.n
    glob, _, _, _ = G.pagerank(oracle.PULL, 0.85, iters=4000, tol=1e-15)
    acc = np.zeros(n)
    for v in range(n):
        e = np.zeros(n)
        e[v] = 1.0
        x, _, _, _ = G.pagerank(oracle.PULL, 0.85, iters=4000, tol=1e-15, personalization=e, x0=e)
        acc += x
    np.testing.assert_allclose(acc / n, glob, rtol=0, atol=1e-13)


def test_ppr_complete_graph():
    """PPR on K_n seeded at 0: by symmetry x_0 = a and x_v = b with
    a = (1-d) + d b and b (n-1-d(n-2)) = d a."""
    n, d = 9, 0.85
    G = og(gg.complete(n))
    e = np.zeros(n)
    e[0] = 1.0
    x, _, _, _ = G.pagerank(oracle.PUSH, d, iters=5000, tol=1e-15, personalization=e)
    c = d / (n - 1 - d * (n - 2))
    a = (1 - d) / (1 - d * c)
    np.testing.assert_allclose(x[0], a, rtol=1e-12)
    np.testing.assert_allclose(x[1:], c * a, rtol=1e-12)


# ----------------------------------------------------------------- BFS

def test_bfs_path_tree_star_disconnected():
    G = og(gg.path(50))
    lv, pa = G.bfs(0)
    assert lv.tolist() == list(range(50))
    assert pa.tolist() == [0] + list(range(49))
    G = og(gg.binary_tree(100))
    lv, _ = G.bfs(0)
    assert lv.tolist() == [int(math.floor(math.log2(i + 1))) for i in range(100)]
    G = og(gg.star(20))
    lv, _ = G.bfs(0)
    assert lv.tolist() == [0] + [1] * 20
    lv, _ = G.bfs(5)
    assert lv[0] == 1 and lv[5] == 0 and (lv[1:5] == 2).all()
    G = og(gg.empty(4))
    lv, pa = G.bfs(2)
    assert lv.tolist() == [-1, -1, 0, -1] and pa.tolist() == [-1, -1, 2, -1]


@pytest.mark.parametrize("seed", range(20))
def test_bfs_brute_force(seed):
    """Levels equal Floyd-Warshall unit distances on tiny directed graphs, for
    the FIFO form and level-synchronous forms with any per-level direction."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 11))
    mask = rng.random((n, n)) < rng.uniform(0.05, 0.5)
    u, v = np.nonzero(mask)
    G = oracle.OracleGraph(n, u, v)
    for root in range(n):
        ref = floyd_warshall_levels(n, u, v, root)
        lv, pa = G.bfs(root)
        assert lv.tolist() == ref.tolist()
        assert check_parents(n, u, v, root, lv, pa) == []
        for dirs in ([0], [1], [0, 1], [1, 0], rng.integers(0, 2, size=12).tolist()):
            lv2, pa2, used = G.bfs_levelsync(root, dirs)
            assert lv2.tolist() == ref.tolist()
            assert check_parents(n, u, v, root, lv2, pa2) == []


def test_bfs_directions_recorded():
    g = gg.rmat(10, 8, seed=5)
    G = og(g)
    lv, _, used = G.bfs_levelsync(0, [0, 1, 1, 0])
    ref, _ = G.bfs(0)
    assert lv.tolist() == ref.tolist()
    dirs = [0, 1, 1, 0]
    assert len(used) == int(ref.max()) + 1
    assert used.tolist() == [dirs[min(i, 3)] for i in range(len(used))]


# ----------------------------------------------------------------- adjoint

@pytest.mark.parametrize("seed", range(6))
def test_adjoint_dense(seed):
    """lambda = (I - d P^T)^-1 g, grad_s = (1-d) lambda, grad_P[v,u] = d lambda_v x_u,
    against LU solves."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 13))
    mask = rng.random((n, n)) < 0.35
    u, v = np.nonzero(mask)
    w = None
    if seed % 2:  # sub-stochastic columns: every source's out-weights sum to one
        w = rng.uniform(0.1, 1.0, size=len(u))
        w = (w / np.bincount(u, weights=w, minlength=n)[u]).astype(np.float32)
    d = 0.85
    G = oracle.OracleGraph(n, u, v, w)
    x, _, _, _ = G.pagerank(oracle.PULL, d, iters=100000, tol=1e-14)
    gvec = rng.normal(size=n)
    lam, gs, gw, _, _ = G.pagerank_adjoint(x, gvec, d)
    P = dense_transition(n, u, v, w)
    lam_ref = np.linalg.solve(np.eye(n) - d * P.T, gvec)
    np.testing.assert_allclose(lam, lam_ref, rtol=0, atol=1e-11)
    np.testing.assert_allclose(gs, (1 - d) * lam_ref, rtol=0, atol=1e-11)
    np.testing.assert_allclose(gw, d * lam_ref[v] * x[u], rtol=0, atol=1e-11)


def test_adjoint_finite_differences():
    """Central differences of L = g . x*(P, s) through the FP64 forward solve."""
    g = gg.rmat(6, 8, seed=11, symmetrize=False).with_weights(12)
    src, dst = g.edges()
    w = g.csr_w.astype(np.float64)
    d = 0.85
    rng = np.random.default_rng(10)
    gvec = rng.normal(size=g.n)
    s0 = np.full(g.n, 1.0 / g.n)

    def loss(wv, s):
        # the forward of the oracle with explicit double weights: rebuild with float32
        # would round the perturbation away, so solve densely at FP64 for FD only
        P = np.zeros((g.n, g.n))
        np.add.at(P, (dst, src), wv)
        x = np.linalg.solve(np.eye(g.n) - d * P, (1 - d) * s)
        return float(gvec @ x)

    G = oracle.OracleGraph(g.n, src, dst, g.csr_w)
    x, _, _, _ = G.pagerank(oracle.PULL, d, iters=100000, tol=1e-15)
    _, gs, gw, _, _ = G.pagerank_adjoint(x, gvec, d)
    h = 1e-4
    for e in rng.choice(g.m, size=12, replace=False):
        wp, wm = w.copy(), w.copy()
        wp[e] += h
        wm[e] -= h
        fd = (loss(wp, s0) - loss(wm, s0)) / (2 * h)
        assert abs(fd - gw[e]) <= 1e-6 * max(1.0, abs(fd)), (e, fd, gw[e])
    for vtx in rng.choice(g.n, size=8, replace=False):
        sp, sm = s0.copy(), s0.copy()
        sp[vtx] += h
        sm[vtx] -= h
        fd = (loss(w, sp) - loss(w, sm)) / (2 * h)
        assert abs(fd - gs[vtx]) <= 1e-7 * max(1.0, abs(fd))


@pytest.mark.parametrize("seed", range(8))
def test_adjoint_raw_weights_forward_mode(seed):
    """Raw weights normalised inside (P = W / S): the oracle's reverse-mode
    gradient against forward-mode derivatives from LU solves.  For each edge
    e = (u -> v) the tangent of P is (E_v - P[:, u]) / S_u in column u only,
    and dx = (I - dP)^-1 d (dP) x; dL = g . dx.  Graphs of n <= 12 with dangling
    vertices, self-loops, a repeated edge and a personalisation vector."""
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(2, 13))
    mask = rng.random((n, n)) < 0.35
    mask[int(rng.integers(n))] = False  # one dangling source
    u, v = np.nonzero(mask)
    if len(u):  # a parallel copy of one edge: S and P must count both
        k = int(rng.integers(len(u)))
        u, v = np.append(u, u[k]), np.append(v, v[k])
    W = rng.uniform(0.1, 2.0, size=len(u))
    d = float(rng.uniform(0.6, 0.9))
    s = rng.random(n)
    s /= s.sum()
    gvec = rng.normal(size=n)
    G = oracle.OracleGraph(n, u, v, W)
    x, lam, gs, gW, conv = G.pagerank_adjoint_raw(gvec, d, personalization=s)
    assert conv
    A = np.zeros((n, n))
    np.add.at(A, (v, u), W)
    S = A.sum(axis=0)
    P = np.divide(A, S, out=np.zeros_like(A), where=S > 0)
    M = np.eye(n) - d * P
    x_ref = np.linalg.solve(M, (1 - d) * s)
    np.testing.assert_allclose(x, x_ref, rtol=0, atol=1e-12)
    np.testing.assert_allclose(lam, np.linalg.solve(M.T, gvec), rtol=0, atol=1e-11)
    np.testing.assert_allclose(gs, (1 - d) * np.linalg.solve(M.T, gvec), rtol=0, atol=1e-11)
    for e in range(len(u)):
        dP = np.zeros((n, n))
        dP[:, u[e]] = -P[:, u[e]] / S[u[e]]
        dP[v[e], u[e]] += 1.0 / S[u[e]]
        dx = np.linalg.solve(M, d * dP @ x_ref)
        assert abs(gW[e] - gvec @ dx) <= 1e-11, (e, gW[e], gvec @ dx)


def test_adjoint_raw_weights_finite_differences():
    """Central differences (h = 1e-4) of L = g . x*(W / S) where every
    perturbation of a raw weight is renormalised inside the loss, through an
    FP64 dense solve, on an R-MAT scale-6 graph with raw weights in (0, 1]."""
    g = gg.rmat(6, 8, seed=13, symmetrize=False).with_weights(14, normalize=False)
    src, dst = g.edges()
    W = g.csr_w.astype(np.float64)
    d = 0.85
    rng = np.random.default_rng(15)
    gvec = rng.normal(size=g.n)

    def loss(Wv):
        S = np.bincount(src, weights=Wv, minlength=g.n)
        P = np.zeros((g.n, g.n))
        np.add.at(P, (dst, src), Wv / S[src])
        return float(gvec @ np.linalg.solve(np.eye(g.n) - d * P, np.full(g.n, (1 - d) / g.n)))

    G = oracle.OracleGraph(g.n, src, dst, g.csr_w)
    _, _, _, gW, conv = G.pagerank_adjoint_raw(gvec, d)
    assert conv
    h = 1e-4
    for e in rng.choice(g.m, size=16, replace=False):
        Wp, Wm = W.copy(), W.copy()
        Wp[e] += h
        Wm[e] -= h
        fd = (loss(Wp) - loss(Wm)) / (2 * h)
        assert abs(fd - gW[e]) <= 1e-7 * max(1.0, abs(fd)), (e, fd, gW[e])


def test_full_size_bfs_checkers_catch_planted_mistakes():
    """The level/parent rules used at full size accept the oracle's BFS and
    reject each kind of planted mistake (a level one too deep, one too shallow,
    a reached vertex marked unreached, a parent from the wrong level)."""
    g = gg.rmat(12, 8, seed=9)
    O = og(g)
    src = int(gg.pick_vertices(g, 1, seed=3)[0])
    level, parent = O.bfs(src)
    esrc = edge_sources(g.csr_off)
    assert check_levels_by_edges(esrc, g.csr_idx, src, level) == 0
    assert check_parents_np(g.csr_off, g.csr_idx, src, level, parent) == 0
    deep = np.nonzero(level == level.max())[0][0]
    mid = np.nonzero(level == 2)[0][0]
    for v, delta in ((deep, 1), (mid, -1)):
        bad = level.copy()
        bad[v] += delta
        assert check_levels_by_edges(esrc, g.csr_idx, src, bad) + \
            check_parents_np(g.csr_off, g.csr_idx, src, bad, parent) > 0
    bad = level.copy()
    bad[mid] = -1
    assert check_levels_by_edges(esrc, g.csr_idx, src, bad) > 0
    badp = parent.copy()
    badp[deep] = src
    assert check_parents_np(g.csr_off, g.csr_idx, src, level, badp) > 0


# ------------------------------------------------------------------ SSSP (Delta-Stepping, Section 3 listing)

def test_sssp_worked_example():
    n, s, d, w, cases = parse_sssp_cases()
    G = oracle.OracleGraph(n, np.array(s), np.array(d), np.array(w, dtype=np.float32))
    for src, dist, pred in cases:
        got, p = G.sssp(src)
        assert np.array_equal(got, np.array(dist)), (src, got)
        assert list(p) == pred
        for delta in (1.0, 2.0, 3.5, 100.0):
            for dirs in ([0], [1], [0, 1], [1, 0, 0]):
                dd, _, _ = G.sssp_delta(src, delta, dirs)
                assert np.array_equal(dd, np.array(dist)), (src, delta, dirs)


@pytest.mark.parametrize("seed", range(8))
def test_sssp_dijkstra_matches_floyd_warshall(seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(2, 11))
    ne = int(rng.integers(0, 3 * n))
    u = rng.integers(0, n, size=ne)
    v = rng.integers(0, n, size=ne)
    w = rng.integers(0, 10, size=ne).astype(np.float32)  # zero weights and parallel edges included
    G = oracle.OracleGraph(n, u, v, w)
    D = floyd_warshall_dist(n, u, v, w)
    for src in range(n):
        dist, pred = G.sssp(src)
        assert np.array_equal(dist, D[src]), (seed, src)
        for t in range(n):  # every predecessor lies on a shortest path
            if np.isfinite(dist[t]) and t != src:
                p = pred[t]
                assert any(a == p and b == t and dist[p] + x == dist[t] for a, b, x in zip(u, v, w))


def test_sssp_unit_weights_are_bfs_levels():
    g = gg.rmat(9, 8, seed=12, symmetrize=False)
    G = og(g)
    for src in gg.pick_vertices(g, 4, seed=13):
        dist, _ = G.sssp(int(src))
        lv, _ = G.bfs(int(src))
        assert np.array_equal(np.where(np.isfinite(dist), dist, -1).astype(np.int64), lv.astype(np.int64))


def test_sssp_path_and_star_closed_forms():
    w = np.array([3, 1, 4, 1, 5, 9, 2, 6], dtype=np.float32)
    n = len(w) + 1
    G = oracle.OracleGraph(n, np.arange(n - 1), np.arange(1, n), w)
    dist, _ = G.sssp(0)
    assert np.array_equal(dist, np.concatenate([[0.0], np.cumsum(w)]))
    k = 6  # star: hub 0, leaves 1..k, edges both ways with weights a_i (out) and b_i (in)
    a = np.arange(1, k + 1, dtype=np.float32)
    b = 10 * a
    src = np.concatenate([np.zeros(k, int), np.arange(1, k + 1)])
    dst = np.concatenate([np.arange(1, k + 1), np.zeros(k, int)])
    G = oracle.OracleGraph(k + 1, src, dst, np.concatenate([a, b]))
    d0, _ = G.sssp(0)
    assert np.array_equal(d0, np.concatenate([[0.0], a]))
    d3, _ = G.sssp(3)  # leaf 3 -> hub (b_3) -> leaf j (a_j)
    want = np.concatenate([[b[2]], b[2] + a])
    want[3] = 0.0
    assert np.array_equal(d3, want)


@pytest.mark.parametrize("delta", [1.0, 7.0, 32.0, 1000.0, 1e9])
def test_sssp_delta_stepping_equals_dijkstra(delta):
    """Delta-Stepping reaches the shortest distances for any bucket width and any
    push/pull sequence (integer weights: sums are exact)."""
    g = gg.with_int_weights(gg.rmat(8, 8, seed=14, symmetrize=False), seed=15, lo=1, hi=64)
    G = og(g)
    rng = np.random.default_rng(16)
    for src in gg.pick_vertices(g, 3, seed=17):
        ref, _ = G.sssp(int(src))
        for dirs in ([0], [1], [0, 1], [1, 0], list(rng.integers(0, 2, size=40))):
            dist, iters, epochs = G.sssp_delta(int(src), delta, dirs)
            assert np.array_equal(dist, ref), (delta, dirs)
            assert iters >= epochs >= 1


def test_sssp_delta_epochs_follow_bucket_width():
    """Unit weights on a path: with delta = 1 every vertex is its own bucket (one
    epoch per distance); with a huge delta everything is one epoch whose push
    iterations advance one hop each (Bellman-Ford)."""
    n = 12
    G = oracle.OracleGraph(n, np.arange(n - 1), np.arange(1, n), np.ones(n - 1, dtype=np.float32))
    dist, iters, epochs = G.sssp_delta(0, 1.0, [0])
    assert epochs == n and np.array_equal(dist, np.arange(n, dtype=np.float64))
    dist, iters, epochs = G.sssp_delta(0, 1e9, [0])
    assert epochs == 1 and iters == n  # n - 1 hops, then one iteration that changes nothing


def test_sssp_certificate_catches_planted_mistakes():
    """The size-independent shortest-path certificate accepts the oracle's
    distances and rejects a distance too long, one too short, a wrong
    predecessor and a reached vertex marked unreachable."""
    g = gg.with_int_weights(gg.rmat(10, 8, seed=18, symmetrize=False), seed=19, lo=1, hi=20)
    G = og(g)
    src = int(gg.pick_vertices(g, 1, seed=20)[0])
    dist, _ = G.sssp(src)
    d32 = dist.astype(np.float32)
    pred = smallest_tight_pred(g.csr_off, g.csr_idx, g.csr_w, src, d32)
    assert check_sssp_certificate(g.csr_off, g.csr_idx, g.csr_w, src, d32, pred) == 0
    far = int(np.nanargmax(np.where(np.isfinite(d32), d32, -1)))
    for delta in (1.0, -1.0):
        bad = d32.copy()
        bad[far] += delta
        assert check_sssp_certificate(g.csr_off, g.csr_idx, g.csr_w, src, bad, pred) > 0
    badp = pred.copy()
    badp[far] = src if pred[far] != src else far
    assert check_sssp_certificate(g.csr_off, g.csr_idx, g.csr_w, src, d32, badp) > 0
    bad = d32.copy()
    bad[far] = np.inf
    assert check_sssp_certificate(g.csr_off, g.csr_idx, g.csr_w, src, bad, pred) > 0


def test_smallest_tight_pred_matches_definition():
    n, s, d, w, cases = parse_sssp_cases()
    csr = gg.from_edges(n, np.array(s), np.array(d), dedup=False)
    order = np.lexsort((np.array(d), np.array(s)))
    wcsr = np.array(w, dtype=np.float32)[order]
    for src, dist, pred in cases:
        got = smallest_tight_pred(csr.csr_off, csr.csr_idx, wcsr, src, np.array(dist, dtype=np.float32))
        assert list(got) == pred


# ------------------------------------------------------------------ triangle counting (NodeIterator, Section 3 listing)

def brute_triangles(n, u, v):
    """Per-vertex triangle counts from the adjacency matrix: tc[i] = sum over
    j < k of A[i,j] A[i,k] A[j,k]; the total is trace(A^3) / 6."""
    A = np.zeros((n, n), dtype=np.int64)
    A[u, v] = 1
    A[v, u] = 1
    np.fill_diagonal(A, 0)
    A3 = A @ A @ A
    return np.diag(A3) // 2, int(np.trace(A3) // 6)


@pytest.mark.parametrize("variant", [oracle.PUSH, oracle.PULL])
@pytest.mark.parametrize("seed", range(6))
def test_triangles_match_adjacency_cube(variant, seed):
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(3, 40))
    g = gg.random_small(n, float(rng.uniform(0.05, 0.6)), seed=700 + seed, directed=False)
    src, dst = g.edges()
    tc, total = og(g).triangles(variant)
    ref, rtot = brute_triangles(n, src, dst)
    assert np.array_equal(tc, ref) and total == rtot


def test_triangles_closed_forms():
    from math import comb

    for k in (3, 4, 7, 12):  # K_k: every vertex in C(k-1, 2) triangles
        tc, total = og(gg.complete(k)).triangles(oracle.PULL)
        assert (tc == comb(k - 1, 2)).all() and total == comb(k, 3)
    a, b = 5, 7  # complete bipartite: no triangles
    u = np.repeat(np.arange(a), b)
    v = np.tile(np.arange(a, a + b), a)
    tc, total = og(gg.from_edges(a + b, u, v, symmetrize=True)).triangles(oracle.PUSH)
    assert total == 0 and not tc.any()
    r = 9  # wheel: hub 0 and a rim cycle 1..r: hub in r triangles, each rim vertex in 2
    rim = np.arange(1, r + 1)
    u = np.concatenate([np.zeros(r, int), rim])
    v = np.concatenate([rim, np.roll(rim, -1)])
    tc, total = og(gg.from_edges(r + 1, u, v, symmetrize=True)).triangles(oracle.PULL)
    assert tc[0] == r and (tc[1:] == 2).all() and total == r
    tc, total = og(gg.binary_tree(100)).triangles(oracle.PULL)  # trees have none
    assert total == 0


def test_triangles_push_equals_pull_and_threads():
    g = gg.rmat(12, 8, seed=22)
    G = og(g)
    a, ta = G.triangles(oracle.PULL, nthreads=1)
    b, tb = G.triangles(oracle.PUSH)
    c, tcn = G.triangles(oracle.PULL, nthreads=4)
    assert np.array_equal(a, b) and np.array_equal(a, c) and ta == tb == tcn > 0
    assert a.sum() == 3 * ta


# ------------------------------------------------------------------ Frontier-Exploit PageRank (residual form)

def test_fe_pagerank_all_active_is_jacobi():
    """eps < 0 keeps every vertex in the frontier: k iterations give the iterate
    of k Jacobi sweeps from the uniform start (the plain PageRank iteration,
    pinned above), and from s when personalised."""
    g = gg.rmat(9, 8, seed=30, symmetrize=False)
    G = og(g)
    s = np.random.default_rng(3).uniform(0.1, 1.0, size=g.n)
    s /= s.sum()
    for k in (0, 1, 2, 7, 20):
        for dirs in ([0], [1], [0, 1]):
            x, _, it = G.pagerank_fe(0.85, -1.0, iters=k, dirs=dirs)
            ref, _, _, _ = G.pagerank(oracle.PULL, 0.85, iters=k) if k else (np.full(g.n, 1.0 / g.n), 0, 0, 0)
            assert it == k and np.abs(x - ref).max() < 1e-15
            x, _, _ = G.pagerank_fe(0.85, -1.0, iters=k, dirs=dirs, personalization=s)
            ref = G.pagerank(oracle.PULL, 0.85, iters=k, personalization=s, x0=s)[0] if k else s
            assert np.abs(x - ref).max() < 1e-15


@pytest.mark.parametrize("seed", range(6))
def test_fe_pagerank_invariant_and_bound(seed):
    """x + (I - dP)^-1 r equals the fixed point (dense LU) at every stopping
    point, the error is within ||r||_1 / (1-d), and every final |r_u| <= eps."""
    rng = np.random.default_rng(800 + seed)
    n = int(rng.integers(3, 13))
    g = gg.random_small(n, float(rng.uniform(0.2, 0.7)), seed=800 + seed)
    src, dst = g.edges()
    w = None
    if seed % 2:
        w = rng.uniform(0.1, 1.0, size=len(src))
        w = (w / np.bincount(src, weights=w, minlength=n)[src]).astype(np.float32)
    G = oracle.OracleGraph(n, src, dst, w)
    P = dense_transition(n, src, dst, w)
    s = rng.uniform(0.1, 1.0, size=n)
    s /= s.sum()
    xs = np.linalg.solve(np.eye(n) - 0.85 * P, 0.15 * s)
    for eps in (1e-3, 1e-6, 1e-10):
        for iters in (3, 1000):
            x, r, it = G.pagerank_fe(0.85, eps, iters=iters, personalization=s,
                                     dirs=list(rng.integers(0, 2, size=40)))
            inv = x + np.linalg.solve(np.eye(n) - 0.85 * P, r)
            np.testing.assert_allclose(inv, xs, rtol=0, atol=1e-13)
            if iters == 1000:
                assert np.abs(r).max() <= eps
                # ||(I - dP)^-1 r||_1 <= ||r||_1 / (1 - d ||P||_1), ||P||_1 the largest column
                # sum (equality for a column-stochastic P and one-signed r)
                pn = P.sum(axis=0).max()
                assert np.abs(x - xs).sum() <= np.abs(r).sum() / (1 - 0.85 * pn) * (1 + 1e-12) + 1e-13


def test_fe_pagerank_frontier_shrinks():
    """On a graph with a fast-converging part and a slow one, later iterations
    propagate from fewer vertices: the final result is reached with fewer edge
    visits than full sweeps would take."""
    g = gg.rmat(10, 8, seed=31, symmetrize=False)
    G = og(g)
    x, r, it = G.pagerank_fe(0.85, 1e-9, iters=1000)
    ref, _, _, _ = G.pagerank(oracle.PULL, 0.85, iters=100000, tol=1e-15)
    assert np.abs(r).max() <= 1e-9
    assert np.abs(x - ref).sum() <= np.abs(r).sum() / 0.15 * (1 + 1e-12) + 1e-12


# ------------------------------------------------------------------ betweenness centrality (Brandes, Section 3 listing)

def brute_bc(n, u, v, sources):
    """sum over s in sources, t != s, v not in {s, t} of sigma_st(v) / sigma_st,
    with distances and path counts from repeated matrix products (unit
    weights): sigma_st(v) = sigma_sv sigma_vt when d(s,v) + d(v,t) = d(s,t)."""
    A = np.zeros((n, n), dtype=np.int64)
    A[u, v] = 1
    np.fill_diagonal(A, 0)
    D = np.full((n, n), -1, dtype=np.int64)
    S = np.zeros((n, n), dtype=np.float64)
    np.fill_diagonal(D, 0)
    np.fill_diagonal(S, 1.0)
    P = np.eye(n, dtype=np.float64)  # number of walks of length k
    for k in range(1, n):
        P = P @ A
        new = (D < 0) & (P > 0)
        D[new] = k
        S[new] = P[new]  # first length with a walk: those walks are the shortest paths
    bc = np.zeros(n)
    for s in sources:
        for t in range(n):
            if t == s or D[s, t] < 0:
                continue
            for w in range(n):
                if w in (s, t) or D[s, w] < 0 or D[w, t] < 0:
                    continue
                if D[s, w] + D[w, t] == D[s, t]:
                    bc[w] += S[s, w] * S[w, t] / S[s, t]
    return bc


@pytest.mark.parametrize("seed", range(6))
def test_bc_matches_path_counting(seed):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(3, 13))
    g = gg.random_small(n, float(rng.uniform(0.15, 0.6)), seed=900 + seed, directed=bool(seed % 2))
    src, dst = g.edges()
    sources = rng.choice(n, size=int(rng.integers(1, n + 1)), replace=False)
    np.testing.assert_allclose(og(g).bc(sources), brute_bc(n, src, dst, sources), rtol=1e-12, atol=1e-12)


def test_bc_closed_forms():
    n = 9  # undirected path, all sources: vertex i lies on 2 i (n-1-i) ordered shortest paths
    bc = og(gg.path(n)).bc(np.arange(n))
    np.testing.assert_allclose(bc, [2 * i * (n - 1 - i) for i in range(n)], atol=1e-12)
    k = 7  # star: the hub is on every path between two leaves, (k)(k-1) ordered pairs
    bc = og(gg.star(k)).bc(np.arange(k + 1))
    assert bc[0] == k * (k - 1) and not bc[1:].any()
    bc = og(gg.complete(6)).bc(np.arange(6))  # complete graph: no vertex is between two others
    assert not bc.any()


@pytest.mark.parametrize("seed", range(4))
def test_bc_dependency_sum_is_path_interior_count(seed):
    # for one source the dependencies add up to the interior vertices of one shortest path per target:
    # sum_v delta_s(v) = sum over reached t != s of (d(s, t) - 1)
    g = gg.rmat(9, 8, seed=40 + seed, symmetrize=bool(seed % 2))
    O = og(g)
    for s in gg.pick_vertices(g, 5, seed=seed):
        lv, _ = O.bfs(int(s))
        want = np.maximum(lv[lv > 0] - 1, 0).sum()
        assert abs(O.bc([int(s)]).sum() - want) <= 1e-9 * max(1, want)


def _brandes_py(off, idx, n, s, variant=""):
    """Brandes for one source in plain Python, with a planted mistake on request:
    'no_one' drops the 1 of (1 + delta), 'ratio' inverts sigma_u / sigma_w,
    'self' adds the source's own dependency."""
    from collections import deque
    dist = [-1] * n
    sigma = [0.0] * n
    dist[s], sigma[s] = 0, 1.0
    order, q = [], deque([s])
    while q:
        u = q.popleft()
        order.append(u)
        for w in idx[off[u]:off[u + 1]]:
            if dist[w] < 0:
                dist[w] = dist[u] + 1
                q.append(w)
            if dist[w] == dist[u] + 1:
                sigma[w] += sigma[u]
    delta = [0.0] * n
    bc = np.zeros(n)
    for u in reversed(order):
        for w in idx[off[u]:off[u + 1]]:
            if dist[w] == dist[u] + 1:
                r = sigma[w] / sigma[u] if variant == "ratio" else sigma[u] / sigma[w]
                delta[u] += r * ((0.0 if variant == "no_one" else 1.0) + delta[w])
        if u != s or variant == "self":
            bc[u] += delta[u]
    return bc, dist


@pytest.mark.parametrize("variant", ["no_one", "ratio", "self"])
def test_bc_dependency_sum_check_catches_planted_mistakes(variant):
    # the full-size BC test checks sum_v bc(v) = sum_t (d(s,t) - 1) per source; this pins that the
    # check rejects the plausible mistakes in the accumulation, while the correct form passes it
    g = gg.rmat(8, 8, seed=5)
    off, idx = list(g.csr_off), list(g.csr_idx)
    O = og(g)
    caught = False
    for s in gg.pick_vertices(g, 6, seed=1):
        good, dist = _brandes_py(off, idx, g.n, int(s))
        d = np.array(dist)
        want = np.maximum(d[d > 0] - 1, 0).sum()
        assert abs(good.sum() - want) <= 1e-9 * max(1, want)
        np.testing.assert_allclose(good, O.bc([int(s)]), rtol=1e-12, atol=1e-12)
        bad, _ = _brandes_py(off, idx, g.n, int(s), variant)
        caught |= abs(bad.sum() - want) > 1e-6 * max(1, want)
    assert caught, variant
