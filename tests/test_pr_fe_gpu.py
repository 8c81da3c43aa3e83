"""Frontier-Exploit PageRank (gp_pagerank_fe) against the oracle.

Tolerances follow from the arithmetic of the residual form:
- eps < 0 keeps every vertex in the frontier, so k iterations are k Jacobi
  sweeps from the uniform start: max-abs 1e-6 and L1 1e-5 against the oracle,
  as for PageRank itself;
- a converged run (empty frontier) is within its own a-posteriori bound
  ||r||_1 / (1 - d) of the FP64 fixed point, plus FP32 rounding (L1 1e-5);
- against the oracle's run of the same algorithm: within the sum of both
  bounds plus the same rounding allowance."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

ROUND_L1 = 1e-5


@pytest.fixture(scope="module")
def gp():
    import torch

    import paper_2010_16012_gb300 as gp

    assert torch.cuda.is_available()
    gp.load()
    return gp


ZOO = [
    lambda: gg.rmat(10, 8, seed=1),
    lambda: gg.rmat(11, 16, seed=2, symmetrize=False),
    lambda: gg.rmat(12, 8, seed=3).with_weights(4),
    lambda: gg.star(3000),
    lambda: gg.erdos_renyi(4000, 20000, seed=5),
    lambda: gg.path(300),
]


def np_(t):
    return t.cpu().numpy().astype(np.float64)


def fixed_point(O, s=None):
    x, _, _, conv = O.pagerank(oracle.PULL, 0.85, iters=100000, tol=1e-12, personalization=s)
    assert conv
    return x


@pytest.mark.parametrize("gi", range(len(ZOO)))
@pytest.mark.parametrize("mode", ["push", "pull", "auto"])
def test_fe_all_active_is_jacobi(gp, gi, mode):
    g = ZOO[gi]()
    G = gp.Graph.from_graphgen(g)
    O = oracle.OracleGraph.from_graph(g)
    m = {"push": gp.PUSH, "pull": gp.PULL, "auto": gp.AUTO}[mode]
    for k in (1, 5, 20):
        x, st = gp.pagerank_fe(G, m, 0.85, eps=-1.0, iters=k)
        ref, _, it = O.pagerank_fe(0.85, -1.0, iters=k)
        err = np.abs(np_(x) - ref)
        assert st["iterations"] == it == k
        assert err.max() <= 1e-6 and err.sum() <= 1e-5, (g.name, mode, k, err.max(), err.sum())


@pytest.mark.parametrize("gi", range(len(ZOO)))
@pytest.mark.parametrize("mode", ["push", "pull", "auto"])
def test_fe_converged_within_bound(gp, gi, mode):
    g = ZOO[gi]()
    G = gp.Graph.from_graphgen(g)
    O = oracle.OracleGraph.from_graph(g)
    xs = fixed_point(O)
    m = {"push": gp.PUSH, "pull": gp.PULL, "auto": gp.AUTO}[mode]
    for eps in (1e-7, 1e-9):
        x, st = gp.pagerank_fe(G, m, 0.85, eps=eps, iters=1000)
        assert st["frontier_left"] == 0
        one_minus_d = 1.0 - float(np.float32(0.85))  # the damping is passed as FP32
        assert abs(st["error_bound"] - st["residual_l1"] / one_minus_d) <= 1e-12 * max(1.0, st["error_bound"])
        assert np.abs(np_(x) - xs).sum() <= st["error_bound"] + ROUND_L1, (g.name, mode, eps)
        xo, ro, _ = O.pagerank_fe(0.85, eps, iters=1000)
        bound = st["error_bound"] + np.abs(ro).sum() / 0.15
        assert np.abs(np_(x) - xo).sum() <= bound + ROUND_L1


def test_fe_forced_directions_and_shrinking_frontier(gp):
    g = gg.rmat(12, 16, seed=6, symmetrize=False)
    G = gp.Graph.from_graphgen(g)
    xs = fixed_point(oracle.OracleGraph.from_graph(g))
    rng = np.random.default_rng(7)
    for dirs in ([0, 1], [1, 0, 0], list(rng.integers(0, 2, size=50))):
        x, st = gp.pagerank_fe(G, gp.AUTO, 0.85, eps=1e-9, iters=1000, dirs=dirs)
        L = min(len(dirs), st["iterations"])
        assert st["direction"][:L] == [int(d) for d in dirs[:L]]
        assert np.abs(np_(x) - xs).sum() <= st["error_bound"] + ROUND_L1
    x, st = gp.pagerank_fe(G, gp.AUTO, 0.85, eps=1e-9, iters=1000)
    fr = st["frontier"]
    assert fr[0] > g.n / 2 and fr[-1] < fr[0] / 4  # the frontier thins out
    assert st["pushes"] > 0 and st["pulls"] > 0  # the switch used both directions


def test_fe_personalized_and_host_output(gp):
    g = gg.rmat(11, 8, seed=8)
    G = gp.Graph.from_graphgen(g)
    O = oracle.OracleGraph.from_graph(g)
    seed = int(gg.pick_vertices(g, 1, seed=9)[0])
    e = np.zeros(g.n, dtype=np.float32)
    e[seed] = 1.0
    xs = fixed_point(O, s=e.astype(np.float64))
    out = np.zeros(g.n, dtype=np.float32)
    _, st = gp.pagerank_fe(G, gp.AUTO, 0.85, eps=1e-9, iters=1000, personalization=e, out=out)
    assert np.abs(out.astype(np.float64) - xs).sum() <= st["error_bound"] + ROUND_L1


def test_fe_cap_and_bad_input(gp):
    G = gp.Graph.from_graphgen(gg.rmat(10, 8, seed=10))
    x, st = gp.pagerank_fe(G, gp.AUTO, 0.85, eps=1e-12, iters=3)
    assert st["iterations"] == 3 and st["frontier_left"] > 0
    with pytest.raises(gp.GpError):
        gp.pagerank_fe(G, gp.AUTO, 0.85, eps=1e-12, iters=3, raise_not_converged=True)
    for kw in (dict(mode=7), dict(damping=1.0), dict(eps=float("nan")), dict(iters=-1), dict(dirs=[0, 3])):
        args = dict(mode=gp.AUTO, damping=0.85, eps=1e-9, iters=10)
        args.update(kw)
        with pytest.raises(gp.GpError):
            gp.pagerank_fe(G, **args)
