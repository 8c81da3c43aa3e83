"""Adjoint of the PageRank fixed point (gp_pagerank_backward and the autograd
Function) against the FP64 oracle adjoint and against central finite
differences of the FP64 forward solve.  Tolerance (the contract of the
differentiation form): 1e-4 relative, max|gpu - ref| / max|ref|."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

REL = 1e-4


@pytest.fixture(scope="module")
def gp():
    import torch

    import paper_2010_16012_gb300 as gp

    assert torch.cuda.is_available()
    gp.load()
    return gp


def rel_err(a, ref):
    a = a.cpu().numpy().astype(np.float64) if hasattr(a, "cpu") else np.asarray(a, dtype=np.float64)
    return float(np.abs(a - ref).max() / max(np.abs(ref).max(), 1e-300))


def fixed_point(O, d=0.85, s=None):
    x, _, _, conv = O.pagerank(oracle.PULL, d, iters=100000, tol=1e-14, personalization=s)
    assert conv
    return x


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("symmetric", [False, True])
def test_adjoint_matches_oracle(gp, mode, weighted, symmetric):
    import torch

    g = gg.rmat(10, 8, seed=21, symmetrize=symmetric)
    if weighted:
        g = g.with_weights(22)
    G = gp.Graph.from_graphgen(g, validate=True)
    O = oracle.OracleGraph.from_graph(g)
    x = fixed_point(O)
    rng = np.random.default_rng(3)
    gvec = rng.normal(size=g.n)
    _, gs_ref, gw_ref, _, _ = O.pagerank_adjoint(x, gvec, 0.85)
    xt = torch.from_numpy(x.astype(np.float32)).cuda()
    gt = torch.from_numpy(gvec.astype(np.float32)).cuda()
    gw, gs, st = gp.pagerank_backward(G, xt, gt, mode=mode, iters=2000, tol=1e-9)
    assert rel_err(gs, gs_ref) <= REL, rel_err(gs, gs_ref)
    assert rel_err(gw, gw_ref) <= REL, rel_err(gw, gw_ref)


def test_adjoint_host_buffers(gp):
    g = gg.rmat(9, 8, seed=5, symmetrize=False).with_weights(6)
    G = gp.Graph.from_graphgen(g)
    O = oracle.OracleGraph.from_graph(g)
    x = fixed_point(O)
    gvec = np.random.default_rng(1).normal(size=g.n)
    _, gs_ref, gw_ref, _, _ = O.pagerank_adjoint(x, gvec, 0.85)
    lib = gp.load()
    import ctypes

    gw = np.zeros(g.m, dtype=np.float32)
    gs = np.zeros(g.n, dtype=np.float32)
    x32, g32 = x.astype(np.float32), gvec.astype(np.float32)  # host inputs, kept alive across the call
    st = gp.gp_pr_stats()
    rc = lib.gp_pagerank_backward(G.handle, gp.PULL, ctypes.c_float(0.85), gp._ptr(x32), gp._ptr(g32), gp._ptr(gw),
                                  gp._ptr(gs), 2000, ctypes.c_double(1e-9), ctypes.byref(st), gp._stream_ptr(None))
    assert rc == gp.OK, lib.gp_last_error()
    assert rel_err(gs, gs_ref) <= REL and rel_err(gw, gw_ref) <= REL


def test_raw_weight_gradient_with_normalize(gp):
    """GP_UPLOAD_NORMALIZE: the gradient with respect to the raw weights (P = W / S
    normalised inside) against the oracle's own raw-weight adjoint, which is
    pinned on CPU by forward-mode LU derivatives and renormalising finite
    differences."""
    import torch

    g = gg.rmat(9, 8, seed=7, symmetrize=False).with_weights(8, normalize=False)
    G = gp.Graph.from_graphgen(g, normalize=True)
    O = oracle.OracleGraph.from_graph(g)  # raw weights; the oracle normalises them itself
    gvec = np.random.default_rng(2).normal(size=g.n)
    x, _, gs_ref, gw_ref, conv = O.pagerank_adjoint_raw(gvec, 0.85)
    assert conv
    gw, gs, _ = gp.pagerank_backward(G, torch.from_numpy(x.astype(np.float32)).cuda(),
                                     torch.from_numpy(gvec.astype(np.float32)).cuda(), iters=2000, tol=1e-9)
    assert rel_err(gw, gw_ref) <= REL, rel_err(gw, gw_ref)
    assert rel_err(gs, gs_ref) <= REL, rel_err(gs, gs_ref)
    # the forward pass of the normalised upload reaches the oracle's fixed point
    xg, st = gp.pagerank(G, gp.PULL, 0.85, 1000, 1e-9)
    assert st["converged"] and float(np.abs(xg.cpu().numpy().astype(np.float64) - x).max()) <= 1e-6


def test_finite_differences_scale10(gp):
    """Central differences (h = 1e-3) of L = g.x*(P, s) through the FP64 oracle
    forward solve, on a weighted scale-10 R-MAT copy; the GPU gradient comes from
    the GPU forward pass followed by the GPU adjoint."""
    import torch

    g = gg.rmat(10, 16, seed=11, symmetrize=False).with_weights(12)
    G = gp.Graph.from_graphgen(g)
    src, dst = g.edges()
    w = g.csr_w.astype(np.float64)
    d = 0.85
    rng = np.random.default_rng(10)
    gvec = rng.normal(size=g.n)
    s0 = np.full(g.n, 1.0 / g.n)

    def loss(wv, s):
        O = oracle.OracleGraph(g.n, src, dst, wv)
        x, _, _, conv = O.pagerank(oracle.PULL, d, iters=100000, tol=1e-14, personalization=s)
        assert conv
        return float(gvec @ x)

    x, st = gp.pagerank(G, gp.PULL, d, 1000, 1e-9)
    assert st["converged"]
    gw, gs, _ = gp.pagerank_backward(G, x, torch.from_numpy(gvec.astype(np.float32)).cuda(), iters=2000, tol=1e-9)
    gw, gs = gw.cpu().numpy().astype(np.float64), gs.cpu().numpy().astype(np.float64)
    h = 1e-3
    fd_w, fd_s = [], []
    edges = rng.choice(g.m, size=16, replace=False)
    verts = rng.choice(g.n, size=8, replace=False)
    for e in edges:
        wp, wm = w.copy(), w.copy()
        wp[e] += h
        wm[e] -= h
        fd_w.append((loss(wp, s0) - loss(wm, s0)) / (2 * h))
    for v in verts:
        sp, sm = s0.copy(), s0.copy()
        sp[v] += h
        sm[v] -= h
        fd_s.append((loss(w, sp) - loss(w, sm)) / (2 * h))
    fd_w, fd_s = np.array(fd_w), np.array(fd_s)
    assert np.abs(gw[edges] - fd_w).max() <= REL * np.abs(fd_w).max(), (gw[edges], fd_w)
    assert np.abs(gs[verts] - fd_s).max() <= REL * np.abs(fd_s).max(), (gs[verts], fd_s)


def test_autograd_function(gp):
    import torch

    g = gg.rmat(10, 8, seed=31, symmetrize=False).with_weights(32)
    perm = torch.from_numpy(gg._transpose_perm(g)).cuda()
    G = gp.Graph.from_graphgen(g)
    w = torch.from_numpy(g.csr_w.copy()).cuda().requires_grad_(True)
    s = torch.full((g.n,), 1.0 / g.n, device="cuda", requires_grad=True)
    coef = torch.from_numpy(np.random.default_rng(4).normal(size=g.n).astype(np.float32)).cuda()
    x = gp.pagerank_autograd(G, w, s, csc_perm=perm, iters=1000, tol=1e-9, adj_tol=1e-9)
    (coef * x).sum().backward()
    src, dst = g.edges()
    O = oracle.OracleGraph(g.n, src, dst, g.csr_w)
    xr = fixed_point(O, s=np.full(g.n, 1.0 / g.n))
    _, gs_ref, gw_ref, _, _ = O.pagerank_adjoint(xr, coef.cpu().numpy().astype(np.float64), 0.85)
    assert rel_err(w.grad, gw_ref) <= REL and rel_err(s.grad, gs_ref) <= REL
    # one gradient step: the next forward pass uses the new weights
    with torch.no_grad():
        w2 = (w - 0.01 * w.grad).clamp_min(1e-6)
    x2 = gp.pagerank_autograd(G, w2, None, csc_perm=perm, iters=1000, tol=1e-9)
    O2 = oracle.OracleGraph(g.n, src, dst, w2.cpu().numpy())
    xr2 = fixed_point(O2)
    assert np.abs(x2.detach().cpu().numpy() - xr2).max() < 1e-6


def test_autograd_graphs_sharing_one_graph(gp):
    """Two forward passes with different weights on one Graph, then the first
    one's backward: its gradient is taken at its own weights."""
    import torch

    g = gg.rmat(9, 8, seed=41, symmetrize=False).with_weights(42)
    perm = torch.from_numpy(gg._transpose_perm(g)).cuda()
    G = gp.Graph.from_graphgen(g)
    src, dst = g.edges()
    coef = torch.from_numpy(np.random.default_rng(5).normal(size=g.n).astype(np.float32)).cuda()
    w1 = torch.from_numpy(g.csr_w.copy()).cuda().requires_grad_(True)
    w2_host = (g.csr_w * np.random.default_rng(6).uniform(0.2, 1.0, size=g.m)).astype(np.float32)
    w2 = torch.from_numpy(w2_host).cuda().requires_grad_(True)
    x1 = gp.pagerank_autograd(G, w1, None, csc_perm=perm, iters=1000, tol=1e-9, adj_tol=1e-9)
    x2 = gp.pagerank_autograd(G, w2, None, csc_perm=perm, iters=1000, tol=1e-9, adj_tol=1e-9)
    (coef * x1).sum().backward()
    (coef * x2).sum().backward()
    for w, wh in ((w1, g.csr_w), (w2, w2_host)):
        O = oracle.OracleGraph(g.n, src, dst, wh)
        xr = fixed_point(O)
        _, _, gw_ref, _, _ = O.pagerank_adjoint(xr, coef.cpu().numpy().astype(np.float64), 0.85)
        assert rel_err(w.grad, gw_ref) <= REL
