"""gp_pull_sweep_noalloc: one pull PageRank sweep that allocates no device memory.

Some callers may not allocate device memory while they run -- code inside a
framework hook that only gets the buffers the framework hands it, pipelines
that reserve all device memory at start-up, or processes whose memory another
allocator already holds.  For them the library offers this sweep, whose
intermediate data lives in a fixed array compiled into libgp.

Here it is called through the C ABI, twice in a row (the second call starting
from the first call's output, so stale contents of the shared array would
show), and each result is compared element by element with the CPU oracle's
single sweep from the same iterate and with the regular gp_pagerank entry point
doing the same sweep, within the parity tolerance the other tests use (max-abs
1e-6, L1 1e-5).  Also covered: edge weights with a per-source normaliser, a
personalisation vector, a graph of exactly GP_NOALLOC_MAX_VERTICES vertices,
malformed offsets and indices (a NaN residual, no fault), and that a call
leaves the library's memory pool and PyTorch's allocator untouched.  This file
is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

MAX_ABS, L1 = 1e-6, 1e-5
D = 0.85


@pytest.fixture(scope="module")
def gp():
    import torch

    import paper_2010_16012_gb300 as gp

    assert torch.cuda.is_available()
    gp.load()
    return gp


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _vp(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _sweep(gp, n, m, off, idx, w, inv, x, s=None):
    """One call through the C ABI; returns (status, y, residual) after a sync."""
    import torch

    lib = gp.load()
    y = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
    res = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    before_pool = gp.pool_usage()
    before_torch = torch.cuda.memory_allocated()
    st = lib.gp_pull_sweep_noalloc(n, m, _vp(off), _vp(idx), _vp(w), _vp(inv), _vp(x), ctypes.c_float(D), _vp(s),
                                   _vp(y), _vp(res), ctypes.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    # the call itself allocated nothing: neither from the library's pool nor through torch
    assert gp.pool_usage() == before_pool
    assert torch.cuda.memory_allocated() == before_torch
    return st, y, res.item()


def _inv_out_degree(g):
    dout = g.out_degree()
    return np.where(dout > 0, np.float32(1.0) / np.maximum(dout, 1).astype(np.float32), 0).astype(np.float32)


def _close(y, ref, what):
    err = np.abs(y.cpu().numpy().astype(np.float64) - ref)
    assert err.max() <= MAX_ABS and err.sum() <= L1, (what, err.max(), err.sum())


def test_noalloc_sweep_matches_oracle_and_gp_pagerank_twice(gp):
    lib = gp.load()
    g = gg.rmat(13, 16, seed=3, symmetrize=False)  # directed: in- and out-degrees differ
    n, m = g.n, g.m
    off, idx, inv = _dev(g.csc_off), _dev(g.csc_idx), _dev(_inv_out_degree(g))
    G = gp.Graph.from_graphgen(g)
    O = oracle.OracleGraph.from_graph(g, weighted=False)
    rng = np.random.default_rng(4)
    xh = rng.random(n).astype(np.float32)
    xh /= xh.sum()
    x = _dev(xh)
    for call in range(2):
        st, y, res = _sweep(gp, n, m, off, idx, None, inv, x)
        assert st == gp.OK, lib.gp_last_error()
        ref, k, rref, _ = O.pagerank(oracle.PULL, D, iters=1, x0=x.cpu().numpy())
        assert k == 1
        _close(y, ref, ("oracle", call))
        assert abs(res - rref) <= L1, (call, res, rref)
        yg, rst = gp.pagerank(G, gp.PULL, D, iters=1, x0=x)
        _close(y, yg.cpu().numpy().astype(np.float64), ("gp_pagerank", call))
        assert abs(res - rst["residual"]) <= L1, (call, res, rst["residual"])
        x = y  # the second call starts from the first call's output


def test_noalloc_weighted_with_normaliser_and_personalization(gp):
    """csc_w = raw weights, inv_deg = 1/S_u (the per-source weight sum): the
    sweep applies P_vu = w_uv / S_u; the oracle is given P in FP64."""
    lib = gp.load()
    g = gg.rmat(12, 16, seed=5, symmetrize=False).with_weights(6, normalize=False)
    n, m = g.n, g.m
    src, dst = g.edges()
    S = np.bincount(src, weights=g.csr_w.astype(np.float64), minlength=n)
    inv = np.where(S > 0, 1.0 / np.where(S > 0, S, 1.0), 0.0).astype(np.float32)
    O = oracle.OracleGraph(n, src, dst, g.csr_w.astype(np.float64) / S[src])
    rng = np.random.default_rng(7)
    s = rng.random(n)
    s /= s.sum()
    xh = rng.random(n).astype(np.float32)
    xh /= xh.sum()
    x, sd = _dev(xh), _dev(s.astype(np.float32))
    off, idx, w, invd = _dev(g.csc_off), _dev(g.csc_idx), _dev(g.csc_w), _dev(inv)
    for call in range(2):
        st, y, res = _sweep(gp, n, m, off, idx, w, invd, x, sd)
        assert st == gp.OK, lib.gp_last_error()
        ref, _, rref, _ = O.pagerank(oracle.PULL, D, iters=1, x0=x.cpu().numpy(),
                                     personalization=sd.cpu().numpy())
        _close(y, ref, ("weighted", call))
        assert abs(res - rref) <= L1
        x = y


def test_noalloc_at_its_maximum_size(gp):
    """n = GP_NOALLOC_MAX_VERTICES exactly (R-MAT scale 20, directed)."""
    lib = gp.load()
    g = gg.rmat(20, 8, seed=9, symmetrize=False)
    assert g.n == gp.NOALLOC_MAX_VERTICES
    O = oracle.OracleGraph.from_graph(g, weighted=False)
    xh = np.full(g.n, 1.0 / g.n, dtype=np.float32)
    st, y, res = _sweep(gp, g.n, g.m, _dev(g.csc_off), _dev(g.csc_idx), None, _dev(_inv_out_degree(g)), _dev(xh))
    assert st == gp.OK, lib.gp_last_error()
    ref, _, rref, _ = O.pagerank(oracle.PULL, D, iters=1, x0=xh, nthreads=oracle.max_threads())
    _close(y, ref, "max size")
    assert abs(res - rref) <= L1


def test_noalloc_flags_malformed_input_without_reading_it(gp):
    """Out-of-range indices and offsets give a NaN residual (the bad entries are
    skipped), and the next well-formed call is correct again."""
    import torch

    lib = gp.load()
    g = gg.rmat(10, 8, seed=11, symmetrize=False)
    n, m = g.n, g.m
    inv = _dev(_inv_out_degree(g))
    xh = np.full(n, 1.0 / n, dtype=np.float32)
    x = _dev(xh)
    for bad in (n, -1, 2**31 - 1):
        idx = g.csc_idx.copy()
        idx[m // 2] = bad
        st, _, res = _sweep(gp, n, m, _dev(g.csc_off), _dev(idx), None, inv, x)
        assert st == gp.OK and np.isnan(res), (bad, res)
    off = g.csc_off.copy()
    off[n // 2] = m + 5  # one offset beyond m: both pairs that share it are rejected
    st, _, res = _sweep(gp, n, m, _dev(off), _dev(g.csc_idx), None, inv, x)
    assert st == gp.OK and np.isnan(res)
    off = g.csc_off.copy()
    off[n // 3] = -3
    st, _, res = _sweep(gp, n, m, _dev(off), _dev(g.csc_idx), None, inv, x)
    assert st == gp.OK and np.isnan(res)
    # offsets that rise and fall: every pair (0, M) is in range on its own, but a
    # warp's 32 degrees sum past 2^31; the tile must be refused, not scanned
    M = (1 << 27) + 1024
    nn = 64
    off = np.zeros(nn + 1, dtype=np.int64)
    off[1::2] = M
    idx = torch.zeros(M, dtype=torch.int32, device="cuda")
    st, _, res = _sweep(gp, nn, M, _dev(off), idx, None, _dev(np.ones(nn, np.float32)),
                        _dev(np.full(nn, 1.0 / nn, np.float32)))
    assert st == gp.OK and np.isnan(res)
    del idx
    # a well-formed call after the bad ones
    O = oracle.OracleGraph.from_graph(g, weighted=False)
    st, y, res = _sweep(gp, n, m, _dev(g.csc_off), _dev(g.csc_idx), None, inv, x)
    assert st == gp.OK and np.isfinite(res)
    ref, _, _, _ = O.pagerank(oracle.PULL, D, iters=1, x0=xh)
    _close(y, ref, "after bad input")


def test_noalloc_rejects_sizes_beyond_its_scratch(gp):
    lib = gp.load()
    st = lib.gp_pull_sweep_noalloc(gp.NOALLOC_MAX_VERTICES + 1, 0, None, None, None, None, None,
                                   ctypes.c_float(D), None, None, None, None)
    assert st == gp.ERR_INVALID
    assert b"GP_NOALLOC_MAX_VERTICES" in lib.gp_last_error()
    st = lib.gp_pull_sweep_noalloc(0, 0, None, None, None, None, None, ctypes.c_float(D), None, None, None, None)
    assert st == gp.ERR_INVALID
    st = lib.gp_pull_sweep_noalloc(16, 1 << 31, None, None, None, None, None, ctypes.c_float(D), None, None, None,
                                   None)
    assert st == gp.ERR_INVALID
