"""gp_pull_sweep_noalloc: one pull PageRank sweep that allocates no device memory.

Some callers may not allocate device memory while they run -- code inside a
framework hook that only gets the buffers the framework hands it, pipelines
that reserve all device memory at start-up, or processes whose memory another
allocator already holds.  For them the library offers this sweep, whose
intermediate data lives in a fixed array compiled into libgp.  Here it is
called through the C ABI, twice in a row (the second call starting from the
first call's output, so stale contents of the shared array would show), and
each result is compared with the regular gp_pagerank entry point doing the same
single sweep, within the parity tolerance the other tests use (max-abs 1e-6,
L1 1e-5).  This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu

MAX_ABS, L1 = 1e-6, 1e-5


@pytest.fixture(scope="module")
def gp():
    import torch

    import paper_2010_16012_gb300 as gp

    assert torch.cuda.is_available()
    gp.load()
    return gp


def test_noalloc_sweep_matches_gp_pagerank_twice(gp):
    import torch

    lib = gp.load()
    g = gg.rmat(13, 16, seed=3, symmetrize=False)  # directed: in- and out-degrees differ
    n, m = g.n, g.m
    dout = g.out_degree()
    inv = np.where(dout > 0, np.float32(1.0) / np.maximum(dout, 1).astype(np.float32), 0).astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    csc_off, csc_idx, inv_d = dev(g.csc_off), dev(g.csc_idx), dev(inv)
    G = gp.Graph.from_graphgen(g)
    rng = np.random.default_rng(4)
    x = rng.random(n).astype(np.float32)
    x /= x.sum()
    x = dev(x)
    stream = torch.cuda.current_stream()
    for call in range(2):
        y = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
        res = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.gp_pull_sweep_noalloc(n, m, ctypes.c_void_p(csc_off.data_ptr()), ctypes.c_void_p(csc_idx.data_ptr()),
                                       None, ctypes.c_void_p(inv_d.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                       ctypes.c_float(0.85), None, ctypes.c_void_p(y.data_ptr()),
                                       ctypes.c_void_p(res.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert st == gp.OK, lib.gp_last_error()
        torch.cuda.synchronize()
        ref, rst = gp.pagerank(G, gp.PULL, 0.85, iters=1, x0=x)
        err = np.abs(y.cpu().numpy().astype(np.float64) - ref.cpu().numpy().astype(np.float64))
        assert err.max() <= MAX_ABS and err.sum() <= L1, (call, err.max(), err.sum())
        assert abs(res.item() - rst["residual"]) <= L1, (call, res.item(), rst["residual"])
        x = y  # the second call starts from the first call's output


def test_noalloc_rejects_graphs_beyond_its_scratch(gp):
    lib = gp.load()
    st = lib.gp_pull_sweep_noalloc(gp.NOALLOC_MAX_VERTICES + 1, 0, None, None, None, None, None,
                                   ctypes.c_float(0.85), None, None, None, None)
    assert st == gp.ERR_INVALID
    assert b"GP_NOALLOC_MAX_VERTICES" in lib.gp_last_error()
