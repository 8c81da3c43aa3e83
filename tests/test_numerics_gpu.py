"""Device self-checks.  The library's integer-arithmetic binary64 -> binary32
rounding (the push epilogue rounds its FP64 sums with it) against the hardware
conversion on the same device: identical bits over the binary32 normal range --
random encodings across the whole binary64 range, exact ties in both parities,
carries into the exponent, the overflow edge -- and signed zero below 2^-126.
The bounded grid barrier: a missing block makes the others time out with an
error status instead of hanging."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MIN_NORMAL = 2.0 ** -126


@pytest.fixture(scope="module")
def gp():
    import torch

    import paper_2010_16012_gb300 as gp

    assert torch.cuda.is_available()
    gp.load()
    return gp


def cases():
    rng = np.random.default_rng(0)
    out = [rng.integers(0, 2 ** 64, size=1 << 18, dtype=np.uint64).view(np.float64)]  # any encoding
    f = (rng.uniform(-1.0, 1.0, size=1 << 16) * 2.0 ** rng.integers(-120, 120, size=1 << 16)).astype(np.float32)
    f64 = f.astype(np.float64)
    half = np.abs(np.spacing(f).astype(np.float64)) / 2
    out += [f64, f64 + half, f64 - half, f64 + half * 0.999, f64 + half * 1.001, f64 * (1 + 2.0 ** -30)]
    edge = [0.0, -0.0, MIN_NORMAL, -MIN_NORMAL, MIN_NORMAL * (1 - 2.0 ** -30), MIN_NORMAL * (1 - 2.0 ** -25),
            float(np.finfo(np.float32).max), float(np.finfo(np.float32).max) * (1 + 2.0 ** -25),
            float(np.finfo(np.float32).max) * (1 + 2.0 ** -26), 1.0 - 2.0 ** -25, 1.0 - 2.0 ** -26, 2.0 - 2.0 ** -24,
            np.inf, -np.inf, np.nan, 1e-300, -1e300, 5e-324]
    out.append(np.array(edge))
    return np.concatenate(out)


def test_narrow_matches_hardware(gp):
    import torch

    v = cases()
    ours, hw = gp.selftest_narrow(torch.from_numpy(v).cuda())
    ours, hw = ours.cpu().numpy(), hw.cpu().numpy()
    nan = np.isnan(v)
    assert np.isnan(ours[nan]).all() and np.isnan(hw[nan]).all()
    small = ~nan & (np.abs(v) < MIN_NORMAL)
    assert (ours[small] == 0).all() and (np.signbit(ours[small]) == np.signbit(v[small])).all()
    assert (np.abs(hw[small]) <= MIN_NORMAL).all()
    rest = ~nan & ~small
    diff = np.nonzero(ours[rest].view(np.uint32) != hw[rest].view(np.uint32))[0]
    assert diff.size == 0, (v[rest][diff[:5]], ours[rest][diff[:5]], hw[rest][diff[:5]])
    assert rest.sum() > 300000


def test_narrow_rejects_bad_arguments(gp):
    lib = gp.load()
    assert lib.gp_selftest_narrow(-1, None, None, None, None) == gp.ERR_INVALID
    assert lib.gp_selftest_narrow(4, None, None, None, None) == gp.ERR_INVALID
    assert lib.gp_selftest_narrow(0, None, None, None, None) == gp.OK


def test_grid_barrier_timeout_is_reported_and_context_survives(gp):
    """A block that never reaches the grid barrier: the others give up after
    their bounded wait, the call reports GP_ERR_TIMEOUT, and the device context
    keeps working (a BFS afterwards is correct)."""
    import graphgen as gg
    import oracle

    lib = gp.load()
    assert lib.gp_selftest_barrier(-1, None) == gp.OK
    assert lib.gp_selftest_barrier(3, None) == gp.ERR_TIMEOUT
    assert b"ran out" in lib.gp_last_error()
    assert lib.gp_selftest_barrier(1 << 30, None) == gp.ERR_INVALID
    assert lib.gp_selftest_barrier(-1, None) == gp.OK
    g = gg.rmat(10, 8, seed=3)
    level, _, _ = gp.bfs(gp.Graph.from_graphgen(g), 0, gp.AUTO)
    ref, _ = oracle.OracleGraph.from_graph(g).bfs(0)
    assert np.array_equal(level.cpu().numpy(), ref)
