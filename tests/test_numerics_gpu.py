"""The library's integer-arithmetic binary64 -> binary32 rounding (the push
epilogue rounds its FP64 sums with it) against the hardware conversion on the
same device: identical bits over the binary32 normal range -- random encodings
across the whole binary64 range, exact ties in both parities, carries into the
exponent, the overflow edge -- and signed zero below 2^-126."""
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
