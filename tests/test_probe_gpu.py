"""gp_probe_rates: every kind runs, and the work it times is the work it
claims -- the add kinds leave exactly one unit per operation in their tables,
the gathers read the zeroed tables (sum 0)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gp():
    import torch

    import paper_2010_16012_gb300 as gp

    assert torch.cuda.is_available()
    gp.load()
    return gp


@pytest.mark.parametrize("kind", ["gather_global", "gather_shared", "gather_cluster", "red_f64", "red_f32",
                                  "atom_shared_f64", "atom_shared_f32"])
def test_probe_kinds(gp, kind):
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    grid = 2 * sms - (2 * sms) % 8
    iters = 64
    rate, check = gp.probe_rates(kind, iters)
    assert rate > 1e9
    if kind.startswith("gather"):
        assert check == 0.0
    else:
        assert check == grid * 1024 * iters


def test_probe_bad_input(gp):
    for kind, iters in ((7, 16), (-1, 16), (0, 0), (0, 70000)):
        with pytest.raises(gp.GpError):
            gp.probe_rates(kind, iters)
