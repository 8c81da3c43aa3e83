"""Autotuner cache (host logic, no GPU): keys separate graphs, tuning scopes and GPU
models; entries round-trip through the JSON file; the env var selects the file."""
import os


def test_key_and_roundtrip(tmp_path, monkeypatch):
    import paper_2010_16012_gb300 as gp

    info = {"n": 10, "m": 20, "max_out_degree": 5, "max_in_degree": 6, "isolated": 1, "symmetric": 0, "weighted": 0}
    k1 = gp.tune_key(info, gp.TUNE_ALL, "GB300")
    assert k1 != gp.tune_key(dict(info, m=21), gp.TUNE_ALL, "GB300")
    assert k1 != gp.tune_key(info, gp.TUNE_PULL, "GB300")
    assert k1 != gp.tune_key(info, gp.TUNE_ALL, "B200")
    path = str(tmp_path / "sub" / "tune.json")
    opts = gp.options_dict(gp.default_options())
    assert set(opts) == set(gp.OPTION_FIELDS)
    # every field of gp_options is cached (a tuned value left out would be lost on a cache hit)
    assert set(opts) == {f for f, _ in gp.gp_options._fields_ if not f.startswith("reserved")}
    assert opts["bfs_groups"] == 0 and opts["bfs_light_max"] == 32 and opts["pull_hot_slots"] == 20480
    gp.tune_cache_store(path, k1, {"options": opts, "evaluated": 3})
    gp.tune_cache_store(path, "other", {"options": opts, "evaluated": 1})
    data = gp.tune_cache_load(path)
    assert data[k1]["options"] == opts and data[k1]["evaluated"] == 3 and "other" in data
    assert gp.tune_cache_load(str(tmp_path / "missing.json")) == {}
    monkeypatch.setenv("GP_TUNE_CACHE", path)
    assert gp.tune_cache_path() == path
    assert gp.tune_cache_path(str(tmp_path / "x.json")) == str(tmp_path / "x.json")


def test_struct_layouts():
    import ctypes

    import paper_2010_16012_gb300 as gp

    assert ctypes.sizeof(gp.gp_tune_result) == 80
    assert ctypes.sizeof(gp.gp_batch_stats) == 24
    assert ctypes.sizeof(gp.gp_batch_options) == 32
