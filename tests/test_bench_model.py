"""The benchmark's roofline byte models and traffic lookup (host logic, no GPU):
the pull sweep's compulsory bytes are 4m + 28n + 8, the push sweep's 4m + 24n + 8
(+4m weighted); the two pull kernels' index streams together cover every edge
once; a BFS level's bytes follow its per-level counts; a traffic row counts only
while its source key matches."""
import types

import bench
import graphgen as gg


def _opts(**kw):
    o = dict(pull_light_max=16, push_light_max=16, chunk_edges=256)
    o.update(kw)
    return types.SimpleNamespace(**o)


def test_sweep_bytes_closed_forms():
    g = gg.rmat(10, 8, seed=3)
    n, m = g.n, g.m
    assert bench.sweep_bytes(g) == 4 * m + 28 * n + 8
    assert bench.pr_sweep_bytes(g, 1) == bench.sweep_bytes(g)
    assert bench.pr_sweep_bytes(g, 0) == 4 * m + 24 * n + 8
    assert bench.pr_sweep_bytes(g, 1, weighted=True) - bench.pr_sweep_bytes(g, 1) == 4 * m
    assert bench.pr_sweep_bytes(g, 0, weighted=True) - bench.pr_sweep_bytes(g, 0) == 4 * m


def test_pull_kernels_split_the_index_stream():
    """Whatever the light limit, the big kernel's index bytes plus the light
    kernel's equal 4m, and the big kernel's chunk count follows the chunk size."""
    g = gg.rmat(11, 16, seed=5)
    din = g.in_degree()
    n, m = g.n, g.m
    for light in (0, 4, 16, 64, 1 << 20):
        for C in (32, 256):
            kb = bench.kernel_bytes(g, _opts(pull_light_max=light, chunk_edges=C))
            big = din > light
            e_big = int(din[big].sum())
            ch = int(((din[big] + C - 1) // C).sum())
            assert kb["pull_big"] == 4 * e_big + 20 * ch
            light_index = kb["pull_light"] - (8 * (n + 1) + 20 * n + 4 * ch + 12 * int(big.sum()))
            assert light_index + 4 * e_big == 4 * m
    # every vertex light: no big kernel bytes at all
    kb = bench.kernel_bytes(g, _opts(pull_light_max=int(din.max())))
    assert kb["pull_big"] == 0
    # the push epilogue: FP64 accumulator (default) 32n, FP32 24n, as the library's rule picks
    assert kb["push_epilogue"] == 32 * n
    assert bench.kernel_bytes(g, _opts(push_fp64_accum=0))["push_epilogue"] == 24 * n
    assert bench.kernel_bytes(g, _opts(push_fp64_accum=1), l2_bytes=1024)["push_epilogue"] == 32 * n
    small_l2 = 8 * n  # the FP64 array is twice half the L2
    want = 24 if int(din.max()) <= 4096 else 32
    assert bench.kernel_bytes(g, _opts(), l2_bytes=small_l2)["push_epilogue"] == want * n


def test_push_kernel_counts_every_out_edge():
    g = gg.star(300)  # one hub with 299 out-edges, 299 leaves with one
    dout = g.out_degree()
    kb = bench.kernel_bytes(g, _opts(push_light_max=16, chunk_edges=32))
    ch = int(((dout[dout > 16] + 31) // 32).sum())
    assert ch == (int(dout.max()) + 31) // 32
    assert kb["push_scatter"] == 4 * g.m + 8 * (g.n + 1) + 12 * g.n + 16 * ch


def test_bfs_level_bytes():
    n = 1 << 12
    name, by = bench.bfs_level_bytes(n, 0, frontier=10, examined=100, candidates=0, new=7)
    assert name == "bfs_topdown" and by == 20 * 10 + 4 * 100 + 48 * 7
    name, by = bench.bfs_level_bytes(n, 1, frontier=10, examined=100, candidates=50, new=7)
    assert name == "bfs_bottomup" and by == 2 * (n // 8) + 20 * 50 + 4 * 100 + 8 * 7
    # a level that finds nothing still reads its frontier (top-down) or its bitmaps (bottom-up)
    assert bench.bfs_level_bytes(n, 0, 1, 0, 0, 0)[1] == 20
    assert bench.bfs_level_bytes(n, 1, 1, 0, 0, 0)[1] == n // 4


def test_captured_traffic_follows_the_source_key(monkeypatch):
    assert bench.captured_traffic("no_such_kernel") is None
    got = bench.captured_traffic("pull_big")
    if got is not None:  # the committed row matches the current source
        assert isinstance(got, int) and got > 4 * 4_000_000
    monkeypatch.setattr(bench, "source_key", lambda cu: "0" * 16)
    assert bench.captured_traffic("pull_big") is None


def test_source_key_covers_kernel_and_shared_header(tmp_path, monkeypatch):
    """The key changes with either file: a copy of the tree with one byte added to
    the shared header gives another key."""
    import shutil

    src = tmp_path / "paper_2010_16012_gb300" / "csrc"
    src.mkdir(parents=True)
    real = bench.ROOT
    for f in ("pagerank.cu", "gp_internal.cuh"):
        shutil.copy(f"{real}/paper_2010_16012_gb300/csrc/{f}", src / f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    k1 = bench.source_key("pagerank.cu")
    with open(src / "gp_internal.cuh", "a") as fh:
        fh.write("\n")
    assert bench.source_key("pagerank.cu") != k1
