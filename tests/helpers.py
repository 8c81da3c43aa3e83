"""Test helpers: golden-file parsing and independent reference computations
(numpy linear algebra, brute-force shortest paths) used to pin the oracle."""
from __future__ import annotations

import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _frac(tok: str) -> Fraction:
    return Fraction(tok)


def parse_pagerank_cases(path=os.path.join(GOLDEN, "pagerank_worked_examples.txt")):
    cases, cur = [], None
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        key, *vals = line.split()
        if key == "case":
            cur = {"name": vals[0]}
        elif key == "end":
            cases.append(cur)
            cur = None
        elif key == "n":
            cur["n"] = int(vals[0])
        elif key == "d":
            cur["d"] = _frac(vals[0])
        elif key == "edges":
            src, dst, w = [], [], []
            for tok in vals:
                uv, _, wt = tok.partition(":")
                u, v = uv.split(">")
                src.append(int(u))
                dst.append(int(v))
                w.append(_frac(wt) if wt else None)
            cur["src"], cur["dst"] = src, dst
            cur["w"] = None if all(x is None for x in w) else w
        elif key in ("sweep1", "sweep2", "fixed"):
            cur[key] = [_frac(t) for t in vals]
        elif key in ("res1", "res2"):
            cur[key] = _frac(vals[0])
    return cases


def parse_bfs_case(path=os.path.join(GOLDEN, "bfs_worked_example.txt")):
    out = {}
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        key, *vals = line.split()
        if key == "edges":
            out["src_e"] = [int(t.split(">")[0]) for t in vals]
            out["dst_e"] = [int(t.split(">")[1]) for t in vals]
        elif key in ("n", "src"):
            out[key] = int(vals[0])
        else:
            out[key] = [int(t) for t in vals]
    return out


def dense_transition(n, src, dst, w=None):
    """Column-stochastic-or-leaky P with P[v, u] = w_e or 1/deg_out(u) for edge e=(u->v)."""
    src = np.asarray(src)
    dst = np.asarray(dst)
    P = np.zeros((n, n))
    deg = np.bincount(src, minlength=n) if len(src) else np.zeros(n, dtype=np.int64)
    for e in range(len(src)):
        u, v = src[e], dst[e]
        P[v, u] += (float(w[e]) if w is not None else 1.0 / deg[u])
    return P


def dense_pagerank(n, src, dst, d, s=None, w=None):
    """Fixed point of x = (1-d)s + dPx by LU with partial pivoting (numpy.linalg.solve)."""
    P = dense_transition(n, src, dst, w)
    s = np.full(n, 1.0 / n) if s is None else np.asarray(s, dtype=np.float64)
    return np.linalg.solve(np.eye(n) - d * P, (1 - d) * s)


def floyd_warshall_levels(n, src, dst, root):
    """Unit-weight all-pairs shortest paths by Floyd-Warshall; row `root` as BFS levels."""
    INF = np.inf
    D = np.full((n, n), INF)
    np.fill_diagonal(D, 0.0)
    for u, v in zip(src, dst):
        if u != v:
            D[u, v] = min(D[u, v], 1.0)
    for k in range(n):
        D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])
    row = D[root]
    return np.where(np.isinf(row), -1, row).astype(np.int64)


def check_parents(n, src_e, dst_e, root, level, parent):
    """BFS-tree validity: root is its own parent at level 0; every reached v != root
    has an edge parent[v] -> v and level[parent[v]] == level[v] - 1; unreached
    vertices have parent -1.  Returns a list of violations (empty when valid)."""
    edges = set(zip(np.asarray(src_e).tolist(), np.asarray(dst_e).tolist()))
    bad = []
    if level[root] != 0 or parent[root] != root:
        bad.append(("root", root))
    for v in range(n):
        if v == root:
            continue
        if level[v] == -1:
            if parent[v] != -1:
                bad.append(("unreached-has-parent", v))
            continue
        p = parent[v]
        if p < 0 or (p, v) not in edges or level[p] != level[v] - 1:
            bad.append(("bad-parent", v, p))
    return bad


def check_parents_np(csr_off, csr_idx, root, level, parent):
    """Vectorised check_parents for large graphs (edge existence by searching the
    sorted CSR row of the parent).  Returns the number of violations."""
    n = level.shape[0]
    level = level.astype(np.int64)
    parent = parent.astype(np.int64)
    bad = 0
    bad += int(level[root] != 0) + int(parent[root] != root)
    reached = level >= 0
    reached[root] = False
    bad += int(np.count_nonzero(parent[level < 0] != -1))
    v = np.nonzero(reached)[0]
    p = parent[v]
    okp = (p >= 0) & (p < n)
    bad += int(np.count_nonzero(~okp))
    v, p = v[okp], p[okp]
    bad += int(np.count_nonzero(level[p] != level[v] - 1))
    beg = csr_off[p]
    end = csr_off[p + 1]
    # edge p->v exists iff v appears in sorted row p
    found = np.zeros(v.shape[0], dtype=bool)
    # vectorised binary search over rows
    lo, hi = beg.copy(), end.copy()
    while True:
        active = lo < hi
        if not active.any():
            break
        mid = (lo + hi) // 2
        mv = np.where(active, csr_idx[np.minimum(mid, len(csr_idx) - 1)], 0)
        less = active & (mv < v)
        lo = np.where(less, mid + 1, lo)
        hi = np.where(active & ~less, mid, hi)
    inrow = lo < end
    found[inrow] = csr_idx[lo[inrow]] == v[inrow]
    bad += int(np.count_nonzero(~found))
    return bad


def edge_sources(csr_off):
    """Tail of every CSR edge slot (int32[m])."""
    deg = np.diff(csr_off)
    return np.repeat(np.arange(deg.shape[0], dtype=np.int32), deg)


def check_levels_by_edges(csr_src, csr_idx, root, level):
    """Edge conditions that, together with valid parents (check_parents_np),
    make `level` exactly the BFS distance from `root` at any graph size: the
    root has level 0, and no edge u->v leaves a reached u towards an unreached
    v or a v more than one level below u.  (Parents give a path of length
    level[v], so level >= distance; the edge rule along a shortest path gives
    level <= distance.)  Returns the number of violations."""
    lv = level.astype(np.int64)
    lu = lv[csr_src]
    lh = lv[csr_idx]
    bad = int(lv[root] != 0)
    bad += int(np.count_nonzero((lu >= 0) & ((lh < 0) | (lh > lu + 1))))
    return bad


def parse_sssp_cases(path=os.path.join(GOLDEN, "sssp_worked_example.txt")):
    """(n, src_e, dst_e, w_e, [(src, dist, pred), ...]) from the SSSP fixture."""
    n, cases, cur = 0, [], None
    src_e, dst_e, w_e = [], [], []
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        key, *vals = line.split()
        if key == "n":
            n = int(vals[0])
        elif key == "edges":
            for t in vals:
                uv, w = t.split(":")
                u, v = uv.split(">")
                src_e.append(int(u))
                dst_e.append(int(v))
                w_e.append(float(w))
        elif key == "src":
            cur = [int(vals[0]), None, None]
            cases.append(cur)
        elif key == "dist":
            cur[1] = [float("inf") if t == "inf" else float(t) for t in vals]
        elif key == "pred":
            cur[2] = [int(t) for t in vals]
    return n, src_e, dst_e, w_e, cases


def floyd_warshall_dist(n, src, dst, w):
    """All-pairs shortest path weights by Floyd-Warshall (min-plus closure), inf if none."""
    D = np.full((n, n), np.inf)
    np.fill_diagonal(D, 0.0)
    for u, v, x in zip(src, dst, w):
        D[u, v] = min(D[u, v], float(x))
    for k in range(n):
        D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])
    return D


def check_sssp_certificate(csr_off, csr_idx, csr_w, src, dist, pred):
    """Conditions that make `dist` the exact shortest distances at any size:
    dist[src] = 0; every edge u->v with finite dist[u] satisfies dist[v] <=
    dist[u] + w (so no path is shorter than dist: dist is a lower bound); every
    reached v != src has a tight predecessor edge, dist[v] = dist[pred] + w, and
    the predecessors lead back to src (so dist[v] is the length of a real path);
    unreached vertices have dist inf and pred -1.
    Weights are compared in FP32 as the library forms the sums.  Returns the
    number of violations."""
    dist = np.asarray(dist, dtype=np.float32)
    pred = np.asarray(pred, dtype=np.int64)
    n = dist.shape[0]
    deg = np.diff(csr_off)
    u = np.repeat(np.arange(n, dtype=np.int64), deg)
    w = np.ones(csr_idx.shape[0], dtype=np.float32) if csr_w is None else np.asarray(csr_w, dtype=np.float32)
    bad = int(dist[src] != 0) + int(pred[src] != src)
    fin = np.isfinite(dist[u])
    relax = (dist[u] + w).astype(np.float32)
    bad += int(np.count_nonzero(fin & (dist[csr_idx] > relax)))
    reached = np.isfinite(dist)
    bad += int(np.count_nonzero(~reached & (pred != -1)))
    v = np.nonzero(reached)[0]
    v = v[v != src]
    p = pred[v]
    ok = (p >= 0) & (p < n)
    bad += int(np.count_nonzero(~ok))
    v, p = v[ok], p[ok]
    # tight predecessor edge p->v: the slot of v in p's sorted row (vectorised
    # binary search), whose weight makes dist[p] + w == dist[v]
    lo, hi = csr_off[p].copy(), csr_off[p + 1].copy()
    while True:
        active = lo < hi
        if not active.any():
            break
        mid = (lo + hi) // 2
        mv = np.where(active, csr_idx[np.minimum(mid, len(csr_idx) - 1)], 0)
        less = active & (mv < v)
        lo = np.where(less, mid + 1, lo)
        hi = np.where(active & ~less, mid, hi)
    found = (lo < csr_off[p + 1]) & (csr_idx[np.minimum(lo, len(csr_idx) - 1)] == v)
    wv = w[np.minimum(lo, len(w) - 1)]
    tight = found & ((dist[p] + wv).astype(np.float32) == dist[v])
    bad += int(np.count_nonzero(~tight))
    # the predecessor pointers reach src from every reached vertex (no cycle of
    # zero-weight tight edges): follow them by pointer doubling
    hop = np.where(reached, pred, -1)
    hop[src] = src
    cur = np.where(reached, hop, -1)
    for _ in range(int(np.ceil(np.log2(max(n, 2)))) + 1):
        nxt = np.where(cur >= 0, hop[np.maximum(cur, 0)], -1)
        cur = nxt
    bad += int(np.count_nonzero(reached & (cur != src)))
    return bad


def smallest_tight_pred(csr_off, csr_idx, csr_w, src, dist):
    """For each reached v != src, the smallest u with an edge u->v and dist[u] + w == dist[v] (FP32)."""
    dist = np.asarray(dist, dtype=np.float32)
    n = dist.shape[0]
    u = np.repeat(np.arange(n, dtype=np.int64), np.diff(csr_off))
    w = np.ones(csr_idx.shape[0], dtype=np.float32) if csr_w is None else np.asarray(csr_w, dtype=np.float32)
    tight = np.isfinite(dist[u]) & ((dist[u] + w).astype(np.float32) == dist[csr_idx])
    out = np.full(n, -1, dtype=np.int64)
    best = np.full(n, np.iinfo(np.int64).max, dtype=np.int64)
    np.minimum.at(best, csr_idx[tight].astype(np.int64), u[tight])
    has = best != np.iinfo(np.int64).max
    out[has] = best[has]
    out[src] = src
    return out
