"""Seeded synthetic graph inputs for the push/pull sweeps.

This package only manufactures inputs (R-MAT and Erdos-Renyi graphs, hand-made
small graphs, edge weights and random vertex picks) in the paper's adjacency
layout (Section 2.2: one contiguous neighbour array plus per-vertex offsets, for
out-edges = CSR and for in-edges = CSC).  It contains none of PageRank's or
BFS's arithmetic.  Both the CPU oracle and the CUDA library consume what it
returns; they share nothing else.

The sampling code is plain C (``graphgen.c``), compiled on first use with gcc,
so a graph is bit-identical on x86-64 and AArch64 and independent of the number
of threads.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_SO = os.path.join(_HERE, "_graphgen.so")
_lock = threading.Lock()
_lib = None

RMAT_A, RMAT_B, RMAT_C = 0.57, 0.19, 0.19


def build(force: bool = False) -> str:
    """Compile graphgen.c into _graphgen.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _get():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
            i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
            f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
            c = ctypes
            lib.gg_key.restype = c.c_uint64
            lib.gg_key.argtypes = [c.c_uint64]
            lib.gg_draw.restype = c.c_uint64
            lib.gg_draw.argtypes = [c.c_uint64, c.c_uint64]
            lib.gg_rmat_edges.restype = None
            lib.gg_rmat_edges.argtypes = [c.c_int, c.c_int64, c.c_double, c.c_double, c.c_double,
                                          c.c_uint64, i32p, i32p, c.c_int]
            lib.gg_er_edges.restype = None
            lib.gg_er_edges.argtypes = [c.c_int64, c.c_int64, c.c_uint64, i32p, i32p, c.c_int]
            lib.gg_build_csr.restype = c.c_int64
            lib.gg_build_csr.argtypes = [c.c_int64, c.c_int64, i32p, i32p, c.c_int, c.c_int, c.c_int,
                                         i64p, i32p, c.c_int64, c.c_int]
            lib.gg_transpose.restype = None
            lib.gg_transpose.argtypes = [c.c_int64, i64p, i32p, c.c_void_p, i64p, i32p, c.c_void_p,
                                         c.c_void_p]
            lib.gg_uniform_weights.restype = None
            lib.gg_uniform_weights.argtypes = [c.c_int64, c.c_uint64, f32p, c.c_int]
            lib.gg_normalize_rows.restype = None
            lib.gg_normalize_rows.argtypes = [c.c_int64, i64p, f32p, c.c_int]
            lib.gg_int_weights.argtypes = [c.c_int64, c.c_uint64, c.c_int32, c.c_int32, f32p, c.c_int]
            lib.gg_pick_vertices.restype = c.c_int64
            lib.gg_pick_vertices.argtypes = [c.c_int64, i64p, c.c_int64, c.c_int64, c.c_uint64, i32p]
            _lib = lib
    return _lib


@dataclass
class Graph:
    """A directed graph in both adjacency directions.

    ``csr_off``/``csr_idx``: out-edges (row u lists the heads v of u->v, ascending).
    ``csc_off``/``csc_idx``: in-edges (column v lists the tails u of u->v, ascending).
    ``csr_w``/``csc_w``: optional FP32 weights of the same edges in each order.
    An undirected graph is stored as its symmetric directed version, where the
    two directions coincide (``symmetric`` is True and the arrays are shared).
    """

    name: str
    n: int
    csr_off: np.ndarray
    csr_idx: np.ndarray
    csc_off: np.ndarray
    csc_idx: np.ndarray
    symmetric: bool = False
    csr_w: Optional[np.ndarray] = None
    csc_w: Optional[np.ndarray] = None
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.csr_off[-1])

    def out_degree(self) -> np.ndarray:
        return np.diff(self.csr_off)

    def in_degree(self) -> np.ndarray:
        return np.diff(self.csc_off)

    def edges(self):
        """(src, dst) int32 arrays of all edges, in CSR order."""
        src = np.repeat(np.arange(self.n, dtype=np.int32), np.diff(self.csr_off))
        return src, self.csr_idx

    def with_weights(self, seed: int, normalize: bool = True, nthreads: int = 0) -> "Graph":
        """Copy of the graph with weights uniform in (0, 1] (one draw per CSR edge),
        optionally scaled so every source's out-weights sum to one."""
        lib = _get()
        w = np.empty(self.m, dtype=np.float32)
        lib.gg_uniform_weights(self.m, seed, w, nthreads)
        if normalize:
            lib.gg_normalize_rows(self.n, self.csr_off, w, nthreads)
        perm = _transpose_perm(self)
        return Graph(self.name + f"+w{seed}", self.n, self.csr_off, self.csr_idx, self.csc_off,
                     self.csc_idx, self.symmetric, w, np.ascontiguousarray(w[perm]),
                     dict(self.meta, weight_seed=seed, normalized=normalize))


def with_int_weights(g: Graph, seed: int, lo: int = 1, hi: int = 255, symmetric_weights: bool = False,
                     nthreads: int = 0) -> Graph:
    """Copy of the graph with integer-valued weights uniform in [lo, hi] (stored
    as float32; path sums are exact in FP32 below 2^24).  One draw per CSR edge;
    with symmetric_weights (symmetric graphs only) the edge u->v takes the draw
    of its u < v direction, so w(u->v) = w(v->u)."""
    lib = _get()
    w = np.empty(g.m, dtype=np.float32)
    lib.gg_int_weights(g.m, seed, lo, hi, w, nthreads)
    perm = _transpose_perm(g)
    if symmetric_weights:
        if not g.symmetric:
            raise ValueError("symmetric weights need a symmetric graph")
        src, dst = g.edges()
        swap = src > dst  # take the weight of the reverse edge: CSC slot perm maps CSR edge -> reverse
        w = np.where(swap, w[perm], w).astype(np.float32)
    return Graph(g.name + f"+iw{seed}", g.n, g.csr_off, g.csr_idx, g.csc_off, g.csc_idx, g.symmetric, w,
                 np.ascontiguousarray(w[perm]), dict(g.meta, weight_seed=seed, int_weights=(lo, hi)))


def _transpose_perm(g: Graph) -> np.ndarray:
    lib = _get()
    toff = np.empty(g.n + 1, dtype=np.int64)
    tidx = np.empty(g.m, dtype=np.int32)
    perm = np.empty(g.m, dtype=np.int64)
    lib.gg_transpose(g.n, g.csr_off, g.csr_idx, None, toff, tidx, None, perm.ctypes.data)
    return perm


def from_edges(n: int, src, dst, *, symmetrize: bool = False, drop_self: bool = True,
               dedup: bool = True, name: str = "edges", nthreads: int = 0) -> Graph:
    """Build CSR + CSC from an edge list (sorted rows; optional symmetrise,
    self-loop removal and de-duplication)."""
    lib = _get()
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    ne = int(src.shape[0])
    cap = max(1, (2 if symmetrize else 1) * ne)
    off = np.empty(n + 1, dtype=np.int64)
    idx = np.empty(cap, dtype=np.int32)
    m = lib.gg_build_csr(n, ne, src, dst, int(symmetrize), int(drop_self), int(dedup), off, idx, cap,
                         nthreads)
    if m < 0:
        raise ValueError("edge endpoint outside [0, n)")
    idx = np.ascontiguousarray(idx[:m]) if m < cap else idx
    if symmetrize:
        return Graph(name, n, off, idx, off, idx, True)
    toff = np.empty(n + 1, dtype=np.int64)
    tidx = np.empty(m, dtype=np.int32)
    lib.gg_transpose(n, off, idx, None, toff, tidx, None, None)
    return Graph(name, n, off, idx, toff, tidx, False)


def rmat(scale: int, edgefactor: int = 16, a: float = RMAT_A, b: float = RMAT_B, c: float = RMAT_C,
         seed: int = 1, symmetrize: bool = True, nthreads: int = 0) -> Graph:
    """R-MAT graph with 2^scale vertices from edgefactor * 2^scale sampled edges,
    self-loops and duplicates removed, symmetrised by default."""
    lib = _get()
    n = 1 << scale
    ne = edgefactor * n
    src = np.empty(ne, dtype=np.int32)
    dst = np.empty(ne, dtype=np.int32)
    lib.gg_rmat_edges(scale, ne, a, b, c, seed, src, dst, nthreads)
    g = from_edges(n, src, dst, symmetrize=symmetrize, name=f"rmat{scale}_ef{edgefactor}_s{seed}",
                   nthreads=nthreads)
    g.meta.update(kind="rmat", scale=scale, edgefactor=edgefactor, a=a, b=b, c=c, seed=seed)
    return g


def erdos_renyi(n: int, samples: int, seed: int, nthreads: int = 0) -> Graph:
    """Directed Erdos-Renyi G(n, m) graph from `samples` uniform (src, dst)
    pairs, self-loops and duplicates removed."""
    lib = _get()
    src = np.empty(samples, dtype=np.int32)
    dst = np.empty(samples, dtype=np.int32)
    lib.gg_er_edges(n, samples, seed, src, dst, nthreads)
    g = from_edges(n, src, dst, symmetrize=False, name=f"er{n}_m{samples}_s{seed}", nthreads=nthreads)
    g.meta.update(kind="er", samples=samples, seed=seed)
    return g


def pick_vertices(g: Graph, count: int, seed: int, min_out_degree: int = 1) -> np.ndarray:
    """`count` distinct vertices with out-degree >= min_out_degree (seeded)."""
    lib = _get()
    out = np.empty(max(count, 1), dtype=np.int32)
    got = lib.gg_pick_vertices(g.n, g.csr_off, count, min_out_degree, seed, out)
    return out[:got].copy()


def draw(seed: int, i: int) -> int:
    """Draw i (a 64-bit integer) of the stream for `seed`."""
    lib = _get()
    return int(lib.gg_draw(lib.gg_key(seed), i))


# ---------------------------------------------------------------- hand-made graphs

def path(n: int, directed: bool = False) -> Graph:
    """0 - 1 - ... - (n-1)."""
    s = np.arange(max(n - 1, 0), dtype=np.int32)
    return from_edges(n, s, s + 1, symmetrize=not directed, name=f"path{n}")


def cycle(n: int, directed: bool = True) -> Graph:
    """0 -> 1 -> ... -> n-1 -> 0."""
    s = np.arange(n, dtype=np.int32)
    return from_edges(n, s, (s + 1) % n, symmetrize=not directed, name=f"cycle{n}")


def complete(n: int) -> Graph:
    """K_n: every ordered pair (u, v), u != v."""
    u, v = np.meshgrid(np.arange(n, dtype=np.int32), np.arange(n, dtype=np.int32), indexing="ij")
    keep = u != v
    return from_edges(n, u[keep], v[keep], name=f"K{n}")


def star(k: int) -> Graph:
    """Undirected star: centre 0 joined to leaves 1..k."""
    leaves = np.arange(1, k + 1, dtype=np.int32)
    return from_edges(k + 1, np.zeros(k, dtype=np.int32), leaves, symmetrize=True, name=f"star{k}")


def binary_tree(n: int) -> Graph:
    """Undirected heap-ordered binary tree: i joined to 2i+1 and 2i+2."""
    child = np.arange(1, n, dtype=np.int32)
    return from_edges(n, (child - 1) // 2, child, symmetrize=True, name=f"btree{n}")


def empty(n: int) -> Graph:
    """n isolated vertices."""
    z = np.zeros(0, dtype=np.int32)
    return from_edges(n, z, z, name=f"empty{n}")


def random_small(n: int, p: float, seed: int, directed: bool = True) -> Graph:
    """Small G(n, p) graph for fuzzing: pair (u, v) kept when draw u*n+v < p."""
    key_draws = np.array([draw(seed, i) for i in range(n * n)], dtype=np.uint64)
    keep = (key_draws >> np.uint64(11)).astype(np.float64) * 2.0 ** -53 < p
    u, v = np.divmod(np.nonzero(keep)[0], n)
    return from_edges(n, u.astype(np.int32), v.astype(np.int32), symmetrize=not directed,
                      name=f"gnp{n}_{p}_{seed}")
