"""Plain FP64 CPU oracle for push/pull PageRank and BFS (ctypes over oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The CUDA library never
imports this package and this package never imports the library; they share no
code.  Inputs come from the ``graphgen`` package, which holds no method
arithmetic.

What each function computes, with the paper passage it follows, is documented
in ``oracle.c``.  Parity status: every function here is pinned by the
``-m "not gpu"`` tests in ``tests/test_oracle_pins.py`` (closed forms, a dense
linear solve, brute-force shortest paths, a hand-derived worked example and
finite differences).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None

PUSH, PULL = 0, 1
TOPDOWN, BOTTOMUP = 0, 1


def build(force: bool = False) -> str:
    """Compile oracle.c into _oracle.so (gcc -O2, OpenMP, strict IEEE: no -ffast-math)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _get():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            c = ctypes
            vp = c.c_void_p
            lib.or_graph_new.restype = vp
            lib.or_graph_new.argtypes = [c.c_int64, c.c_int64, vp, vp, vp]
            lib.or_graph_free.restype = None
            lib.or_graph_free.argtypes = [vp]
            lib.or_pagerank.restype = c.c_int
            lib.or_pagerank.argtypes = [vp, c.c_int, c.c_double, c.c_int, c.c_double, vp, vp, vp,
                                        c.POINTER(c.c_int), c.POINTER(c.c_double), c.c_int]
            lib.or_bfs_fifo.restype = c.c_int64
            lib.or_bfs_fifo.argtypes = [vp, c.c_int32, vp, vp]
            lib.or_bfs_levelsync.restype = c.c_int
            lib.or_bfs_levelsync.argtypes = [vp, c.c_int32, vp, c.c_int, vp, vp, vp, c.c_int]
            lib.or_pagerank_adjoint.restype = c.c_int
            lib.or_pagerank_adjoint.argtypes = [vp, c.c_double, vp, vp, c.c_int, c.c_double, vp, vp, vp,
                                                c.POINTER(c.c_double), c.c_int]
            lib.or_pagerank_adjoint_raw.restype = c.c_int
            lib.or_pagerank_adjoint_raw.argtypes = [vp, c.c_double, vp, vp, c.c_int, c.c_double, vp, vp, vp, vp]
            lib.or_sssp_dijkstra.restype = c.c_int64
            lib.or_sssp_dijkstra.argtypes = [vp, c.c_int32, vp, vp]
            lib.or_sssp_delta.restype = c.c_int64
            lib.or_sssp_delta.argtypes = [vp, c.c_int32, c.c_double, vp, c.c_int, vp, c.POINTER(c.c_int64)]
            lib.or_pagerank_fe.restype = c.c_int
            lib.or_pagerank_fe.argtypes = [vp, c.c_double, c.c_double, c.c_int, vp, vp, c.c_int, vp, vp]
            lib.or_bc.restype = c.c_int
            lib.or_bc.argtypes = [vp, vp, c.c_int64, vp]
            lib.or_triangles.restype = c.c_int64
            lib.or_triangles.argtypes = [vp, c.c_int, vp, c.c_int]
            lib.or_max_threads.restype = c.c_int
            lib.or_max_threads.argtypes = []
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class OracleGraph:
    """The oracle's own adjacency, rebuilt from an edge list (src[e] -> dst[e],
    optional per-edge weight w[e] = P_{dst,src}, taken in double precision)."""

    def __init__(self, n: int, src, dst, w=None):
        self._lib = _get()
        self.n = int(n)
        self._src = np.ascontiguousarray(src, dtype=np.int32)
        self._dst = np.ascontiguousarray(dst, dtype=np.int32)
        self.m = int(self._src.shape[0])
        if self.m and (self._src.min() < 0 or self._src.max() >= n or self._dst.min() < 0
                       or self._dst.max() >= n):
            raise ValueError("edge endpoint outside [0, n)")
        # weights in double precision (float32 inputs convert exactly)
        self._w = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
        self._h = self._lib.or_graph_new(self.n, self.m, _ptr(self._src), _ptr(self._dst), _ptr(self._w))

    @classmethod
    def from_graph(cls, g, weighted: bool = True):
        """From a graphgen.Graph: its edge list in CSR order (and CSR weights)."""
        src, dst = g.edges()
        return cls(g.n, src, dst, g.csr_w if weighted else None)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.or_graph_free(h)
            self._h = None

    # ------------------------------------------------------------ PageRank
    def pagerank(self, variant: int = PULL, damping: float = 0.85, iters: int = 20, tol: float = 0.0,
                 personalization=None, x0=None, nthreads: int = 1):
        """Power iteration (Algorithm 1).  Returns (x, iters_done, residual, converged)."""
        x = np.empty(self.n, dtype=np.float64)
        s = None if personalization is None else np.ascontiguousarray(personalization, dtype=np.float64)
        x0a = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
        k = ctypes.c_int(0)
        r = ctypes.c_double(0.0)
        rc = self._lib.or_pagerank(self._h, int(variant), float(damping), int(iters), float(tol),
                                   _ptr(s), _ptr(x0a), _ptr(x), ctypes.byref(k), ctypes.byref(r),
                                   int(nthreads))
        return x, k.value, r.value, rc == 0

    # ------------------------------------------------------------ BFS
    def bfs(self, src: int):
        """FIFO BFS over out-edges.  Returns (level, parent) int32 arrays."""
        level = np.empty(self.n, dtype=np.int32)
        parent = np.empty(self.n, dtype=np.int32)
        self._lib.or_bfs_fifo(self._h, int(src), _ptr(level), _ptr(parent))
        return level, parent

    def bfs_levelsync(self, src: int, dirs=(TOPDOWN,), max_levels: int = 4096):
        """Level-synchronous BFS (Algorithm 3, ready = 1) with one direction per
        level (0 top-down/push, 1 bottom-up/pull; the last entry repeats).
        Returns (level, parent, dirs_used)."""
        level = np.empty(self.n, dtype=np.int32)
        parent = np.empty(self.n, dtype=np.int32)
        d = np.ascontiguousarray(np.asarray(dirs, dtype=np.int8))
        used = np.full(max_levels, -1, dtype=np.int8)
        L = self._lib.or_bfs_levelsync(self._h, int(src), _ptr(d), int(d.shape[0]), _ptr(level),
                                       _ptr(parent), _ptr(used), max_levels)
        return level, parent, used[:min(L, max_levels)].copy()

    # ------------------------------------------------------------ adjoint
    def pagerank_adjoint(self, x, g, damping: float = 0.85, iters: int = 10000, tol: float = 1e-14,
                         nthreads: int = 1):
        """Adjoint of the fixed point for L = g.x.  Returns (lambda, grad_s,
        grad_w in input edge order, iters_done, residual)."""
        lam = np.empty(self.n, dtype=np.float64)
        gs = np.empty(self.n, dtype=np.float64)
        gw = np.empty(self.m, dtype=np.float64)
        r = ctypes.c_double(0.0)
        xa = np.ascontiguousarray(x, dtype=np.float64)
        ga = np.ascontiguousarray(g, dtype=np.float64)
        k = self._lib.or_pagerank_adjoint(self._h, float(damping), _ptr(xa), _ptr(ga), int(iters),
                                          float(tol), _ptr(lam), _ptr(gs), _ptr(gw), ctypes.byref(r),
                                          int(nthreads))
        return lam, gs, gw, k, r.value

    def pagerank_adjoint_raw(self, g, damping: float = 0.85, personalization=None, iters: int = 100000,
                             tol: float = 1e-14):
        """Gradient of L = g.x* with respect to the RAW weights this graph was
        built with, normalised per source inside (P_vu = W_uv / S_u).  Returns
        (x*, lambda, grad_s, grad_W in input edge order, converged)."""
        n, m = self.n, self.m
        x, lam, gs = (np.empty(n, dtype=np.float64) for _ in range(3))
        gW = np.empty(m, dtype=np.float64)
        s = None if personalization is None else np.ascontiguousarray(personalization, dtype=np.float64)
        ga = np.ascontiguousarray(g, dtype=np.float64)
        rc = self._lib.or_pagerank_adjoint_raw(self._h, float(damping), _ptr(s), _ptr(ga), int(iters), float(tol),
                                               _ptr(x), _ptr(lam), _ptr(gs), _ptr(gW))
        return x, lam, gs, gW, rc == 0

    # ------------------------------------------------------------ SSSP
    def sssp(self, src: int):
        """Dijkstra (FP64).  Returns (dist float64 with inf unreached, pred int32)."""
        dist = np.empty(self.n, dtype=np.float64)
        pred = np.empty(self.n, dtype=np.int32)
        self._lib.or_sssp_dijkstra(self._h, int(src), _ptr(dist), _ptr(pred))
        return dist, pred

    def sssp_delta(self, src: int, delta: float, dirs=(PUSH,)):
        """Delta-Stepping, one direction per relaxation iteration (0 push,
        1 pull; the last entry repeats).  Returns (dist, iterations, epochs)."""
        dist = np.empty(self.n, dtype=np.float64)
        d = np.ascontiguousarray(np.asarray(dirs, dtype=np.int8))
        ep = ctypes.c_int64(0)
        it = self._lib.or_sssp_delta(self._h, int(src), float(delta), _ptr(d), int(d.shape[0]), _ptr(dist),
                                     ctypes.byref(ep))
        return dist, int(it), ep.value


    # ------------------------------------------------------------ Frontier-Exploit PageRank
    def pagerank_fe(self, damping: float = 0.85, eps: float = 1e-9, iters: int = 1000, personalization=None,
                    dirs=(PULL,)):
        """Residual-propagation PageRank from a frontier (|r| > eps).  Returns
        (x, r, iterations)."""
        x = np.empty(self.n, dtype=np.float64)
        r = np.empty(self.n, dtype=np.float64)
        s = None if personalization is None else np.ascontiguousarray(personalization, dtype=np.float64)
        d = np.ascontiguousarray(np.asarray(dirs, dtype=np.int8))
        k = self._lib.or_pagerank_fe(self._h, float(damping), float(eps), int(iters), _ptr(s), _ptr(d),
                                     int(d.shape[0]), _ptr(x), _ptr(r))
        return x, r, int(k)

    # ------------------------------------------------------------ betweenness centrality
    def bc(self, sources):
        """Brandes betweenness centrality summed over `sources` (FP64)."""
        src = np.ascontiguousarray(np.asarray(sources, dtype=np.int32))
        out = np.empty(self.n, dtype=np.float64)
        self._lib.or_bc(self._h, _ptr(src), int(src.shape[0]), _ptr(out))
        return out

    # ------------------------------------------------------------ triangles
    def triangles(self, variant: int = PULL, nthreads: int = 1):
        """NodeIterator triangle counts (the graph must be symmetric, simple).
        Returns (tc int64[n], total triangles)."""
        tc = np.empty(self.n, dtype=np.int64)
        total = self._lib.or_triangles(self._h, int(variant), _ptr(tc), int(nthreads))
        return tc, int(total)


def max_threads() -> int:
    return int(_get().or_max_threads())
