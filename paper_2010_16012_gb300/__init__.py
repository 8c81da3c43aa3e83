"""Push/pull graph sweeps on GB300: Python binding of libgp.

Thin ctypes layer over the C ABI declared in include/gp.h, with the same names
and argument marshalling only: every step of PageRank and BFS runs in libgp's
CUDA kernels.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if libgp.so is missing, load() raises.

    import paper_2010_16012_gb300 as gp
    G = gp.Graph.from_arrays(n, csr_off, csr_idx, csc_off, csc_idx)   # torch CUDA tensors
    ranks, st = gp.pagerank(G, gp.PULL, damping=0.85, iters=300, tol=1e-7)
    level, parent, st = gp.bfs(G, src=0, mode=gp.AUTO)
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgp.so")

PUSH, PULL, AUTO = 0, 1, 2
TUNE_PULL, TUNE_PUSH, TUNE_AUTO, TUNE_BFS, TUNE_ALL = 0x1, 0x2, 0x4, 0x8, 0xF
UPLOAD_VALIDATE, UPLOAD_SYMMETRIC, UPLOAD_COPY, UPLOAD_NORMALIZE = 0x1, 0x2, 0x4, 0x8
OK, ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
BFS_MAX_LEVELS = 512

_lock = threading.Lock()
_lib = None


class GpError(RuntimeError):
    def __init__(self, status: int, what: str, message: str):
        super().__init__(f"{what}: status {status} ({message})")
        self.status = status


class gp_options(ctypes.Structure):
    _fields_ = [("pull_light_max", ctypes.c_int32), ("push_light_max", ctypes.c_int32),
                ("chunk_edges", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("poll_interval", ctypes.c_int32), ("pr_auto_mode", ctypes.c_int32),
                ("bfs_alpha", ctypes.c_float), ("bfs_beta", ctypes.c_float),
                ("push_fp64_accum", ctypes.c_int32), ("pull_hot_slots", ctypes.c_int32),
                ("push_hot_slots", ctypes.c_int32), ("sssp_alpha", ctypes.c_float), ("fe_alpha", ctypes.c_float),
                ("bc_alpha", ctypes.c_float), ("bfs_light_max", ctypes.c_int32), ("bfs_groups", ctypes.c_int32)]


class gp_graph_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("max_out_degree", ctypes.c_int64),
                ("max_in_degree", ctypes.c_int64), ("pull_big_vertices", ctypes.c_int64),
                ("pull_big_chunks", ctypes.c_int64), ("push_big_vertices", ctypes.c_int64),
                ("push_big_chunks", ctypes.c_int64), ("isolated", ctypes.c_int64),
                ("symmetric", ctypes.c_int32), ("weighted", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64)]


class gp_pr_stats(ctypes.Structure):
    _fields_ = [("iters_done", ctypes.c_int32), ("mode_used", ctypes.c_int32), ("residual", ctypes.c_double),
                ("ms", ctypes.c_float), ("converged", ctypes.c_int32), ("push_updates_l2", ctypes.c_int64),
                ("push_updates_shared", ctypes.c_int64), ("push_updates_merged", ctypes.c_int64),
                ("push_flush_l2", ctypes.c_int64)]


class gp_bfs_stats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("switches", ctypes.c_int32), ("reached", ctypes.c_int64),
                ("edges_examined", ctypes.c_int64), ("edges_reached", ctypes.c_int64), ("ms", ctypes.c_float),
                ("direction", ctypes.c_int8 * BFS_MAX_LEVELS), ("frontier", ctypes.c_int64 * BFS_MAX_LEVELS),
                ("examined", ctypes.c_int64 * BFS_MAX_LEVELS), ("init_ns", ctypes.c_int32),
                ("level_ns", ctypes.c_int32 * BFS_MAX_LEVELS)]


class gp_bfs_summary(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("switches", ctypes.c_int32), ("reached", ctypes.c_int64),
                ("edges_examined", ctypes.c_int64), ("edges_reached", ctypes.c_int64)]


SSSP_MAX_ITERS = 1024


class gp_sssp_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("epochs", ctypes.c_int32), ("reached", ctypes.c_int64),
                ("edges_examined", ctypes.c_int64), ("pushes", ctypes.c_int32), ("pulls", ctypes.c_int32),
                ("ms", ctypes.c_float), ("init_ns", ctypes.c_int32), ("direction", ctypes.c_int8 * SSSP_MAX_ITERS),
                ("bucket", ctypes.c_int64 * SSSP_MAX_ITERS), ("active", ctypes.c_int64 * SSSP_MAX_ITERS),
                ("examined", ctypes.c_int64 * SSSP_MAX_ITERS), ("iter_ns", ctypes.c_int32 * SSSP_MAX_ITERS)]


FE_MAX_ITERS = 1024


class gp_fe_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("pushes", ctypes.c_int32), ("pulls", ctypes.c_int32),
                ("residual_l1", ctypes.c_double), ("error_bound", ctypes.c_double),
                ("frontier_left", ctypes.c_int64), ("ms", ctypes.c_float), ("init_ns", ctypes.c_int32),
                ("direction", ctypes.c_int8 * FE_MAX_ITERS), ("frontier", ctypes.c_int64 * FE_MAX_ITERS),
                ("examined", ctypes.c_int64 * FE_MAX_ITERS), ("iter_ns", ctypes.c_int32 * FE_MAX_ITERS)]


class gp_tc_stats(ctypes.Structure):
    _fields_ = [("triangles", ctypes.c_int64), ("probes", ctypes.c_int64), ("ms", ctypes.c_float),
                ("mode_used", ctypes.c_int32)]


BC_MAX_STEPS = 1024


class gp_bc_stats(ctypes.Structure):
    _fields_ = [("sources", ctypes.c_int64), ("levels", ctypes.c_int64), ("reached", ctypes.c_int64),
                ("edges_examined", ctypes.c_int64), ("pushes", ctypes.c_int64), ("pulls", ctypes.c_int64),
                ("ms", ctypes.c_float), ("steps", ctypes.c_int32), ("direction", ctypes.c_int8 * BC_MAX_STEPS),
                ("phase", ctypes.c_int8 * BC_MAX_STEPS), ("level", ctypes.c_int32 * BC_MAX_STEPS),
                ("frontier", ctypes.c_int64 * BC_MAX_STEPS), ("examined", ctypes.c_int64 * BC_MAX_STEPS),
                ("step_ns", ctypes.c_int32 * BC_MAX_STEPS)]


class gp_batch_stats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int32), ("levels", ctypes.c_int32), ("ms", ctypes.c_float),
                ("blocks", ctypes.c_int32), ("jobs", ctypes.c_int32), ("packed", ctypes.c_int32)]


class gp_batch_options(ctypes.Structure):
    _fields_ = [("big_in_degree", ctypes.c_int32), ("chunk_edges", ctypes.c_int32), ("l2_budget_mb", ctypes.c_int32),
                ("msbfs_alpha", ctypes.c_float), ("msbfs_beta", ctypes.c_float), ("ppr_start", ctypes.c_int32),
                ("ppr_pack", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]


class gp_batch_tune_result(ctypes.Structure):
    _fields_ = [("options", gp_batch_options), ("ppr_ms", ctypes.c_float), ("msbfs_ms", ctypes.c_float),
                ("trials", ctypes.c_int32)]


class gp_tune_result(ctypes.Structure):
    _fields_ = [("best", gp_options), ("pull_ms_per_sweep", ctypes.c_float), ("push_ms_per_sweep", ctypes.c_float),
                ("bfs_ms", ctypes.c_float), ("evaluated", ctypes.c_int32)]


class gp_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

# (name, restype, argtypes) of every entry point of include/gp.h
_VP, _I32, _I64, _F, _D, _U = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double, ctypes.c_uint
SIGNATURES = [
    ("gp_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("gp_last_error", ctypes.c_char_p, []),
    ("gp_version", ctypes.c_int, []),
    ("gp_set_allocator", ctypes.c_int, [ALLOC_FN, FREE_FN, _VP]),
    ("gp_pool_usage", ctypes.c_int, [ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    ("gp_pool_trim", ctypes.c_int, [_I64]),
    ("gp_graph_upload", ctypes.c_int, [ctypes.POINTER(_VP), _I64, _I64, _VP, _VP, _VP, _VP, _VP, _VP, _U, _VP]),
    ("gp_graph_free", ctypes.c_int, [_VP]),
    ("gp_graph_info_get", ctypes.c_int, [_VP, ctypes.POINTER(gp_graph_info)]),
    ("gp_options_default", ctypes.c_int, [ctypes.POINTER(gp_options)]),
    ("gp_graph_set_options", ctypes.c_int, [_VP, ctypes.POINTER(gp_options), _VP]),
    ("gp_graph_get_options", ctypes.c_int, [_VP, ctypes.POINTER(gp_options)]),
    ("gp_pagerank", ctypes.c_int, [_VP, ctypes.c_int, _F, ctypes.c_int, _D, _VP, _VP, _VP,
                                   ctypes.POINTER(gp_pr_stats), _VP]),
    ("gp_pagerank_backward", ctypes.c_int, [_VP, ctypes.c_int, _F, _VP, _VP, _VP, _VP, ctypes.c_int, _D,
                                            ctypes.POINTER(gp_pr_stats), _VP]),
    ("gp_graph_set_weights", ctypes.c_int, [_VP, _VP, _VP, _VP]),
    ("gp_bfs", ctypes.c_int, [_VP, _I32, ctypes.c_int, _VP, _VP, ctypes.POINTER(gp_bfs_stats), _VP]),
    ("gp_bfs_multi", ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, _VP, _VP, ctypes.c_int,
                                    ctypes.POINTER(gp_bfs_summary), _VP]),
    ("gp_bfs_directed", ctypes.c_int, [_VP, _I32, _VP, ctypes.c_int, _VP, _VP, ctypes.POINTER(gp_bfs_stats),
                                       _VP]),
    ("gp_sssp", ctypes.c_int, [_VP, _I32, _F, ctypes.c_int, _VP, ctypes.c_int, _VP, _VP,
                               ctypes.POINTER(gp_sssp_stats), _VP]),
    ("gp_pagerank_fe", ctypes.c_int, [_VP, ctypes.c_int, _F, _D, ctypes.c_int, _VP, ctypes.c_int, _VP, _VP,
                                      ctypes.POINTER(gp_fe_stats), _VP]),
    ("gp_triangles", ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, ctypes.POINTER(gp_tc_stats), _VP]),
    ("gp_bc", ctypes.c_int, [_VP, _VP, ctypes.c_int64, ctypes.c_int, _VP, ctypes.c_int, _VP,
                             ctypes.POINTER(gp_bc_stats), _VP]),
    ("gp_batch_create", ctypes.c_int, [ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.c_int, ctypes.c_int, _VP]),
    ("gp_batch_free", ctypes.c_int, [_VP]),
    ("gp_batch_options_default", ctypes.c_int, [ctypes.POINTER(gp_batch_options)]),
    ("gp_batch_set_options", ctypes.c_int, [_VP, ctypes.POINTER(gp_batch_options), _VP]),
    ("gp_batch_get_options", ctypes.c_int, [_VP, ctypes.POINTER(gp_batch_options)]),
    ("gp_batch_autotune", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(gp_batch_tune_result), _VP]),
    ("gp_ppr_batched", ctypes.c_int, [_VP, _VP, _F, ctypes.c_int, _D, ctypes.POINTER(_VP), _VP,
                                      ctypes.POINTER(gp_batch_stats), _VP]),
    ("gp_msbfs_batched", ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.POINTER(_VP), ctypes.POINTER(gp_batch_stats),
                                        _VP]),
    ("gp_pull_sweep_noalloc", ctypes.c_int, [_I64, _I64, _VP, _VP, _VP, _VP, _VP, _F, _VP, _VP, _VP, _VP]),
    ("gp_autotune", ctypes.c_int, [_VP, _U, _VP, ctypes.c_int, ctypes.POINTER(gp_tune_result), _VP]),
    ("gp_profile_enable", ctypes.c_int, [ctypes.c_int]),
    ("gp_profile_read", ctypes.c_int, [ctypes.POINTER(gp_kernel_time), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    ("gp_selftest_narrow", ctypes.c_int, [_I64, _VP, _VP, _VP, _VP]),
    ("gp_selftest_barrier", ctypes.c_int, [ctypes.c_int, _VP]),
]


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libgp.so (raises if it has not been built: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"libgp CUDA library not built ({path} missing): run "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            lib = ctypes.CDLL(path)
            for name, res, args in SIGNATURES:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(status: int, what: str, allow=()):
    if status != OK and status not in allow:
        lib = load()
        msg = lib.gp_last_error().decode() or lib.gp_status_string(status).decode()
        raise GpError(status, what, msg)
    return status


def _torch():
    import torch

    return torch


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    """Device or host address of a torch tensor / numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return ctypes.c_void_p(t.ctypes.data)
    assert t.is_contiguous()
    return ctypes.c_void_p(t.data_ptr())


def default_options() -> gp_options:
    o = gp_options()
    _check(load().gp_options_default(ctypes.byref(o)), "gp_options_default")
    return o


class Graph:
    """A graph uploaded to the GPU (the gp_graph handle).

    Arrays are int64 offsets / int32 indices (/ float32 weights) in CSR
    (out-edges) and CSC (in-edges) order.  CUDA tensors are read in place and
    kept referenced by this object; numpy arrays (or copy=True) are copied into
    library-owned device memory by gp_graph_upload.
    """

    def __init__(self, n, csr_off, csr_idx, csc_off=None, csc_idx=None, csr_w=None, csc_w=None, *,
                 symmetric=False, validate=False, normalize=False, copy=None, stream=None):
        lib = load()
        host = any(isinstance(a, np.ndarray) for a in (csr_off, csr_idx, csc_off, csc_idx, csr_w, csc_w))
        if copy is None:
            copy = host
        flags = (UPLOAD_VALIDATE if validate else 0) | (UPLOAD_SYMMETRIC if symmetric else 0) | \
                (UPLOAD_COPY if copy else 0) | (UPLOAD_NORMALIZE if normalize else 0)
        self._keep = None if copy else (csr_off, csr_idx, csc_off, csc_idx, csr_w, csc_w)
        self.n = int(n)
        self.m = int(csr_idx.shape[0])
        self.symmetric = symmetric
        self.weighted = csr_w is not None
        self._stream = stream
        h = ctypes.c_void_p()
        _check(lib.gp_graph_upload(ctypes.byref(h), self.n, self.m, _ptr(csr_off), _ptr(csr_idx), _ptr(csr_w),
                                   _ptr(csc_off), _ptr(csc_idx), _ptr(csc_w), flags, _stream_ptr(stream)),
               "gp_graph_upload")
        self._h = h

    @classmethod
    def from_graphgen(cls, g, device="cuda", validate=False, normalize=False, copy=False, stream=None):
        """Upload a graphgen.Graph (host numpy arrays): moved to CUDA tensors
        first unless copy=True (then gp_graph_upload copies from host)."""
        # a symmetric structure with per-source weights is not a symmetric graph:
        # its CSC weights differ, so it is uploaded with both directions
        sym = g.symmetric and g.csr_w is None
        if copy:
            return cls(g.n, g.csr_off, g.csr_idx, None if sym else g.csc_off, None if sym else g.csc_idx, g.csr_w,
                       None if sym else g.csc_w, symmetric=sym, validate=validate, normalize=normalize, copy=True,
                       stream=stream)
        torch = _torch()
        t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(device)
        csr_off, csr_idx = t(g.csr_off), t(g.csr_idx)
        csr_w = t(g.csr_w)
        if sym:
            return cls(g.n, csr_off, csr_idx, None, None, csr_w, None, symmetric=True, validate=validate,
                       normalize=normalize, stream=stream)
        return cls(g.n, csr_off, csr_idx, t(g.csc_off), t(g.csc_idx), csr_w, t(g.csc_w), validate=validate,
                   normalize=normalize, stream=stream)

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("graph already freed")
        return self._h

    def free(self):
        if getattr(self, "_h", None):
            _check(load().gp_graph_free(self._h), "gp_graph_free")
            self._h = None
            self._keep = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def info(self) -> dict:
        i = gp_graph_info()
        _check(load().gp_graph_info_get(self.handle, ctypes.byref(i)), "gp_graph_info_get")
        return {f: getattr(i, f) for f, _ in gp_graph_info._fields_}

    def options(self) -> gp_options:
        o = gp_options()
        _check(load().gp_graph_get_options(self.handle, ctypes.byref(o)), "gp_graph_get_options")
        return o

    def set_weights(self, csr_w, csc_w=None, stream=None):
        """gp_graph_set_weights: point the graph at new (device) weight arrays."""
        self._wkeep = (csr_w, csc_w)
        _check(load().gp_graph_set_weights(self.handle, _ptr(csr_w), _ptr(csc_w), _stream_ptr(stream)),
               "gp_graph_set_weights")

    def set_options(self, opt: gp_options = None, stream=None, **kw):
        o = opt if opt is not None else self.options()
        for k, v in kw.items():
            setattr(o, k, v)
        _check(load().gp_graph_set_options(self.handle, ctypes.byref(o), _stream_ptr(stream)),
               "gp_graph_set_options")


def pagerank(g: Graph, mode=PULL, damping=0.85, iters=20, tol=0.0, personalization=None, x0=None, out=None,
             stream=None, raise_not_converged=False):
    """gp_pagerank.  Returns (ranks, stats dict).  `out` may be a CUDA tensor
    or a host (numpy / CPU tensor) array; by default a new CUDA tensor."""
    torch = _torch()
    if out is None:
        out = torch.empty(g.n, dtype=torch.float32, device="cuda")
    st = gp_pr_stats()
    allow = () if raise_not_converged else (ERR_NOT_CONVERGED,)
    _check(load().gp_pagerank(g.handle, int(mode), float(damping), int(iters), float(tol), _ptr(personalization),
                              _ptr(x0), _ptr(out), ctypes.byref(st), _stream_ptr(stream)), "gp_pagerank", allow)
    return out, {"iters_done": st.iters_done, "mode_used": st.mode_used, "residual": st.residual, "ms": st.ms,
                 "converged": bool(st.converged), "push_updates_l2": st.push_updates_l2,
                 "push_updates_shared": st.push_updates_shared, "push_updates_merged": st.push_updates_merged,
                 "push_flush_l2": st.push_flush_l2}


def pagerank_backward(g: Graph, ranks, grad_ranks, mode=PULL, damping=0.85, iters=1000, tol=1e-7,
                      want_weights=True, want_personalization=True, stream=None, raise_not_converged=False):
    """gp_pagerank_backward.  Returns (grad_weights [CSR order] or None,
    grad_personalization or None, stats dict)."""
    torch = _torch()
    gw = torch.empty(g.m, dtype=torch.float32, device="cuda") if want_weights else None
    gs = torch.empty(g.n, dtype=torch.float32, device="cuda") if want_personalization else None
    st = gp_pr_stats()
    allow = () if raise_not_converged else (ERR_NOT_CONVERGED,)
    _check(load().gp_pagerank_backward(g.handle, int(mode), float(damping), _ptr(ranks), _ptr(grad_ranks), _ptr(gw),
                                       _ptr(gs), int(iters), float(tol), ctypes.byref(st), _stream_ptr(stream)),
           "gp_pagerank_backward", allow)
    return gw, gs, {"iters_done": st.iters_done, "residual": st.residual, "ms": st.ms,
                    "converged": bool(st.converged)}


def _autograd_function():
    torch = _torch()

    class PageRankFunction(torch.autograd.Function):
        """x = PageRank(csr_w, s) with gradients by the adjoint kernels (implicit
        differentiation of the fixed point; nothing is checkpointed)."""

        @staticmethod
        def forward(ctx, csr_w, personalization, graph, csc_perm, damping, iters, tol, mode, adj_iters, adj_tol):
            ctx.weights = None
            if csr_w is not None:
                csc_w = None if csc_perm is None else csr_w.detach().index_select(0, csc_perm).contiguous()
                ctx.weights = (csr_w.detach().contiguous(), csc_w)
                graph.set_weights(*ctx.weights)
            s = None if personalization is None else personalization.detach().contiguous()
            x, _ = pagerank(graph, mode, damping, iters, tol, personalization=s)
            ctx.graph = graph
            ctx.cfg = (damping, mode, adj_iters, adj_tol)
            ctx.has_w = csr_w is not None
            ctx.has_s = personalization is not None
            ctx.save_for_backward(x)
            return x

        @staticmethod
        def backward(ctx, grad_x):
            (x,) = ctx.saved_tensors
            damping, mode, adj_iters, adj_tol = ctx.cfg
            if ctx.weights is not None:  # another forward may have repointed the shared graph since
                ctx.graph.set_weights(*ctx.weights)
            gw, gs, _ = pagerank_backward(ctx.graph, x, grad_x.contiguous().float(), mode, damping, adj_iters, adj_tol,
                                          want_weights=ctx.has_w, want_personalization=ctx.has_s)
            return gw, gs, None, None, None, None, None, None, None, None

    return PageRankFunction


def pagerank_autograd(graph: Graph, csr_w=None, personalization=None, csc_perm=None, damping=0.85, iters=1000,
                      tol=1e-7, mode=PULL, adj_iters=1000, adj_tol=1e-7):
    """Differentiable PageRank: gradients flow to the CSR edge weights `csr_w`
    (`csc_perm[j]` = CSR position of CSC slot j for non-symmetric graphs) and to
    the personalization vector.

    The graph's weights are replaced in place: after the call `graph` points at
    copies of `csr_w` (and its CSC permutation) made by this forward pass, for
    later gp_pagerank calls too.  Backward points the graph at its own forward's
    weights again before the adjoint, so several autograd graphs may share one
    Graph and run their backward passes in any order, provided they are used
    from one host thread at a time."""
    global _PRF
    if _PRF is None:
        _PRF = _autograd_function()
    return _PRF.apply(csr_w, personalization, graph, csc_perm, damping, iters, tol, mode, adj_iters, adj_tol)


_PRF = None


def bfs(g: Graph, src: int, mode=AUTO, level=None, parent=None, want_parent=True, dirs=None, stream=None,
        want_stats=True):
    """gp_bfs / gp_bfs_directed.  Returns (level, parent or None, stats dict or
    None).  With want_stats=False and device outputs the call returns without
    waiting for the search (a barrier timeout is then reported by the next
    search on the graph)."""
    torch = _torch()
    if level is None:
        level = torch.empty(g.n, dtype=torch.int32, device="cuda")
    if parent is None and want_parent:
        parent = torch.empty(g.n, dtype=torch.int32, device="cuda")
    st = gp_bfs_stats()
    stp = ctypes.byref(st) if want_stats else None
    lib = load()
    if dirs is None:
        _check(lib.gp_bfs(g.handle, int(src), int(mode), _ptr(level), _ptr(parent), stp, _stream_ptr(stream)),
               "gp_bfs")
    else:
        d = np.ascontiguousarray(np.asarray(dirs, dtype=np.int8))
        _check(lib.gp_bfs_directed(g.handle, int(src), _ptr(d), int(d.shape[0]), _ptr(level), _ptr(parent), stp,
                                   _stream_ptr(stream)), "gp_bfs_directed")
    if not want_stats:
        return level, parent, None
    L = min(st.levels, BFS_MAX_LEVELS)
    stats = {"levels": st.levels, "switches": st.switches, "reached": st.reached,
             "edges_examined": st.edges_examined, "edges_reached": st.edges_reached, "ms": st.ms,
             "direction": list(st.direction[:L]), "frontier": list(st.frontier[:L]),
             "examined": list(st.examined[:L]), "init_us": st.init_ns / 1e3,
             "level_us": [x / 1e3 for x in st.level_ns[:L]]}
    return level, parent, stats


def bfs_multi(g: Graph, sources, mode=AUTO, levels=None, parents=None, want_parent=True, groups=0, stream=None,
              want_summary=True):
    """gp_bfs_multi: independent searches from every source in one launch.
    levels / parents: lists of CUDA int32 tensors of n entries (allocated when
    None).  Returns (levels, parents or None, list of summary dicts or None).
    With want_summary=False the call returns without waiting (a barrier
    timeout is then reported by the next gp_bfs_multi on the graph)."""
    torch = _torch()
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.int32).reshape(-1))
    k = int(src.shape[0])
    if levels is None:
        levels = [torch.empty(g.n, dtype=torch.int32, device="cuda") for _ in range(k)]
    if parents is None and want_parent:
        parents = [torch.empty(g.n, dtype=torch.int32, device="cuda") for _ in range(k)]
    if len(levels) != k or (parents is not None and len(parents) != k):
        raise ValueError("bfs_multi: one level (and parent) tensor per source")
    lp = (ctypes.c_void_p * max(k, 1))(*[t.data_ptr() for t in levels])
    pp = None if parents is None else (ctypes.c_void_p * max(k, 1))(*[t.data_ptr() for t in parents])
    sm = (gp_bfs_summary * max(k, 1))() if want_summary else None
    _check(load().gp_bfs_multi(g.handle, _ptr(src), k, int(mode), ctypes.cast(lp, _VP),
                               None if pp is None else ctypes.cast(pp, _VP), int(groups), sm, _stream_ptr(stream)),
           "gp_bfs_multi")
    if not want_summary:
        return levels, parents, None
    out = [{"levels": x.levels, "switches": x.switches, "reached": x.reached, "edges_examined": x.edges_examined,
            "edges_reached": x.edges_reached} for x in sm[:k]]
    return levels, parents, out


def sssp(g: Graph, src: int, delta: float, mode=AUTO, dist=None, pred=None, want_pred=True, dirs=None,
         stream=None, want_stats=True):
    """gp_sssp.  Returns (dist, pred or None, stats dict or None)."""
    torch = _torch()
    if dist is None:
        dist = torch.empty(g.n, dtype=torch.float32, device="cuda")
    if pred is None and want_pred:
        pred = torch.empty(g.n, dtype=torch.int32, device="cuda")
    st = gp_sssp_stats()
    d = None if dirs is None else np.ascontiguousarray(np.asarray(dirs, dtype=np.int8))
    _check(load().gp_sssp(g.handle, int(src), float(delta), int(mode), _ptr(d), 0 if d is None else int(d.shape[0]),
                          _ptr(dist), _ptr(pred), ctypes.byref(st) if want_stats else None, _stream_ptr(stream)),
           "gp_sssp")
    if not want_stats:
        return dist, pred, None
    L = min(st.iterations, SSSP_MAX_ITERS)
    stats = {"iterations": st.iterations, "epochs": st.epochs, "reached": st.reached,
             "edges_examined": st.edges_examined, "pushes": st.pushes, "pulls": st.pulls, "ms": st.ms,
             "init_us": st.init_ns / 1e3, "direction": list(st.direction[:L]), "bucket": list(st.bucket[:L]),
             "active": list(st.active[:L]), "examined": list(st.examined[:L]),
             "iter_us": [x / 1e3 for x in st.iter_ns[:L]]}
    return dist, pred, stats


def pagerank_fe(g: Graph, mode=AUTO, damping=0.85, eps=1e-9, iters=1000, personalization=None, out=None, dirs=None,
                stream=None, raise_not_converged=False):
    """gp_pagerank_fe.  Returns (ranks, stats dict)."""
    torch = _torch()
    if out is None:
        out = torch.empty(g.n, dtype=torch.float32, device="cuda")
    st = gp_fe_stats()
    d = None if dirs is None else np.ascontiguousarray(np.asarray(dirs, dtype=np.int8))
    allow = () if raise_not_converged else (ERR_NOT_CONVERGED,)
    _check(load().gp_pagerank_fe(g.handle, int(mode), float(damping), float(eps), int(iters), _ptr(d),
                                 0 if d is None else int(d.shape[0]), _ptr(personalization), _ptr(out),
                                 ctypes.byref(st), _stream_ptr(stream)), "gp_pagerank_fe", allow)
    L = min(st.iterations, FE_MAX_ITERS)
    return out, {"iterations": st.iterations, "pushes": st.pushes, "pulls": st.pulls,
                 "residual_l1": st.residual_l1, "error_bound": st.error_bound, "frontier_left": st.frontier_left,
                 "ms": st.ms, "init_us": st.init_ns / 1e3, "direction": list(st.direction[:L]),
                 "frontier": list(st.frontier[:L]), "examined": list(st.examined[:L]),
                 "iter_us": [x / 1e3 for x in st.iter_ns[:L]]}


def triangles(g: Graph, mode=PULL, out=None, stream=None):
    """gp_triangles.  Returns (per-vertex counts int64, total, stats dict)."""
    torch = _torch()
    if out is None:
        out = torch.empty(g.n, dtype=torch.int64, device="cuda")
    total = ctypes.c_int64(0)
    st = gp_tc_stats()
    _check(load().gp_triangles(g.handle, int(mode), _ptr(out), ctypes.byref(total), ctypes.byref(st),
                               _stream_ptr(stream)), "gp_triangles")
    return out, total.value, {"triangles": st.triangles, "probes": st.probes, "ms": st.ms,
                              "mode_used": st.mode_used}


def bc(g: Graph, sources, mode=AUTO, dirs=None, out=None, want_stats=True, stream=None):
    """gp_bc: betweenness centrality summed over `sources` (int32, host array or
    device tensor).  Returns (FP64 centralities, stats dict or None)."""
    torch = _torch()
    if out is None:
        out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    if hasattr(sources, "data_ptr"):
        assert sources.dtype == torch.int32 and sources.is_contiguous()
        src, nsrc = sources, int(sources.numel())
    else:
        src = np.ascontiguousarray(np.asarray(sources, dtype=np.int32))
        nsrc = int(src.shape[0])
    d = None if dirs is None else np.ascontiguousarray(np.asarray(dirs, dtype=np.int8))
    st = gp_bc_stats() if want_stats else None
    _check(load().gp_bc(g.handle, _ptr(src) if nsrc else None, nsrc, int(mode), _ptr(d),
                        0 if d is None else int(d.shape[0]), _ptr(out), ctypes.byref(st) if st else None,
                        _stream_ptr(stream)), "gp_bc")
    if st is None:
        return out, None
    L = st.steps
    return out, {"sources": st.sources, "levels": st.levels, "reached": st.reached,
                 "edges_examined": st.edges_examined, "pushes": st.pushes, "pulls": st.pulls, "ms": st.ms,
                 "steps": L, "direction": list(st.direction[:L]), "phase": list(st.phase[:L]),
                 "level": list(st.level[:L]), "frontier": list(st.frontier[:L]), "examined": list(st.examined[:L]),
                 "step_us": [x / 1e3 for x in st.step_ns[:L]]}


def pool_usage():
    """gp_pool_usage: (reserved, used) bytes of the library's default memory pool
    on the current device."""
    r, u = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(load().gp_pool_usage(ctypes.byref(r), ctypes.byref(u)), "gp_pool_usage")
    return r.value, u.value


def pool_trim(keep_bytes=0):
    """gp_pool_trim: return the pool's unused memory to the driver, keeping at
    most keep_bytes reserved."""
    _check(load().gp_pool_trim(int(keep_bytes)), "gp_pool_trim")


class Batch:
    """gp_batch: batched personalised PageRank and multi-source BFS over several graphs."""

    def __init__(self, graphs, k_ppr=256, stream=None):
        lib = load()
        self.graphs = list(graphs)
        self.k = int(k_ppr)
        arr = (ctypes.c_void_p * len(self.graphs))(*[g.handle.value for g in self.graphs])
        h = ctypes.c_void_p()
        _check(lib.gp_batch_create(ctypes.byref(h), arr, len(self.graphs), self.k, _stream_ptr(stream)),
               "gp_batch_create")
        self._h = h

    def free(self):
        if getattr(self, "_h", None):
            _check(load().gp_batch_free(self._h), "gp_batch_free")
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    BATCH_OPTION_FIELDS = ("big_in_degree", "chunk_edges", "l2_budget_mb", "msbfs_alpha", "msbfs_beta", "ppr_start",
                           "ppr_pack")

    def options(self) -> dict:
        o = gp_batch_options()
        _check(load().gp_batch_get_options(self._h, ctypes.byref(o)), "gp_batch_get_options")
        return {f: getattr(o, f) for f in self.BATCH_OPTION_FIELDS}

    def set_options(self, stream=None, **kw):
        o = gp_batch_options()
        _check(load().gp_batch_get_options(self._h, ctypes.byref(o)), "gp_batch_get_options")
        for k, v in kw.items():
            if k not in self.BATCH_OPTION_FIELDS:
                raise KeyError(k)
            setattr(o, k, v)
        _check(load().gp_batch_set_options(self._h, ctypes.byref(o), _stream_ptr(stream)), "gp_batch_set_options")

    def autotune(self, seeds=None, sources=None, ppr_sweeps=16, stream=None) -> dict:
        """gp_batch_autotune: choose and install the fastest options for these
        seeds ([ngraphs][k]) and BFS sources ([ngraphs][nsrc]).  Returns
        {"options", "ppr_ms", "msbfs_ms", "trials"}."""
        sd = None if seeds is None else np.ascontiguousarray(
            np.asarray(seeds, dtype=np.int32).reshape(len(self.graphs), self.k))
        so = None if sources is None else np.ascontiguousarray(np.asarray(sources, dtype=np.int32))
        nsrc = 0 if so is None else int(so.shape[1])
        r = gp_batch_tune_result()
        _check(load().gp_batch_autotune(self._h, _ptr(sd), _ptr(so), nsrc, int(ppr_sweeps), ctypes.byref(r),
                                        _stream_ptr(stream)), "gp_batch_autotune")
        return {"options": {f: getattr(r.options, f) for f in self.BATCH_OPTION_FIELDS}, "ppr_ms": r.ppr_ms,
                "msbfs_ms": r.msbfs_ms, "trials": r.trials}

    def ppr(self, seeds, damping=0.85, iters=1000, tol=1e-6, outs=None, stream=None):
        """seeds: int array [ngraphs][k].  Returns (list of [n_i, k] tensors, iters_done [ngraphs, k], stats)."""
        torch = _torch()
        seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.int32).reshape(len(self.graphs), self.k))
        if outs is None:
            outs = [torch.empty((g.n, self.k), dtype=torch.float32, device="cuda") for g in self.graphs]
        optr = (ctypes.c_void_p * len(outs))(*[o.data_ptr() if hasattr(o, "data_ptr") else o.ctypes.data for o in outs])
        done = np.zeros((len(self.graphs), self.k), dtype=np.int32)
        st = gp_batch_stats()
        _check(load().gp_ppr_batched(self._h, _ptr(seeds), float(damping), int(iters), float(tol), optr, _ptr(done),
                                     ctypes.byref(st), _stream_ptr(stream)), "gp_ppr_batched")
        return outs, done, {"sweeps": st.sweeps, "ms": st.ms, "blocks": st.blocks, "jobs": st.jobs,
                            "packed": st.packed}

    def msbfs(self, sources, outs=None, stream=None):
        """sources: int array [ngraphs][nsrc] (nsrc <= 64).  Returns (list of [n_i, 64] int32 tensors, stats)."""
        torch = _torch()
        sources = np.ascontiguousarray(np.asarray(sources, dtype=np.int32))
        nsrc = sources.shape[1]
        if outs is None:
            outs = [torch.empty((g.n, 64), dtype=torch.int32, device="cuda") for g in self.graphs]
        optr = (ctypes.c_void_p * len(outs))(*[o.data_ptr() if hasattr(o, "data_ptr") else o.ctypes.data for o in outs])
        st = gp_batch_stats()
        _check(load().gp_msbfs_batched(self._h, _ptr(sources), int(nsrc), optr, ctypes.byref(st), _stream_ptr(stream)),
               "gp_msbfs_batched")
        return outs, {"levels": st.levels, "ms": st.ms, "blocks": st.blocks}


OPTION_FIELDS = ["pull_light_max", "push_light_max", "chunk_edges", "blocks_per_sm", "poll_interval", "pr_auto_mode",
                 "bfs_alpha", "bfs_beta", "push_fp64_accum", "pull_hot_slots", "push_hot_slots", "sssp_alpha",
                 "fe_alpha", "bc_alpha", "bfs_light_max", "bfs_groups"]


def options_dict(o: gp_options) -> dict:
    return {f: getattr(o, f) for f in OPTION_FIELDS}


def tune_key(info: dict, what: int, device_name: str = "") -> str:
    """Cache key of a tuning result: the graph's shape statistics, what was tuned
    and the GPU model."""
    return "|".join(str(x) for x in (device_name, info["n"], info["m"], info["max_out_degree"], info["max_in_degree"],
                                     info["isolated"], info["symmetric"], info["weighted"], what))


def tune_cache_path(path=None) -> str:
    """The JSON cache file: `path`, else $GP_TUNE_CACHE, else ~/.cache/gp_tune.json."""
    return path or os.environ.get("GP_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "gp_tune.json")


def tune_cache_load(path) -> dict:
    import json

    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune_cache_store(path, key: str, entry: dict):
    import json

    data = tune_cache_load(path)
    data[key] = entry
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def autotune(g: Graph, what: int = TUNE_ALL, sources=None, cache=None, use_cache: bool = True, stream=None) -> dict:
    """gp_autotune with a JSON cache keyed by graph statistics and GPU model.
    Returns {"options": {...}, "cached": bool, ...timings}."""
    torch = _torch()
    path = tune_cache_path(cache)
    key = tune_key(g.info(), what, torch.cuda.get_device_name())
    if use_cache:
        hit = tune_cache_load(path).get(key)
        if hit:
            g.set_options(stream=stream, **hit["options"])
            return dict(hit, cached=True)
    src = None
    n_src = 0
    if what & TUNE_BFS:
        src = np.ascontiguousarray(np.asarray(sources, dtype=np.int32))
        n_src = int(src.shape[0])
    res = gp_tune_result()
    _check(load().gp_autotune(g.handle, int(what), _ptr(src), n_src, ctypes.byref(res), _stream_ptr(stream)),
           "gp_autotune")
    entry = {"options": options_dict(res.best), "pull_ms_per_sweep": res.pull_ms_per_sweep,
             "push_ms_per_sweep": res.push_ms_per_sweep, "bfs_ms": res.bfs_ms, "evaluated": res.evaluated}
    if use_cache:
        tune_cache_store(path, key, entry)
    return dict(entry, cached=False)


NOALLOC_MAX_VERTICES = 1 << 20


def pull_sweep_noalloc(n, m, csc_off, csc_idx, inv_deg, x, y, residual, damping=0.85, csc_w=None,
                       personalization=None, stream=None):
    """gp_pull_sweep_noalloc: one pull sweep into caller-owned `y` (float32[n])
    and `residual` (float64[1]), with no device allocation by the library."""
    _check(load().gp_pull_sweep_noalloc(int(n), int(m), _ptr(csc_off), _ptr(csc_idx), _ptr(csc_w), _ptr(inv_deg),
                                        _ptr(x), float(damping), _ptr(personalization), _ptr(y), _ptr(residual),
                                        _stream_ptr(stream)), "gp_pull_sweep_noalloc")


def profile_enable(on: bool = True):
    _check(load().gp_profile_enable(int(on)), "gp_profile_enable")


def selftest_narrow(values, stream=None):
    """gp_selftest_narrow on a CUDA float64 tensor: (library rounding, hardware rounding)."""
    torch = _torch()
    ours = torch.empty(values.shape[0], dtype=torch.float32, device=values.device)
    hw = torch.empty_like(ours)
    _check(load().gp_selftest_narrow(int(values.shape[0]), _ptr(values), _ptr(ours), _ptr(hw), _stream_ptr(stream)),
           "gp_selftest_narrow")
    return ours, hw


def profile_read(reset: bool = True) -> list:
    """[(kernel name, launches, total ms)] sorted by total time."""
    buf = (gp_kernel_time * 64)()
    cnt = ctypes.c_int(0)
    _check(load().gp_profile_read(buf, 64, ctypes.byref(cnt), int(reset)), "gp_profile_read")
    return [(buf[i].name.decode(), buf[i].launches, buf[i].total_ms) for i in range(cnt.value)]
