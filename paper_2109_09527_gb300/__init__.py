"""GB300 (sm_103a) PageRank: Python binding of the C ABI in ``include/pagerank.h``.

This module only marshals arguments: every step of the computation runs in the
CUDA library ``_build/libpagerank_gb300.so``.  The functions named ``pr_*``
mirror the C entry points one to one (a non-OK status raises
:class:`PageRankError`, except ``PR_NOT_CONVERGED`` which is returned); the
:class:`Graph` class wraps a ``pr_graph`` handle for convenience.

Array arguments may be numpy arrays (host memory), torch tensors (host or
CUDA), or raw integer addresses.  Device tensors are used in place; host
arrays are copied by the library.  ``stream=None`` means torch's current CUDA
stream when torch has initialised CUDA, else the legacy default stream.

If the library is missing or stale it is built with nvcc on first use; if
that fails, import-time use raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

PR_OK = 0
PR_ERR_INVALID_ARG = 1
PR_ERR_CUDA = 2
PR_ERR_OOM = 3
PR_NOT_CONVERGED = 4
PR_ERR_UNSUPPORTED = 5
PR_ERR_INVALID_GRAPH = 6
PR_ERR_DEVICE_TIMEOUT = 7

PR_IN_CSR = 0
PR_OUT_CSR = 1
PR_JACOBI = 0
PR_NONBLOCKING = 1
PR_EDGE = 2

PR_OPT_HEAVY_DEGREE = 1
PR_OPT_USE_GRAPH = 2
PR_OPT_CTAS_PER_SM = 3
PR_OPT_INDEX64 = 4
PR_OPT_HOT_VERTICES = 5
PR_OPT_HOT_CACHE = 6
PR_OPT_STAGED_TILES = 7
PR_OPT_NB_HUBS = 8
PR_OPT_NB_L1_HUBS = 9
PR_OPT_BATCH_BF16 = 10
PR_OPT_PERFORATION = 11
PR_OPT_DYNAMIC_TILES = 12
PR_OPT_DELAY_NS = 13
PR_OPT_TMA_TILES = 14
PR_OPT_TEST_WITHHOLD_COPY = 15
PR_OPT_NB_FAIL_AFTER = 16
PR_OPT_LIGHT_LANES = 17
PR_OPT_BATCH_DC = 18
PR_OPT_FUSED_SEGMENTS = 19
PR_OPT_BATCH_ASYNC = 20
PR_OPT_IMPLICIT_ZERO_ROWS = 21
PR_OPT_SYNC_DC = 22
PR_OPT_TMA_HOT_VERTICES = 23
PR_OPT_NB_PIPELINE = 24

LIB_PATH = _build.LIB_PATH


class PageRankError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_status_name(status)}: {message}")
        self.status = status


class pr_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("residual_l1", ctypes.c_double), ("sum_x", ctypes.c_double),
                ("dangling_mass", ctypes.c_double), ("edge_visits", ctypes.c_double),
                ("ms_device", ctypes.c_float), ("launches", ctypes.c_int32),
                ("loop_edge_visits", ctypes.c_double), ("ms_loop", ctypes.c_float),
                ("frozen_rows", ctypes.c_int32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class pr_graph_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("n_dangling", ctypes.c_int64),
                ("n_zero_indeg", ctypes.c_int64), ("n_heavy", ctypes.c_int64),
                ("n_segments", ctypes.c_int64), ("n_tiles", ctypes.c_int64),
                ("max_indeg", ctypes.c_int64), ("rowptr_bytes", ctypes.c_int32),
                ("sm_count", ctypes.c_int32), ("device_bytes", ctypes.c_int64),
                ("setup_ms", ctypes.c_float), ("n_tma_tiles", ctypes.c_int64),
                ("hub_prefix_edges", ctypes.c_int64), ("n_isolated", ctypes.c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes) of every entry point declared in include/pagerank.h
_VP, _I64, _I32, _D, _F = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_float
SIGNATURES = {
    "pr_create_graph": (ctypes.c_int, [_I64, _I64, _VP, ctypes.c_int, _VP, _VP, ctypes.c_int, _VP,
                                       ctypes.POINTER(_VP)]),
    "pr_destroy_graph": (ctypes.c_int, [_VP]),
    "pr_trim_memory": (ctypes.c_int, []),
    "pr_solve": (ctypes.c_int, [_VP, _F, _D, _I32, ctypes.c_int, _VP, _VP, _VP,
                                ctypes.POINTER(pr_info), _VP]),
    "pr_iterate": (ctypes.c_int, [_VP, _F, _VP, _VP, _I32, _VP, ctypes.POINTER(pr_info), _VP]),
    "pr_graph_get_stats": (ctypes.c_int, [_VP, ctypes.POINTER(pr_graph_stats)]),
    "pr_set_option": (ctypes.c_int, [_VP, ctypes.c_int, _I64]),
    "pr_step_noalloc": (ctypes.c_int, [_I64, _VP, _VP, _VP, _F, _VP, _VP, _VP, _VP]),
    "pr_solve_batched": (ctypes.c_int, [_VP, _F, _D, _I32, _I32, _VP, _VP, ctypes.POINTER(_D),
                                        ctypes.POINTER(_I32), ctypes.POINTER(pr_info), _VP]),
    "pr_graph_set_partition": (ctypes.c_int, [_VP, _I32, _VP, _VP]),
    "pr_create_wgraph": (ctypes.c_int, [_I64, _I64, _VP, _VP, _VP, _VP, ctypes.POINTER(_VP)]),
    "pr_destroy_wgraph": (ctypes.c_int, [_VP]),
    "pr_wgraph_set_weights": (ctypes.c_int, [_VP, _VP, _VP]),
    "pr_solve_weighted": (ctypes.c_int, [_VP, _F, _D, _I32, _VP, _VP, ctypes.POINTER(pr_info), _VP]),
    "pr_adjoint": (ctypes.c_int, [_VP, _F, _D, _I32, _VP, _VP, _VP, _VP, ctypes.POINTER(pr_info), _VP]),
    "pr_solve_set": (ctypes.c_int, [_VP, _F, _D, _I32, _VP, ctypes.POINTER(_D), ctypes.POINTER(_I32),
                                    ctypes.POINTER(pr_info), _VP]),
    "pr_measure_gather_rate": (ctypes.c_int, [_I64, _I64, ctypes.c_int, ctypes.c_int, _I32,
                                              ctypes.c_uint64, ctypes.POINTER(_D), _VP]),
    "pr_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "pr_last_error": (ctypes.c_char_p, []),
}


def load(path: str | None = None):
    """The ctypes handle of the CUDA library (built on first use if missing or stale)."""
    global _lib
    with _lock:
        if _lib is None or path is not None:
            if path is None:
                path = _build.build()
            if not os.path.exists(path):
                raise ImportError(f"CUDA library not found at {path}")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            if path == LIB_PATH:
                _lib = lib
            else:
                return lib
    return _lib


def _status_name(s: int) -> str:
    try:
        return load().pr_status_string(s).decode()
    except Exception:  # noqa: BLE001 - naming only
        return f"status {s}"


def _check(status: int, allow_not_converged: bool = False) -> int:
    if status == PR_OK or (allow_not_converged and status == PR_NOT_CONVERGED):
        return status
    raise PageRankError(status, load().pr_last_error().decode())


def _addr(obj, dtype=None):
    """Address of an array argument: None, int, numpy array or torch tensor."""
    if obj is None:
        return None
    if isinstance(obj, int):
        return obj
    if isinstance(obj, np.ndarray):
        if dtype is not None and obj.dtype != dtype:
            raise TypeError(f"expected dtype {np.dtype(dtype)}, got {obj.dtype}")
        if not obj.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return obj.ctypes.data
    if hasattr(obj, "data_ptr"):  # torch.Tensor
        if not obj.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if dtype is not None:
            want = {np.float32: "torch.float32", np.int32: "torch.int32",
                    np.int64: "torch.int64"}[np.dtype(dtype).type]
            if str(obj.dtype) != want:
                raise TypeError(f"expected {want}, got {obj.dtype}")
        return obj.data_ptr()
    raise TypeError(f"unsupported array argument {type(obj)}")


def _stream(stream):
    if stream is not None:
        return int(stream) if not hasattr(stream, "cuda_stream") else stream.cuda_stream
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


# ---------------------------------------------------------------- C entry points --

def pr_create_graph(n, nnz, rowptr, rowptr_is_64, colidx, weights=None, layout=PR_IN_CSR,
                    stream=None):
    out = _VP()
    _check(load().pr_create_graph(int(n), int(nnz), _addr(rowptr), int(bool(rowptr_is_64)),
                                  _addr(colidx, np.int32), _addr(weights), int(layout),
                                  _stream(stream), ctypes.byref(out)))
    return out.value


def pr_destroy_graph(g):
    return _check(load().pr_destroy_graph(g))


def pr_trim_memory():
    """Return the device memory the library's pool keeps for reuse to the system."""
    return _check(load().pr_trim_memory())


def pr_solve(g, damping, tol, max_iter, variant, teleport, x0, x_out, stream=None):
    """Returns (status, pr_info); status is PR_OK or PR_NOT_CONVERGED."""
    info = pr_info()
    st = _check(load().pr_solve(g, float(damping), float(tol), int(max_iter), int(variant),
                                _addr(teleport, np.float32), _addr(x0, np.float32),
                                _addr(x_out, np.float32), ctypes.byref(info), _stream(stream)),
                allow_not_converged=True)
    return st, info


def pr_iterate(g, damping, teleport, x_in, n_iter, x_out, stream=None):
    info = pr_info()
    _check(load().pr_iterate(g, float(damping), _addr(teleport, np.float32),
                             _addr(x_in, np.float32), int(n_iter), _addr(x_out, np.float32),
                             ctypes.byref(info), _stream(stream)))
    return info


def pr_solve_batched(g, damping, tol, max_iter, k, teleport, x_out, stream=None):
    """Returns (status, pr_info, col_residual[k], col_iterations[k]); status is PR_OK or
    PR_NOT_CONVERGED.  teleport: n x k row-major float32 (host or device) or None."""
    info = pr_info()
    res = (ctypes.c_double * int(k))()
    its = (ctypes.c_int32 * int(k))()
    st = _check(load().pr_solve_batched(g, float(damping), float(tol), int(max_iter), int(k),
                                        _addr(teleport, np.float32), _addr(x_out, np.float32),
                                        res, its, ctypes.byref(info), _stream(stream)),
                allow_not_converged=True)
    return st, info, np.array(res[:], dtype=np.float64), np.array(its[:], dtype=np.int32)


def pr_graph_set_partition(g, offsets, stream=None):
    """Declare g as the disjoint union of graphs on caller-id ranges offsets[i]..offsets[i+1]."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    return _check(load().pr_graph_set_partition(g, int(off.size - 1), off.ctypes.data, _stream(stream)))


def pr_solve_set(g, count, damping, tol, max_iter, x_out, stream=None):
    """Returns (status, pr_info, graph_residual[count], graph_iterations[count])."""
    info = pr_info()
    res = (ctypes.c_double * int(count))()
    its = (ctypes.c_int32 * int(count))()
    st = _check(load().pr_solve_set(g, float(damping), float(tol), int(max_iter),
                                    _addr(x_out, np.float32), res, its, ctypes.byref(info),
                                    _stream(stream)),
                allow_not_converged=True)
    return st, info, np.array(res[:], dtype=np.float64), np.array(its[:], dtype=np.int32)


def pr_graph_get_stats(g):
    s = pr_graph_stats()
    _check(load().pr_graph_get_stats(g, ctypes.byref(s)))
    return s.as_dict()


def pr_set_option(g, key, value):
    return _check(load().pr_set_option(g, int(key), int(value)))


def pr_step_noalloc(n, rowptr, colidx, inv_outdeg, damping, x_in, x_out, sums_out, stream=None):
    """One synchronous update on a caller-owned plain CSR without any allocation (all
    arrays device memory; sums_out holds 3 doubles).  Asynchronous on the stream."""
    return _check(load().pr_step_noalloc(int(n), _addr(rowptr, np.int32), _addr(colidx, np.int32),
                                         _addr(inv_outdeg, np.float32), float(damping),
                                         _addr(x_in, np.float32), _addr(x_out, np.float32),
                                         _addr(sums_out), _stream(stream)))


def pr_measure_gather_rate(n_values, n_indices, cached, blocks_per_sm, chunks, seed=1, stream=None):
    """Random 4-byte loads per second from an n_values-float vector (see the header):
    returns {"gathers_per_s", "ms", "gathers"} of one timed launch."""
    out = (_D * 3)()
    _check(load().pr_measure_gather_rate(int(n_values), int(n_indices), int(cached), int(blocks_per_sm),
                                         int(chunks), int(seed), out, _stream(stream)))
    return {"gathers_per_s": out[0], "ms": out[1], "gathers": out[2]}


def pr_status_string(status):
    return load().pr_status_string(int(status)).decode()


def pr_last_error():
    return load().pr_last_error().decode()


# ------------------------------------------------------------------- convenience --

class Graph:
    """Owns a pr_graph built from an in-edge CSR (row v lists the sources of v's in-edges)."""

    def __init__(self, rowptr, colidx, stream=None, layout=PR_IN_CSR):
        """layout PR_IN_CSR: row v lists the sources of v's in-edges; PR_OUT_CSR: row u
        lists the targets of u's out-edges (transposed on the device at creation)."""
        n = (rowptr.shape[0] if hasattr(rowptr, "shape") else len(rowptr)) - 1
        nnz = colidx.shape[0] if hasattr(colidx, "shape") else len(colidx)
        is64 = str(getattr(rowptr, "dtype", "")) in ("int64", "torch.int64")
        if not is64 and str(getattr(rowptr, "dtype", "")) not in ("int32", "torch.int32"):
            raise TypeError("rowptr must be int32 or int64")
        self.n, self.nnz = int(n), int(nnz)
        self.handle = pr_create_graph(n, nnz, rowptr, is64, colidx, layout=layout, stream=stream)

    def close(self):
        if getattr(self, "handle", None):
            pr_destroy_graph(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def stats(self):
        return pr_graph_get_stats(self.handle)

    def solve(self, damping=0.85, tol=1e-6, max_iter=200, variant=PR_JACOBI, teleport=None,
              x0=None, out=None, stream=None):
        """PageRank vector; `out` defaults to a host float32 numpy array.  Returns (out, info)."""
        if out is None:
            out = np.empty(self.n, dtype=np.float32)
        if isinstance(variant, str):
            variant = {"jacobi": PR_JACOBI, "nonblocking": PR_NONBLOCKING, "edge": PR_EDGE}[variant]
        status, info = pr_solve(self.handle, damping, tol, max_iter, variant, teleport, x0, out,
                                stream=stream)
        return out, info

    def solve_batched(self, k, teleport=None, damping=0.85, tol=1e-6, max_iter=200, out=None,
                      stream=None):
        """k personalised PageRank vectors at once (teleport: n x k row-major, or None for
        uniform).  `out` defaults to a host float32 numpy array of shape (n, k).
        Returns (out, info, col_residual, col_iterations)."""
        if out is None:
            out = np.empty((self.n, k), dtype=np.float32)
        status, info, res, its = pr_solve_batched(self.handle, damping, tol, max_iter, k, teleport,
                                                  out, stream=stream)
        return out, info, res, its

    def set_partition(self, offsets, stream=None):
        """Treat the graph as independent graphs on caller-id ranges [offsets[i], offsets[i+1])."""
        pr_graph_set_partition(self.handle, offsets, stream=stream)
        self.set_count = len(offsets) - 1

    def solve_set(self, damping=0.85, tol=1e-6, max_iter=200, out=None, stream=None):
        """PageRank of every graph of the partition.  Returns (out, info, residuals, iterations)."""
        if out is None:
            out = np.empty(self.n, dtype=np.float32)
        status, info, res, its = pr_solve_set(self.handle, self.set_count, damping, tol, max_iter,
                                              out, stream=stream)
        return out, info, res, its

    def iterate(self, x_in, n_iter=1, damping=0.85, teleport=None, out=None, stream=None):
        """Exactly n_iter synchronous updates from x_in (no stopping test, no rescaling)."""
        if out is None:
            out = np.empty(self.n, dtype=np.float32)
        info = pr_iterate(self.handle, damping, teleport, x_in, n_iter, out, stream=stream)
        return out, info

    def set_option(self, key, value):
        pr_set_option(self.handle, key, value)


DEFAULT_HEAVY_DEGREE = 256   # the library's default heavy in-degree threshold


def set_heavy_degree(value: int):
    """Heavy in-degree threshold for graphs created next on this thread (power of two;
    DEFAULT_HEAVY_DEGREE restores the default)."""
    pr_set_option(None, PR_OPT_HEAVY_DEGREE, value)


# ------------------------------------------------------ weighted graphs, adjoint --

def pr_create_wgraph(n, nnz, rowptr, colidx, weights, stream=None):
    out = _VP()
    _check(load().pr_create_wgraph(int(n), int(nnz), _addr(rowptr, np.int64), _addr(colidx, np.int32),
                                   _addr(weights, np.float32), _stream(stream), ctypes.byref(out)))
    return out.value


def pr_destroy_wgraph(g):
    return _check(load().pr_destroy_wgraph(g))


def pr_wgraph_set_weights(g, weights, stream=None):
    return _check(load().pr_wgraph_set_weights(g, _addr(weights, np.float32), _stream(stream)))


def pr_solve_weighted(g, damping, tol, max_iter, teleport, x_out, stream=None):
    info = pr_info()
    st = _check(load().pr_solve_weighted(g, float(damping), float(tol), int(max_iter),
                                         _addr(teleport, np.float32), _addr(x_out, np.float32),
                                         ctypes.byref(info), _stream(stream)),
                allow_not_converged=True)
    return st, info


def pr_adjoint(g, damping, tol, max_iter, x, dL_dx, dL_dteleport, dL_dweights, stream=None):
    info = pr_info()
    st = _check(load().pr_adjoint(g, float(damping), float(tol), int(max_iter), _addr(x, np.float32),
                                  _addr(dL_dx, np.float32), _addr(dL_dteleport, np.float32),
                                  _addr(dL_dweights, np.float32), ctypes.byref(info), _stream(stream)),
                allow_not_converged=True)
    return st, info


class WeightedGraph:
    """Owns a pr_wgraph: an in-edge CSR with positive edge weights (row-normalised by
    source into transition probabilities), for the weighted solve and its adjoint."""

    def __init__(self, rowptr, colidx, weights, stream=None):
        self.n = (rowptr.shape[0] if hasattr(rowptr, "shape") else len(rowptr)) - 1
        self.nnz = colidx.shape[0] if hasattr(colidx, "shape") else len(colidx)
        self.handle = pr_create_wgraph(self.n, self.nnz, rowptr, colidx, weights, stream=stream)

    def close(self):
        if getattr(self, "handle", None):
            pr_destroy_wgraph(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    def set_weights(self, weights, stream=None):
        pr_wgraph_set_weights(self.handle, weights, stream=stream)

    def solve(self, damping=0.85, tol=1e-6, max_iter=200, teleport=None, out=None, stream=None):
        if out is None:
            out = np.empty(self.n, dtype=np.float32)
        _, info = pr_solve_weighted(self.handle, damping, tol, max_iter, teleport, out, stream=stream)
        return out, info

    def adjoint(self, x, dL_dx, damping=0.85, tol=1e-6, max_iter=500, grad_teleport=None,
                grad_weights=None, stream=None):
        """dL/dteleport and dL/dweights (numpy arrays unless buffers are given)."""
        if grad_teleport is None:
            grad_teleport = np.empty(self.n, dtype=np.float32)
        if grad_weights is None:
            grad_weights = np.empty(self.nnz, dtype=np.float32)
        _, info = pr_adjoint(self.handle, damping, tol, max_iter, x, dL_dx, grad_teleport,
                             grad_weights, stream=stream)
        return grad_teleport, grad_weights, info


def weighted_pagerank(graph, teleport, weights, damping=0.85, tol=1e-6, max_iter=200,
                      adjoint_tol=1e-6, adjoint_max_iter=500):
    """Differentiable weighted PageRank: x = PageRank(graph with edge weights, teleport), as
    a torch.autograd.Function whose backward runs the library's adjoint solve (implicit
    differentiation of the fixed point).  teleport (n) and weights (nnz) are CUDA float32
    tensors; returns x (n).  The graph's weights are set from `weights` on every call."""
    import torch

    class _WeightedPageRank(torch.autograd.Function):
        @staticmethod
        def forward(ctx, t, w):
            t = t.detach().contiguous()
            w = w.detach().contiguous()
            graph.set_weights(w)
            x = torch.empty_like(t)
            graph.solve(damping, tol, max_iter, teleport=t, out=x)
            ctx.save_for_backward(x, w)
            return x

        @staticmethod
        def backward(ctx, grad_x):
            x, w = ctx.saved_tensors
            graph.set_weights(w)
            gt = torch.empty_like(x)
            gw = torch.empty_like(w)
            graph.adjoint(x, grad_x.contiguous(), damping, adjoint_tol, adjoint_max_iter,
                          grad_teleport=gt, grad_weights=gw)
            return gt, gw

    return _WeightedPageRank.apply(teleport, weights)
