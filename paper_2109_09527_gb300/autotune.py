"""Autotuner for the layout and launch options of a graph.

The library's defaults (heavy-row threshold 256, 48K L1-cached hub ranks, occupancy-sized
grids) were measured on R-MAT and Erdos-Renyi graphs of 2^24 vertices.  A caller with
another graph can let `tune` time the synchronous update on that graph under each candidate
and keep the fastest:

  * the heavy in-degree threshold (rows at or above it are gathered in 2048-edge segments
    by whole warps) -- a layout choice, so each candidate builds the graph once;
  * the number of binned vertex ids whose ranks the gathers cache in L1 (the rest are read
    from L2 only);
  * blocks per SM of the persistent iteration kernels.

Every candidate is timed by the library itself (CUDA events around `iterations`
synchronous updates, `pr_info.ms_loop`), after one untimed warm-up run; the result is a
dict of the winning options and the measured times of every candidate.  `build_tuned`
builds a graph with a result, `apply` sets its launch options on a built graph.
`tune_batched` does the same for the batched solver's row binning (its k-tile is fixed at
32 columns, one 128-byte row per gathered edge).
"""
from __future__ import annotations

import numpy as np

from . import (DEFAULT_HEAVY_DEGREE, PR_OPT_CTAS_PER_SM, PR_OPT_HOT_VERTICES,
               PR_OPT_TMA_HOT_VERTICES, Graph, pr_iterate, set_heavy_degree)

HEAVY_CANDIDATES = (128, 256, 512, 1024, 2048, 4096)
HOT_CANDIDATES = (16384, 49152, 131072)
TMA_HOT_CANDIDATES = (4096, 16384, 32768)   # the pipelined row kernel's own hub count
DEFAULT_TMA_HOT = 16384
CTAS_CANDIDATES = (0, 2, 3)
POLICY_L1_HUBS = 4   # see PR_OPT_HOT_VERTICES: hubs through L1, the rest L2-only


def _time(g: Graph, x, out, iterations: int, damping: float) -> float:
    pr_iterate(g.handle, damping, None, x, iterations, out)          # warm-up
    info = pr_iterate(g.handle, damping, None, x, iterations, out)
    return info.ms_loop / iterations


def tune(rowptr, colidx, iterations: int = 6, damping: float = 0.85,
         heavy=HEAVY_CANDIDATES, hot=HOT_CANDIDATES, ctas=CTAS_CANDIDATES,
         tma_hot=TMA_HOT_CANDIDATES) -> dict:
    """Time candidate options on this graph (rowptr/colidx as for Graph: host arrays or CUDA
    tensors).  The search is coordinate-wise: the heavy threshold first (with default launch
    options), then the hub count, then the pipelined row kernel's own hub count, then blocks
    per SM, each with the best of the previous.  Returns {"heavy_degree", "hot_vertices",
    "tma_hot_vertices", "ctas_per_sm", "ms_per_iteration", "trials"}."""
    n = (rowptr.shape[0] if hasattr(rowptr, "shape") else len(rowptr)) - 1
    try:
        import torch
        on_device = hasattr(rowptr, "is_cuda") and rowptr.is_cuda
    except ImportError:  # pragma: no cover - torch is always present with the tests
        on_device = False
    if on_device:
        x = torch.full((n,), 1.0 / n, dtype=torch.float32, device=rowptr.device)
        out = torch.empty_like(x)
    else:
        x = np.full(n, 1.0 / n, dtype=np.float32)
        out = np.empty(n, dtype=np.float32)
    trials = []
    best = {"heavy_degree": DEFAULT_HEAVY_DEGREE, "hot_vertices": 49152, "tma_hot_vertices": DEFAULT_TMA_HOT,
            "ctas_per_sm": 0, "ms_per_iteration": float("inf")}
    graphs = {}
    try:
        for h in heavy:
            set_heavy_degree(h)
            try:
                graphs[h] = Graph(rowptr, colidx)
            finally:
                set_heavy_degree(DEFAULT_HEAVY_DEGREE)
            ms = _time(graphs[h], x, out, iterations, damping)
            trials.append({"heavy_degree": h, "hot_vertices": 49152, "ctas_per_sm": 0, "ms": ms})
            if ms < best["ms_per_iteration"]:
                best.update(heavy_degree=h, ms_per_iteration=ms)
        g = graphs[best["heavy_degree"]]
        for hv in hot:
            g.set_option(PR_OPT_HOT_VERTICES, (POLICY_L1_HUBS << 28) | min(hv, (1 << 28) - 1))
            ms = _time(g, x, out, iterations, damping)
            trials.append({"heavy_degree": best["heavy_degree"], "hot_vertices": hv, "ctas_per_sm": 0, "ms": ms})
            if ms < best["ms_per_iteration"]:
                best.update(hot_vertices=hv, ms_per_iteration=ms)
        g.set_option(PR_OPT_HOT_VERTICES, (POLICY_L1_HUBS << 28) | best["hot_vertices"])
        for th in tma_hot:
            g.set_option(PR_OPT_TMA_HOT_VERTICES, th)
            ms = _time(g, x, out, iterations, damping)
            trials.append({"heavy_degree": best["heavy_degree"], "hot_vertices": best["hot_vertices"],
                           "tma_hot_vertices": th, "ctas_per_sm": 0, "ms": ms})
            if ms < best["ms_per_iteration"]:
                best.update(tma_hot_vertices=th, ms_per_iteration=ms)
        g.set_option(PR_OPT_TMA_HOT_VERTICES, best["tma_hot_vertices"])
        for c in ctas:
            g.set_option(PR_OPT_CTAS_PER_SM, c)
            ms = _time(g, x, out, iterations, damping)
            trials.append({"heavy_degree": best["heavy_degree"], "hot_vertices": best["hot_vertices"],
                           "ctas_per_sm": c, "ms": ms})
            if ms < best["ms_per_iteration"]:
                best.update(ctas_per_sm=c, ms_per_iteration=ms)
    finally:
        for gg in graphs.values():
            gg.close()
    best["trials"] = trials
    return best


def tune_batched(rowptr, colidx, teleport, k: int, damping: float = 0.85, tol: float = 1e-6,
                 heavy=HEAVY_CANDIDATES) -> dict:
    """Time the batched solver (pr_solve_batched with these k teleport columns, n x k row-major,
    host or device) on this graph under each heavy threshold -- the row binning of its
    gathers: rows at or above it are walked in 2048-edge segments, the rest as light-row
    tasks -- one untimed warm-up solve each, and keep the fastest.  The k-tile is fixed: one
    gathered row of the batched matrices is always 32 columns (128 bytes), so fewer
    columns per solve would move the same bytes.  Returns {"heavy_degree",
    "ms_per_solve", "trials"}."""
    import numpy as np
    n = (rowptr.shape[0] if hasattr(rowptr, "shape") else len(rowptr)) - 1
    trials = []
    best = {"heavy_degree": DEFAULT_HEAVY_DEGREE, "ms_per_solve": float("inf")}
    out = np.empty((n, k), dtype=np.float32)
    for h in heavy:
        set_heavy_degree(h)
        try:
            g = Graph(rowptr, colidx)
        finally:
            set_heavy_degree(DEFAULT_HEAVY_DEGREE)
        with g:
            g.solve_batched(k, teleport, damping=damping, tol=tol, out=out)     # warm-up
            _, info, _, _ = g.solve_batched(k, teleport, damping=damping, tol=tol, out=out)
        trials.append({"heavy_degree": h, "ms": info.ms_device, "iterations": info.iterations})
        if info.ms_device < best["ms_per_solve"]:
            best.update(heavy_degree=h, ms_per_solve=info.ms_device)
    best["trials"] = trials
    return best


def apply(g: Graph, result: dict) -> Graph:
    """Set a tuning result's launch options on a graph built with its heavy threshold."""
    g.set_option(PR_OPT_HOT_VERTICES, (POLICY_L1_HUBS << 28) | int(result["hot_vertices"]))
    g.set_option(PR_OPT_TMA_HOT_VERTICES, int(result.get("tma_hot_vertices", DEFAULT_TMA_HOT)))
    g.set_option(PR_OPT_CTAS_PER_SM, int(result["ctas_per_sm"]))
    return g


def build_tuned(rowptr, colidx, result: dict) -> Graph:
    """A graph built and configured with a tuning result."""
    set_heavy_degree(int(result["heavy_degree"]))
    try:
        g = Graph(rowptr, colidx)
    finally:
        set_heavy_degree(DEFAULT_HEAVY_DEGREE)
    return apply(g, result)
