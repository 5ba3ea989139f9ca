"""Seeded synthetic directed graphs as in-edge CSR (row v lists the sources u of u -> v).

This module builds inputs only; it holds none of the PageRank arithmetic.  The
CUDA library (through its C ABI) and the CPU oracle are both fed from it.

Large generators (R-MAT, ER with dangling vertices) run in C (``graphgen.c``),
compiled on first use with gcc into ``graphgen/_build``.  The small fixture
graphs used for closed-form checks are written out here in numpy.

All outputs are ``(rowptr: int64[n+1], colidx: int32[nnz])`` with every row's
sources sorted ascending, self-loops and duplicate edges removed (unless a
fixture asks otherwise).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_OUT = os.path.join(_HERE, "_build", "libgraphgen.so")
_lock = threading.Lock()
_lib = None

# Graph500 quadrant probabilities (a, b, c); d = 1 - a - b - c = 0.05.
GRAPH500_ABC = (0.57, 0.19, 0.19)


def build(force: bool = False) -> str:
    """Compile graphgen.c into a shared library (gcc, -O2, no FMA contraction)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    tmp = _OUT + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-pthread",
           "-ffp-contract=off", "-fvisibility=hidden", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, u64, dbl, vp = (ctypes.c_int64, ctypes.c_int, ctypes.c_uint64,
                                      ctypes.c_double, ctypes.c_void_p)
            lib.gg_rmat.restype = i64
            lib.gg_rmat.argtypes = [i32, i32, dbl, dbl, dbl, u64, i32, i32, vp, vp, i64]
            lib.gg_rmat_n.restype = i64
            lib.gg_rmat_n.argtypes = [i64, i32, dbl, dbl, dbl, u64, i32, i32, vp, vp, i64]
            lib.gg_er_dangling.restype = i64
            lib.gg_er_dangling.argtypes = [i64, dbl, dbl, u64, i32, vp, vp, i64]
            lib.gg_uniform.restype = None
            lib.gg_uniform.argtypes = [u64, u64, i64, vp]
            lib.gg_permutation.restype = None
            lib.gg_permutation.argtypes = [u64, u64, i64, vp]
            lib.gg_random_u64.restype = u64
            lib.gg_random_u64.argtypes = [u64, u64, u64]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def rmat(scale: int, edge_factor: int = 16, a: float = GRAPH500_ABC[0], b: float = GRAPH500_ABC[1],
         c: float = GRAPH500_ABC[2], seed: int = 1, permute: bool = True, nthreads: int = 0):
    """R-MAT digraph, 2^scale vertices, edge_factor * 2^scale drawn edges, Graph500
    quadrant probabilities by default, seeded relabelling, no self-loops or duplicates."""
    lib = _load()
    n = 1 << scale
    cap = lib.gg_rmat(scale, edge_factor, a, b, c, seed, int(permute), nthreads, None, None, 0)
    if cap < 0:
        raise ValueError(f"gg_rmat: bad arguments (code {cap})")
    rowptr = np.empty(n + 1, dtype=np.int64)
    colidx = np.empty(max(cap, 1), dtype=np.int32)
    nnz = lib.gg_rmat(scale, edge_factor, a, b, c, seed, int(permute), nthreads,
                      _ptr(rowptr), _ptr(colidx), cap)
    if nnz < 0:
        raise MemoryError(f"gg_rmat failed (code {nnz})")
    return rowptr, colidx[:nnz]


def rmat_n(n: int, edge_factor: int = 8, a: float = GRAPH500_ABC[0], b: float = GRAPH500_ABC[1],
           c: float = GRAPH500_ABC[2], seed: int = 1, permute: bool = True, nthreads: int = 0):
    """R-MAT digraph on any n >= 2 vertices: edge_factor * n draws of the R-MAT recursion at
    scale ceil(log2 n), a draw with an endpoint >= n redrawn from a retry stream, seeded
    relabelling of range(n), no self-loops or duplicates."""
    lib = _load()
    cap = lib.gg_rmat_n(n, edge_factor, a, b, c, seed, int(permute), nthreads, None, None, 0)
    if cap < 0:
        raise ValueError(f"gg_rmat_n: bad arguments (code {cap})")
    rowptr = np.empty(n + 1, dtype=np.int64)
    colidx = np.empty(max(cap, 1), dtype=np.int32)
    nnz = lib.gg_rmat_n(n, edge_factor, a, b, c, seed, int(permute), nthreads,
                        _ptr(rowptr), _ptr(colidx), cap)
    if nnz < 0:
        raise MemoryError(f"gg_rmat_n failed (code {nnz})")
    return rowptr, colidx[:nnz]


def multi_rmat(count: int = 64, n_lo: float = 1e3, n_hi: float = 1e6, edge_factor: int = 8,
               seed: int = 1):
    """`count` independent R-MAT digraphs whose vertex counts are log-uniform in
    [n_lo, n_hi] (rounded to integers), graph g drawn with seed (seed << 8) + g."""
    u = uniform(seed, 1, count)
    sizes = np.rint(n_lo * (n_hi / n_lo) ** u).astype(np.int64)
    return [rmat_n(int(sizes[g]), edge_factor, seed=(seed << 8) + g) for g in range(count)]


def block_diagonal(graphs):
    """One in-edge CSR holding the graphs side by side (graph g's vertex v becomes
    offsets[g] + v).  Returns (rowptr int64, colidx int32, offsets int64[count + 1])."""
    offsets = np.zeros(len(graphs) + 1, dtype=np.int64)
    for g, (rp, ci) in enumerate(graphs):
        offsets[g + 1] = offsets[g] + (rp.size - 1)
    nnz = sum(ci.size for _, ci in graphs)
    rowptr = np.zeros(offsets[-1] + 1, dtype=np.int64)
    colidx = np.empty(nnz, dtype=np.int32)
    e = 0
    for g, (rp, ci) in enumerate(graphs):
        o = offsets[g]
        rowptr[o + 1: offsets[g + 1] + 1] = e + rp[1:]
        colidx[e: e + ci.size] = ci + o
        e += ci.size
    return rowptr, colidx, offsets


def seed_teleports(n: int, k: int, per_column: int = 8, seed: int = 1):
    """k personalisation vectors as an n x k row-major float32 matrix: column j is uniform
    (1/per_column) over per_column distinct seeded random vertices."""
    if per_column > n:
        raise ValueError("more seed vertices than vertices")
    t = np.zeros((n, k), dtype=np.float32)
    for j in range(k):
        picked = []
        draw = 0
        while len(picked) < per_column:
            u = uniform(seed, 2 + j, per_column + draw)[draw:]
            for v in np.minimum((u * n).astype(np.int64), n - 1):
                if v not in picked and len(picked) < per_column:
                    picked.append(int(v))
            draw += per_column
        t[picked, j] = 1.0 / per_column
    return t


def er_dangling(n: int, mean_deg: float = 16.0, frac_dangling: float = 0.2, seed: int = 1,
                nthreads: int = 0):
    """Digraph with round(frac_dangling*n) vertices forced dangling and Poisson out-degrees
    (mean mean_deg over all n) with uniform destinations for the rest."""
    lib = _load()
    cap = lib.gg_er_dangling(n, mean_deg, frac_dangling, seed, nthreads, None, None, 0)
    if cap < 0:
        raise ValueError(f"gg_er_dangling: bad arguments (code {cap})")
    rowptr = np.empty(n + 1, dtype=np.int64)
    colidx = np.empty(max(cap, 1), dtype=np.int32)
    nnz = lib.gg_er_dangling(n, mean_deg, frac_dangling, seed, nthreads,
                             _ptr(rowptr), _ptr(colidx), cap)
    if nnz < 0:
        raise MemoryError(f"gg_er_dangling failed (code {nnz})")
    return rowptr, colidx[:nnz]


def uniform(seed: int, stream: int, count: int) -> np.ndarray:
    """`count` seeded uniform doubles in (0, 1) (counter-based; stream selects the sequence)."""
    out = np.empty(count, dtype=np.float64)
    _load().gg_uniform(seed, stream, count, _ptr(out))
    return out


def permutation(seed: int, stream: int, n: int) -> np.ndarray:
    """Seeded random permutation of range(n) (Fisher-Yates on the counter-based generator)."""
    out = np.empty(n, dtype=np.int32)
    _load().gg_permutation(seed, stream, n, _ptr(out))
    return out


def edges_to_in_csr(n: int, src, dst, dedup: bool = True, drop_self_loops: bool = True):
    """In-edge CSR of the edge list (src[i] -> dst[i]): rows are destinations, each row's
    sources sorted ascending.  With dedup=False repeated edges are kept (multi-edges)."""
    src = np.asarray(src, dtype=np.int64).ravel()
    dst = np.asarray(dst, dtype=np.int64).ravel()
    if src.shape != dst.shape:
        raise ValueError("src and dst differ in length")
    if src.size and (src.min() < 0 or dst.min() < 0 or src.max() >= n or dst.max() >= n):
        raise ValueError("vertex id out of range")
    if drop_self_loops:
        keep = src != dst
        src, dst = src[keep], dst[keep]
    key = dst * n + src
    key = np.unique(key) if dedup else np.sort(key)
    d = key // n
    s = key % n
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, d + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr.astype(np.int64), s.astype(np.int32)


def in_csr_edges(rowptr, colidx):
    """(src, dst) arrays of the edges held in an in-edge CSR."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    n = rowptr.size - 1
    dst = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    return np.asarray(colidx, dtype=np.int64), dst


def permute_in_csr(rowptr, colidx, perm):
    """The same graph with vertex v renamed perm[v]."""
    src, dst = in_csr_edges(rowptr, colidx)
    perm = np.asarray(perm, dtype=np.int64)
    return edges_to_in_csr(rowptr.size - 1, perm[src], perm[dst], dedup=False, drop_self_loops=False)


# ---------------------------------------------------------------- fixtures --

def cycle(n: int):
    """Directed n-cycle 0 -> 1 -> ... -> n-1 -> 0."""
    u = np.arange(n)
    return edges_to_in_csr(n, u, (u + 1) % n)


def complete(n: int):
    """Complete digraph without self-loops."""
    s, d = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return edges_to_in_csr(n, s.ravel(), d.ravel())


def empty(n: int):
    """n isolated vertices (all dangling)."""
    return np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32)


def in_star(n: int):
    """Leaves 1..n-1 each link to hub 0; the hub has no out-edges."""
    leaves = np.arange(1, n)
    return edges_to_in_csr(n, leaves, np.zeros_like(leaves))


def out_star(n: int):
    """Hub 0 links to each leaf 1..n-1; leaves have no out-edges."""
    leaves = np.arange(1, n)
    return edges_to_in_csr(n, np.zeros_like(leaves), leaves)


def bi_star(n: int):
    """Hub 0 and every leaf 1..n-1 link to each other."""
    leaves = np.arange(1, n)
    hub = np.zeros_like(leaves)
    return edges_to_in_csr(n, np.concatenate([hub, leaves]), np.concatenate([leaves, hub]))


def random_digraph(n: int, m: int, seed: int, allow_multi: bool = False, self_loops: bool = False):
    """m seeded uniform edges on n vertices (duplicates kept only with allow_multi)."""
    r = uniform(seed, 7, 2 * m)
    src = np.minimum((r[:m] * n).astype(np.int64), n - 1)
    dst = np.minimum((r[m:] * n).astype(np.int64), n - 1)
    return edges_to_in_csr(n, src, dst, dedup=not allow_multi, drop_self_loops=not self_loops)
