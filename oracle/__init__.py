"""FP64 CPU oracle for PageRank -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``pagerank_oracle.c`` (plain,
single-threaded C in double precision, compiled with gcc into
``oracle/_build``) with numpy-facing functions.  Nothing here imports, links or
shares code with the CUDA library under test.

Every function takes the graph as in-edge CSR: ``rowptr`` int64[n+1] and
``colidx`` int32[nnz], row v holding the sources u of the edges u -> v.
The functions and the paper passages they follow are listed in the C file's
header; in short:

* :func:`outdeg`            -- out-degrees counted from colidx.
* :func:`jacobi_step`       -- one synchronous update (Eq. 1 with the uniform
                               dangling share; inner loops of Alg. 1).
* :func:`pagerank_jacobi`   -- Alg. 1 (Barrier baseline) to a tolerance.
* :func:`vertex_update`     -- one vertex's update from a given vector.
* :func:`dense_solve`       -- the fixed point by Gaussian elimination.
* :func:`nosync`            -- Alg. 3 (No-Sync) with simulated threads.
* :func:`nosync_perforated` -- the same with the loop perforation of Alg. 5.
* :func:`fixed_point`       -- Alg. 1 run until the change stops shrinking.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pagerank_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libpagerank_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False, src: str = _SRC, out: str = _OUT) -> str:
    """Compile the oracle with gcc (-O2, IEEE double, no FMA contraction, no fast-math)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-fvisibility=hidden", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _declare(lib):
    i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
    lib.or_outdeg.restype = ctypes.c_int
    lib.or_outdeg.argtypes = [i64, vp, vp, vp]
    lib.or_vertex_update.restype = dbl
    lib.or_vertex_update.argtypes = [i64, i64, vp, vp, vp, dbl, vp, dbl, vp]
    lib.or_jacobi_step.restype = ctypes.c_int
    lib.or_jacobi_step.argtypes = [i64, vp, vp, vp, dbl, vp, ctypes.c_int, vp, vp, vp, vp, vp]
    lib.or_pagerank_jacobi.restype = ctypes.c_int
    lib.or_pagerank_jacobi.argtypes = [i64, vp, vp, dbl, vp, ctypes.c_int, dbl, i32, vp, vp,
                                       vp, vp, vp]
    lib.or_dense_solve.restype = ctypes.c_int
    lib.or_dense_solve.argtypes = [i64, vp, vp, dbl, vp, ctypes.c_int, vp]
    lib.or_pagerank_perforated.restype = ctypes.c_int
    lib.or_pagerank_perforated.argtypes = [i64, vp, vp, dbl, vp, dbl, i32, dbl, vp, vp, vp, vp]
    lib.or_w_outweight.restype = ctypes.c_int
    lib.or_w_outweight.argtypes = [i64, vp, vp, vp, vp]
    lib.or_w_jacobi.restype = ctypes.c_int
    lib.or_w_jacobi.argtypes = [i64, vp, vp, vp, dbl, vp, dbl, i32, vp, vp, vp, vp]
    lib.or_w_adjoint.restype = ctypes.c_int
    lib.or_w_adjoint.argtypes = [i64, vp, vp, vp, dbl, vp, vp, dbl, i32, vp, vp, vp, vp, vp, vp]
    lib.or_w_adjoint_step.restype = ctypes.c_int
    lib.or_w_adjoint_step.argtypes = [i64, vp, vp, vp, dbl, vp, vp, vp, vp]
    lib.or_nosync.restype = ctypes.c_int
    lib.or_nosync.argtypes = [i64, vp, vp, dbl, vp, ctypes.c_int, ctypes.c_int, i32, vp,
                              ctypes.c_int, dbl, i32, vp, vp, vp, vp, vp, dbl, vp]
    return lib


def load(path: str | None = None):
    """The oracle's ctypes handle (compiles on first use).  `path` loads another build of
    the same source, e.g. a deliberately broken copy used to show that the pins bite."""
    global _lib
    if path is not None:
        return _declare(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
    return _lib


class OracleError(RuntimeError):
    pass


def _csr(rowptr, colidx):
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colidx = np.ascontiguousarray(colidx, dtype=np.int32)
    if colidx.size == 0:
        colidx = np.zeros(1, dtype=np.int32)  # a valid pointer; never read
    return rowptr, colidx


def _vec(a, n):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != (n,):
        raise ValueError(f"expected a vector of length {n}")
    return a


def _p(a):
    return None if a is None else a.ctypes.data


def _check(rc, what):
    if rc != 0:
        raise OracleError(f"{what} failed with code {rc}")


def outdeg(rowptr, colidx, lib=None):
    lib = lib or load()
    rowptr, colidx = _csr(rowptr, colidx)
    n = rowptr.size - 1
    out = np.empty(n, dtype=np.int64)
    _check(lib.or_outdeg(n, _p(rowptr), _p(colidx), _p(out)), "or_outdeg")
    return out


def jacobi_step(rowptr, colidx, x, d=0.85, t=None, redistribute=True, lib=None):
    """One synchronous update.  Returns (x_new, dangling_mass_of_x, l1_change, max_change)."""
    lib = lib or load()
    rowptr, colidx = _csr(rowptr, colidx)
    n = rowptr.size - 1
    x = _vec(x, n)
    t = _vec(t, n)
    deg = outdeg(rowptr, colidx, lib)
    xn = np.empty(n, dtype=np.float64)
    D, l1, linf = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib.or_jacobi_step(n, _p(rowptr), _p(colidx), _p(deg), d, _p(t), int(redistribute),
                              _p(x), _p(xn), ctypes.byref(D), ctypes.byref(l1),
                              ctypes.byref(linf)), "or_jacobi_step")
    return xn, D.value, l1.value, linf.value


def pagerank_jacobi(rowptr, colidx, d=0.85, tol=1e-10, max_iter=1000, t=None, x0=None,
                    redistribute=True, history=False, lib=None):
    """Alg. 1 from x0 (default t).  Returns (x, iterations, last_l1_change[, history])."""
    lib = lib or load()
    rowptr, colidx = _csr(rowptr, colidx)
    n = rowptr.size - 1
    t = _vec(t, n)
    x0 = _vec(x0, n)
    x = np.empty(n, dtype=np.float64)
    it, res = ctypes.c_int32(), ctypes.c_double()
    hist = np.zeros(max(max_iter, 1), dtype=np.float64) if history else None
    _check(lib.or_pagerank_jacobi(n, _p(rowptr), _p(colidx), d, _p(t), int(redistribute), tol,
                                  max_iter, _p(x0), _p(x), ctypes.byref(it), ctypes.byref(res),
                                  _p(hist)), "or_pagerank_jacobi")
    if history:
        return x, it.value, res.value, hist[: it.value]
    return x, it.value, res.value


def fixed_point(rowptr, colidx, d=0.85, t=None, redistribute=True, tol=1e-13, max_iter=5000,
                lib=None):
    """The fixed point to FP64 accuracy: Alg. 1 until the L1 change is below tol (default
    1e-13) or max_iter.  The error to the exact fixed point is at most d/(1-d) times the
    last change (contraction bound)."""
    x, it, res = pagerank_jacobi(rowptr, colidx, d=d, tol=tol, max_iter=max_iter, t=t,
                                 redistribute=redistribute, lib=lib)
    return x, it, res


def vertex_update(v, rowptr, colidx, x, dangling_mass, d=0.85, t=None, deg=None, lib=None):
    """The updated rank of vertex v computed from vector x and the given dangling mass."""
    lib = lib or load()
    rowptr, colidx = _csr(rowptr, colidx)
    n = rowptr.size - 1
    x = _vec(x, n)
    t = _vec(t, n)
    if deg is None:
        deg = outdeg(rowptr, colidx, lib)
    return lib.or_vertex_update(int(v), n, _p(rowptr), _p(colidx), _p(deg), d, _p(t),
                                float(dangling_mass), _p(x))


def dangling_mass(rowptr, colidx, x, deg=None, lib=None):
    if deg is None:
        deg = outdeg(rowptr, colidx, lib)
    x = np.asarray(x, dtype=np.float64)
    return float(np.sum(x[deg == 0], dtype=np.float64)) if deg.size else 0.0


def dense_solve(rowptr, colidx, d=0.85, t=None, redistribute=True, lib=None):
    lib = lib or load()
    rowptr, colidx = _csr(rowptr, colidx)
    n = rowptr.size - 1
    t = _vec(t, n)
    x = np.empty(n, dtype=np.float64)
    _check(lib.or_dense_solve(n, _p(rowptr), _p(colidx), d, _p(t), int(redistribute), _p(x)),
           "or_dense_solve")
    return x


def nosync(rowptr, colidx, d=0.85, p=4, tol=1e-10, max_sweeps=1000, t=None, x0=None,
           speed=None, norm="l1", redistribute=True, dangling="complement", lib=None):
    """Alg. 3 with p simulated threads.  ``dangling`` picks the form of the dangling share:
    "mass" (running dangling mass D) or "complement" (sum(t) minus the running mass of the
    vertices with out-edges).  Returns (x, sweeps_per_thread, updates, estimate)."""
    x, sweeps, upd, est, _ = nosync_perforated(rowptr, colidx, d=d, p=p, tol=tol,
                                               max_sweeps=max_sweeps, t=t, x0=x0, speed=speed,
                                               norm=norm, redistribute=redistribute,
                                               dangling=dangling, eps=0.0, lib=lib)
    return x, sweeps, upd, est


def nosync_perforated(rowptr, colidx, d=0.85, p=4, tol=1e-10, max_sweeps=1000, t=None, x0=None,
                      speed=None, norm="l1", redistribute=True, dangling="complement", eps=0.0,
                      lib=None):
    """Alg. 3 with the loop perforation of Alg. 5: a vertex whose change is nonzero and below
    eps is no longer recomputed (eps = 0: plain Alg. 3).  Returns (x, sweeps_per_thread,
    updates_computed, estimate, frozen_count)."""
    if dangling not in ("mass", "complement"):
        raise ValueError("dangling must be 'mass' or 'complement'")
    lib = lib or load()
    rowptr, colidx = _csr(rowptr, colidx)
    n = rowptr.size - 1
    t = _vec(t, n)
    x0 = _vec(x0, n)
    sp = None if speed is None else np.ascontiguousarray(speed, dtype=np.int32)
    if sp is not None and sp.shape != (p,):
        raise ValueError("speed needs one entry per thread")
    x = np.empty(n, dtype=np.float64)
    sweeps = np.zeros(p, dtype=np.int32)
    upd, est, nf = ctypes.c_int64(), ctypes.c_double(), ctypes.c_int64()
    _check(lib.or_nosync(n, _p(rowptr), _p(colidx), d, _p(t), int(redistribute),
                         1 if dangling == "complement" else 0, p, _p(sp),
                         0 if norm == "l1" else 1, tol, max_sweeps, _p(x0), _p(x), _p(sweeps),
                         ctypes.byref(upd), ctypes.byref(est), float(eps), ctypes.byref(nf)),
           "or_nosync")
    return x, sweeps, upd.value, est.value, nf.value


# ------------------------------------------------------------ weighted graphs --

def _weights(w, nnz):
    w = np.ascontiguousarray(w, dtype=np.float64)
    if w.shape != (nnz,):
        raise ValueError(f"expected {nnz} edge weights")
    if nnz == 0:
        w = np.ones(1, dtype=np.float64)
    return w


def w_outweight(rowptr, colidx, w, lib=None):
    """W(u) = sum of the weights of u's out-edges (edges given as an in-edge CSR)."""
    lib = lib or load()
    rowptr, colidx = _csr(rowptr, colidx)
    n = rowptr.size - 1
    W = np.empty(n, dtype=np.float64)
    _check(lib.or_w_outweight(n, _p(rowptr), _p(colidx), _p(_weights(w, int(rowptr[-1]))), _p(W)),
           "or_w_outweight")
    return W


def w_pagerank(rowptr, colidx, w, d=0.85, t=None, tol=1e-13, max_iter=5000, x0=None, lib=None):
    """Alg. 1 on the weighted graph (P(u,v) = w(u,v)/W(u)).  Returns (x, iterations, last_l1)."""
    lib = lib or load()
    rowptr, colidx = _csr(rowptr, colidx)
    n = rowptr.size - 1
    x = np.empty(n, dtype=np.float64)
    it, res = ctypes.c_int32(), ctypes.c_double()
    _check(lib.or_w_jacobi(n, _p(rowptr), _p(colidx), _p(_weights(w, int(rowptr[-1]))), d,
                           _p(_vec(t, n)), tol, max_iter, _p(_vec(x0, n)), _p(x), ctypes.byref(it),
                           ctypes.byref(res)), "or_w_jacobi")
    return x, it.value, res.value


def w_adjoint(rowptr, colidx, w, x, c, d=0.85, tol=1e-14, max_iter=5000, lib=None):
    """Adjoint of L = c^T x at the weighted fixed point x.  Returns a dict with lambda, mu,
    grad_t (dL/dt) and grad_w (dL/dw per edge, aligned with colidx), iterations, residual."""
    lib = lib or load()
    rowptr, colidx = _csr(rowptr, colidx)
    n = rowptr.size - 1
    nnz = int(rowptr[-1])
    lam, mu, gt = (np.empty(n, dtype=np.float64) for _ in range(3))
    gw = np.empty(max(nnz, 1), dtype=np.float64)
    it, res = ctypes.c_int32(), ctypes.c_double()
    _check(lib.or_w_adjoint(n, _p(rowptr), _p(colidx), _p(_weights(w, nnz)), d, _p(_vec(x, n)),
                            _p(_vec(c, n)), tol, max_iter, _p(lam), _p(mu), _p(gt), _p(gw),
                            ctypes.byref(it), ctypes.byref(res)), "or_w_adjoint")
    return {"lambda": lam, "mu": mu, "grad_t": gt, "grad_w": gw[:nnz], "iterations": it.value,
            "residual": res.value}


def w_adjoint_step(rowptr, colidx, w, c, lam, d=0.85, lib=None):
    """One update of the adjoint system from lam: returns (lambda_out, l1_change)."""
    lib = lib or load()
    rowptr, colidx = _csr(rowptr, colidx)
    n = rowptr.size - 1
    out = np.empty(n, dtype=np.float64)
    l1 = ctypes.c_double()
    _check(lib.or_w_adjoint_step(n, _p(rowptr), _p(colidx), _p(_weights(w, int(rowptr[-1]))), d,
                                 _p(_vec(c, n)), _p(_vec(lam, n)), _p(out), ctypes.byref(l1)),
           "or_w_adjoint_step")
    return out, l1.value


def dense_adjoint(rowptr, colidx, w, c, d=0.85, t=None):
    """The same gradients by dense linear algebra (small n): M = I - d P^T - (d/n) 1 a^T is
    assembled explicitly, x = (1-d) M^-1 t and lambda = M^-T c by numpy's solver, and each
    edge weight's gradient is -lambda^T (dM/dw_e) x with dM/dw_e assembled from the
    quotient rule on P(u,.) = w(u,.)/W(u).  Returns (x, lambda, grad_t, grad_w)."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    colidx = np.asarray(colidx, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    n = rowptr.size - 1
    t = np.full(n, 1.0 / n) if t is None else np.asarray(t, dtype=np.float64)
    dst = np.repeat(np.arange(n), np.diff(rowptr))
    W = np.zeros(n)
    np.add.at(W, colidx, w)
    P = np.zeros((n, n))                      # P[u, v]
    for e in range(colidx.size):
        P[colidx[e], dst[e]] += w[e] / W[colidx[e]]
    a = (W == 0.0).astype(np.float64)
    M = np.eye(n) - d * P.T - (d / n) * np.outer(np.ones(n), a)
    x = np.linalg.solve(M, (1.0 - d) * t)
    lam = np.linalg.solve(M.T, np.asarray(c, dtype=np.float64))
    grad_t = (1.0 - d) * lam
    grad_w = np.empty(colidx.size)
    for e in range(colidx.size):
        u, v = colidx[e], dst[e]
        dP = np.zeros((n, n))                 # d P / d w_e: row u only
        dP[u, :] = -P[u, :] / W[u]
        dP[u, v] += 1.0 / W[u]
        dM = -d * dP.T
        grad_w[e] = -lam @ dM @ x
    return x, lam, grad_t, grad_w


def pagerank_perforated(rowptr, colidx, d=0.85, tol=1e-10, max_iter=1000, eps=0.0, t=None, lib=None):
    """Alg. 5 (loop perforation): a vertex whose change is nonzero and below eps stops being
    recomputed.  Returns (x, iterations, last_l1_change, frozen_count)."""
    lib = lib or load()
    rowptr, colidx = _csr(rowptr, colidx)
    n = rowptr.size - 1
    x = np.empty(n, dtype=np.float64)
    it, res, nf = ctypes.c_int32(), ctypes.c_double(), ctypes.c_int64()
    _check(lib.or_pagerank_perforated(n, _p(rowptr), _p(colidx), d, _p(_vec(t, n)), tol, max_iter, eps,
                                      _p(x), ctypes.byref(it), ctypes.byref(res), ctypes.byref(nf)),
           "or_pagerank_perforated")
    return x, it.value, res.value, nf.value
