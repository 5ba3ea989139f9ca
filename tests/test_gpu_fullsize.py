"""Parity at the full benchmark sizes, in the benchmark's launch configuration.

Graphs: R-MAT scale 24 and the Erdos-Renyi digraph of 2^24 vertices with 20%
dangling vertices (the two graphs the benchmark solves, same seeds), and R-MAT
scale 26 with 64-bit row offsets solved by the barrier-free variant.  Each
graph is created from device arrays with default options, as the benchmark
does.

At these sizes the FP64 oracle cannot follow a whole solve, so each result is
checked by what the oracle can compute in seconds:

  * matching mode over a few iterations (all vertices): three synchronous GPU
    updates from the uniform vector against three oracle iterations, L1 <= 1e-6
    and per-vertex relative error <= 1e-4 (FP32 against FP64);
  * a residual certificate for every converged solve: one FP64 oracle update
    T(x) of the returned vector gives r = ||T(x) - x||_1, and the contraction of
    Eq. 1 (factor d in L1) bounds the distance to the fixed point by r/(1-d).
    The solves stop when the L1 change of a synchronous update is below 1e-6,
    so r must be below that plus the FP32 rounding of x (about 2^-24 per unit
    of mass per rounding; 5e-7 is ample);
  * sampled vertices, one by one: the oracle's single-vertex update (Eq. 1 at
    one row) at 2048 seeded random vertices and the 64 vertices of largest
    rank agrees with the full oracle update, and changes x_v by at most 1e-3
    relative;
  * invariants: sum(x) = 1 and x_v >= (1-d)/n for every vertex.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pr = pytest.importorskip("paper_2109_09527_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

D = 0.85
TOL = 1e-6
SEEDS = {"rmat24": 24, "er24": 1024, "rmat26": 26}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    yield


_graphs = {}


def graph(name):
    if name not in _graphs:
        if name == "rmat24":
            _graphs[name] = gg.rmat(24, 16, seed=SEEDS[name])
        elif name == "er24":
            _graphs[name] = gg.er_dangling(1 << 24, 16.0, 0.2, seed=SEEDS[name])
        elif name == "rmat26":
            _graphs.clear()   # host memory: keep one graph at a time at this size
            _graphs[name] = gg.rmat(26, 16, seed=SEEDS[name])
        else:
            raise KeyError(name)
    return _graphs[name]


def device_graph(rp, ci):
    dev = torch.device("cuda", 0)
    return pr.Graph(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev))


def certify(rp, ci, x, deg):
    """Residual certificate and sampled single-vertex checks of a converged result."""
    n = rp.size - 1
    x64 = np.asarray(x, np.float64)
    assert abs(x64.sum() - 1.0) < 1e-5
    assert x64.min() >= (1.0 - D) / n * (1.0 - 1e-5)
    xn, dmass, r, _ = oracle.jacobi_step(rp, ci, x64, d=D)
    assert r < TOL + 5e-7, f"one FP64 update moves the result by {r:.3e} in L1"
    rng = np.random.default_rng(7)
    sample = np.unique(np.concatenate([rng.integers(0, n, 2048), np.argsort(x64)[-64:]]))
    for v in sample:
        xv = oracle.vertex_update(int(v), rp, ci, x64, dmass, d=D, deg=deg)
        assert xv == pytest.approx(xn[v], rel=1e-12, abs=1e-300)
        assert abs(xv - x64[v]) <= 1e-3 * x64[v], (int(v), xv, x64[v])
    return r


@pytest.mark.parametrize("name", ["rmat24", "er24"])
def test_fullsize_iterations_match_oracle(name):
    """Three synchronous updates at full size: every vertex against the oracle."""
    rp, ci = graph(name)
    n = rp.size - 1
    dev = torch.device("cuda", 0)
    x0 = torch.full((n,), 1.0 / n, dtype=torch.float32, device=dev)
    out = torch.empty_like(x0)
    with device_graph(rp, ci) as g:
        info = pr.pr_iterate(g.handle, D, None, x0, 3, out)
        torch.cuda.synchronize()
    assert info.iterations == 3
    x = out.cpu().numpy().astype(np.float64)
    xo, it, _ = oracle.pagerank_jacobi(rp, ci, d=D, tol=0, max_iter=3)
    assert it == 3
    assert float(np.abs(x - xo).sum()) <= 1e-6
    assert float(np.max(np.abs(x - xo) / xo)) <= 1e-4


@pytest.mark.parametrize("name", ["rmat24", "er24"])
def test_fullsize_solves_certified(name):
    """Both variants to L1 < 1e-6 as the benchmark runs them; each result certified by
    the oracle, and the two results within the sum of their certificates."""
    rp, ci = graph(name)
    n = rp.size - 1
    deg = oracle.outdeg(rp, ci)
    dev = torch.device("cuda", 0)
    out = torch.empty(n, dtype=torch.float32, device=dev)
    results = {}
    with device_graph(rp, ci) as g:
        for variant in ("jacobi", "nonblocking"):
            _, info = g.solve(damping=D, tol=TOL, max_iter=200, variant=variant, out=out)
            torch.cuda.synchronize()
            assert info.converged == 1, variant
            assert info.residual_l1 < TOL
            x = out.cpu().numpy()
            r = certify(rp, ci, x, deg)
            results[variant] = (x.astype(np.float64), r)
    (xj, rj), (xn, rn) = results["jacobi"], results["nonblocking"]
    bound = (rj + rn) / (1.0 - D) + 4e-7
    assert float(np.abs(xj - xn).sum()) <= bound


def test_massive_rmat26_nonblocking_int64():
    """R-MAT scale 26 (67.1M vertices, about 1.07e9 edges), 64-bit row offsets kept on
    the device, barrier-free variant to L1 < 1e-6, certified by the oracle."""
    rp, ci = graph("rmat26")
    n = rp.size - 1
    assert rp.dtype == np.int64 and n == 1 << 26 and ci.size > 1_000_000_000
    pr.pr_set_option(None, pr.PR_OPT_INDEX64, 1)
    try:
        g = device_graph(rp, ci)
    finally:
        pr.pr_set_option(None, pr.PR_OPT_INDEX64, 0)
    with g:
        assert g.stats()["rowptr_bytes"] == 8
        out = torch.empty(n, dtype=torch.float32, device=torch.device("cuda", 0))
        _, info = g.solve(damping=D, tol=TOL, max_iter=200, variant="nonblocking", out=out)
        torch.cuda.synchronize()
        assert info.converged == 1
        x = out.cpu().numpy()
    certify(rp, ci, x, oracle.outdeg(rp, ci))
    _graphs.clear()
