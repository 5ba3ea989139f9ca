"""Weighted PageRank and its adjoint (pr_create_wgraph, pr_solve_weighted, pr_adjoint, and
the torch.autograd.Function on top) against the FP64 oracle.

  * tiny graphs (n <= 12): forward, dL/dt and dL/dw against the dense adjoint (explicit
    matrices, numpy's solver);
  * R-MAT scale 12: every gradient entry against the oracle's iterative adjoint, and 32
    teleport and 32 weight entries (64 sampled entries) against central differences
    (h = 1e-3) of the FP64 forward at tol 1e-14;
  * graphs whose rows reach the block-per-row class of the weighted kernels (rows with
    >= 2048 edges) in the in-edge direction (forward), the out-edge direction (adjoint) or
    both: an in-star and an out-star with 4096 leaves, their union, and R-MAT scale 16
    with edge factor 16 (17 rows of each kind) -- x, dL/dt and dL/dw element by element
    against the oracle;
  * the adjoint workload at full size (weighted R-MAT scale 20, weights U(0.1, 1],
    L = sum_i c_i x_i with c ~ N(0, 1)): x against the oracle's Alg. 1 after the same
    number of iterations, dL/dt and dL/dw element by element against the oracle's adjoint
    evaluated at the same x; the identities (1-d) lambda^T t = c^T x and sum over u's
    out-edges of w(e) dL/dw(e) = 0, and the adjoint equation at sampled vertices.
FP32 against FP64: the forward within the single-vector bar (L1 <= 1e-6, per-vertex
relative <= 1e-4).  Gradients three ways: within 1e-4 of the largest entry (absolute),
relative L1 <= 1e-4, and every entry within 1e-3 of the magnitude of the terms it is
made of (for dL/dw(e), e = (u, v): d x(u)/W(u) (|lambda(v)| + sum_v' P(u,v') |lambda(v')|);
for dL/dt(u): (1-d) (|c(u)| + d sum_v P(u,v) |lambda(v)| + d a(u) |sum lambda|/n)), plus
1e-6 of the largest entry for the error the stopping test leaves.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pr = pytest.importorskip("paper_2109_09527_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

D = 0.85


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    yield


def weighted(rp, ci, seed):
    return (0.1 + 0.9 * gg.uniform(seed, 11, ci.size)).astype(np.float32)


def loss_weights(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n).astype(np.float32)


def close_to(a, b, scale_rel=1e-4):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b))) <= scale_rel * max(float(np.max(np.abs(b))), 1e-30)


def rel_l1(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.abs(a - b).sum() / max(float(np.abs(b).sum()), 1e-300))


def term_scales(rp, ci, w64, x64, lam64, d=D):
    """Per-entry magnitude of the terms each gradient is made of (see the module doc)."""
    n = rp.size - 1
    dst = np.repeat(np.arange(n), np.diff(rp))
    W = np.zeros(n)
    np.add.at(W, ci, w64)
    P = w64 / W[ci]
    mu_abs = np.zeros(n)
    np.add.at(mu_abs, ci, P * np.abs(lam64[dst]))
    dangling = W == 0
    lam_abs = np.abs(lam64)
    scale_t = (1 - d) * (np.abs(lam64) + d * mu_abs + d * dangling * abs(lam64.sum()) / n)
    scale_w = d * x64[ci] / W[ci] * (lam_abs[dst] + mu_abs[ci])
    return scale_t, scale_w


def check_gradients(rp, ci, w64, x64, c64, gt, gw, d=D):
    """dL/dt and dL/dw from the GPU against the oracle's adjoint at the same x."""
    adj = oracle.w_adjoint(rp, ci, w64, x64, c64, d=d, tol=1e-11)
    scale_t, scale_w = term_scales(rp, ci, w64, x64, adj["lambda"], d)
    scale_t = np.maximum(scale_t, (1 - d) * np.abs(c64))
    for got, ref, sc, name in ((gt, adj["grad_t"], scale_t, "dL/dt"), (gw, adj["grad_w"], scale_w, "dL/dw")):
        got = np.asarray(got, np.float64)
        err = np.abs(got - ref)
        bound = 1e-3 * sc + 1e-6 * np.max(np.abs(ref))
        worst = int(np.argmax(err / np.maximum(bound, 1e-300)))
        assert close_to(got, ref), (name, float(np.max(err)), float(np.max(np.abs(ref))))
        assert rel_l1(got, ref) <= 1e-4, (name, rel_l1(got, ref))
        assert np.all(err <= bound), (name, worst, float(err[worst]), float(bound[worst]), float(ref[worst]))
    return adj


def star_graph(kind, leaves=4096):
    """In-star (leaves -> hub 0), out-star (hub 0 -> leaves) or both, as in-edge CSR."""
    n = leaves + 1
    lv = np.arange(1, n)
    hub = np.zeros(leaves, dtype=np.int64)
    if kind == "in":
        src, dst = lv, hub
    elif kind == "out":
        src, dst = hub, lv
    else:
        src, dst = np.concatenate([lv, hub]), np.concatenate([hub, lv])
    return gg.edges_to_in_csr(n, src, dst)


@pytest.mark.parametrize("graph", ["in_star", "out_star", "bi_star", "rmat16"])
def test_block_per_row_class_against_the_oracle(graph):
    """Rows with >= 2048 edges are gathered by a whole block each (forward over in-edges,
    adjoint and per-edge gradients over out-edges); these graphs put such rows on the
    forward side (in-star), the adjoint side (out-star) or both."""
    if graph == "rmat16":
        rp, ci = gg.rmat(16, 16, seed=16)
    else:
        rp, ci = star_graph(graph.split("_")[0])
    n = rp.size - 1
    indeg, outdeg = np.diff(rp), np.bincount(ci, minlength=n)
    if graph in ("in_star", "bi_star", "rmat16"):
        assert indeg.max() >= 2048
    if graph in ("out_star", "bi_star", "rmat16"):
        assert outdeg.max() >= 2048
    w = weighted(rp, ci, 7)
    c = loss_weights(n, 7)
    w64, c64 = w.astype(np.float64), c.astype(np.float64)
    with pr.WeightedGraph(rp, ci, w) as g:
        # The stars' FP32 iterates end in a rounding 2-cycle: the hub (~46% of the mass)
        # and its 4096 identical leaves flip by a few ulps each iteration, an L1 change of
        # ~6e-7 in an FP32 emulation of the kernel's arithmetic; their tolerance sits above
        # that floor.
        x, info = g.solve(D, 2e-6 if graph.endswith("star") else 1e-6, 500)
        assert info.converged == 1
        # forward: the oracle's Alg. 1 after the same iterations (matching mode)
        xo, _, _ = oracle.w_pagerank(rp, ci, w64, d=D, tol=0.0, max_iter=info.iterations)
        assert np.abs(x - xo).sum() <= 1e-6
        assert np.max(np.abs(x - xo) / xo) <= 1e-4
        # and the fixed point, within the bound of the stopping test
        xs, _, _ = oracle.w_pagerank(rp, ci, w64, d=D, tol=1e-15)
        assert np.abs(x - xs).sum() <= info.residual_l1 / (1 - D) + 2e-7
        gt, gw, ainfo = g.adjoint(x, c, D, 1e-6, 2000)
        assert ainfo.converged == 1
    check_gradients(rp, ci, w64, x.astype(np.float64), c64, gt, gw)


@pytest.mark.parametrize("seed", range(5))
def test_tiny_graphs_match_the_dense_adjoint(seed):
    n = 4 + 2 * seed
    rp, ci = gg.random_digraph(n, 3 * n, seed=20 + seed, allow_multi=seed % 2 == 0)
    w = weighted(rp, ci, seed)
    t = (0.05 + gg.uniform(seed, 12, n)).astype(np.float32)
    t /= t.sum()
    c = loss_weights(n, seed)
    xd, lamd, gtd, gwd = oracle.dense_adjoint(rp, ci, w.astype(np.float64), c.astype(np.float64), d=D,
                                              t=t.astype(np.float64))
    with pr.WeightedGraph(rp, ci, w) as g:
        x, info = g.solve(D, 1e-7, 500, teleport=t)
        assert info.converged == 1
        gt, gw, ainfo = g.adjoint(x, c, D, 1e-6, 1000)
        assert ainfo.converged == 1
    assert np.abs(x - xd).sum() <= 1e-6
    assert close_to(gt, gtd) and close_to(gw, gwd)


def test_rmat12_against_the_oracle_adjoint_and_central_differences():
    rp, ci = gg.rmat(12, 8, seed=12)
    n = rp.size - 1
    w = weighted(rp, ci, 3)
    c = loss_weights(n, 3)
    t = np.full(n, 1.0 / n, dtype=np.float32)
    with pr.WeightedGraph(rp, ci, w) as g:
        x, info = g.solve(D, 1e-7, 500)
        gt, gw, ainfo = g.adjoint(x, c, D, 1e-6, 2000)
    assert info.converged == 1 and ainfo.converged == 1
    w64, c64 = w.astype(np.float64), c.astype(np.float64)
    xo, _, _ = oracle.w_pagerank(rp, ci, w64, d=D, tol=1e-15)
    assert np.abs(x - xo).sum() <= 1e-6
    assert np.max(np.abs(x - xo) / xo) <= 1e-4
    adj = oracle.w_adjoint(rp, ci, w64, xo, c64, d=D)
    assert close_to(gt, adj["grad_t"]) and close_to(gw, adj["grad_w"])
    h = 1e-3

    def L(tt, ww):
        xx, _, _ = oracle.w_pagerank(rp, ci, ww, d=D, t=tt, tol=1e-14, x0=xo)
        return c64 @ xx

    rng = np.random.default_rng(1)
    t64 = t.astype(np.float64)
    for i in rng.integers(0, n, 32):
        tp, tm = t64.copy(), t64.copy()
        tp[i] += h
        tm[i] -= h
        fd = (L(tp, w64) - L(tm, w64)) / (2 * h)
        assert abs(gt[i] - fd) <= 1e-4 * np.max(np.abs(adj["grad_t"])), i
    for e in rng.integers(0, ci.size, 32):
        wp, wm = w64.copy(), w64.copy()
        wp[e] += h
        wm[e] -= h
        fd = (L(t64, wp) - L(t64, wm)) / (2 * h)
        assert abs(gw[e] - fd) <= 1e-4 * np.max(np.abs(adj["grad_w"])) + 1e-8, e


def test_autograd_function_matches_the_adjoint_and_set_weights():
    rp, ci = gg.rmat(11, 8, seed=2)
    n = rp.size - 1
    w = weighted(rp, ci, 5)
    c = loss_weights(n, 5)
    dev = torch.device("cuda", 0)
    with pr.WeightedGraph(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev),
                          torch.from_numpy(w).to(dev)) as g:
        t = torch.full((n,), 1.0 / n, device=dev, requires_grad=True)
        wt = torch.from_numpy(w * 1.5).to(dev).requires_grad_(True)   # the call sets these weights
        x = pr.weighted_pagerank(g, t, wt, damping=D, tol=1e-7, adjoint_tol=1e-6)
        L = (torch.from_numpy(c).to(dev) * x).sum()
        L.backward()
        torch.cuda.synchronize()
        xh, _ = g.solve(D, 1e-7, 500)           # graph holds w * 1.5 now
        gt, gw, _ = g.adjoint(xh, c, D, 1e-6, 500)
    assert np.array_equal(x.detach().cpu().numpy(), xh)
    assert np.array_equal(t.grad.cpu().numpy(), gt)
    assert np.array_equal(wt.grad.cpu().numpy(), gw)
    # scaling all weights changes nothing: P is row-normalised
    xo, _, _ = oracle.w_pagerank(rp, ci, w.astype(np.float64), d=D, tol=1e-15)
    assert np.abs(xh - xo).sum() <= 1e-6


def test_invalid_weights_and_arguments():
    rp, ci = gg.rmat(8, 8, seed=1)
    w = weighted(rp, ci, 1)
    bad = w.copy()
    bad[3] = 0.0
    with pytest.raises(pr.PageRankError):
        pr.WeightedGraph(rp, ci, bad)
    with pr.WeightedGraph(rp, ci, w) as g:
        bad[3] = np.nan
        with pytest.raises(pr.PageRankError):
            g.set_weights(bad)
        g.set_weights(w)
        x, info = g.solve()
        assert info.converged == 1
        with pytest.raises(pr.PageRankError):
            pr.pr_adjoint(g.handle, D, 1e-6, 10, x, x, None, None)


def test_fullsize_weighted_rmat20_identities_and_sampled_adjoint_equation():
    """Config: weighted R-MAT scale 20, weights U(0.1, 1], L = c^T x with c ~ N(0, 1)."""
    rp, ci = gg.rmat(20, 16, seed=20)
    n = rp.size - 1
    w = weighted(rp, ci, 20)
    c = loss_weights(n, 20)
    dev = torch.device("cuda", 0)
    with pr.WeightedGraph(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev),
                          torch.from_numpy(w).to(dev)) as g:
        assert np.diff(rp).max() >= 2048 and np.bincount(ci, minlength=n).max() >= 2048
        x, info = g.solve(D, 1e-6, 200)
        gt, gw, ainfo = g.adjoint(x, c, D, 1e-6, 1000)
    assert info.converged == 1 and ainfo.converged == 1
    x64, c64, w64 = x.astype(np.float64), c.astype(np.float64), w.astype(np.float64)
    # x against the oracle's Alg. 1 after the same number of iterations
    xo, _, _ = oracle.w_pagerank(rp, ci, w64, d=D, tol=0.0, max_iter=info.iterations)
    assert np.abs(x64 - xo).sum() <= 1e-6
    assert np.max(np.abs(x64 - xo) / xo) <= 1e-4
    # every gradient entry against the oracle's adjoint at the same x
    check_gradients(rp, ci, w64, x64, c64, gt, gw)
    lam = gt.astype(np.float64) / (1 - D)
    # (1-d) lambda^T t = c^T x  (t uniform)
    assert abs(gt.astype(np.float64).sum() / n - c64 @ x64) <= 1e-4 * np.abs(c64) @ x64
    # the weighted gradients of each vertex's out-edges sum to zero, to within the FP32
    # rounding of the terms d x(u)/W(u) w(e) lambda(v) they are made of
    W = np.zeros(n)
    np.add.at(W, ci, w64)
    dst = np.repeat(np.arange(n), np.diff(rp))
    per_src = np.zeros(n)
    np.add.at(per_src, ci, w64 * gw.astype(np.float64))
    scale = np.zeros(n)
    np.add.at(scale, ci, w64 * np.abs(lam[dst]))
    has_out = W > 0
    scale[has_out] *= D * x64[has_out] / W[has_out]
    assert np.all(np.abs(per_src) <= 1e-5 * scale + 1e-15)
    # the adjoint equation lambda(u) = c(u) + d (mu(u) + a(u) sum(lambda)/n), one vertex at a time
    order = np.argsort(ci, kind="stable")
    out_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(out_ptr, ci.astype(np.int64) + 1, 1)
    out_ptr = np.cumsum(out_ptr)
    L = lam.sum()
    rng = np.random.default_rng(2)
    for u in rng.integers(0, n, 512):
        es = order[out_ptr[u]: out_ptr[u + 1]]
        mu = float((w64[es] / W[u] * lam[dst[es]]).sum()) if es.size else 0.0
        rhs = c64[u] + D * (mu + (L / n if W[u] == 0 else 0.0))
        assert abs(lam[u] - rhs) <= 1e-4 * max(1.0, abs(rhs)), u
