"""Many independent graphs in one solve (pr_graph_set_partition + pr_solve_set) against
the FP64 oracle run on each graph alone.

Graph i of the set is an ordinary PageRank problem on its own vertices (teleport 1/n_i,
its own dangling share), so the oracle solves each graph's sub-CSR separately, for the
number of iterations the library reports for that graph (matching mode): L1 <= 1e-6 and
per-vertex relative error <= 1e-4.  At the full size of the multi-graph workload (64
R-MAT graphs with 1e3..1e6 vertices, edge factor 8) every graph is certified by one FP64
oracle update of its own result.
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


def mixed_set():
    graphs = [gg.rmat_n(n, 8, seed=100 + n) for n in (300, 1000, 2500, 5000, 777)]
    graphs.append(gg.er_dangling(3000, 6.0, 0.25, seed=4))
    graphs.append(gg.cycle(50))                       # already at its fixed point
    graphs.append(gg.empty(10))                       # every vertex dangling
    graphs.append(gg.in_star(40))
    return graphs


def sub_graph(rp, ci, off, i):
    lo, hi = off[i], off[i + 1]
    return rp[lo: hi + 1] - rp[lo], ci[rp[lo]: rp[hi]] - lo


def check_graphs(graphs, x, off, its, tol):
    for i, (grp, gci) in enumerate(graphs):
        xi = x[off[i]: off[i + 1]].astype(np.float64)
        xo, it, _ = oracle.pagerank_jacobi(grp, gci, d=D, tol=0, max_iter=int(its[i]))
        xo /= xo.sum()
        assert np.abs(xi - xo).sum() <= 1e-6, i
        assert np.max(np.abs(xi - xo) / xo) <= 1e-4, i
        _, it_o, _ = oracle.pagerank_jacobi(grp, gci, d=D, tol=tol, max_iter=500)
        assert abs(it_o - int(its[i])) <= 1, (i, it_o, its[i])


@pytest.mark.parametrize("heavy", [1024, 64])
def test_set_matches_each_graph_alone(heavy):
    graphs = mixed_set()
    rp, ci, off = gg.block_diagonal(graphs)
    pr.set_heavy_degree(heavy)
    try:
        g = pr.Graph(rp, ci)
    finally:
        pr.set_heavy_degree(pr.DEFAULT_HEAVY_DEGREE)
    with g:
        g.set_partition(off)
        x, info, res, its = g.solve_set(tol=1e-6, max_iter=300)
        # the same graphs one at a time through the single-graph solver
        singles = []
        for grp, gci in graphs:
            with pr.Graph(grp, gci) as gi:
                singles.append(gi.solve(tol=1e-6, max_iter=300))
    assert info.converged == 1 and np.all(res < 1e-6)
    assert info.iterations == its.max()
    assert its[6] == 1                               # the cycle stops after one iteration
    for i, (xs, infos) in enumerate(singles):
        assert infos.iterations == its[i], i
        np.testing.assert_allclose(x[off[i]: off[i + 1]], xs, rtol=1e-5, err_msg=str(i))
        assert abs(float(x[off[i]: off[i + 1]].astype(np.float64).sum()) - 1.0) < 1e-6
    check_graphs(graphs, x, off, its, 1e-6)


def test_set_is_deterministic_with_and_without_the_loop_graph():
    graphs = mixed_set()
    rp, ci, off = gg.block_diagonal(graphs)
    with pr.Graph(rp, ci) as g:
        g.set_partition(off)
        x1, _, _, its1 = g.solve_set()
        x2, _, _, its2 = g.solve_set()
        g.set_option(pr.PR_OPT_USE_GRAPH, 0)
        x3, _, _, its3 = g.solve_set()
    assert np.array_equal(x1, x2) and np.array_equal(x1, x3)
    assert np.array_equal(its1, its2) and np.array_equal(its1, its3)


def test_set_partition_errors():
    graphs = [gg.rmat_n(200, 8, seed=1), gg.rmat_n(300, 8, seed=2)]
    rp, ci, off = gg.block_diagonal(graphs)
    with pr.Graph(rp, ci) as g:
        for bad in ([0, 200], [0, 300, 500], [0, 200, 200, 500], [1, 200, 500]):
            with pytest.raises(pr.PageRankError):
                g.set_partition(bad)
        # an edge across the two graphs
        src, dst = gg.in_csr_edges(rp, ci)
        rp2, ci2 = gg.edges_to_in_csr(500, np.append(src, 10), np.append(dst, 400))
        with pr.Graph(rp2, ci2) as g2:
            with pytest.raises(pr.PageRankError) as e:
                g2.set_partition(off)
            assert e.value.status == pr.PR_ERR_INVALID_GRAPH
            with pytest.raises(pr.PageRankError):
                pr.pr_solve_set(g2.handle, 2, D, 1e-6, 10, np.empty(500, np.float32))
        # the valid partition works after the failures
        g.set_partition(off)
        x, info, res, its = g.solve_set()
        assert info.converged == 1


def test_sixty_four_rmat_graphs_fullsize_certified():
    """The multi-graph workload at full size: 64 R-MAT graphs, vertex counts log-uniform in
    [1e3, 1e6], edge factor 8, one block-diagonal graph on the device; every graph's result
    is certified by one FP64 oracle update of that graph."""
    graphs = gg.multi_rmat(64, 1e3, 1e6, 8, seed=64)
    rp, ci, off = gg.block_diagonal(graphs)
    dev = torch.device("cuda", 0)
    with pr.Graph(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev)) as g:
        g.set_partition(off)
        out = torch.empty(rp.size - 1, dtype=torch.float32, device=dev)
        _, info, res, its = g.solve_set(tol=1e-6, out=out)
        torch.cuda.synchronize()
        x = out.cpu().numpy()
    assert info.converged == 1 and np.all(res < 1e-6)
    for i, (grp, gci) in enumerate(graphs):
        xi = x[off[i]: off[i + 1]].astype(np.float64)
        assert abs(xi.sum() - 1.0) < 1e-5
        _, _, r, _ = oracle.jacobi_step(grp, gci, xi, d=D)
        assert r < 1e-6 + 5e-7, (i, r)
