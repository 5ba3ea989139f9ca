"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (FP32 ranks against FP64):
  * matching mode -- GPU Jacobi and the oracle's Alg. 1 after the same number of
    iterations from the same start: L1 <= 1e-6 and per-vertex relative error
    <= 1e-4 (the target stated for FP32 ranks);
  * one synchronous update from the same input: L1 <= 1e-6, relative <= 1e-4;
  * any variant against the fixed point x*: ||x - x*||_1 <= r/(1-d) + 2e-7,
    where r is the L1 change of the verifying synchronous update reported by
    the library (contraction bound of Eq. 1 with factor d) and 2e-7 covers the
    FP32 rounding of x itself (about 2^-24 of sum(x) per rounding).
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


def l1(a, b):
    return float(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)).sum())


def max_rel(a, b):
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(np.asarray(a, np.float64) - b) / np.abs(b)))


def solve(rp, ci, **kw):
    with pr.Graph(rp, ci) as g:
        x, info = g.solve(**kw)
        return x, info, g.stats()


def matching(rp, ci, x, info, t=None, x0=None):
    xo, it, _ = oracle.pagerank_jacobi(rp, ci, d=D, tol=0, max_iter=info.iterations, t=t, x0=x0)
    return xo


# ------------------------------------------------------------------ fixtures --

@pytest.mark.parametrize("n", [1, 2, 5, 64, 300])
def test_closed_form_graphs(n):
    L = n - 1
    cases = [(gg.cycle, np.full(n, 1.0 / n)), (gg.complete, np.full(n, 1.0 / n)),
             (gg.empty, np.full(n, 1.0 / n))]
    if n >= 2:
        cases += [(gg.in_star, np.array([(1 + D * L) / (n + D * L)] + [1.0 / (n + D * L)] * L)),
                  (gg.out_star, np.array([1.0 / (n + D)] + [(L + D) / (L * (n + D))] * L))]
    for build, expect in cases:
        if n == 1 and build is not gg.empty:
            continue
        rp, ci = build(n)
        for variant in ("jacobi", "nonblocking"):
            x, info, _ = solve(rp, ci, tol=1e-6, max_iter=500, variant=variant)
            assert info.converged == 1, (build.__name__, variant)
            np.testing.assert_allclose(x, expect, rtol=2e-5, err_msg=f"{build.__name__} {variant}")


# ---------------------------------------------------- R-MAT, matching mode --

@pytest.mark.parametrize("scale,heavy,index64", [(10, 1024, 0), (12, 64, 0), (14, 1024, 0),
                                                 (14, 64, 1), (12, 4096, 0)])
def test_rmat_jacobi_matches_oracle(scale, heavy, index64):
    """Each layout path in turn: default bins; heavy threshold 64 (segments for most edges);
    64-bit row offsets on device; threshold 4096 (no heavy rows at scale 12)."""
    rp, ci = gg.rmat(scale, seed=scale)
    pr.set_heavy_degree(heavy)
    pr.pr_set_option(None, pr.PR_OPT_INDEX64, index64)
    try:
        x, info, st = solve(rp, ci, tol=1e-6, max_iter=200)
    finally:
        pr.set_heavy_degree(pr.DEFAULT_HEAVY_DEGREE)
        pr.pr_set_option(None, pr.PR_OPT_INDEX64, 0)
    assert st["rowptr_bytes"] == (8 if index64 else 4)
    if heavy == 64:
        assert st["n_heavy"] > 0 and st["n_segments"] > 0
    if heavy == 4096:
        assert st["n_heavy"] == 0
    xo = matching(rp, ci, x, info)
    _, it_oracle, _ = oracle.pagerank_jacobi(rp, ci, d=D, tol=1e-6, max_iter=200)
    assert abs(info.iterations - it_oracle) <= 1
    assert info.converged == 1 and info.residual_l1 < 1e-6
    assert l1(x, xo) <= 1e-6
    assert max_rel(x, xo) <= 1e-4
    assert abs(np.sum(x, dtype=np.float64) - 1.0) < 1e-5


def test_er_dangling_jacobi_matches_oracle():
    rp, ci = gg.er_dangling(20000, seed=3)
    x, info, st = solve(rp, ci, tol=1e-6, max_iter=200)
    assert st["n_dangling"] == 4000
    xo = matching(rp, ci, x, info)
    assert l1(x, xo) <= 1e-6 and max_rel(x, xo) <= 1e-4


def test_small_config_scale16_budget():
    """R-MAT scale 16, tol 1e-10 or 200 iterations: 1e-10 is below the FP32 floor of the
    L1 change, so the budget ends the run; the vector still matches the oracle's 200th
    iterate."""
    rp, ci = gg.rmat(16, seed=1)
    with pr.Graph(rp, ci) as g:
        x = np.empty(rp.size - 1, np.float32)
        status, info = pr.pr_solve(g.handle, D, 1e-10, 200, pr.PR_JACOBI, None, None, x)
    assert status in (pr.PR_NOT_CONVERGED, pr.PR_OK)
    if status == pr.PR_NOT_CONVERGED:
        assert info.iterations == 200 and info.converged == 0
    assert np.isfinite(info.residual_l1) and info.residual_l1 < 1e-6
    xo = matching(rp, ci, x, info)
    assert l1(x, xo) <= 1e-6 and max_rel(x, xo) <= 1e-4


# ------------------------------------------------------------ one update --

@pytest.mark.parametrize("scale,heavy", [(13, 1024), (13, 64)])
def test_one_synchronous_update(scale, heavy):
    rp, ci = gg.rmat(scale, seed=21)
    n = rp.size - 1
    x_in = gg.uniform(5, 1, n) + 0.1
    x_in = (x_in / x_in.sum()).astype(np.float32)
    t = gg.uniform(6, 1, n).astype(np.float32)
    t /= t.sum()
    pr.set_heavy_degree(heavy)
    try:
        with pr.Graph(rp, ci) as g:
            for tt in (None, t):
                x1, info = g.iterate(x_in, n_iter=1, teleport=tt)
                xo, Dm, l1o, _ = oracle.jacobi_step(rp, ci, x_in.astype(np.float64), d=D,
                                                    t=None if tt is None else tt.astype(np.float64))
                assert l1(x1, xo) <= 1e-6 and max_rel(x1, xo) <= 1e-4
                assert info.residual_l1 == pytest.approx(l1o, rel=1e-3, abs=1e-9)
                assert info.dangling_mass == pytest.approx(
                    oracle.dangling_mass(rp, ci, xo), rel=1e-5)
            # three updates equal three oracle steps
            x3, _ = g.iterate(x_in, n_iter=3)
            xo3, _, _ = oracle.pagerank_jacobi(rp, ci, d=D, tol=0, max_iter=3, x0=x_in)
            assert l1(x3, xo3) <= 1e-6
    finally:
        pr.set_heavy_degree(pr.DEFAULT_HEAVY_DEGREE)


def test_personalised_teleport_and_warm_start():
    rp, ci = gg.rmat(12, seed=8)
    n = rp.size - 1
    t = np.zeros(n, np.float32)
    seeds = gg.permutation(8, 3, n)[:8]
    t[seeds] = 1.0 / 8
    x, info, _ = solve(rp, ci, tol=1e-7, max_iter=300, teleport=t)
    xo = matching(rp, ci, x, info, t=t.astype(np.float64))
    assert l1(x, xo) <= 1e-6
    assert abs(np.sum(x, dtype=np.float64) - 1.0) < 1e-5
    # warm start from the answer: converges at once
    x2, info2, _ = solve(rp, ci, tol=1e-6, max_iter=300, teleport=t, x0=x)
    assert info2.iterations <= 3 and l1(x2, x) < 1e-6


def test_host_and_device_buffers_agree_and_runs_are_bitwise_reproducible():
    rp, ci = gg.rmat(13, seed=4)
    n = rp.size - 1
    dev = torch.device("cuda:0")
    with pr.Graph(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev)) as g:
        out_d = torch.empty(n, dtype=torch.float32, device=dev)
        g.solve(tol=1e-6, out=out_d)
        torch.cuda.synchronize()
        out_h, _ = g.solve(tol=1e-6)
        out_h2, _ = g.solve(tol=1e-6)
        g.set_option(pr.PR_OPT_USE_GRAPH, 0)
        out_h3, info3 = g.solve(tol=1e-6)
    assert np.array_equal(out_d.cpu().numpy(), out_h)
    assert np.array_equal(out_h, out_h2)
    assert np.array_equal(out_h, out_h3)          # host-driven loop, same iterates


# ---------------------------------------------------------- barrier-free --

@pytest.mark.parametrize("build", ["rmat12", "rmat14_heavy64", "rmat13_heavy64_index64", "er"])
def test_nonblocking_reaches_the_fixed_point(build):
    if build == "er":
        rp, ci = gg.er_dangling(30000, seed=9)
    elif build == "rmat12":
        rp, ci = gg.rmat(12, seed=2)
    elif build == "rmat14_heavy64":
        rp, ci = gg.rmat(14, seed=3)
        pr.set_heavy_degree(64)
    else:   # 64-bit row offsets on the device, segments for most edges
        rp, ci = gg.rmat(13, seed=4)
        pr.set_heavy_degree(64)
        pr.pr_set_option(None, pr.PR_OPT_INDEX64, 1)
    try:
        xstar, _, _ = oracle.fixed_point(rp, ci, d=D)
        for tol in (1e-6, 2e-7):
            x, info, _ = solve(rp, ci, tol=tol, max_iter=500, variant="nonblocking")
            assert info.converged == 1 and info.residual_l1 < tol
            err = l1(x, xstar)
            assert err <= info.residual_l1 / (1 - D) + 2e-7, (tol, err, info.residual_l1)
            assert max_rel(x, xstar) <= 1e-4
            xj, infoj, _ = solve(rp, ci, tol=tol, max_iter=500, variant="jacobi")
            assert l1(x, xj) <= (info.residual_l1 + infoj.residual_l1) / (1 - D) + 4e-7
    finally:
        pr.set_heavy_degree(pr.DEFAULT_HEAVY_DEGREE)
        pr.pr_set_option(None, pr.PR_OPT_INDEX64, 0)


@pytest.mark.parametrize("fail_after", [1, 3])
def test_nonblocking_recovers_from_a_failing_block(fail_after):
    """The paper's failing thread (Fig. 9) on the GPU: block 0 of the first persistent launch
    stops after `fail_after` sweeps and leaves the other blocks' stopping test.  The verifying
    synchronous update sees its stale rows, the solve resumes with every block, and the
    result still meets tol and the fixed-point bound -- in more sweeps than without the
    failure."""
    rp, ci = gg.rmat(14, seed=3)
    xstar, _, _ = oracle.fixed_point(rp, ci, d=D)
    with pr.Graph(rp, ci) as g:
        x0, info0 = g.solve(tol=1e-6, max_iter=500, variant="nonblocking")
        g.set_option(pr.PR_OPT_NB_FAIL_AFTER, fail_after)
        x, info = g.solve(tol=1e-6, max_iter=500, variant="nonblocking")
        g.set_option(pr.PR_OPT_NB_FAIL_AFTER, 0)
    assert info0.converged == 1 and info.converged == 1
    assert info.residual_l1 < 1e-6
    assert info.launches > info0.launches          # a second persistent launch
    assert info.iterations > info0.iterations
    assert l1(x, xstar) <= info.residual_l1 / (1 - D) + 2e-7
    assert max_rel(x, xstar) <= 1e-4


@pytest.mark.parametrize("build", ["rmat12", "rmat12_heavy64", "er", "cycle", "in_star"])
def test_edge_centric_variant_matches_jacobi_and_oracle(build):
    """Barriers-Edge (Alg. 2, PR_EDGE): the same synchronous iterates as the vertex form up to
    FP32 rounding -- against the oracle in matching mode, against PR_JACOBI, with a uniform
    and a personalised teleport, on the default layout and with heavy threshold 64."""
    heavy = pr.DEFAULT_HEAVY_DEGREE
    if build == "rmat12":
        rp, ci = gg.rmat(12, seed=4)
    elif build == "rmat12_heavy64":
        rp, ci = gg.rmat(12, seed=5)
        heavy = 64
    elif build == "er":
        rp, ci = gg.er_dangling(20001, seed=7)
    elif build == "cycle":
        rp, ci = gg.cycle(37)
    else:
        rp, ci = gg.in_star(3001)
    n = rp.size - 1
    t = (gg.uniform(8, 3, n) + 0.05).astype(np.float32)
    t /= t.sum()
    pr.set_heavy_degree(heavy)
    try:
        g = pr.Graph(rp, ci)
    finally:
        pr.set_heavy_degree(pr.DEFAULT_HEAVY_DEGREE)
    with g:
        for tt in (None, t):
            xj, ij = g.solve(tol=1e-6, max_iter=300, variant="jacobi", teleport=tt)
            xe, ie = g.solve(tol=1e-6, max_iter=300, variant="edge", teleport=tt)
            assert ie.converged == 1 and abs(ie.iterations - ij.iterations) <= 1, (ie.iterations, ij.iterations)
            assert max_rel(xe, xj) <= 1e-5
            xo = matching(rp, ci, xe, ie, t=None if tt is None else tt.astype(np.float64))
            assert l1(xe, xo) <= 1e-6 and max_rel(xe, xo) <= 1e-4
            assert ie.edge_visits == ie.iterations * ci.size


def test_edge_centric_variant_needs_32_bit_offsets():
    rp, ci = gg.rmat(10, seed=2)
    pr.pr_set_option(None, pr.PR_OPT_INDEX64, 1)
    try:
        g = pr.Graph(rp, ci)
    finally:
        pr.pr_set_option(None, pr.PR_OPT_INDEX64, 0)
    with g:
        with pytest.raises(pr.PageRankError) as e:
            g.solve(variant="edge")
        assert e.value.status == pr.PR_ERR_UNSUPPORTED
        x, info = g.solve(variant="jacobi")
        assert info.converged == 1


def test_nonblocking_budget_of_one_sweep_returns():
    rp, ci = gg.rmat(12, seed=5)
    with pr.Graph(rp, ci) as g:
        x = np.empty(rp.size - 1, np.float32)
        status, info = pr.pr_solve(g.handle, D, 1e-9, 1, pr.PR_NONBLOCKING, None, None, x)
    assert status == pr.PR_NOT_CONVERGED and info.converged == 0
    assert np.isfinite(info.residual_l1) and np.all(np.isfinite(x))


# ------------------------------------------------------------- boundary --

def test_invalid_graphs_are_rejected():
    ci = np.array([1, 0], np.int32)
    for rp, why in [(np.array([0, 2, 1], np.int64), "decreasing"),
                    (np.array([1, 1, 2], np.int64), "rowptr[0]"),
                    (np.array([0, 1, 2], np.int64), None)]:
        if why is None:
            bad = np.array([1, 5], np.int32)   # colidx out of range
            with pytest.raises(pr.PageRankError) as e:
                pr.Graph(rp, bad)
        else:
            with pytest.raises(pr.PageRankError) as e:
                pr.Graph(rp, ci)
        assert e.value.status == pr.PR_ERR_INVALID_GRAPH
    rp = np.array([0, 1, 3], np.int64)   # rowptr[n] != nnz
    with pytest.raises(pr.PageRankError) as e:
        pr.pr_create_graph(2, 2, rp, True, ci)
    assert e.value.status == pr.PR_ERR_INVALID_GRAPH


def test_invalid_solve_arguments():
    rp, ci = gg.cycle(8)
    with pr.Graph(rp, ci) as g:
        x = np.empty(8, np.float32)
        for damping, tol, it, var in [(1.0, 1e-6, 10, 0), (-0.1, 1e-6, 10, 0), (0.85, 0.0, 10, 0),
                                      (0.85, 1e-6, 0, 0), (0.85, 1e-6, 10, 7)]:
            with pytest.raises(pr.PageRankError) as e:
                pr.pr_solve(g.handle, damping, tol, it, var, None, None, x)
            assert e.value.status == pr.PR_ERR_INVALID_ARG
        status, info = pr.pr_solve(g.handle, 0.85, 1e-12, 1, pr.PR_JACOBI, None, None, x)
        assert info.iterations == 1 and np.isfinite(info.residual_l1)


def test_damping_zero_is_the_teleport():
    rp, ci = gg.rmat(10, seed=1)
    x, info, _ = solve(rp, ci, damping=0.0, tol=1e-9, max_iter=10)
    np.testing.assert_allclose(x, 1.0 / (rp.size - 1), rtol=1e-6)


# ------------------------------------------------------ light-tile modes --

@pytest.mark.parametrize("build", ["rmat14", "rmat12_heavy64_index64", "er"])
def test_staged_tiles_match_oracle(build):
    """Edge-parallel (staged) light tiles, both variants: the synchronous solve in matching
    mode and the barrier-free solve against the fixed point; the staged and row-by-row
    synchronous solves agree to FP32 summation-order rounding."""
    index64 = 0
    if build == "er":
        rp, ci = gg.er_dangling(40000, seed=11)
    elif build == "rmat14":
        rp, ci = gg.rmat(14, seed=6)
    else:
        rp, ci = gg.rmat(12, seed=7)
        pr.set_heavy_degree(64)
        index64 = 1
    pr.pr_set_option(None, pr.PR_OPT_INDEX64, index64)
    try:
        g = pr.Graph(rp, ci)
    finally:
        pr.pr_set_option(None, pr.PR_OPT_INDEX64, 0)
        pr.set_heavy_degree(pr.DEFAULT_HEAVY_DEGREE)
    xstar, _, _ = oracle.fixed_point(rp, ci, d=D)
    with g:
        g.set_option(pr.PR_OPT_STAGED_TILES, 0)
        x_rows, info_rows = g.solve(tol=1e-6, max_iter=200, variant="jacobi")
        g.set_option(pr.PR_OPT_STAGED_TILES, 3)
        x, info = g.solve(tol=1e-6, max_iter=200, variant="jacobi")
        assert info.converged == 1
        xo = matching(rp, ci, x, info)
        assert l1(x, xo) <= 1e-6 and max_rel(x, xo) <= 1e-4
        assert info.iterations == info_rows.iterations
        assert max_rel(x, x_rows) <= 1e-5
        xn, infon = g.solve(tol=1e-6, max_iter=500, variant="nonblocking")
        assert infon.converged == 1 and infon.residual_l1 < 1e-6
        assert l1(xn, xstar) <= infon.residual_l1 / (1 - D) + 2e-7
        assert max_rel(xn, xstar) <= 1e-4


@pytest.mark.parametrize("build", ["rmat14", "rmat12_heavy64", "rmat13_heavy2048", "er", "small"])
def test_pipelined_row_kernel_matches_row_kernel_and_oracle(build):
    """The pipelined synchronous row kernel (bulk asynchronous copies of each tile into
    shared memory, PR_OPT_TMA_TILES = 1, the default) against the row-by-row kernel (0)
    and the oracle: the solve in matching mode, one update with a personalised teleport,
    and the layouts at the edges of its stage sizes (heavy threshold 2048: single light
    rows of up to 2047 edges; graphs whose sizes are not multiples of 4)."""
    heavy = 1024
    if build == "rmat14":
        rp, ci = gg.rmat(14, seed=6)
    elif build == "rmat12_heavy64":
        rp, ci = gg.rmat(12, seed=7)
        heavy = 64
    elif build == "rmat13_heavy2048":
        rp, ci = gg.rmat(13, seed=9)
        heavy = 2048
    elif build == "er":
        rp, ci = gg.er_dangling(40001, seed=11)
    else:
        rp, ci = gg.rmat_n(4099, 8, seed=5)
    n = rp.size - 1
    pr.set_heavy_degree(heavy)
    try:
        g = pr.Graph(rp, ci)
    finally:
        pr.set_heavy_degree(pr.DEFAULT_HEAVY_DEGREE)
    t = (gg.uniform(3, 7, n) + 0.05).astype(np.float32)
    t /= t.sum()
    x_in = (gg.uniform(4, 7, n) + 0.1).astype(np.float32)
    x_in /= x_in.sum()
    with g:
        assert g.stats()["n_tma_tiles"] > 0
        res = {}
        for tma in (1, 0):
            g.set_option(pr.PR_OPT_TMA_TILES, tma)
            x, info = g.solve(tol=1e-6, max_iter=200, variant="jacobi")
            x1, info1 = g.iterate(x_in, n_iter=1, teleport=t)
            res[tma] = (x, info, x1, info1)
    x, info, x1, info1 = res[1]
    xr, infor, x1r, info1r = res[0]
    assert info.converged == 1 and info.iterations == infor.iterations
    assert max_rel(x, xr) <= 1e-5 and max_rel(x1, x1r) <= 1e-5
    xo = matching(rp, ci, x, info)
    assert l1(x, xo) <= 1e-6 and max_rel(x, xo) <= 1e-4
    xo1, _, l1o, _ = oracle.jacobi_step(rp, ci, x_in.astype(np.float64), d=D, t=t.astype(np.float64))
    assert l1(x1, xo1) <= 1e-6 and max_rel(x1, xo1) <= 1e-4
    assert info1.residual_l1 == pytest.approx(l1o, rel=1e-3, abs=1e-9)


@pytest.mark.parametrize("build", ["rmat15", "rmat13_heavy64", "rmat14_heavy2048", "rmat18"])
def test_fused_segments_match_the_separate_kernel_and_oracle(build):
    """Heavy-row segments as tiles of the pipelined kernel (PR_OPT_FUSED_SEGMENTS = 1),
    interleaved with the light tiles, the block that gathers a row's last segment updating
    the row: against the separate segment kernel (0, the default) and the oracle -- the
    solve in matching mode, one update with a personalised teleport, bitwise reproducible
    runs (the heavy rows' L1 change and dangling mass are added in row order).  The layouts
    cover heavy thresholds 64, 256 and 2048 and rows of up to about 20,000 in-edges."""
    heavy = 256
    if build == "rmat15":
        rp, ci = gg.rmat(15, seed=61)
    elif build == "rmat13_heavy64":
        rp, ci = gg.rmat(13, seed=62)
        heavy = 64
    elif build == "rmat14_heavy2048":
        rp, ci = gg.rmat(14, seed=63)
        heavy = 2048
    else:
        rp, ci = gg.rmat(18, seed=64)
    n = rp.size - 1
    pr.set_heavy_degree(heavy)
    try:
        g = pr.Graph(rp, ci)
    finally:
        pr.set_heavy_degree(pr.DEFAULT_HEAVY_DEGREE)
    t = (gg.uniform(5, 7, n) + 0.05).astype(np.float32)
    t /= t.sum()
    x_in = (gg.uniform(6, 7, n) + 0.1).astype(np.float32)
    x_in /= x_in.sum()
    with g:
        assert g.stats()["n_segments"] > 0 and g.stats()["n_tma_tiles"] > 0
        res = {}
        for fused in (1, 0):
            g.set_option(pr.PR_OPT_FUSED_SEGMENTS, fused)
            x, info = g.solve(tol=1e-6, max_iter=200, variant="jacobi")
            x1, info1 = g.iterate(x_in, n_iter=1, teleport=t)
            res[fused] = (x, info, x1, info1)
        g.set_option(pr.PR_OPT_FUSED_SEGMENTS, 1)
        x_again, _ = g.solve(tol=1e-6, max_iter=200, variant="jacobi")
        xb, infob = g.solve(tol=1e-6, max_iter=200, variant="nonblocking")   # its verifying update fused
    x, info, x1, info1 = res[1]
    xr, infor, x1r, info1r = res[0]
    assert np.array_equal(x, x_again)
    assert info.converged == 1 and abs(info.iterations - infor.iterations) <= 1
    assert max_rel(x, xr) <= 1e-5 and max_rel(x1, x1r) <= 1e-5
    xo = matching(rp, ci, x, info)
    assert l1(x, xo) <= 1e-6 and max_rel(x, xo) <= 1e-4
    xo1, d_in, l1o, _ = oracle.jacobi_step(rp, ci, x_in.astype(np.float64), d=D, t=t.astype(np.float64))
    assert l1(x1, xo1) <= 1e-6 and max_rel(x1, xo1) <= 1e-4
    assert info1.residual_l1 == pytest.approx(l1o, rel=1e-3, abs=1e-9)
    assert info1.dangling_mass == pytest.approx(oracle.dangling_mass(rp, ci, xo1), rel=1e-5, abs=1e-12)
    xs, _, _ = oracle.fixed_point(rp, ci, d=D)
    assert infob.converged == 1 and l1(xb, xs) <= infob.residual_l1 / (1 - D) + 2e-7


@pytest.mark.parametrize("build", ["rmat15", "er", "rmat12_heavy64"])
def test_light_lane_mappings_match_the_oracle(build):
    """Both lane mappings of the light-row tiles (PR_OPT_LIGHT_LANES: by degree class, or
    by the tile's row count with four edges per lane and row in flight), on the pipelined
    kernel, the row kernel and the barrier-free kernel: the synchronous solve in matching
    mode against the oracle, the barrier-free solve against the fixed point.  The mapping
    changes only the summation order."""
    heavy = 64 if build == "rmat12_heavy64" else 256
    if build == "rmat15":
        rp, ci = gg.rmat(15, seed=15)
    elif build == "er":
        rp, ci = gg.er_dangling(30011, seed=12)
    else:
        rp, ci = gg.rmat(12, seed=8)
    pr.set_heavy_degree(heavy)
    try:
        g = pr.Graph(rp, ci)
    finally:
        pr.set_heavy_degree(pr.DEFAULT_HEAVY_DEGREE)
    xstar, _, _ = oracle.fixed_point(rp, ci, d=D)
    with g:
        for mode in (0, 1):
            g.set_option(pr.PR_OPT_LIGHT_LANES, mode)
            for tma in (1, 0):
                g.set_option(pr.PR_OPT_TMA_TILES, tma)
                x, info = g.solve(tol=1e-6, max_iter=200, variant="jacobi")
                assert info.converged == 1
                xo = matching(rp, ci, x, info)
                assert l1(x, xo) <= 1e-6 and max_rel(x, xo) <= 1e-4, (mode, tma)
            g.set_option(pr.PR_OPT_TMA_TILES, 1)
            x, info = g.solve(tol=1e-6, max_iter=200, variant="nonblocking")
            assert info.converged == 1
            assert l1(x, xstar) <= info.residual_l1 / (1 - D) + 2e-7, mode
        with pytest.raises(pr.PageRankError):
            g.set_option(pr.PR_OPT_LIGHT_LANES, 2)


@pytest.mark.parametrize("batch", range(4))
def test_random_small_graphs_both_variants(batch):
    """Forty seeded random digraphs (1 to 600 vertices, 0 to 8 edges per vertex on average,
    duplicates and self-loops in half of them, so multiplicities and dangling vertices of
    every kind occur): the synchronous solve in matching mode and the barrier-free solve
    against the fixed point, on the default layout and with heavy threshold 64 (short
    rows gathered in segments)."""
    rng = np.random.default_rng(1000 + batch)
    for case in range(10):
        n = int(rng.integers(1, 601))
        m = int(rng.integers(0, 8 * n + 1))
        seed = 10000 * batch + case
        rp, ci = gg.random_digraph(n, m, seed=seed, allow_multi=case % 2 == 0, self_loops=case % 2 == 0)
        xstar, _, _ = oracle.fixed_point(rp, ci, d=D)
        heavy = 64 if case % 3 == 0 else pr.DEFAULT_HEAVY_DEGREE
        pr.set_heavy_degree(heavy)
        try:
            g = pr.Graph(rp, ci)
        finally:
            pr.set_heavy_degree(pr.DEFAULT_HEAVY_DEGREE)
        with g:
            x, info = g.solve(tol=1e-6, max_iter=300)
            xn, infon = g.solve(tol=1e-6, max_iter=500, variant="nonblocking")
        assert info.converged == 1 and infon.converged == 1, (n, m, seed)
        xo = matching(rp, ci, x, info)
        assert l1(x, xo) <= 1e-6 and max_rel(x, xo) <= 1e-4, (n, m, seed)
        assert l1(xn, xstar) <= infon.residual_l1 / (1 - D) + 2e-7, (n, m, seed)
        assert abs(float(np.sum(xn, dtype=np.float64)) - 1.0) < 1e-5


def test_pipelined_row_kernel_bounded_wait_reports_a_timeout():
    """Failure detection without a fault: the test hook makes block 0's producer announce a
    tile copy that never comes, so the gathering warps' mbarrier wait runs out after about
    a second; the solve returns PR_ERR_DEVICE_TIMEOUT, and the same graph (same context)
    then solves normally."""
    import time
    rp, ci = gg.rmat(16, seed=6)
    with pr.Graph(rp, ci) as g:
        st = g.stats()
        # one block per SM, so that block 0 owns at least three tiles (the hook counts them)
        assert st["n_tma_tiles"] > 2 * st["sm_count"]
        g.set_option(pr.PR_OPT_CTAS_PER_SM, 1)
        for k in (1, 2, 3):
            g.set_option(pr.PR_OPT_TEST_WITHHOLD_COPY, k)
            t0 = time.perf_counter()
            with pytest.raises(pr.PageRankError) as e:
                g.solve(tol=1e-6, max_iter=50)
            assert e.value.status == pr.PR_ERR_DEVICE_TIMEOUT
            assert time.perf_counter() - t0 < 30
        g.set_option(pr.PR_OPT_TEST_WITHHOLD_COPY, 0)
        g.set_option(pr.PR_OPT_CTAS_PER_SM, 0)
        x, info = g.solve(tol=1e-6, max_iter=200)
    assert info.converged == 1
    xo = matching(rp, ci, x, info)
    assert l1(x, xo) <= 1e-6 and max_rel(x, xo) <= 1e-4


def test_pipelined_row_kernel_not_used_where_it_cannot_apply():
    """Heavy threshold 4096 (light rows longer than a stage) and 64-bit offsets: no
    pipelined tiles; the solve still matches the oracle."""
    rp, ci = gg.rmat(12, seed=3)
    for heavy, idx64 in ((4096, 0), (1024, 1)):
        pr.set_heavy_degree(heavy)
        pr.pr_set_option(None, pr.PR_OPT_INDEX64, idx64)
        try:
            g = pr.Graph(rp, ci)
        finally:
            pr.set_heavy_degree(pr.DEFAULT_HEAVY_DEGREE)
            pr.pr_set_option(None, pr.PR_OPT_INDEX64, 0)
        with g:
            assert g.stats()["n_tma_tiles"] == 0
            x, info = g.solve(tol=1e-6, max_iter=200)
        xo = matching(rp, ci, x, info)
        assert l1(x, xo) <= 1e-6 and max_rel(x, xo) <= 1e-4


@pytest.mark.parametrize("hubs", [0, 4, 1000, 8192])
def test_nonblocking_hub_snapshot_sizes(hubs):
    """The barrier-free kernel with no hub snapshot, a tiny one, one that is not a
    multiple of 4 (rounded down) and the largest: the fixed point is reached."""
    rp, ci = gg.rmat(14, seed=8)
    xstar, _, _ = oracle.fixed_point(rp, ci, d=D)
    with pr.Graph(rp, ci) as g:
        g.set_option(pr.PR_OPT_NB_HUBS, hubs)
        x, info = g.solve(tol=1e-6, max_iter=500, variant="nonblocking")
    assert info.converged == 1 and info.residual_l1 < 1e-6
    assert l1(x, xstar) <= info.residual_l1 / (1 - D) + 2e-7
    assert max_rel(x, xstar) <= 1e-4


@pytest.mark.parametrize("l1_hubs", [0, 64, 49152, 1 << 30])
def test_nonblocking_l1_hub_gathers(l1_hubs):
    """Barrier-free kernel with no weak hub gathers (every gather a relaxed load), a few,
    the default and all vertices: each run reaches the fixed point."""
    rp, ci = gg.rmat(14, seed=12)
    xstar, _, _ = oracle.fixed_point(rp, ci, d=D)
    with pr.Graph(rp, ci) as g:
        g.set_option(pr.PR_OPT_NB_L1_HUBS, l1_hubs)
        x, info = g.solve(tol=1e-6, max_iter=500, variant="nonblocking")
    assert info.converged == 1 and info.residual_l1 < 1e-6
    assert l1(x, xstar) <= info.residual_l1 / (1 - D) + 2e-7
    assert max_rel(x, xstar) <= 1e-4


# ------------------------------------------------------- loop perforation --

@pytest.mark.parametrize("heavy", [1024, 64])
def test_loop_perforation(heavy):
    """Alg. 5 in the synchronous solver.  A bound no FP32 change goes below freezes nothing,
    so the solve is the plain one, bit for bit; with eps = 1e-11 rows freeze, the solve
    needs no more iterations, and its distance to the fixed point is of the size the FP64
    oracle's own perforated run reaches (within 5x, plus the FP32 rounding)."""
    rp, ci = gg.rmat(14, seed=21)
    pr.set_heavy_degree(heavy)
    try:
        g = pr.Graph(rp, ci)
    finally:
        pr.set_heavy_degree(pr.DEFAULT_HEAVY_DEGREE)
    xstar, _, _ = oracle.fixed_point(rp, ci, d=D)
    with g:
        # the perforated solve runs on the row kernel: compare with the same kernel
        g.set_option(pr.PR_OPT_TMA_TILES, 0)
        x0, info0 = g.solve(tol=1e-7, max_iter=300)
        g.set_option(pr.PR_OPT_PERFORATION, 30)
        x1, info1 = g.solve(tol=1e-7, max_iter=300)
        assert np.array_equal(x0, x1) and info1.iterations == info0.iterations
        g.set_option(pr.PR_OPT_PERFORATION, 11)
        x2, info2 = g.solve(tol=1e-7, max_iter=300)
        g.set_option(pr.PR_OPT_PERFORATION, 0)
        x3, info3 = g.solve(tol=1e-7, max_iter=300)
    assert np.array_equal(x0, x3)                      # off again: the plain solve
    assert info1.frozen_rows == 0 and info0.frozen_rows == 0
    assert info2.converged == 1 and info2.iterations <= info0.iterations
    assert info2.frozen_rows > 0
    xo, _, _, nf = oracle.pagerank_perforated(rp, ci, d=D, tol=1e-7, max_iter=300, eps=1e-11)
    assert nf > 0
    err_gpu = l1(x2, xstar)
    err_oracle = l1(xo, xstar)
    assert err_gpu <= 5 * err_oracle + info2.residual_l1 / (1 - D) + 2e-7, (err_gpu, err_oracle)


@pytest.mark.parametrize("graph", ["rmat14", "er14"])
def test_nosync_opt_perforated_barrier_free(graph):
    """Alg. 5 applied to the barrier-free solver (the paper's No-Sync-Opt).  A bound no FP32
    change goes below freezes nothing: the solve is the plain barrier-free one, certified
    like it.  With eps = 1e-9 rows freeze (reported in frozen_rows), the verifying
    synchronous update certifies the perforated vector, and its distance to the fixed
    point is of the scale a frozen row can contribute, (frozen rows * eps + residual) /
    (1 - d): each row froze on a change below eps, and the map contracts by d.  Which
    rows freeze, and when, depends on the update order: the FP64 oracle's perforated
    No-Sync runs (1 to 1024 simulated threads) reach at most 0.16 of that scale (its own
    pin), the GPU's thousands of warps updating in place about 1.0 of it (measured
    0.85-1.03 on R-MAT-14), so the test allows twice the scale."""
    rp, ci = gg.rmat(14, seed=21) if graph == "rmat14" else gg.er_dangling(1 << 14, seed=5)
    xstar, _, _ = oracle.fixed_point(rp, ci, d=D)
    with pr.Graph(rp, ci) as g:
        x0, info0 = g.solve(tol=1e-6, max_iter=300, variant="nonblocking")
        g.set_option(pr.PR_OPT_PERFORATION, 30)
        x1, info1 = g.solve(tol=1e-6, max_iter=300, variant="nonblocking")
        g.set_option(pr.PR_OPT_PERFORATION, 9)
        x2, info2 = g.solve(tol=1e-6, max_iter=300, variant="nonblocking")
        g.set_option(pr.PR_OPT_PERFORATION, 0)
        x3, info3 = g.solve(tol=1e-6, max_iter=300, variant="nonblocking")
    for x, info in ((x0, info0), (x1, info1), (x3, info3)):
        assert info.converged == 1 and info.frozen_rows == 0
        assert l1(x, xstar) <= info.residual_l1 / (1 - D) + 2e-7
    assert info2.converged == 1 and info2.frozen_rows > 0
    err_gpu = l1(x2, xstar)
    scale = (info2.frozen_rows * 1e-9 + info2.residual_l1) / (1 - D)
    assert err_gpu <= 2 * scale + 2e-7, (err_gpu, scale)
    # the freezes moved the result: the perforated vector is no longer the plain one's
    assert l1(x2, x0) > 0
    assert abs(float(np.sum(x2, dtype=np.float64)) - 1.0) < 1e-5


def test_nosync_opt_rejects_the_diagnostics_form():
    rp, ci = gg.rmat(10, seed=3)
    with pr.Graph(rp, ci) as g:
        g.set_option(pr.PR_OPT_PERFORATION, 9)
        g.set_option(pr.PR_OPT_NB_FAIL_AFTER, 2)
        with pytest.raises(pr.PageRankError) as e:
            g.solve(tol=1e-6, variant="nonblocking")
        assert e.value.status == pr.PR_ERR_UNSUPPORTED


# ------------------------------------------------ helping and slow blocks --

def test_dynamic_tiles_take_over_a_slow_block():
    """Barrier-Helper's GPU form: with block 0 slowed (a bounded sleep before it takes each
    tile), dynamic tile assignment lets the other blocks take its share, so the solve is
    faster than with the static assignment.  A delay changes no arithmetic: the static run
    is bit for bit the undelayed one; the dynamic run differs only in the order of the
    per-block partial sums (last-bit changes of D and r)."""
    rp, ci = gg.rmat(20, seed=23)     # several tiles per block
    with pr.Graph(rp, ci) as g:
        assert g.stats()["n_tiles"] > 3 * 608
        # the reference is the row kernel the delayed runs use (the pipelined kernel's
        # smaller tiles give its light rows other lane groups: other rounding)
        g.set_option(pr.PR_OPT_TMA_TILES, 0)
        x_ref, info_ref = g.solve(tol=1e-6, max_iter=200)
        g.set_option(pr.PR_OPT_DELAY_NS, 100000)
        times, xs = {}, {}
        for dyn in (0, 1):
            g.set_option(pr.PR_OPT_DYNAMIC_TILES, dyn)
            best = None
            for _ in range(2):
                x, info = g.solve(tol=1e-6, max_iter=200)
                best = info.ms_loop if best is None else min(best, info.ms_loop)
            assert info.converged == 1
            times[dyn], xs[dyn] = best, x
    assert np.array_equal(xs[0], x_ref)
    assert max_rel(xs[1], x_ref) <= 1e-5
    assert times[1] < 0.7 * times[0], times


# ------------------------------------------------------ out-edge CSR input --

def out_csr(rp, ci, n):
    """The out-edge CSR (row u lists the targets of u's edges) of an in-edge CSR."""
    dst = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    return gg.edges_to_in_csr(n, dst, ci.astype(np.int64), dedup=False, drop_self_loops=False)


@pytest.mark.parametrize("build", ["rmat13", "er", "multi", "small", "index64"])
def test_out_csr_layout_is_transposed_on_the_device(build):
    """PR_OUT_CSR: the library sorts the edges by target on the device (stable, so every
    in-row lists its sources in increasing order).  The in-edge CSR built from it is the
    one the caller would have given, so both solves agree bit for bit, and the result
    matches the oracle run on the in-edge CSR."""
    index64 = 0
    if build == "rmat13":
        rp, ci = gg.rmat(13, seed=44)
    elif build == "er":
        rp, ci = gg.er_dangling(20011, seed=45)
    elif build == "multi":
        rp, ci = gg.random_digraph(700, 5000, seed=46, allow_multi=True, self_loops=True)
    elif build == "small":
        rp, ci = gg.random_digraph(3, 4, seed=47, allow_multi=True, self_loops=True)
    else:
        rp, ci = gg.rmat(12, seed=48)
        index64 = 1
    n = rp.size - 1
    orp, oci = out_csr(rp, ci, n)
    assert orp[-1] == ci.size
    pr.pr_set_option(None, pr.PR_OPT_INDEX64, index64)
    try:
        g_in = pr.Graph(rp, ci)
        g_out = pr.Graph(orp, oci, layout=pr.PR_OUT_CSR)
    finally:
        pr.pr_set_option(None, pr.PR_OPT_INDEX64, 0)
    with g_in, g_out:
        assert g_out.stats()["nnz"] == ci.size and g_out.stats()["max_indeg"] == g_in.stats()["max_indeg"]
        for variant in ("jacobi", "nonblocking"):
            x_in, info_in = g_in.solve(tol=1e-6, variant=variant)
            x_out, info_out = g_out.solve(tol=1e-6, variant=variant)
            if variant == "jacobi":
                assert np.array_equal(x_in, x_out)
                xo = matching(rp, ci, x_out, info_out)
                assert l1(x_out, xo) <= 1e-6 and max_rel(x_out, xo) <= 1e-4
            else:
                xs, _, _ = oracle.fixed_point(rp, ci, d=D)
                assert l1(x_out, xs) <= info_out.residual_l1 / (1 - D) + 2e-7


def test_out_csr_validation_and_weights():
    rp, ci = gg.rmat(8, seed=2)
    n = rp.size - 1
    orp, oci = out_csr(rp, ci, n)
    bad = oci.copy()
    bad[5] = n                                        # a target out of range
    with pytest.raises(pr.PageRankError) as e:
        pr.Graph(orp, bad, layout=pr.PR_OUT_CSR)
    assert e.value.status == pr.PR_ERR_INVALID_GRAPH
    with pytest.raises(pr.PageRankError) as e:
        pr.pr_create_graph(n, ci.size, rp, 1, ci, weights=np.ones(ci.size, np.float32))
    assert e.value.status == pr.PR_ERR_UNSUPPORTED
    assert "pr_create_wgraph" in str(e.value)


@pytest.mark.parametrize("build", ["rmat12", "er_isolated", "all_isolated", "rmat14_heavy64"])
def test_implicit_zero_rows_in_the_synchronous_iteration(build):
    """PR_OPT_IMPLICIT_ZERO_ROWS in the pipelined row kernel: after the first update the
    ranks of rows without in-edges are (1-d) t_v + d D/n (Eq. 1 with nothing gathered), so
    the tiles of isolated vertices are skipped, the other such rows store their quotient
    only, and the ranks are written after the loop.  Against the full update (option 0)
    and the oracle: the converged solve in matching mode, a personalised teleport, and
    exactly 1, 2 and 5 updates from a given vector (pr_iterate), whose last L1 change
    includes the analytic part."""
    heavy = 64 if build == "rmat14_heavy64" else 256
    if build == "rmat12":
        rp, ci = gg.rmat(12, seed=31)
    elif build == "rmat14_heavy64":
        rp, ci = gg.rmat(14, seed=32)
    elif build == "er_isolated":
        # ER on the first 3000 vertices, 2001 isolated vertices after them
        rp0, ci0 = gg.er_dangling(3000, 6.0, 0.2, seed=33)
        rp = np.concatenate([rp0, np.full(2001, rp0[-1], rp0.dtype)])
        ci = ci0
    else:
        rp, ci = np.zeros(1001, np.int64), np.zeros(0, np.int32)
    n = rp.size - 1
    iso = int(((np.diff(rp) == 0) & (np.bincount(ci, minlength=n) == 0)).sum())
    t = (gg.uniform(5, 9, n) + 0.05).astype(np.float32)
    t /= t.sum()
    x_in = (gg.uniform(6, 9, n) + 0.1).astype(np.float32)
    x_in /= x_in.sum()
    pr.set_heavy_degree(heavy)
    try:
        g = pr.Graph(rp, ci)
    finally:
        pr.set_heavy_degree(pr.DEFAULT_HEAVY_DEGREE)
    with g:
        assert g.stats()["n_isolated"] == iso and g.stats()["n_tma_tiles"] > 0
        res = {}
        for imp in (1, 0):
            g.set_option(pr.PR_OPT_IMPLICIT_ZERO_ROWS, imp)
            r = [g.solve(tol=1e-6, max_iter=200), g.solve(tol=1e-6, max_iter=200, teleport=t)]
            for k in (1, 2, 5):
                r.append(g.iterate(x_in, n_iter=k, teleport=t))
            res[imp] = r
        g.set_option(pr.PR_OPT_IMPLICIT_ZERO_ROWS, 1)
    for (x1, i1), (x0, i0) in zip(res[1], res[0]):
        assert abs(i1.iterations - i0.iterations) <= 1
        assert max_rel(x1, x0) <= 1e-5
        # near convergence the L1 change is a few FP32 units of each rank, which the
        # analytic change of the implicit rows (exact, not rounded to FP32) does not
        # reproduce: there the two agree to a tenth of the tolerance 1e-6
        assert i1.residual_l1 == pytest.approx(i0.residual_l1, rel=1e-4, abs=1e-7)
        assert i1.dangling_mass == pytest.approx(i0.dangling_mass, rel=1e-6, abs=1e-12)
    (x, info), (xt, infot) = res[1][0], res[1][1]
    assert info.converged == 1 and infot.converged == 1
    xo = matching(rp, ci, x, info)
    assert l1(x, xo) <= 1e-6 and max_rel(x, xo) <= 1e-4
    xo = matching(rp, ci, xt, infot, t=t.astype(np.float64))
    assert l1(xt, xo) <= 1e-6 and max_rel(xt, xo) <= 1e-4
    for (xk, ik), k in zip(res[1][2:], (1, 2, 5)):
        xo, _, _ = oracle.pagerank_jacobi(rp, ci, d=D, tol=0, max_iter=k, t=t.astype(np.float64),
                                          x0=x_in.astype(np.float64))
        assert l1(xk, xo) <= 1e-6 and max_rel(xk, xo) <= 1e-4, k
        xp, _, _ = oracle.pagerank_jacobi(rp, ci, d=D, tol=0, max_iter=k - 1, t=t.astype(np.float64),
                                          x0=x_in.astype(np.float64)) if k > 1 else (x_in, 0, 0)
        assert ik.residual_l1 == pytest.approx(l1(xo, xp), rel=1e-3, abs=1e-7), k
    if build == "all_isolated":
        np.testing.assert_allclose(x, 1.0 / n, rtol=1e-6)
        assert info.iterations == 1


@pytest.mark.parametrize("build,sweeps", [("rmat14", 4), ("rmat13_heavy64", 2), ("er", 4), ("er", 1),
                                          ("rmat12_idx64", 3)])
def test_sync_bf16_defect_correction_reaches_the_fixed_point(build, sweeps):
    """PR_OPT_SYNC_DC: BF16 storage of the quotient vector in the synchronous solver by
    defect correction.  Each FP32 step x' = F(x) (Eq. 1) is followed by `sweeps` sweeps
    delta <- r + d (P^T delta + L/n) gathering BF16 quotients (heavy rows through the
    segment kernel), then x <- x + delta.  The stopping test is the FP32 step's L1 change,
    so the result is an FP32 iterate: against the FP64 fixed point it is within the L1 bound
    r/(1-d) its residual gives, one oracle update of it changes it by less than 2e-6, and it
    takes fewer FP32 steps than the plain solve, for the uniform and a personalised
    teleport."""
    heavy, idx64 = 256, 0
    if build == "rmat14":
        rp, ci = gg.rmat(14, seed=41)
    elif build == "rmat13_heavy64":
        rp, ci = gg.rmat(13, seed=42)
        heavy = 64
    elif build == "rmat12_idx64":
        rp, ci = gg.rmat(12, seed=43)
        idx64 = 1
    else:
        rp, ci = gg.er_dangling(30011, 8.0, 0.2, seed=44)
    n = rp.size - 1
    t = (gg.uniform(8, 3, n) + 0.05).astype(np.float32)
    t /= t.sum()
    pr.set_heavy_degree(heavy)
    pr.pr_set_option(None, pr.PR_OPT_INDEX64, idx64)
    try:
        g = pr.Graph(rp, ci)
    finally:
        pr.set_heavy_degree(pr.DEFAULT_HEAVY_DEGREE)
        pr.pr_set_option(None, pr.PR_OPT_INDEX64, 0)
    with g:
        plain = [g.solve(tol=1e-6, max_iter=200), g.solve(tol=1e-6, max_iter=200, teleport=t)]
        g.set_option(pr.PR_OPT_SYNC_DC, sweeps)
        dcs = [g.solve(tol=1e-6, max_iter=200), g.solve(tol=1e-6, max_iter=200, teleport=t)]
        g.set_option(pr.PR_OPT_SYNC_DC, 0)
        again, _ = g.solve(tol=1e-6, max_iter=200)
    assert np.array_equal(again, plain[0][0])            # off again: the plain solve
    for (x, info), (xp, infop), tt in zip(dcs, plain, (None, t)):
        t64 = None if tt is None else tt.astype(np.float64)
        assert info.converged == 1 and info.residual_l1 < 1e-6
        assert info.iterations < infop.iterations
        assert info.edge_visits == (info.iterations + sweeps * (info.iterations - 1)) * ci.size
        assert x.astype(np.float64).sum() == pytest.approx(1.0, abs=1e-6)
        xstar, _, _ = oracle.fixed_point(rp, ci, d=D, t=t64)
        assert l1(x, xstar) <= info.residual_l1 / (1 - D) + 2e-7
        _, _, r_or, _ = oracle.jacobi_step(rp, ci, x.astype(np.float64), d=D, t=t64)
        assert r_or < 2e-6


@pytest.mark.parametrize("build", ["er_isolated", "rmat13", "all_isolated"])
def test_nonblocking_leaves_isolated_vertices_to_the_end(build):
    """The barrier-free kernel does not sweep isolated vertices (no in- and no out-edges):
    with the complement form of the dangling share their ranks enter no other row's update,
    so they are written once from the final mass of the other vertices, before the
    verifying synchronous update.  The solve still reaches the FP64 fixed point within the
    bound its certified residual gives, for the uniform and a personalised teleport (seeds
    on isolated vertices included)."""
    if build == "er_isolated":
        rp0, ci0 = gg.er_dangling(3000, 6.0, 0.2, seed=51)
        rp = np.concatenate([rp0, np.full(2001, rp0[-1], rp0.dtype)])
        ci = ci0
    elif build == "rmat13":
        rp, ci = gg.rmat(13, seed=52)
    else:
        rp, ci = np.zeros(1001, np.int64), np.zeros(0, np.int32)
    n = rp.size - 1
    iso = np.flatnonzero((np.diff(rp) == 0) & (np.bincount(ci, minlength=n) == 0))
    assert iso.size > 0
    t = (gg.uniform(9, 4, n) + 0.05).astype(np.float32)
    t[iso[: max(1, iso.size // 10)]] += 1.0          # heavier teleport on some isolated vertices
    t /= t.sum()
    with pr.Graph(rp, ci) as g:
        assert g.stats()["n_isolated"] == iso.size
        for tt in (None, t):
            x, info = g.solve(tol=1e-6, max_iter=200, variant="nonblocking", teleport=tt)
            assert info.converged == 1 and info.residual_l1 < 1e-6
            t64 = None if tt is None else tt.astype(np.float64)
            xstar, _, _ = oracle.fixed_point(rp, ci, d=D, t=t64)
            assert l1(x, xstar) <= info.residual_l1 / (1 - D) + 2e-7
            _, _, r_or, _ = oracle.jacobi_step(rp, ci, x.astype(np.float64), d=D, t=t64)
            assert r_or < 2e-6


@pytest.mark.parametrize("build", ["rmat14", "er", "rmat13_teleport"])
def test_pipelined_nonblocking_reaches_the_fixed_point(build):
    """PR_OPT_NB_PIPELINE: the barrier-free sweeps with the light-row tiles' offsets,
    column indices, 1/outdeg and teleport staged in shared memory by a producer warp (bulk
    asynchronous copies) reach the FP64 fixed point within the bound of their certified
    residual, as the default form does."""
    if build == "rmat14":
        rp, ci = gg.rmat(14, seed=61)
    elif build == "er":
        rp, ci = gg.er_dangling(40000, 8.0, 0.2, seed=62)
    else:
        rp, ci = gg.rmat(13, seed=63)
    n = rp.size - 1
    t = None
    if build == "rmat13_teleport":
        t = (gg.uniform(11, 5, n) + 0.05).astype(np.float32)
        t /= t.sum()
    with pr.Graph(rp, ci) as g:
        g.set_option(pr.PR_OPT_NB_PIPELINE, 1)
        x, info = g.solve(tol=1e-6, max_iter=200, variant="nonblocking", teleport=t)
        g.set_option(pr.PR_OPT_NB_PIPELINE, 0)
    assert info.converged == 1 and info.residual_l1 < 1e-6
    t64 = None if t is None else t.astype(np.float64)
    xstar, _, _ = oracle.fixed_point(rp, ci, d=D, t=t64)
    assert l1(x, xstar) <= info.residual_l1 / (1 - D) + 2e-7
