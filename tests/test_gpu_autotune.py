"""The option autotuner: it times every candidate on the caller's graph and returns the
fastest; a graph built with its choice still solves to the oracle's fixed point."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pr = pytest.importorskip("paper_2109_09527_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    yield


def test_tune_picks_a_timed_candidate_and_the_tuned_graph_is_correct():
    from paper_2109_09527_gb300 import autotune
    rp, ci = gg.rmat(15, 16, seed=15)
    res = autotune.tune(rp, ci, iterations=4, heavy=(256, 1024), hot=(16384, 49152), ctas=(0, 2),
                        tma_hot=(4096, 16384))
    trials = res["trials"]
    assert len(trials) == 2 + 2 + 2 + 2
    assert all(t["ms"] > 0 for t in trials)
    assert res["ms_per_iteration"] == min(t["ms"] for t in trials)
    assert res["heavy_degree"] in (256, 1024) and res["hot_vertices"] in (16384, 49152)
    assert res["tma_hot_vertices"] in (4096, 16384)
    xstar, _, _ = oracle.fixed_point(rp, ci, d=0.85)
    with autotune.build_tuned(rp, ci, res) as g:
        x, info = g.solve(tol=1e-6)
        assert g.stats()["n_heavy"] >= 0
    assert info.converged == 1
    assert float(np.abs(x.astype(np.float64) - xstar).sum()) <= info.residual_l1 / 0.15 + 2e-7


def test_tune_batched_picks_a_timed_threshold_and_solves_correctly():
    from paper_2109_09527_gb300 import autotune
    rp, ci = gg.rmat(13, 16, seed=13)
    n = rp.size - 1
    t = gg.seed_teleports(n, 8, 8, seed=13)
    res = autotune.tune_batched(rp, ci, t, 8, heavy=(64, 256, 1024))
    assert [tr["heavy_degree"] for tr in res["trials"]] == [64, 256, 1024]
    assert all(tr["ms"] > 0 for tr in res["trials"])
    assert res["ms_per_solve"] == min(tr["ms"] for tr in res["trials"])
    pr.set_heavy_degree(res["heavy_degree"])
    try:
        g = pr.Graph(rp, ci)
    finally:
        pr.set_heavy_degree(pr.DEFAULT_HEAVY_DEGREE)
    with g:
        xb, info, res_cols, its = g.solve_batched(8, t, tol=1e-6)
    assert info.converged == 1
    for j in range(8):
        xj, _, _ = oracle.fixed_point(rp, ci, d=0.85, t=t[:, j].astype(np.float64))
        assert float(np.abs(xb[:, j] - xj).sum()) <= res_cols[j] / 0.15 + 2e-7, j
