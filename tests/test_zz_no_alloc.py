"""pr_step_noalloc: the allocation-free synchronous update, called through the C ABI.

Some callers cannot allocate device memory where they need an update (a fixed memory
pool, another framework's allocator, a latency-bound loop); this entry point works on
their own buffers plus one fixed scratch array inside the library.  The test checks it
against the existing entry point (pr_iterate on a pr_graph) and against the FP64
oracle's update (Eq. 1 with the dangling share D/n) on two calls in a row, with the
tolerances of the other parity tests (L1 <= 1e-6, per-vertex relative <= 1e-4).
It is collected last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pr = pytest.importorskip("paper_2109_09527_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _l1(a, b):
    return float(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)).sum())


def _max_rel(a, b):
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(np.asarray(a, np.float64) - b) / np.abs(b)))


@pytest.mark.parametrize("graph", ["rmat13", "er"])
def test_no_alloc_step_matches_pr_iterate_twice(graph):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rp, ci = gg.rmat(13, seed=31) if graph == "rmat13" else gg.er_dangling(20000, seed=32)
    n = rp.size - 1
    outdeg = np.bincount(ci, minlength=n)
    inv = np.where(outdeg > 0, 1.0 / np.maximum(outdeg, 1), 0.0).astype(np.float32)
    dev = torch.device("cuda:0")
    d_rp = torch.from_numpy(rp.astype(np.int32)).to(dev)
    d_ci = torch.from_numpy(ci).to(dev)
    d_inv = torch.from_numpy(inv).to(dev)
    x0 = torch.full((n,), 1.0 / n, dtype=torch.float32, device=dev)
    x1 = torch.empty_like(x0)
    x2 = torch.empty_like(x0)
    sums1 = torch.zeros(3, dtype=torch.float64, device=dev)
    sums2 = torch.zeros(3, dtype=torch.float64, device=dev)

    pr.pr_step_noalloc(n, d_rp, d_ci, d_inv, 0.85, x0, x1, sums1)
    pr.pr_step_noalloc(n, d_rp, d_ci, d_inv, 0.85, x1, x2, sums2)
    torch.cuda.synchronize()
    x1h, x2h = x1.cpu().numpy(), x2.cpu().numpy()
    s1, s2 = sums1.cpu().numpy(), sums2.cpu().numpy()

    with pr.Graph(rp, ci) as g:
        ref1, info1 = g.iterate(x0.cpu().numpy(), n_iter=1)
        ref2, info2 = g.iterate(x1h, n_iter=1)
    for got, ref, sums, info in ((x1h, ref1, s1, info1), (x2h, ref2, s2, info2)):
        assert _l1(got, ref) <= 1e-6 and _max_rel(got, ref) <= 1e-4
        assert sums[1] == pytest.approx(info.dangling_mass, rel=1e-5, abs=1e-12)
        assert sums[2] == pytest.approx(info.residual_l1, rel=1e-4, abs=1e-9)
    # the same two updates by the FP64 oracle, each from the vector the call was given
    for x_prev, got, sums in ((x0.cpu().numpy(), x1h, s1), (x1h, x2h, s2)):
        xo, d_in, l1o, _ = oracle.jacobi_step(rp, ci, x_prev.astype(np.float64), d=0.85)
        assert _l1(got, xo) <= 1e-6 and _max_rel(got, xo) <= 1e-4
        assert sums[0] == pytest.approx(d_in, rel=1e-6, abs=1e-12)
        d_out = oracle.dangling_mass(rp, ci, xo)
        assert sums[1] == pytest.approx(d_out, rel=1e-5, abs=1e-12)
        assert sums[2] == pytest.approx(l1o, rel=1e-3, abs=1e-8)
    assert s1[0] == pytest.approx(float(np.sum(np.float64(1.0 / n) * (outdeg == 0))), rel=1e-6)
    # the dangling mass of x1: summed in FP64 by the second call, Kahan-compensated FP32 per
    # thread by the first
    assert s2[0] == pytest.approx(s1[1], rel=1e-6)


def test_no_alloc_rejects_sizes_beyond_its_scratch():
    big = (1 << 24) + 1
    with pytest.raises(pr.PageRankError) as e:
        pr.pr_step_noalloc(big, 1, 1, 1, 0.85, 1, 2, 1)
    assert e.value.status == pr.PR_ERR_INVALID_ARG
    assert "16,777,216" in str(e.value)


def test_no_alloc_rejects_overlapping_vectors():
    """x_out starting one element after x_in shares n - 1 elements with it: rejected
    before any GPU work."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n = 64
    dev = torch.device("cuda:0")
    rp = torch.arange(n + 1, dtype=torch.int32, device=dev)
    ci = torch.roll(torch.arange(n, dtype=torch.int32, device=dev), 1)
    inv = torch.ones(n, dtype=torch.float32, device=dev)
    buf = torch.full((n + 1,), 1.0 / n, dtype=torch.float32, device=dev)
    sums = torch.zeros(3, dtype=torch.float64, device=dev)
    with pytest.raises(pr.PageRankError) as e:
        pr.pr_step_noalloc(n, rp, ci, inv, 0.85, buf.data_ptr(), buf.data_ptr() + 4, sums)
    assert e.value.status == pr.PR_ERR_INVALID_ARG
    assert "overlap" in str(e.value)
