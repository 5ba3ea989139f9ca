"""The seeded input generators: canonical CSR, determinism, workload shape."""
import numpy as np
import pytest

import graphgen as gg


def _canonical(rowptr, colidx, n):
    assert rowptr.dtype == np.int64 and colidx.dtype == np.int32
    assert rowptr.shape == (n + 1,) and rowptr[0] == 0 and rowptr[-1] == colidx.size
    assert np.all(np.diff(rowptr) >= 0)
    assert colidx.size == 0 or (colidx.min() >= 0 and colidx.max() < n)
    src, dst = gg.in_csr_edges(rowptr, colidx)
    assert not np.any(src == dst), "self-loop survived"
    key = dst * n + src
    assert np.all(np.diff(key) > 0), "rows not sorted or duplicate edge"


@pytest.mark.parametrize("scale", [4, 8, 12])
def test_rmat_canonical_and_thread_independent(scale):
    a = gg.rmat(scale, seed=11, nthreads=1)
    b = gg.rmat(scale, seed=11, nthreads=4)
    _canonical(*a, 1 << scale)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    c = gg.rmat(scale, seed=12)
    assert not np.array_equal(a[1], c[1])


def test_rmat_shape_of_workload():
    n = 1 << 14
    rowptr, colidx = gg.rmat(14, seed=1)
    nnz = colidx.size
    # 16 * 2^14 drawn edges; self-loops and duplicates remove a minority
    assert 0.6 * 16 * n < nnz < 16 * n
    indeg = np.diff(rowptr)
    outdeg = np.bincount(colidx, minlength=n)
    # power law: heavy hubs, many isolated vertices, a max far above the mean
    assert indeg.max() > 50 * indeg.mean() and outdeg.max() > 50 * outdeg.mean()
    assert 0.2 < np.mean(outdeg == 0) < 0.6
    # b = c: in- and out-degree sequences have the same scale
    assert 0.5 < indeg.max() / outdeg.max() < 2.0


def test_rmat_unpermuted_hub_is_vertex_zero():
    rowptr, colidx = gg.rmat(10, seed=3, permute=False)
    indeg = np.diff(rowptr)
    outdeg = np.bincount(colidx, minlength=1 << 10)
    assert indeg.argmax() == 0 and outdeg.argmax() == 0


def test_er_dangling_fraction_and_mean_degree():
    n = 50000
    rowptr, colidx = gg.er_dangling(n, mean_deg=16, frac_dangling=0.2, seed=5)
    _canonical(rowptr, colidx, n)
    outdeg = np.bincount(colidx, minlength=n)
    assert abs(np.mean(outdeg == 0) - 0.2) < 1e-3
    assert abs(colidx.size / n - 16.0) < 0.2
    nz = outdeg[outdeg > 0]
    assert abs(nz.mean() - 20.0) < 0.2 and abs(nz.var() - 20.0) < 1.5  # Poisson(20)
    b = gg.er_dangling(n, seed=5, nthreads=1)
    assert np.array_equal(b[1], colidx)


def test_fixtures():
    rp, ci = gg.cycle(5)
    assert list(ci) == [4, 0, 1, 2, 3]
    rp, ci = gg.complete(4)
    assert np.all(np.diff(rp) == 3)
    rp, ci = gg.in_star(5)
    assert rp[1] == 4 and rp[-1] == 4
    rp, ci = gg.out_star(5)
    assert rp[1] == 0 and np.all(ci == 0)
    rp, ci = gg.bi_star(5)
    assert ci.size == 8
    rp, ci = gg.empty(3)
    assert ci.size == 0
    rp, ci = gg.edges_to_in_csr(3, [0, 0, 1], [1, 1, 2], dedup=False)
    assert list(ci) == [0, 0, 1]


def test_uniform_and_permutation():
    u = gg.uniform(1, 0, 1000)
    assert np.all((u > 0) & (u < 1)) and abs(u.mean() - 0.5) < 0.05
    assert np.array_equal(u, gg.uniform(1, 0, 1000))
    p = gg.permutation(1, 9, 1000)
    assert np.array_equal(np.sort(p), np.arange(1000))


def test_rmat_n_any_size_deterministic_and_clean():
    for n in (2, 3, 1000, 4097):
        rp, ci = gg.rmat_n(n, 8, seed=12)
        assert rp.size == n + 1 and rp[0] == 0 and rp[-1] == ci.size
        assert np.all(np.diff(rp) >= 0)
        if ci.size:
            assert ci.min() >= 0 and ci.max() < n
        src, dst = gg.in_csr_edges(rp, ci)
        assert np.all(src != dst)                                  # no self-loops
        assert np.unique(dst * n + src).size == src.size           # no duplicates
        rp2, ci2 = gg.rmat_n(n, 8, seed=12, nthreads=1)
        assert np.array_equal(rp, rp2) and np.array_equal(ci, ci2)  # thread-count independent
    rp, ci = gg.rmat_n(5000, 8, seed=1)
    assert 0.8 * 8 * 5000 < ci.size <= 8 * 5000                    # few draws lost to dedup
    # skew: the in-degree distribution is heavy-tailed like R-MAT's
    indeg = np.diff(rp)
    assert indeg.max() > 10 * indeg.mean()


def test_multi_rmat_sizes_and_block_diagonal():
    graphs = gg.multi_rmat(16, 1e3, 1e5, 8, seed=4)
    sizes = np.array([rp.size - 1 for rp, _ in graphs])
    assert sizes.min() >= 1000 and sizes.max() <= 100000
    assert np.array_equal(sizes, [rp.size - 1 for rp, _ in gg.multi_rmat(16, 1e3, 1e5, 8, seed=4)])
    rp, ci, off = gg.block_diagonal(graphs)
    assert off[-1] == sizes.sum() and rp[-1] == ci.size == sum(c.size for _, c in graphs)
    for g, (grp, gci) in enumerate(graphs):
        lo, hi = off[g], off[g + 1]
        sub_rp = rp[lo: hi + 1] - rp[lo]
        sub_ci = ci[rp[lo]: rp[hi]] - lo
        assert np.array_equal(sub_rp, grp) and np.array_equal(sub_ci, gci)


def test_seed_teleports():
    t = gg.seed_teleports(1000, 32, 8, seed=3)
    assert t.shape == (1000, 32) and t.dtype == np.float32
    assert np.all((t > 0).sum(axis=0) == 8)
    np.testing.assert_allclose(t.sum(axis=0), 1.0, rtol=1e-6)
    assert np.array_equal(t, gg.seed_teleports(1000, 32, 8, seed=3))
    assert not np.array_equal(t, gg.seed_teleports(1000, 32, 8, seed=4))
