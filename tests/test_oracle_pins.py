"""Pins for the FP64 oracle against facts fixed independently of its code.

Each pin is something the paper or the mathematics fixes without reference to the oracle:
a hand-worked example (tests/golden), closed forms derived by substitution, the random
surfer's stationary distribution (a Markov-chain description of the same quantity,
solved as an eigenproblem), a library PageRank (networkx), brute force over every
digraph on up to 4 vertices, and invariants/bounds that any correct solution obeys.
The last test compiles deliberately broken copies of the oracle and checks that each
plausible mistake (dropped term, wrong sign, transposed operand) fails a pin.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import graphgen as gg
import oracle

D85 = 0.85
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ helpers --

def surfer_stationary(n, src, dst, d, t=None):
    """Stationary distribution of the random surfer, written from its description:
    from page u the surfer teleports with probability 1-d to a page drawn from t
    (uniform by default); otherwise it follows one of u's out-links chosen uniformly
    (a repeated link is proportionally more likely) or, if u has none, jumps to a
    uniformly random page.  Solved as the eigenvector of eigenvalue 1 of P^T."""
    t = np.full(n, 1.0 / n) if t is None else np.asarray(t, dtype=np.float64) / np.sum(t)
    P = np.zeros((n, n))
    links = np.zeros((n, n))
    for u, v in zip(src, dst):
        links[u, v] += 1
    for u in range(n):
        P[u, :] += (1 - d) * t
        k = links[u].sum()
        if k > 0:
            P[u, :] += d * links[u] / k
        else:
            P[u, :] += d / n
    w, V = np.linalg.eig(P.T)
    i = np.argmin(np.abs(w - 1.0))
    pi = np.real(V[:, i])
    return pi / pi.sum()


def load_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *rest = line.split()
            vals[key] = rest
    return vals


def frac_list(tokens):
    return [float(Fraction(x)) for x in tokens]


# --------------------------------------------------------- worked example --

def test_worked_example_one_step(oracle_lib):
    g = load_golden("worked_example_4v.txt")
    n = int(g["n"][0])
    d = float(Fraction(g["d"][0]))
    rp, ci = gg.edges_to_in_csr(n, [int(s) for s in g["src"]], [int(s) for s in g["dst"]])
    x = np.array(frac_list(g["x"]))
    t = np.array(frac_list(g["t"]))
    xn, D, l1, _ = oracle.jacobi_step(rp, ci, x, d=d)
    assert D == pytest.approx(float(Fraction(g["dangling_mass"][0])), abs=1e-15)
    np.testing.assert_allclose(xn, frac_list(g["x_next"]), rtol=0, atol=1e-15)
    assert l1 == pytest.approx(float(Fraction(g["l1_change"][0])), abs=1e-15)
    xl, _, _, _ = oracle.jacobi_step(rp, ci, x, d=d, redistribute=False)
    np.testing.assert_allclose(xl, frac_list(g["x_next_literal"]), rtol=0, atol=1e-15)
    xt, _, _, _ = oracle.jacobi_step(rp, ci, x, d=d, t=t)
    np.testing.assert_allclose(xt, frac_list(g["x_next_teleport"]), rtol=0, atol=1e-15)
    # the single-vertex form agrees with the whole-vector step
    for v in range(n):
        assert oracle.vertex_update(v, rp, ci, x, D, d=d) == pytest.approx(xn[v], abs=1e-16)
        assert oracle.vertex_update(v, rp, ci, x, D, d=d, t=t) == pytest.approx(xt[v], abs=1e-16)


def test_outdeg_counts_multiplicity():
    rp, ci = gg.edges_to_in_csr(4, [0, 0, 0, 1, 2], [1, 1, 2, 2, 0], dedup=False)
    assert list(oracle.outdeg(rp, ci)) == [3, 1, 1, 0]


# ------------------------------------------------------------ closed forms --

def _both(rp, ci, d, t=None):
    xs = oracle.dense_solve(rp, ci, d=d, t=t)
    xj, it, res = oracle.fixed_point(rp, ci, d=d, t=t)
    return xs, xj


@pytest.mark.parametrize("n", [2, 3, 7, 50])
@pytest.mark.parametrize("d", [0.0, 0.5, 0.85, 0.99])
def test_closed_forms(n, d):
    L = n - 1
    for build, expect in [
        (gg.cycle, np.full(n, 1.0 / n)),
        (gg.complete, np.full(n, 1.0 / n)),
        (gg.empty, np.full(n, 1.0 / n)),
        (gg.in_star, np.array([(1 + d * L) / (n + d * L)] + [1.0 / (n + d * L)] * L)),
        (gg.out_star, np.array([1.0 / (n + d)] + [(L + d) / (L * (n + d))] * L)),
        (gg.bi_star, None),
    ]:
        rp, ci = build(n)
        if expect is None:  # bidirectional star
            hub = (1 + d * L) / (n * (1 + d))
            expect = np.array([hub] + [(1 - d) / n + d * hub / L] * L)
        for x in _both(rp, ci, d):
            np.testing.assert_allclose(x, expect, rtol=1e-11, atol=1e-14,
                                       err_msg=f"{build.__name__} n={n} d={d}")


def test_literal_eq1_leaks_mass():
    # single edge 0 -> 1 on two vertices, Eq. 1 without a dangling share:
    # x0 = (1-d)/2,  x1 = (1-d)/2 + d*x0
    d = 0.85
    rp, ci = gg.edges_to_in_csr(2, [0], [1])
    x = oracle.dense_solve(rp, ci, d=d, redistribute=False)
    np.testing.assert_allclose(x, [(1 - d) / 2, (1 - d) / 2 + d * (1 - d) / 2], atol=1e-15)
    xj, _, _ = oracle.fixed_point(rp, ci, d=d, redistribute=False)
    np.testing.assert_allclose(xj, x, atol=1e-14)
    assert x.sum() < 1.0


def test_literal_equals_redistributed_without_dangling():
    rp, ci = gg.cycle(9)
    rp2, ci2 = gg.rmat(9, seed=2)
    for r, c in [(rp, ci), (rp2, ci2)]:
        if np.any(oracle.outdeg(r, c) == 0):
            x1, _, _ = oracle.pagerank_jacobi(r, c, tol=0, max_iter=30)
            x2, _, _ = oracle.pagerank_jacobi(r, c, tol=0, max_iter=30, redistribute=False)
            assert x2.sum() < x1.sum()
        else:
            x1, _, _ = oracle.pagerank_jacobi(r, c, tol=0, max_iter=30)
            x2, _, _ = oracle.pagerank_jacobi(r, c, tol=0, max_iter=30, redistribute=False)
            assert np.array_equal(x1, x2)


# ------------------------------------------------------------ random surfer --

@pytest.mark.parametrize("seed", range(6))
def test_random_surfer_stationary_distribution(seed):
    n = 5 + 7 * seed
    m = 3 * n
    multi = seed % 2 == 1
    rp, ci = gg.random_digraph(n, m, seed=seed, allow_multi=multi, self_loops=multi)
    src, dst = gg.in_csr_edges(rp, ci)
    t = gg.uniform(seed, 3, n) if seed >= 3 else None
    if t is not None:
        t = t / t.sum()
    for d in (0.5, 0.85):
        pi = surfer_stationary(n, src, dst, d, t)
        xs, xj = _both(rp, ci, d, t)
        np.testing.assert_allclose(xs, pi, rtol=1e-9, atol=1e-13)
        np.testing.assert_allclose(xj, pi, rtol=1e-9, atol=1e-13)


def test_library_pagerank():
    nx = pytest.importorskip("networkx")
    for seed in range(4):
        rp, ci = gg.rmat(8, edge_factor=4, seed=100 + seed)
        n = rp.size - 1
        src, dst = gg.in_csr_edges(rp, ci)
        G = nx.DiGraph()
        G.add_nodes_from(range(n))
        G.add_edges_from(zip(src.tolist(), dst.tolist()))
        ref = nx.pagerank(G, alpha=D85, tol=1e-15, max_iter=100000)
        ref = np.array([ref[v] for v in range(n)])
        x, _, _ = oracle.fixed_point(rp, ci)
        np.testing.assert_allclose(x, ref, rtol=1e-9, atol=1e-14)
        # personalised teleport (networkx keeps dangling mass uniform when dangling=None)
        t = gg.uniform(seed, 5, n)
        t /= t.sum()
        ref = nx.pagerank(G, alpha=D85, personalization={v: t[v] for v in range(n)},
                          dangling={v: 1.0 / n for v in range(n)}, tol=1e-15, max_iter=100000)
        ref = np.array([ref[v] for v in range(n)])
        x, _, _ = oracle.fixed_point(rp, ci, t=t)
        np.testing.assert_allclose(x, ref, rtol=1e-9, atol=1e-14)


# -------------------------------------------------------------- brute force --

def _all_digraphs(n):
    pairs = [(u, v) for u in range(n) for v in range(n) if u != v]
    for mask in range(1 << len(pairs)):
        es = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
        yield es


@pytest.mark.parametrize("n", [2, 3, 4])
def test_every_digraph(n):
    worst_j, worst_s = 0.0, 0.0
    for es in _all_digraphs(n):
        src = [e[0] for e in es]
        dst = [e[1] for e in es]
        rp, ci = gg.edges_to_in_csr(n, src, dst)
        pi = surfer_stationary(n, src, dst, D85)
        xs = oracle.dense_solve(rp, ci)
        xj, _, _ = oracle.fixed_point(rp, ci)
        worst_s = max(worst_s, np.abs(xs - pi).max())
        worst_j = max(worst_j, np.abs(xj - pi).max())
    assert worst_s < 1e-12 and worst_j < 1e-12


# --------------------------------------------------- invariants and bounds --

@pytest.mark.parametrize("seed", range(3))
def test_invariants_and_contraction_bound(seed):
    rp, ci = gg.rmat(11, seed=seed)
    n = rp.size - 1
    t = gg.uniform(seed, 9, n)
    t = 0.7 * t / t.sum()           # sum(t) = 0.7: the fixed point then sums to 0.7
    for tt, total in [(None, 1.0), (t, 0.7)]:
        xstar, _, _ = oracle.fixed_point(rp, ci, t=tt)
        assert xstar.sum() == pytest.approx(total, rel=1e-12)
        floor = (1 - D85) * (np.full(n, 1.0 / n) if tt is None else tt)
        assert np.all(xstar >= floor * (1 - 1e-12))
        # a-posteriori bound of a contraction with factor d in L1:
        #   ||x_k - x*||_1 <= d/(1-d) * ||x_k - x_{k-1}||_1
        x = np.full(n, 1.0 / n) if tt is None else tt.copy()
        for _ in range(15):
            xn, _, l1, _ = oracle.jacobi_step(rp, ci, x, t=tt)
            err = np.abs(xn - xstar).sum()
            assert err <= D85 / (1 - D85) * l1 * (1 + 1e-9) + 1e-14
            x = xn


def test_permutation_equivariance():
    rp, ci = gg.rmat(10, seed=4)
    n = rp.size - 1
    perm = gg.permutation(4, 1, n)
    rp2, ci2 = gg.permute_in_csr(rp, ci, perm)
    x, _, _ = oracle.fixed_point(rp, ci)
    x2, _, _ = oracle.fixed_point(rp2, ci2)
    np.testing.assert_allclose(x2[perm], x, rtol=1e-10, atol=1e-15)


def test_matching_mode_counts_iterations():
    rp, ci = gg.rmat(12, seed=1)
    x, it, res, hist = oracle.pagerank_jacobi(rp, ci, tol=1e-10, max_iter=200, history=True)
    assert res < 1e-10 and it == hist.size and np.all(hist[:-1] >= 1e-10)
    x1, it1, _ = oracle.pagerank_jacobi(rp, ci, tol=0, max_iter=1)
    assert it1 == 1
    # two single steps equal one two-step run
    xa, _, _ = oracle.pagerank_jacobi(rp, ci, tol=0, max_iter=2)
    xb, _, _ = oracle.pagerank_jacobi(rp, ci, tol=0, max_iter=1, x0=x1)
    assert np.array_equal(xa, xb)


# ------------------------------------------------------- No-Sync (Alg. 3) --

@pytest.mark.parametrize("form", ["mass", "complement"])
@pytest.mark.parametrize("p", [1, 3, 16])
def test_nosync_reaches_the_same_fixed_point(form, p):
    """Lemma 2: the lock-free result equals the sequential one within the threshold."""
    rp, ci = gg.rmat(10, seed=7)
    xstar, _, _ = oracle.fixed_point(rp, ci)
    speed = (1 + np.arange(p) % 3).astype(np.int32)  # unequal thread speeds
    x, sweeps, upd, est = oracle.nosync(rp, ci, p=p, tol=1e-12, max_sweeps=5000, speed=speed,
                                        dangling=form)
    assert est <= 1e-12
    assert np.abs(x - xstar).sum() < 1e-10
    assert sweeps.min() >= 1


def test_nosync_paper_norm_and_literal():
    rp, ci = gg.rmat(9, seed=8)
    for redistribute in (True, False):
        xstar, _, _ = oracle.fixed_point(rp, ci, redistribute=redistribute)
        x, sweeps, _, est = oracle.nosync(rp, ci, p=4, tol=1e-14, max_sweeps=5000, norm="linf",
                                          redistribute=redistribute, dangling="mass")
        assert np.abs(x - xstar).sum() < 1e-11


def test_nosync_fewer_sweeps_than_jacobi_iterations():
    """The paper's iteration-count observation (Fig. 7): in-place updates converge in fewer
    sweeps than synchronous iterations.  With uniform dangling redistribution this needs
    the complement form of the dangling share; the running-mass form is slower."""
    rp, ci = gg.rmat(12, seed=3)
    _, it, _ = oracle.pagerank_jacobi(rp, ci, tol=1e-12, max_iter=1000)
    _, sw_c, _, _ = oracle.nosync(rp, ci, p=8, tol=1e-12, dangling="complement")
    _, sw_m, _, _ = oracle.nosync(rp, ci, p=8, tol=1e-12, dangling="mass")
    assert sw_c.max() < it < sw_m.max()


def test_nosync_single_sweep_on_a_chain():
    """p=1 on the chain 0 -> 1 -> ... -> n-1 with Eq. 1 literal: an in-place sweep in vertex
    order sees each predecessor's new value, so one sweep gives the exact fixed point
    x_k = (1-d)/n * sum_{j<=k} d^j (Jacobi needs n sweeps for the same)."""
    n, d = 6, 0.85
    rp, ci = gg.edges_to_in_csr(n, np.arange(n - 1), np.arange(1, n))
    expect = np.array([(1 - d) / n * sum(d ** j for j in range(k + 1)) for k in range(n)])
    x, sweeps, upd, est = oracle.nosync(rp, ci, d=d, p=1, tol=1e-300, max_sweeps=1,
                                        redistribute=False, dangling="mass")
    np.testing.assert_allclose(x, expect, rtol=1e-14)
    xj, _, _ = oracle.pagerank_jacobi(rp, ci, d=d, tol=0, max_iter=1, redistribute=False)
    assert not np.allclose(xj, expect)


# ------------------------------------------------------ planted mistakes --

def _pins_pass(lib):
    """A compact run of the pins above against a given build of the oracle."""
    g = load_golden("worked_example_4v.txt")
    n = int(g["n"][0])
    d = float(Fraction(g["d"][0]))
    rp, ci = gg.edges_to_in_csr(n, [int(s) for s in g["src"]], [int(s) for s in g["dst"]])
    x = np.array(frac_list(g["x"]))
    t = np.array(frac_list(g["t"]))
    try:
        xn, _, _, _ = oracle.jacobi_step(rp, ci, x, d=d, lib=lib)
        if not np.allclose(xn, frac_list(g["x_next"]), atol=1e-15):
            return False
        xt, _, _, _ = oracle.jacobi_step(rp, ci, x, d=d, t=t, lib=lib)
        if not np.allclose(xt, frac_list(g["x_next_teleport"]), atol=1e-15):
            return False
        for build in (gg.in_star, gg.out_star):
            rps, cis = build(7)
            L = 6
            expect = (np.array([(1 + d * L) / (7 + d * L)] + [1 / (7 + d * L)] * L)
                      if build is gg.in_star else
                      np.array([1 / (7 + d)] + [(L + d) / (L * (7 + d))] * L))
            if not np.allclose(oracle.dense_solve(rps, cis, d=d, lib=lib), expect, atol=1e-12):
                return False
        rp2, ci2 = gg.random_digraph(9, 25, seed=2)
        src, dst = gg.in_csr_edges(rp2, ci2)
        pi = surfer_stationary(9, src, dst, d)
        if not np.allclose(oracle.dense_solve(rp2, ci2, d=d, lib=lib), pi, atol=1e-12):
            return False
        xj, _, _ = oracle.fixed_point(rp2, ci2, d=d, lib=lib)
        if not np.allclose(xj, pi, atol=1e-12):
            return False
        xs, _, _, _ = oracle.nosync(rp2, ci2, d=d, p=3, tol=1e-13, lib=lib)
        if not np.allclose(xs, pi, atol=1e-11):
            return False
        # loop perforation (Alg. 5): with eps = inf every vertex freezes after its first
        # update, so the synchronous form is one Jacobi step and the No-Sync form one sweep;
        # on the cycle nothing changes, so nothing may freeze
        x1, _, _, _ = oracle.jacobi_step(rp2, ci2, np.full(9, 1 / 9), d=d, lib=lib)
        xp, itp, rpf, nfp = oracle.pagerank_perforated(rp2, ci2, d=d, tol=1e-12, eps=np.inf, lib=lib)
        if not (np.array_equal(xp, x1) and itp == 2 and rpf == 0.0 and nfp == 9):
            return False
        xg, _, _, _ = oracle.nosync(rp2, ci2, d=d, p=1, tol=1e-300, max_sweeps=1, lib=lib)
        xq, swq, updq, estq, nfq = oracle.nosync_perforated(rp2, ci2, d=d, p=1, tol=1e-12,
                                                            eps=np.inf, lib=lib)
        if not (np.array_equal(xq, xg) and list(swq) == [2] and updq == 9 and nfq == 9):
            return False
        rpc, cic = gg.cycle(5)
        if oracle.pagerank_perforated(rpc, cic, d=d, tol=1e-12, eps=np.inf, lib=lib)[3] != 0:
            return False
        if oracle.nosync_perforated(rpc, cic, d=d, p=2, tol=1e-12, eps=np.inf, lib=lib)[4] != 0:
            return False
        # weighted forward and adjoint against the dense adjoint (numpy linear algebra)
        rp3, ci3 = gg.random_digraph(8, 16, seed=9)   # three dangling vertices
        w3 = 0.1 + 0.9 * gg.uniform(6, 1, ci3.size)
        c3 = gg.uniform(6, 2, 8) - 0.5
        xd, lamd, gtd, gwd = oracle.dense_adjoint(rp3, ci3, w3, c3, d=d)
        xw, _, _ = oracle.w_pagerank(rp3, ci3, w3, d=d, lib=lib)
        if not np.allclose(xw, xd, atol=1e-12):
            return False
        adj = oracle.w_adjoint(rp3, ci3, w3, xw, c3, d=d, lib=lib)
        if not (np.allclose(adj["grad_t"], gtd, atol=1e-11) and np.allclose(adj["grad_w"], gwd, atol=1e-11)):
            return False
    except oracle.OracleError:
        return False
    return True


MUTATIONS = {
    "drop_dangling_share": ("d * (sum + D / (double)n)", "d * (sum)"),
    "wrong_damping_sign": ("(1.0 - d) * or_teleport(n, t, v)", "(1.0 + d) * or_teleport(n, t, v)"),
    "divide_by_target_degree": ("sum += x[u] / (double)outdeg[u];",
                                "sum += x[u] / (double)(outdeg[v] ? outdeg[v] : 1);"),
    "teleport_index": ("return t ? t[v] : 1.0 / (double)n;",
                       "return t ? t[n - 1 - v] : 1.0 / (double)n;"),
    "transposed_system": ("M[v * n + u] -= d / (double)outdeg[u];",
                          "M[u * n + v] -= d / (double)outdeg[u];"),
    "dangling_from_wrong_set": ("if (outdeg[u] == 0) D += x[u];", "if (outdeg[u] == 1) D += x[u];"),
    "nosync_stale_nondangling_mass": ("else S += tmp - previous;", "else S += 0.0;"),
    "weighted_forward_ignores_weight": ("s += x[u] * w[e] / W[u];", "s += x[u] / W[u];"),
    "adjoint_drops_dangling_term": ("(W[u] == 0.0 ? L / (double)n : 0.0)", "0.0"),
    "adjoint_edge_gradient_sign": ("(lambda[v] - mu[u])", "(mu[u] - lambda[v])"),
    "perforation_recomputes_frozen": ("if (frozen[v]) {", "if (0 && frozen[v]) {"),
    "perforation_freezes_unchanged": ("if (change != 0.0 && change < eps) frozen[v] = 1;",
                                      "if (change < eps) frozen[v] = 1;"),
    "nosync_perforation_recomputes_frozen": ("if (!frozen[u]) {", "if (1) {"),
    "nosync_perforation_freezes_unchanged": ("if (diff != 0.0 && diff < eps) frozen[u] = 1;",
                                             "if (diff < eps) frozen[u] = 1;"),
    "adjoint_pushes_to_target": ("mu[u] += w[e] / W[u] * lambda[v];\n            }\n        r = 0.0;",
                                 "mu[v] += w[e] / W[u] * lambda[u];\n            }\n        r = 0.0;"),
}


def test_pins_pass_on_the_real_oracle(oracle_lib):
    assert _pins_pass(oracle_lib)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_each_planted_mistake_fails_a_pin(name, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "pagerank_oracle.c")).read()
    old, new = MUTATIONS[name]
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mutated = tmp_path / "oracle_mut.c"
    mutated.write_text(src.replace(old, new))
    out = oracle.build(force=True, src=str(mutated), out=str(tmp_path / "liboracle_mut.so"))
    lib = oracle.load(out)
    assert not _pins_pass(lib), f"planted mistake '{name}' was not caught"



# ------------------------------------------------------------ weighted graphs --

def weighted_case(n, m, seed, multi=False):
    rp, ci = gg.random_digraph(n, m, seed=seed, allow_multi=multi)
    w = 0.1 + 0.9 * gg.uniform(seed, 7, ci.size)
    return rp, ci, w


def test_unit_weights_reduce_to_the_unweighted_oracle():
    rp, ci = gg.rmat(10, 16, seed=4)
    x, it, r = oracle.w_pagerank(rp, ci, np.ones(ci.size), tol=1e-13)
    xs, _, _ = oracle.fixed_point(rp, ci)
    assert np.allclose(x, xs, atol=1e-14)


def test_scaling_one_vertex_out_weights_changes_nothing():
    """P(u, .) = w(u, .)/W(u) is invariant under scaling u's out-weights."""
    rp, ci, w = weighted_case(40, 200, seed=3)
    x, _, _ = oracle.w_pagerank(rp, ci, w)
    w2 = w.copy()
    w2[ci == 5] *= 7.0
    x2, _, _ = oracle.w_pagerank(rp, ci, w2)
    assert np.allclose(x, x2, atol=1e-14)
    w3 = w.copy()
    w3[np.flatnonzero(ci == 5)[:1]] *= 7.0      # one edge only: the ranks move
    x3, _, _ = oracle.w_pagerank(rp, ci, w3)
    assert np.abs(x - x3).sum() > 1e-6


@pytest.mark.parametrize("seed", range(6))
def test_weighted_forward_and_adjoint_match_the_dense_adjoint(seed):
    n = 3 + seed
    rp, ci, w = weighted_case(n, 2 * n + seed, seed=seed, multi=seed % 2 == 1)
    t = gg.uniform(seed, 8, n) + 0.05
    t /= t.sum()
    c = gg.uniform(seed, 9, n) - 0.5
    xd, lamd, gtd, gwd = oracle.dense_adjoint(rp, ci, w, c, t=t)
    x, _, _ = oracle.w_pagerank(rp, ci, w, t=t)
    assert np.allclose(x, xd, atol=1e-13)
    adj = oracle.w_adjoint(rp, ci, w, x, c)
    assert np.allclose(adj["lambda"], lamd, atol=1e-12)
    assert np.allclose(adj["grad_t"], gtd, atol=1e-12)
    assert np.allclose(adj["grad_w"], gwd, atol=1e-12)


@pytest.mark.parametrize("graph", ["rmat14", "er14"])
def test_perforated_nosync_error_scale(graph):
    """Alg. 5 on Alg. 3: a frozen row stopped on a change below eps and the update is an L1
    contraction with factor d, so the perforated result sits within about
    (frozen rows * eps + tol) / (1 - d) of the fixed point.  Checked over thread counts 1
    to 1024 and three bounds; a dropped freeze test (nothing frozen) or a frozen row that
    kept being updated would change the frozen count or the error."""
    rp, ci = gg.rmat(14, seed=21) if graph == "rmat14" else gg.er_dangling(1 << 14, seed=5)
    xs, _, _ = oracle.fixed_point(rp, ci)
    for p in (1, 64, 1024):
        for eps in (1e-8, 1e-9, 1e-11):
            x, _, upd, _, nf = oracle.nosync_perforated(rp, ci, p=p, tol=1e-7, eps=eps)
            x0, _, upd0, _, nf0 = oracle.nosync_perforated(rp, ci, p=p, tol=1e-7, eps=0.0)
            assert nf > 0 and nf0 == 0 and upd < upd0
            assert np.abs(x - xs).sum() <= (nf * eps + 1e-7) / (1 - 0.85)


def test_adjoint_step_cycle_closed_form():
    """Directed cycle u -> u+1 (mod n), unit weights, no dangling vertex: P(u, u+1) = 1, so
    one update of the adjoint system is lambda_out(u) = c(u) + d lambda(u+1)."""
    n = 7
    rp, ci = gg.cycle(n)
    w = np.ones(ci.size)
    c = gg.uniform(3, 4, n) - 0.5
    lam = gg.uniform(3, 5, n) * 3.0 - 1.0
    out, l1 = oracle.w_adjoint_step(rp, ci, w, c, lam, d=0.8)
    expect = c + 0.8 * np.roll(lam, -1)
    assert np.allclose(out, expect, atol=1e-15)
    assert l1 == pytest.approx(np.abs(expect - lam).sum(), rel=1e-14)


@pytest.mark.parametrize("seed", range(3))
def test_adjoint_step_fixed_point_and_first_iterate(seed):
    """The dense adjoint's lambda (numpy's solver on M^T) is a fixed point of the step, with
    dangling vertices present; from lambda = c the step gives or_w_adjoint's first iterate."""
    n = 5 + seed
    rp, ci, w = weighted_case(n, 2 * n, seed=10 + seed, multi=False)
    c = gg.uniform(seed, 13, n) - 0.5
    _, lamd, _, _ = oracle.dense_adjoint(rp, ci, w, c)
    out, l1 = oracle.w_adjoint_step(rp, ci, w, c, lamd)
    assert l1 < 1e-12 and np.allclose(out, lamd, atol=1e-13)
    first, _ = oracle.w_adjoint_step(rp, ci, w, c, c)
    x, _, _ = oracle.w_pagerank(rp, ci, w)
    adj1 = oracle.w_adjoint(rp, ci, w, x, c, tol=0.0, max_iter=1)
    assert np.allclose(first, adj1["lambda"], atol=1e-15)


def test_adjoint_identities():
    """L = c^T x is linear in t (so (1-d) lambda^T t = L) and unchanged by scaling one
    vertex's out-weights (so the weight gradients of each vertex's out-edges, weighted by
    the weights, sum to zero)."""
    rp, ci = gg.rmat(11, 8, seed=9)
    w = 0.1 + 0.9 * gg.uniform(9, 1, ci.size)
    n = rp.size - 1
    t = gg.uniform(9, 2, n)
    t /= t.sum()
    c = gg.uniform(9, 3, n) - 0.5
    x, _, _ = oracle.w_pagerank(rp, ci, w, t=t)
    adj = oracle.w_adjoint(rp, ci, w, x, c)
    assert abs(adj["grad_t"] @ t - c @ x) < 1e-12
    per_src = np.zeros(n)
    np.add.at(per_src, ci, w * adj["grad_w"])
    assert np.max(np.abs(per_src)) < 1e-12


def test_adjoint_against_central_differences():
    """Central differences (h = 1e-3) of L through the FP64 forward at tol 1e-14: exact for
    the teleport (L is linear in t), second order for the weights."""
    rp, ci = gg.rmat(9, 8, seed=5)
    n = rp.size - 1
    w = 0.1 + 0.9 * gg.uniform(5, 1, ci.size)
    t = np.full(n, 1.0 / n)
    c = gg.uniform(5, 3, n) - 0.5
    x, _, _ = oracle.w_pagerank(rp, ci, w, t=t, tol=1e-15)
    adj = oracle.w_adjoint(rp, ci, w, x, c)
    h = 1e-3

    def L(tt, ww):
        xx, _, _ = oracle.w_pagerank(rp, ci, ww, t=tt, tol=1e-15, x0=x)
        return c @ xx

    rng = np.random.default_rng(0)
    for i in rng.integers(0, n, 8):
        tp, tm = t.copy(), t.copy()
        tp[i] += h
        tm[i] -= h
        fd = (L(tp, w) - L(tm, w)) / (2 * h)
        assert fd == pytest.approx(adj["grad_t"][i], rel=1e-7, abs=1e-11)
    for e in rng.integers(0, ci.size, 8):
        wp, wm = w.copy(), w.copy()
        wp[e] += h
        wm[e] -= h
        fd = (L(t, wp) - L(t, wm)) / (2 * h)
        assert fd == pytest.approx(adj["grad_w"][e], rel=1e-4, abs=1e-9)



# ------------------------------------------------------------ loop perforation --

def test_perforation_with_eps_zero_is_alg1():
    rp, ci = gg.rmat(11, 16, seed=8)
    x0, it0, r0 = oracle.pagerank_jacobi(rp, ci, tol=1e-12, max_iter=500)
    x1, it1, r1, nf = oracle.pagerank_perforated(rp, ci, tol=1e-12, max_iter=500, eps=0.0)
    assert nf == 0 and it0 == it1 and np.array_equal(x0, x1)


def test_perforation_freezes_and_stays_close():
    """Vertices freeze as their changes shrink (on R-MAT-11 all of them by the end); the
    perforated result stays close to the fixed point, and a larger eps stops sooner and
    errs more."""
    rp, ci = gg.rmat(11, 16, seed=8)
    xs, _, _ = oracle.fixed_point(rp, ci)
    _, it_plain, _ = oracle.pagerank_jacobi(rp, ci, tol=1e-10, max_iter=500)
    errs, iters = [], []
    for eps in (1e-12, 1e-9):
        x, it, r, nf = oracle.pagerank_perforated(rp, ci, tol=1e-10, max_iter=500, eps=eps)
        errs.append(float(np.abs(x - xs).sum()))
        iters.append(it)
        assert r < 1e-10 and nf > 0
        assert abs(x.sum() - 1.0) < 1e-5        # frozen ranks no longer conserve mass exactly
    assert iters[1] < iters[0] <= it_plain
    assert errs[0] < errs[1]
    assert errs[0] < 1e-8 and errs[1] < 1e-5


def test_perforation_with_infinite_eps_is_one_step():
    """Alg. 5 with eps = inf freezes every vertex at its first update: the synchronous form
    returns exactly one Jacobi step from t (its second iteration changes nothing), the No-Sync
    form exactly one Gauss-Seidel sweep, and every vertex is computed once."""
    rp, ci = gg.rmat(10, 16, seed=3)
    n = rp.size - 1
    x1, _, _ = oracle.pagerank_jacobi(rp, ci, tol=0, max_iter=1)
    assert np.all(x1 != 1.0 / n)                 # every vertex changes in the first step
    x, it, r, nf = oracle.pagerank_perforated(rp, ci, tol=1e-12, max_iter=50, eps=np.inf)
    assert np.array_equal(x, x1) and it == 2 and r == 0.0 and nf == n
    xg, _, upd_g, _ = oracle.nosync(rp, ci, p=1, tol=1e-300, max_sweeps=1)
    xq, sw, upd, est, nfq = oracle.nosync_perforated(rp, ci, p=1, tol=1e-12, max_sweeps=50, eps=np.inf)
    assert np.array_equal(xq, xg) and list(sw) == [2] and upd == upd_g == n and est == 0.0 and nfq == n
    # several threads: each vertex is still computed exactly once, then all are frozen.  The
    # threads finish their sweeps in the same rounds, in thread order, so at the end of its
    # second (empty) sweep each thread but the last still sees a later thread's first-sweep
    # error, and makes a third
    xm, sw4, upd4, est4, nf4 = oracle.nosync_perforated(rp, ci, p=4, tol=1e-12, max_sweeps=50, eps=np.inf)
    assert upd4 == n and nf4 == n and est4 == 0.0 and list(sw4) == [3, 3, 3, 2]


def test_nosync_perforation_freezes_and_stays_close():
    """No-Sync with perforation (the paper's No-Sync-Opt): vertices freeze as their changes
    shrink, fewer updates are computed than by plain Alg. 3 to the same tolerance, and the
    result stays close to the fixed point; eps = 0 is plain Alg. 3."""
    rp, ci = gg.rmat(11, 16, seed=8)
    xs, _, _ = oracle.fixed_point(rp, ci)
    x0, sw0, upd0, _ = oracle.nosync(rp, ci, p=4, tol=1e-10)
    xz, swz, updz, _, nfz = oracle.nosync_perforated(rp, ci, p=4, tol=1e-10, eps=0.0)
    assert nfz == 0 and updz == upd0 and np.array_equal(xz, x0)
    x, sw, upd, est, nf = oracle.nosync_perforated(rp, ci, p=4, tol=1e-10, eps=1e-12)
    assert nf > 0 and upd < upd0 and est <= 1e-10
    assert float(np.abs(x - xs).sum()) < 1e-8
    assert float(np.abs(x0 - xs).sum()) < float(np.abs(x - xs).sum()) + 1e-9
