/*
 * pagerank_oracle.c -- plain, slow, single-threaded FP64 PageRank oracle.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header, table or
 * helper with the CUDA library it checks; it reads the same in-edge CSR
 * (row v lists the sources u of the edges u -> v) and derives everything else
 * (out-degrees, dangling set) itself.
 *
 * What it computes (paper: Eedi et al., "An Improved and Optimized Practical
 * Non-Blocking PageRank Algorithm for Massive Graphs"):
 *
 *   Eq. 1:  pr(v) = (1-d)/n + d * sum_{(u,v) in E} pr(u) / outdeg(u)
 *
 * with two readings where the paper is silent:
 *   - dangling vertices (outdeg 0) have their rank mass D = sum of their
 *     ranks spread uniformly, adding d*D/n to every vertex (redistribute=1);
 *     redistribute=0 is Eq. 1 taken literally (mass leaks, sum(x) < 1);
 *   - a teleport vector t (default uniform 1/n) replaces the 1/n of the
 *     first term, giving (1-d)*t(v); the dangling share stays uniform.
 * A repeated edge counts with its multiplicity, in outdeg and in the sum.
 *
 * Functions
 *   or_outdeg          out-degree of every vertex, counted from colidx.
 *   or_jacobi_step     one synchronous update (the inner loops of Alg. 1).
 *   or_pagerank_jacobi the Barrier baseline, Alg. 1: iterate from x0 = t
 *                      until the L1 change of an iteration < tol or max_iter.
 *   or_vertex_update   the update of one vertex from a given vector (used to
 *                      check sampled outputs of very large runs).
 *   or_dense_solve     the fixed point as the solution of the linear system
 *                      (I - d*A - (d/n)*1*a^T) x = (1-d)*t by Gaussian
 *                      elimination with partial pivoting (small n only).
 *   or_pagerank_perforated  Alg. 5 (loop perforation) on the synchronous
 *                      iteration: a vertex whose update changed its rank by
 *                      a nonzero amount below eps is frozen, and from the
 *                      next iteration on keeps its rank without being
 *                      recomputed (its rank still feeds its out-neighbours
 *                      and the dangling mass).  eps = 0 is Alg. 1.
 *   or_w_outweight     weighted graphs: W(u) = sum of the weights of u's
 *                      out-edges (the row normaliser of the transition
 *                      matrix P(u,v) = w(u,v)/W(u)).
 *   or_w_jacobi        Alg. 1 on a weighted graph: x(v) = (1-d) t(v) + d *
 *                      ( sum_{(u,v)} x(u) w(u,v)/W(u) + D/n ).
 *   or_w_adjoint       the adjoint of the weighted fixed point for a loss
 *                      L = c^T x: the solution lambda of M^T lambda = c with
 *                      M = I - d P^T - (d/n) 1 a^T (Jacobi iteration on the
 *                      transposed system), then dL/dt = (1-d) lambda and, for
 *                      an edge e = (u, v), dL/dw(e) = d x(u)/W(u) *
 *                      (lambda(v) - sum_{v'} P(u,v') lambda(v')).
 *   or_w_adjoint_step  one update of that transposed system from a given
 *                      lambda, with its L1 change (a certificate for a
 *                      lambda computed elsewhere).
 *   or_nosync          the lock-free No-Sync scheme, Alg. 3: p simulated
 *                      threads, static equal partitions, in-place updates,
 *                      thread-level convergence; two forms of the dangling
 *                      share (running dangling mass, or total minus the
 *                      running non-dangling mass); with eps > 0 the loop
 *                      perforation of Alg. 5, which the paper applies to
 *                      its No-Sync variants as well (Section 4, the
 *                      optimisation of the Barrier and No-Sync variants).
 *
 * Parity status: or_outdeg, or_jacobi_step, or_pagerank_jacobi,
 * or_vertex_update and or_dense_solve are pinned by closed forms, by the
 * random-surfer stationary distribution and by a library PageRank in the
 * CPU test suite; or_nosync is pinned by Lemma 2 (same fixed point) and by
 * its single-thread case, Gauss-Seidel.  Perforation (or_pagerank_perforated,
 * or_nosync with eps > 0) is pinned by eps = 0 (plain Alg. 1 / Alg. 3), by
 * eps = inf (every vertex frozen at its first update: exactly one Jacobi step,
 * or one Gauss-Seidel sweep), and by a graph whose ranks never change (the
 * directed cycle: nothing freezes).  or_w_jacobi is pinned by unit
 * weights (the unweighted oracle), by invariance under scaling one vertex's
 * out-weights, and by a dense solve; or_w_adjoint by the dense adjoint
 * (numpy linear algebra on explicit dM/dw matrices, n <= 12), by central
 * finite differences of or_w_jacobi, and by the identities
 * (1-d) lambda^T t = c^T x and sum_{e out of u} w(e) dL/dw(e) = 0;
 * or_w_adjoint_step by the directed cycle (lambda_out(u) = c(u) + d
 * lambda(u+1) in closed form), by the dense adjoint's lambda (a fixed point:
 * change ~ 0) and by the first iterate of or_w_adjoint.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_API __attribute__((visibility("default")))

enum { OR_OK = 0, OR_BAD_ARG = -1, OR_BAD_GRAPH = -2, OR_NO_MEM = -3, OR_SINGULAR = -4 };

/* Check the CSR is well formed: rowptr[0] = 0, non-decreasing, colidx in range. */
static int or_check_csr(int64_t n, const int64_t* rowptr, const int32_t* colidx) {
    if (n < 1 || !rowptr) return OR_BAD_ARG;
    if (rowptr[0] != 0) return OR_BAD_GRAPH;
    for (int64_t v = 0; v < n; ++v)
        if (rowptr[v + 1] < rowptr[v]) return OR_BAD_GRAPH;
    if (rowptr[n] > 0 && !colidx) return OR_BAD_ARG;
    for (int64_t e = 0; e < rowptr[n]; ++e)
        if (colidx[e] < 0 || colidx[e] >= n) return OR_BAD_GRAPH;
    return OR_OK;
}

/* Out-degree of u = number of edges u -> v = occurrences of u in colidx. */
OR_API int or_outdeg(int64_t n, const int64_t* rowptr, const int32_t* colidx, int64_t* outdeg) {
    int rc = or_check_csr(n, rowptr, colidx);
    if (rc) return rc;
    for (int64_t u = 0; u < n; ++u) outdeg[u] = 0;
    for (int64_t e = 0; e < rowptr[n]; ++e) outdeg[colidx[e]] += 1;
    return OR_OK;
}

/* Teleport weight of v: t[v], or 1/n when t is NULL. */
static double or_teleport(int64_t n, const double* t, int64_t v) {
    return t ? t[v] : 1.0 / (double)n;
}

/* Dangling mass: sum of x over vertices without out-edges. */
static double or_dangling_mass(int64_t n, const int64_t* outdeg, const double* x) {
    double D = 0.0;
    for (int64_t u = 0; u < n; ++u)
        if (outdeg[u] == 0) D += x[u];
    return D;
}

/* New rank of v from the vector x (Eq. 1, plus the uniform dangling share
 * d*D/n where D is the dangling mass of x). */
OR_API double or_vertex_update(int64_t v, int64_t n, const int64_t* rowptr, const int32_t* colidx,
                               const int64_t* outdeg, double d, const double* t, double D,
                               const double* x) {
    double sum = 0.0;
    for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
        int64_t u = colidx[e];
        sum += x[u] / (double)outdeg[u];
    }
    return (1.0 - d) * or_teleport(n, t, v) + d * (sum + D / (double)n);
}

/* One synchronous (Jacobi) update xn = F(x).  Outputs: the dangling mass of
 * x that was spread, and the L1 and max-abs change |xn - x|. */
OR_API int or_jacobi_step(int64_t n, const int64_t* rowptr, const int32_t* colidx,
                          const int64_t* outdeg, double d, const double* t, int redistribute,
                          const double* x, double* xn, double* dangling_out,
                          double* l1_out, double* linf_out) {
    double D = redistribute ? or_dangling_mass(n, outdeg, x) : 0.0;
    double l1 = 0.0, linf = 0.0;
    for (int64_t v = 0; v < n; ++v) {
        xn[v] = or_vertex_update(v, n, rowptr, colidx, outdeg, d, t, D, x);
        double diff = fabs(xn[v] - x[v]);
        l1 += diff;
        if (diff > linf) linf = diff;
    }
    if (dangling_out) *dangling_out = D;
    if (l1_out) *l1_out = l1;
    if (linf_out) *linf_out = linf;
    return OR_OK;
}

/* Alg. 1 (Barrier baseline): x0 = t (or the given x0); each iteration computes
 * every vertex from the previous vector, then swaps.  Stops when the L1 change
 * of the last iteration is below tol, or after max_iter iterations (tol <= 0:
 * run exactly max_iter).  history, if not NULL, receives the L1 change of each
 * iteration.  Returns OR_OK; *iters and *resid describe the last iteration. */
OR_API int or_pagerank_jacobi(int64_t n, const int64_t* rowptr, const int32_t* colidx, double d,
                              const double* t, int redistribute, double tol, int32_t max_iter,
                              const double* x0, double* x, int32_t* iters, double* resid,
                              double* history) {
    int rc = or_check_csr(n, rowptr, colidx);
    if (rc) return rc;
    if (!(d >= 0.0 && d < 1.0) || max_iter < 0) return OR_BAD_ARG;
    int64_t* outdeg = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    double* xn = (double*)malloc((size_t)n * sizeof(double));
    if (!outdeg || !xn) { free(outdeg); free(xn); return OR_NO_MEM; }
    or_outdeg(n, rowptr, colidx, outdeg);
    for (int64_t v = 0; v < n; ++v) x[v] = x0 ? x0[v] : or_teleport(n, t, v);
    int32_t k = 0;
    double l1 = INFINITY;
    while (k < max_iter) {
        or_jacobi_step(n, rowptr, colidx, outdeg, d, t, redistribute, x, xn, NULL, &l1, NULL);
        memcpy(x, xn, (size_t)n * sizeof(double));
        if (history) history[k] = l1;
        ++k;
        if (tol > 0.0 && l1 < tol) break;
    }
    if (iters) *iters = k;
    if (resid) *resid = l1;
    free(outdeg);
    free(xn);
    return OR_OK;
}

/* Alg. 5: Alg. 1 with loop perforation.  frozen_out (may be NULL) receives
 * how many vertices ended frozen. */
OR_API int or_pagerank_perforated(int64_t n, const int64_t* rowptr, const int32_t* colidx, double d,
                                  const double* t, double tol, int32_t max_iter, double eps, double* x,
                                  int32_t* iters, double* resid, int64_t* frozen_out) {
    int rc = or_check_csr(n, rowptr, colidx);
    if (rc) return rc;
    if (!(d >= 0.0 && d < 1.0) || max_iter < 0 || !(eps >= 0.0)) return OR_BAD_ARG;
    int64_t* outdeg = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    double* xn = (double*)malloc((size_t)n * sizeof(double));
    unsigned char* frozen = (unsigned char*)calloc((size_t)n, 1);
    if (!outdeg || !xn || !frozen) { free(outdeg); free(xn); free(frozen); return OR_NO_MEM; }
    or_outdeg(n, rowptr, colidx, outdeg);
    for (int64_t v = 0; v < n; ++v) x[v] = or_teleport(n, t, v);
    int32_t k = 0;
    double l1 = INFINITY;
    while (k < max_iter) {
        const double D = or_dangling_mass(n, outdeg, x);
        l1 = 0.0;
        for (int64_t v = 0; v < n; ++v) {
            if (frozen[v]) {
                xn[v] = x[v];
                continue;
            }
            xn[v] = or_vertex_update(v, n, rowptr, colidx, outdeg, d, t, D, x);
            const double change = fabs(xn[v] - x[v]);
            l1 += change;
            if (change != 0.0 && change < eps) frozen[v] = 1;
        }
        memcpy(x, xn, (size_t)n * sizeof(double));
        ++k;
        if (tol > 0.0 && l1 < tol) break;
    }
    int64_t nf = 0;
    for (int64_t v = 0; v < n; ++v) nf += frozen[v];
    if (iters) *iters = k;
    if (resid) *resid = l1;
    if (frozen_out) *frozen_out = nf;
    free(outdeg);
    free(xn);
    free(frozen);
    return OR_OK;
}

/* The fixed point as a linear system.  Row v of M is
 *   M[v][v] += 1;  M[v][u] -= d * m(u,v) / outdeg(u)  for each edge u -> v
 *   M[v][a]  -= d / n for each dangling a          (when redistribute)
 * and b[v] = (1-d) * t(v).  Solved by Gaussian elimination with partial
 * pivoting (a textbook dense solve; the matrix is a nonsingular M-matrix). */
OR_API int or_dense_solve(int64_t n, const int64_t* rowptr, const int32_t* colidx, double d,
                          const double* t, int redistribute, double* x) {
    int rc = or_check_csr(n, rowptr, colidx);
    if (rc) return rc;
    if (n > 4096 || !(d >= 0.0 && d < 1.0)) return OR_BAD_ARG;
    int64_t* outdeg = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    double* M = (double*)calloc((size_t)(n * n), sizeof(double));
    double* b = (double*)malloc((size_t)n * sizeof(double));
    if (!outdeg || !M || !b) { free(outdeg); free(M); free(b); return OR_NO_MEM; }
    or_outdeg(n, rowptr, colidx, outdeg);
    for (int64_t v = 0; v < n; ++v) {
        M[v * n + v] += 1.0;
        for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
            int64_t u = colidx[e];
            M[v * n + u] -= d / (double)outdeg[u];
        }
        if (redistribute)
            for (int64_t a = 0; a < n; ++a)
                if (outdeg[a] == 0) M[v * n + a] -= d / (double)n;
        b[v] = (1.0 - d) * or_teleport(n, t, v);
    }
    /* forward elimination */
    for (int64_t k = 0; k < n; ++k) {
        int64_t p = k;
        for (int64_t i = k + 1; i < n; ++i)
            if (fabs(M[i * n + k]) > fabs(M[p * n + k])) p = i;
        if (M[p * n + k] == 0.0) { free(outdeg); free(M); free(b); return OR_SINGULAR; }
        if (p != k) {
            for (int64_t j = 0; j < n; ++j) {
                double tmp = M[k * n + j]; M[k * n + j] = M[p * n + j]; M[p * n + j] = tmp;
            }
            double tmp = b[k]; b[k] = b[p]; b[p] = tmp;
        }
        for (int64_t i = k + 1; i < n; ++i) {
            double f = M[i * n + k] / M[k * n + k];
            if (f == 0.0) continue;
            for (int64_t j = k; j < n; ++j) M[i * n + j] -= f * M[k * n + j];
            b[i] -= f * b[k];
        }
    }
    /* back substitution */
    for (int64_t i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int64_t j = i + 1; j < n; ++j) s -= M[i * n + j] * x[j];
        x[i] = s / M[i * n + i];
    }
    free(outdeg); free(M); free(b);
    return OR_OK;
}

/* Alg. 3 (No-Sync), simulated on one core.  The vertices are split into p
 * contiguous partitions of equal size (static allocation).  Thread i updates
 * its vertices in order, in place: the new value of u is computed from the
 * current ranks of its in-neighbours (whatever sweep they are in) and stored
 * at once -- there is no previous-iteration array and no barrier.  After a
 * sweep over its partition a thread counts one iteration, publishes its error
 * threadErr[i] (L1 = sum of |new - old| over its vertices when norm = 0, the
 * paper's max-abs when norm = 1) and stops when the combination of all
 * published errors (sum for L1, max for max-abs) is at most tol; errors are
 * initialised to +inf so that no thread stops before every thread has
 * published.
 *
 * Dangling share (the paper has none; see the file header).  Two forms with
 * the same fixed point:
 *   dangling_form = 0: d*D/n with D the running dangling mass, kept up to
 *                      date by adding each dangling vertex's change as it is
 *                      written;
 *   dangling_form = 1: d*(T - S)/n with T = sum(t) and S the running mass of
 *                      the vertices that do have out-edges, kept up to date
 *                      the same way.  At the fixed point sum(x) = T, so
 *                      T - S = D; away from it this form restores the total
 *                      mass that in-place updates lose or gain.
 *
 * Interleaving: threads run in rounds; in each round thread i performs
 * speed[i] vertex updates (speed NULL: 1 each), in thread order.  A thread that
 * has stopped does nothing.  The run ends when all threads have stopped or a
 * thread has done max_sweeps sweeps.
 *
 * Loop perforation (eps > 0): a vertex whose update changed its rank by a
 * nonzero amount below eps is frozen; its turn in later sweeps passes without
 * recomputing it (it keeps its rank, which still feeds its out-neighbours and
 * the shares, and adds nothing to its thread's error).  eps = 0 is plain
 * Alg. 3.
 *
 * Outputs: x (in place, initialised to t or x0), sweeps[p] (iterations per
 * thread), *updates (vertex updates actually computed), *est (the final
 * combined error), *frozen_out (vertices frozen at the end; may be NULL). */
OR_API int or_nosync(int64_t n, const int64_t* rowptr, const int32_t* colidx, double d,
                     const double* t, int redistribute, int dangling_form, int32_t p,
                     const int32_t* speed, int norm, double tol, int32_t max_sweeps,
                     const double* x0, double* x, int32_t* sweeps, int64_t* updates,
                     double* est, double eps, int64_t* frozen_out) {
    int rc = or_check_csr(n, rowptr, colidx);
    if (rc) return rc;
    if (p < 1 || p > n || !(d >= 0.0 && d < 1.0) || max_sweeps < 1 || !(eps >= 0.0)) return OR_BAD_ARG;
    if (dangling_form != 0 && dangling_form != 1) return OR_BAD_ARG;
    int64_t* outdeg = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    double* thread_err = (double*)malloc((size_t)p * sizeof(double));
    double* local_err = (double*)malloc((size_t)p * sizeof(double));
    int64_t* pos = (int64_t*)malloc((size_t)p * sizeof(int64_t));
    int* stopped = (int*)calloc((size_t)p, sizeof(int));
    unsigned char* frozen = (unsigned char*)calloc((size_t)n, 1);
    if (!outdeg || !thread_err || !local_err || !pos || !stopped || !frozen) {
        free(outdeg); free(thread_err); free(local_err); free(pos); free(stopped); free(frozen);
        return OR_NO_MEM;
    }
    or_outdeg(n, rowptr, colidx, outdeg);
    for (int64_t v = 0; v < n; ++v) x[v] = x0 ? x0[v] : or_teleport(n, t, v);
    double D = or_dangling_mass(n, outdeg, x);
    double T = 0.0, S = 0.0;
    for (int64_t v = 0; v < n; ++v) {
        T += or_teleport(n, t, v);
        if (outdeg[v] > 0) S += x[v];
    }
    for (int32_t i = 0; i < p; ++i) {
        thread_err[i] = INFINITY;
        local_err[i] = 0.0;
        sweeps[i] = 0;
    }
    /* partition i = [i*n/p, (i+1)*n/p) */
    for (int32_t i = 0; i < p; ++i) pos[i] = (int64_t)i * n / p;
    int64_t total_updates = 0;
    int running = p;
    int hit_budget = 0;
    double combined = INFINITY;
    while (running > 0 && !hit_budget) {
        for (int32_t i = 0; i < p && !hit_budget; ++i) {
            if (stopped[i]) continue;
            int64_t lo = (int64_t)i * n / p, hi = (int64_t)(i + 1) * n / p;
            int32_t steps = speed ? speed[i] : 1;
            for (int32_t s = 0; s < steps; ++s) {
                int64_t u = pos[i];
                double diff = 0.0;
                if (!frozen[u]) {
                    double previous = x[u];
                    double share = !redistribute ? 0.0 : (dangling_form == 1 ? T - S : D);
                    double tmp = or_vertex_update(u, n, rowptr, colidx, outdeg, d, t, share, x);
                    x[u] = tmp;
                    if (outdeg[u] == 0) D += tmp - previous;
                    else S += tmp - previous;
                    diff = fabs(tmp - previous);
                    if (diff != 0.0 && diff < eps) frozen[u] = 1;
                    ++total_updates;
                }
                if (norm == 0) local_err[i] += diff;
                else if (diff > local_err[i]) local_err[i] = diff;
                if (++pos[i] == hi) {                 /* end of a sweep */
                    pos[i] = lo;
                    sweeps[i] += 1;
                    thread_err[i] = local_err[i];
                    local_err[i] = 0.0;
                    combined = 0.0;
                    for (int32_t j = 0; j < p; ++j) {
                        if (norm == 0) combined += thread_err[j];
                        else if (thread_err[j] > combined) combined = thread_err[j];
                    }
                    if (combined <= tol) { stopped[i] = 1; --running; break; }
                    if (sweeps[i] >= max_sweeps) { hit_budget = 1; break; }
                }
            }
        }
    }
    if (updates) *updates = total_updates;
    if (est) *est = combined;
    if (frozen_out) {
        int64_t nf = 0;
        for (int64_t v = 0; v < n; ++v) nf += frozen[v];
        *frozen_out = nf;
    }
    free(outdeg); free(thread_err); free(local_err); free(pos); free(stopped); free(frozen);
    return OR_OK;
}

/* ------------------------------------------------------ weighted graphs -- */

/* W(u) = sum of w(e) over the edges e = (u, v), read from the in-edge CSR
 * (weights w[e] are aligned with colidx). */
OR_API int or_w_outweight(int64_t n, const int64_t* rowptr, const int32_t* colidx, const double* w,
                          double* W) {
    int rc = or_check_csr(n, rowptr, colidx);
    if (rc) return rc;
    for (int64_t u = 0; u < n; ++u) W[u] = 0.0;
    for (int64_t e = 0; e < rowptr[n]; ++e) {
        if (!(w[e] > 0.0)) return OR_BAD_ARG;
        W[colidx[e]] += w[e];
    }
    return OR_OK;
}

/* Alg. 1 on the weighted graph from x0 (default t) until the L1 change of an
 * iteration is below tol or max_iter iterations.  A vertex with W(u) = 0 is
 * dangling; its rank is spread uniformly. */
OR_API int or_w_jacobi(int64_t n, const int64_t* rowptr, const int32_t* colidx, const double* w, double d,
                       const double* t, double tol, int32_t max_iter, const double* x0, double* x,
                       int32_t* iterations, double* residual) {
    int rc = or_check_csr(n, rowptr, colidx);
    if (rc) return rc;
    if (!(d >= 0.0 && d < 1.0) || max_iter < 0) return OR_BAD_ARG;
    double* W = (double*)malloc((size_t)n * sizeof(double));
    double* xn = (double*)malloc((size_t)n * sizeof(double));
    if (!W || !xn) { free(W); free(xn); return OR_NO_MEM; }
    rc = or_w_outweight(n, rowptr, colidx, w, W);
    if (rc) { free(W); free(xn); return rc; }
    for (int64_t v = 0; v < n; ++v) x[v] = x0 ? x0[v] : or_teleport(n, t, v);
    int32_t it = 0;
    double r = INFINITY;
    while (it < max_iter) {
        double D = 0.0;
        for (int64_t u = 0; u < n; ++u)
            if (W[u] == 0.0) D += x[u];
        r = 0.0;
        for (int64_t v = 0; v < n; ++v) {
            double s = 0.0;
            for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
                int64_t u = colidx[e];
                s += x[u] * w[e] / W[u];
            }
            xn[v] = (1.0 - d) * or_teleport(n, t, v) + d * (s + D / (double)n);
            r += fabs(xn[v] - x[v]);
        }
        memcpy(x, xn, (size_t)n * sizeof(double));
        ++it;
        if (r < tol) break;
    }
    if (iterations) *iterations = it;
    if (residual) *residual = r;
    free(W);
    free(xn);
    return OR_OK;
}

/* One synchronous update of the adjoint (transposed) system from a given
 * lambda:
 *   lambda_out(u) = c(u) + d * ( sum_{(u,v)} P(u,v) lambda(v) + a(u) * sum(lambda)/n ),
 * the loop body of or_w_adjoint.  *l1 = ||lambda_out - lambda||_1, which bounds
 * the distance of lambda to the solution of M^T lambda = c by l1 / (1 - d)
 * (the transposed map is an L1 contraction with factor d as well). */
OR_API int or_w_adjoint_step(int64_t n, const int64_t* rowptr, const int32_t* colidx, const double* w,
                             double d, const double* c, const double* lambda, double* lambda_out,
                             double* l1) {
    int rc = or_check_csr(n, rowptr, colidx);
    if (rc) return rc;
    if (!(d >= 0.0 && d < 1.0) || !c || !lambda || !lambda_out) return OR_BAD_ARG;
    double* W = (double*)malloc((size_t)n * sizeof(double));
    double* mu = (double*)malloc((size_t)n * sizeof(double));
    if (!W || !mu) { free(W); free(mu); return OR_NO_MEM; }
    rc = or_w_outweight(n, rowptr, colidx, w, W);
    if (rc) { free(W); free(mu); return rc; }
    double L = 0.0;
    for (int64_t u = 0; u < n; ++u) {
        L += lambda[u];
        mu[u] = 0.0;
    }
    for (int64_t v = 0; v < n; ++v)
        for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
            int64_t u = colidx[e];
            mu[u] += w[e] / W[u] * lambda[v];
        }
    double r = 0.0;
    for (int64_t u = 0; u < n; ++u) {
        lambda_out[u] = c[u] + d * (mu[u] + (W[u] == 0.0 ? L / (double)n : 0.0));
        r += fabs(lambda_out[u] - lambda[u]);
    }
    if (l1) *l1 = r;
    free(W);
    free(mu);
    return OR_OK;
}

/* The adjoint of L = c^T x at the weighted fixed point x: lambda solves
 *   lambda(u) = c(u) + d * ( sum_{(u,v)} P(u,v) lambda(v) + a(u) * sum(lambda)/n ),
 * a(u) = 1 for dangling u (M^T lambda = c), iterated synchronously until the
 * L1 change is below tol * ||c||_1 or max_iter.  Outputs lambda, mu(u) =
 * sum_v P(u,v) lambda(v), dL/dt = (1-d) lambda, and dL/dw for every edge. */
OR_API int or_w_adjoint(int64_t n, const int64_t* rowptr, const int32_t* colidx, const double* w, double d,
                        const double* x, const double* c, double tol, int32_t max_iter, double* lambda,
                        double* mu, double* grad_t, double* grad_w, int32_t* iterations, double* residual) {
    int rc = or_check_csr(n, rowptr, colidx);
    if (rc) return rc;
    if (!(d >= 0.0 && d < 1.0) || max_iter < 0) return OR_BAD_ARG;
    double* W = (double*)malloc((size_t)n * sizeof(double));
    double* ln = (double*)malloc((size_t)n * sizeof(double));
    if (!W || !ln) { free(W); free(ln); return OR_NO_MEM; }
    rc = or_w_outweight(n, rowptr, colidx, w, W);
    if (rc) { free(W); free(ln); return rc; }
    double cnorm = 0.0;
    for (int64_t u = 0; u < n; ++u) {
        lambda[u] = c[u];
        cnorm += fabs(c[u]);
    }
    int32_t it = 0;
    double r = INFINITY;
    while (it < max_iter) {
        double L = 0.0;
        for (int64_t u = 0; u < n; ++u) L += lambda[u];
        for (int64_t u = 0; u < n; ++u) mu[u] = 0.0;
        /* the in-edge (u, v) of row v pushes P(u,v) lambda(v) to u */
        for (int64_t v = 0; v < n; ++v)
            for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
                int64_t u = colidx[e];
                mu[u] += w[e] / W[u] * lambda[v];
            }
        r = 0.0;
        for (int64_t u = 0; u < n; ++u) {
            ln[u] = c[u] + d * (mu[u] + (W[u] == 0.0 ? L / (double)n : 0.0));
            r += fabs(ln[u] - lambda[u]);
        }
        memcpy(lambda, ln, (size_t)n * sizeof(double));
        ++it;
        if (r < tol * cnorm) break;
    }
    /* mu of the final lambda, then the gradients */
    for (int64_t u = 0; u < n; ++u) mu[u] = 0.0;
    for (int64_t v = 0; v < n; ++v)
        for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
            int64_t u = colidx[e];
            mu[u] += w[e] / W[u] * lambda[v];
        }
    for (int64_t u = 0; u < n; ++u) grad_t[u] = (1.0 - d) * lambda[u];
    for (int64_t v = 0; v < n; ++v)
        for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
            int64_t u = colidx[e];
            grad_w[e] = d * x[u] / W[u] * (lambda[v] - mu[u]);
        }
    if (iterations) *iterations = it;
    if (residual) *residual = r;
    free(W);
    free(ln);
    return OR_OK;
}
