/*
 * pagerank.h -- C ABI of the GB300 (sm_103a) PageRank library.
 *
 * The library computes the PageRank vector of a directed graph given as CSR:
 *
 *   Eq. 1:  x(v) = (1-d) t(v) + d * ( sum_{(u,v) in E} x(u)/outdeg(u) + D/n )
 *
 * where t is the teleport vector (uniform 1/n unless given), D is the rank
 * held by dangling vertices (outdeg 0), spread uniformly over all n vertices,
 * and a repeated edge counts with its multiplicity.  Eq. 1 of the paper has
 * t = 1/n and no dangling term; the dangling share is this library's reading
 * (mass is conserved: sum(x) = sum(t)).
 *
 * Three solvers run the same update:
 *   PR_JACOBI       the synchronous iteration of Alg. 1 (Barrier baseline):
 *                   every vertex is recomputed from the previous vector, the
 *                   dangling mass and the L1 change ||x_k - x_{k-1}||_1 are
 *                   reduced in the same pass, and the loop stops when that
 *                   change is below tol or after max_iter iterations.
 *   PR_NONBLOCKING  the barrier-free form of Alg. 3 (No-Sync): one persistent
 *                   launch in which warps update ranks in place, with no grid
 *                   synchronisation and no previous-iteration array; each
 *                   block stops on its own view of the global change
 *                   (thread-level convergence, Section 4.3) once it is below
 *                   4 tol.  The result is then verified with one synchronous
 *                   update, whose L1 change is the reported residual; if it
 *                   is not below tol, the persistent launch resumes with a
 *                   4x tighter internal tolerance, within the budget.
 *   PR_EDGE         the edge-centric synchronous iteration of Alg. 2
 *                   (Barriers-Edge), for comparison: each iteration first
 *                   pushes every source's rank/outdeg into a per-edge array
 *                   along its out-edges, then sums each vertex's in-edge slots;
 *                   same iterates as PR_JACOBI up to rounding, more bytes per
 *                   edge.  32-bit row offsets only (else PR_ERR_UNSUPPORTED);
 *                   its out-edge list (8 bytes per edge) and per-edge array
 *                   (4 bytes per edge) are allocated on first use.
 *
 * Conventions
 *   - All functions return a pr_status.  No function aborts or exits; on an
 *     error the thread-local message from pr_last_error() says what failed.
 *   - Vertex ids are 0..n-1, int32 (n <= 2^31-1).  Row offsets may be int32
 *     or int64; the edge count may exceed 2^31 only with int64 offsets.
 *   - Pointers marked "host or device" are classified with
 *     cudaPointerGetAttributes; host memory (pinned or pageable) is copied
 *     in or out by the call, device memory is used in place.
 *   - Work is enqueued on the given CUDA stream (NULL = the legacy default
 *     stream).  Calls that fill a pr_info synchronise that stream before
 *     returning; calls that do not are asynchronous with respect to the host.
 *   - A pr_graph belongs to the device that was current when it was created;
 *     use it with that device current.  One pr_graph must not be used by two
 *     host threads at the same time.
 */
#ifndef PAGERANK_GB300_H
#define PAGERANK_GB300_H

#include <stdint.h>

#if defined(__GNUC__)
#define PR_API __attribute__((visibility("default")))
#else
#define PR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pr_graph pr_graph; /* opaque; owned by the library */
typedef struct pr_wgraph pr_wgraph; /* opaque weighted graph of the adjoint path */

typedef enum pr_status {
    PR_OK = 0,
    PR_ERR_INVALID_ARG = 1,    /* a bad argument; nothing was changed           */
    PR_ERR_CUDA = 2,           /* a CUDA call failed (message in pr_last_error)  */
    PR_ERR_OOM = 3,            /* device or pinned memory could not be obtained  */
    PR_NOT_CONVERGED = 4,      /* max_iter reached; outputs are still written    */
    PR_ERR_UNSUPPORTED = 5,    /* a valid request this build does not implement  */
    PR_ERR_INVALID_GRAPH = 6,  /* rowptr/colidx failed validation on the device  */
    PR_ERR_DEVICE_TIMEOUT = 7  /* a bounded device-side wait gave up             */
} pr_status;

/* layout argument of pr_create_graph */
#define PR_IN_CSR 0  /* rows are destinations: row v lists the sources u of u -> v */
#define PR_OUT_CSR 1 /* rows are sources: row u lists the destinations v of u -> v */

/* variant argument of pr_solve */
#define PR_JACOBI 0
#define PR_NONBLOCKING 1
#define PR_EDGE 2

typedef struct pr_info {
    int32_t iterations;    /* Jacobi: iterations run.  Non-blocking: the largest
                              number of sweeps any block made, summed over
                              launches, plus the verifying update.            */
    int32_t converged;     /* 1 if the stopping test was met                  */
    double residual_l1;    /* L1 change of the last synchronous update         */
    double sum_x;          /* sum of the final vector before renormalisation   */
    double dangling_mass;  /* dangling mass of the final vector (before any
                              renormalisation)                                 */
    double edge_visits;    /* edges gathered in total (GTEPS numerator)        */
    float ms_device;       /* device time of the call's work, CUDA events      */
    int32_t launches;      /* kernel launches the call enqueued                */
    double loop_edge_visits; /* edges gathered inside the iteration loop alone:
                              Jacobi, every iteration; non-blocking, the sweeps
                              of the persistent launches (not the verifying
                              updates)                                        */
    float ms_loop;         /* device time of that loop alone (CUDA events on
                              the call's stream around the while-graph or the
                              host-driven iterations, or around each
                              persistent launch, summed)                      */
    int32_t frozen_rows;   /* rows frozen by loop perforation at the end of
                              the solve (PR_OPT_PERFORATION); 0 otherwise     */
} pr_info;

typedef struct pr_graph_stats {
    int64_t n;             /* vertices                                         */
    int64_t nnz;           /* edges (with multiplicity)                        */
    int64_t n_dangling;    /* vertices without out-edges                       */
    int64_t n_zero_indeg;  /* vertices without in-edges                        */
    int64_t n_heavy;       /* rows gathered in segments by whole warps         */
    int64_t n_segments;    /* edge segments of those rows                      */
    int64_t n_tiles;       /* row tiles of the per-iteration gather kernel     */
    int64_t max_indeg;
    int32_t rowptr_bytes;  /* 4 or 8: width of the row offsets kept on device  */
    int32_t sm_count;
    int64_t device_bytes;  /* device memory owned by the graph                 */
    float setup_ms;        /* device time of pr_create_graph's kernels         */
    int64_t n_tma_tiles;   /* tiles of the pipelined synchronous row kernel (0:
                              the layout cannot use it; see PR_OPT_TMA_TILES)   */
    int64_t hub_prefix_edges; /* edges whose source is among the first 49,152
                              vertices of the binned order, the hub prefix the
                              synchronous gathers read through L1 by default
                              (the other gathers are L1 misses)             */
    int64_t n_isolated;    /* vertices without in- and out-edges (the last
                              rows of the binned order)                       */
} pr_graph_stats;

/* Build a graph on the current device.
 *   n, nnz        vertex and edge counts (n >= 1, nnz >= 0).
 *   rowptr        host or device, n+1 offsets, int64 if rowptr_is_64 else
 *                 int32; rowptr[0] = 0, non-decreasing, rowptr[n] = nnz.
 *   colidx        host or device, nnz int32 vertex ids in [0, n).
 *   weights       must be NULL: a weighted graph is its own object
 *                 (pr_create_wgraph below), whose weighted forward and
 *                 adjoint solvers keep both edge directions.  Non-NULL
 *                 returns PR_ERR_UNSUPPORTED.
 *   layout        PR_IN_CSR: row v lists the sources u of the edges u -> v
 *                 (the CSR input of Alg. 1, "G = ConvertCsr(V,E)" in Alg.
 *                 2/3, read as in-links).  PR_OUT_CSR: row u lists the
 *                 targets v of the edges u -> v; the library transposes it
 *                 on the device (a stable sort of the edges by target, so
 *                 every in-row lists its sources in increasing order) and
 *                 then proceeds as for PR_IN_CSR; needs nnz < 2^31
 *                 (else PR_ERR_UNSUPPORTED) and about 21 bytes of device
 *                 scratch per edge during the call.
 *   stream        CUDA stream for the copies and set-up kernels.
 *   out           receives the new graph; *out is NULL on failure.
 * The library copies the arrays into memory it owns; the caller may free or
 * reuse them when the call returns.  Validation runs on the device: a
 * malformed CSR returns PR_ERR_INVALID_GRAPH.  The call synchronises the
 * stream.  Set-up computes out-degrees, bins rows by in-degree and relabels
 * vertices so that each bin is a contiguous range (outputs are always in the
 * caller's vertex order). */
PR_API pr_status pr_create_graph(int64_t n, int64_t nnz, const void* rowptr, int rowptr_is_64,
                                 const int32_t* colidx, const float* weights, int layout,
                                 void* stream, pr_graph** out);

/* Free a graph and all device memory it owns.  NULL is accepted.  The call
 * first waits for the device to finish all work (as cudaFree does); the
 * memory goes back to the library's per-device pool, where the next
 * pr_create_graph finds it without mapping new pages. */
PR_API pr_status pr_destroy_graph(pr_graph* g);

/* Return the device memory the library's pool on the current device keeps
 * for reuse (memory freed by pr_destroy_graph and set-up scratch) to the
 * system.  Graphs still alive keep theirs. */
PR_API pr_status pr_trim_memory(void);

/* Solve for the PageRank vector (Eq. 1 with the uniform dangling share).
 *   damping       d, 0 <= d < 1 (the paper uses 0.85, Section 1).
 *   tol           > 0: stop when ||x_k - x_{k-1}||_1 < tol (the paper's
 *                 threshold, Alg. 1, compared in L1 rather than max-abs).
 *   max_iter      >= 1: iteration budget (sweep budget for PR_NONBLOCKING).
 *   variant       PR_JACOBI, PR_NONBLOCKING or PR_EDGE.
 *   teleport      host or device, n floats >= 0, or NULL for uniform 1/n.
 *   x0            host or device, n floats (warm start), or NULL for x0 = t.
 *   x_out         host or device, n floats: the result, rescaled in FP64 so
 *                 that sum(x_out) = sum(teleport) (1 when uniform).
 *   info          may be NULL; filled after the stream is synchronised.
 * Returns PR_OK, or PR_NOT_CONVERGED when the budget ran out (x_out and info
 * are written in both cases); PR_ERR_DEVICE_TIMEOUT if a bounded wait of the
 * pipelined row kernel gave up (see PR_OPT_TEST_WITHHOLD_COPY). */
PR_API pr_status pr_solve(pr_graph* g, float damping, double tol, int32_t max_iter, int variant,
                          const float* teleport, const float* x0, float* x_out, pr_info* info,
                          void* stream);

/* Run exactly n_iter synchronous updates (the loop body of Alg. 1) from x_in,
 * with no stopping test and no renormalisation.
 *   x_in, x_out   host or device, n floats each (may be the same buffer).
 *   teleport      as in pr_solve.
 *   info          may be NULL; residual_l1 is the L1 change of the last
 *                 update and dangling_mass the dangling mass of x_out.
 * n_iter >= 1. */
PR_API pr_status pr_iterate(pr_graph* g, float damping, const float* teleport, const float* x_in,
                            int32_t n_iter, float* x_out, pr_info* info, void* stream);

/* Fill *stats with the graph's sizes and set-up figures. */
PR_API pr_status pr_graph_get_stats(const pr_graph* g, pr_graph_stats* stats);

/* Tuning knobs, mostly for tests that force one code path at a time.
 *   PR_OPT_HEAVY_DEGREE   rows with in-degree >= value are gathered in
 *                         segments (a power of two in [64, 4096]; default
 *                         256).  Takes effect at the next pr_create_graph
 *                         of the same thread (it changes the layout), so it
 *                         is a thread-local default, set with g = NULL.  The
 *                         barrier-free kernel gathers in segments only the
 *                         rows of in-degree >= max(value, 1024) and works
 *                         the others as light rows.
 *   PR_OPT_USE_GRAPH      1 (default): the Jacobi loop runs as one CUDA
 *                         graph with a conditional while node; 0: the host
 *                         enqueues iterations in chunks.
 *   PR_OPT_CTAS_PER_SM    blocks per SM of the persistent kernels (0 =
 *                         from occupancy, else 1..8).
 *   PR_OPT_HOT_VERTICES   L1 policy of the rank gathers: bits 0..27 count
 *                         the first vertices in the library's degree order
 *                         (the hubs); bits 28..31 pick the policy: 0 every
 *                         gather is a plain cached load; 1/2/3 the hubs use
 *                         L1 evict_last and the others plain / evict_first /
 *                         no L1 allocation; 4 (default, with 49152 hubs) the
 *                         hubs are plain cached loads and all others are read
 *                         from L2 only, so they cannot evict the hubs.
 *   PR_OPT_NB_PIPELINE    barrier-free solver (PR_NONBLOCKING): 1 feeds its
 *                         light-row tiles through shared memory
 *                         like the pipelined synchronous kernel (a producer
 *                         warp bulk-copies each tile's row offsets, column
 *                         indices, 1/outdeg and teleport ahead of the
 *                         gathering warps; x and y are read in place as
 *                         before); 0 (default; measured faster): every
 *                         gathering warp loads them itself.
 *                         Needs 32-bit offsets and PR_OPT_TMA_TILES; not used
 *                         with PR_OPT_PERFORATION, PR_OPT_NB_HUBS, the staged
 *                         tiles or the diagnostics form.
 *   PR_OPT_TMA_HOT_VERTICES the hub count of the pipelined row kernel
 *                         (PR_OPT_TMA_TILES), at most PR_OPT_HOT_VERTICES' own:
 *                         the shared-memory stages of its three blocks per SM
 *                         take 132 KB of the SM's SRAM, so its L1 holds fewer
 *                         hub ranks than the other kernels' (default 16384;
 *                         0 = PR_OPT_HOT_VERTICES' count).
 *   PR_OPT_HOT_CACHE      vertices at the front of the library's degree
 *                         order whose quotient values each block of the
 *                         synchronous kernels copies into shared memory and
 *                         gathers from there (0..40960, default 0: off --
 *                         measured slower than letting L1 cache them).
 *   PR_OPT_STAGED_TILES   how the light row tiles are gathered, bit 0 for the
 *                         synchronous kernels, bit 1 for the barrier-free
 *                         kernel: 0 = row by row (groups of lanes per row,
 *                         two rows in flight per group; gathers through L1
 *                         can hit the hub ranks), 1 = edge-parallel (the
 *                         whole block issues every gather of the tile at
 *                         once into a 24.6 KB shared-memory staging area,
 *                         then reduces row by row).  Values 0..3.
 *   PR_OPT_NB_HUBS        vertices at the front of the library's degree order
 *                         (the hubs) whose ranks each block of the
 *                         barrier-free kernel gathers from a shared-memory
 *                         snapshot, re-read every few tiles, instead of from
 *                         L2 (0..8192, rounded down to a multiple of 4;
 *                         default 0).  Measured slower than
 *                         PR_OPT_NB_L1_HUBS, which it takes precedence over.
 *   PR_OPT_NB_L1_HUBS     vertices at the front of the degree order whose ranks
 *                         the barrier-free kernel gathers with weak loads that
 *                         L1 may serve (default 49152; 0 = every gather is a
 *                         relaxed gpu-scope load served by L2).  Each block
 *                         issues fence.acq_rel.gpu at the start of a sweep, so
 *                         a cached hub rank is at most about one sweep old --
 *                         a bounded delay, which the asynchronous iteration
 *                         allows.  Under the PTX memory model these weak reads
 *                         race with the owners' relaxed writes; the value read
 *                         is an old or a new rank (aligned 32-bit accesses),
 *                         and the verifying synchronous update certifies the
 *                         result either way.  Set 0 for a race-free run.
 *   PR_OPT_BATCH_BF16     batched solver only: 0 (default) keeps the quotient
 *                         matrix Y in FP32; m in 1..8 also keeps a BF16 copy
 *                         and gathers from it (half the bytes per gathered
 *                         row, FP32 accumulation) until every active column's
 *                         L1 change is below 10^-m, then gathers from the FP32
 *                         copy to the end.  X stays FP32 throughout, so the
 *                         result meets the same tol; BF16's 2^-9 rounding
 *                         limits how far the BF16 phase can go (m ~ 2..3).
 *   PR_OPT_BATCH_DC       batched solver only: 0 (default) off; M in 1..32
 *                         runs BF16 storage by defect correction instead:
 *                         every FP32 step X' = F(X) (whose L1 change per
 *                         column is the stopping test, as in the plain form)
 *                         is followed by M sweeps delta <- r + A delta on the
 *                         error equation, r = X' - X, gathering delta / outdeg
 *                         from a BF16 copy (FP32 sums), and X <- X + delta.
 *                         BF16 rounds the correction, not the ranks, so the
 *                         columns reach the same tol.  info.iterations counts
 *                         the FP32 steps; edge_visits counts both kinds of
 *                         sweep.  Takes precedence over PR_OPT_BATCH_BF16; a
 *                         host-driven loop (no CUDA graph).
 *   PR_OPT_BATCH_ASYNC    batched solver: 1 (default) gathers the rows of a
 *                         32-edge window into shared memory with asynchronous
 *                         copies while the previous window is summed (64 rows
 *                         in flight per warp); 0 loads them into registers
 *                         (16 or 32 rows per warp).  Same sums, same order.
 *   PR_OPT_SYNC_DC        synchronous solver (PR_JACOBI): BF16 storage of the
 *                         quotient vector by defect correction.  0 (default)
 *                         off; M in 1..32: after each FP32 step x' = F(x)
 *                         (Eq. 1; its L1 change is the stopping test, so the
 *                         result is an FP32 iterate) the error e = x* - x is
 *                         approximated by M sweeps delta <- r + d (P^T delta +
 *                         L/n) from delta = r = x' - x, each gathering
 *                         delta/outdeg from a BF16 copy (FP32 sums); L, the
 *                         mass the rounded quotients do not pass on (dangling
 *                         rows and rounding), keeps every sweep mass-
 *                         conserving; then x <- x + delta.  iterations counts
 *                         the FP32 steps, edge_visits both kinds of sweep.
 *                         A host-driven loop (no CUDA graph); not with
 *                         PR_OPT_PERFORATION or PR_EDGE.
 *   PR_OPT_IMPLICIT_ZERO_ROWS the batched solver's FP32 form and the
 *                         synchronous solver's pipelined row kernel (PR_JACOBI,
 *                         pr_iterate; PR_OPT_TMA_TILES, not with
 *                         PR_OPT_FUSED_SEGMENTS): 1 (default) keeps the ranks
 *                         of rows without in-edges implicit after the first
 *                         iteration.  By Eq. 1 such a row's rank is
 *                         (1-d) t_v + d D/n, where D is the column's dangling
 *                         mass, so the update writes only the quotient rank /
 *                         outdeg of those with out-edges and nothing for
 *                         isolated vertices; their L1 change, n_z d |D - D'|/n
 *                         over the n_z such rows, and the isolated vertices'
 *                         share of the next dangling mass are added in FP64,
 *                         and their ranks are written once after the loop.
 *                         Same iterates and quotients up to the rounding of
 *                         the dangling mass; 0 updates every row every
 *                         iteration.  Not used by PR_OPT_BATCH_BF16 or
 *                         PR_OPT_BATCH_DC.
 *   PR_OPT_PERFORATION    loop perforation (Alg. 5) in the synchronous solver
 *                         (PR_JACOBI, pr_iterate) and in the barrier-free one
 *                         (PR_NONBLOCKING: the paper's No-Sync-Opt, Section
 *                         4): 0 (default) off; m in 1..30 freezes a vertex
 *                         once an update changes its rank by a nonzero amount
 *                         below 10^-m -- it is no longer recomputed (its rank
 *                         still feeds its out-neighbours and the dangling
 *                         mass).  An approximation: the result differs from
 *                         the fixed point by more than the contraction bound
 *                         of the residual; frozen rows count as changes of 0
 *                         in the residual, also in the barrier-free solver's
 *                         verifying synchronous update.  pr_info.frozen_rows
 *                         reports how many rows froze.  Row-by-row tiles only
 *                         (PR_OPT_STAGED_TILES is ignored); in the
 *                         barrier-free solver not together with
 *                         PR_OPT_NB_FAIL_AFTER or PR_TRACE_NB
 *                         (PR_ERR_UNSUPPORTED).
 *   PR_OPT_DYNAMIC_TILES  synchronous solver: 0 (default) each block owns a
 *                         fixed round-robin share of the row tiles; 1 blocks
 *                         take tiles from a shared counter, so a slow block's
 *                         work is taken over by the others (the GPU form of
 *                         Barrier-Helper, Alg. 6).
 *   PR_OPT_DELAY_NS       synchronous solver, for experiments: block 0 sleeps
 *                         this many nanoseconds (0..1e6, __nanosleep, bounded)
 *                         before taking each tile -- a slowed processor, as
 *                         in the paper's delayed-thread experiments.  0 = off.
 *   PR_OPT_TMA_TILES      synchronous solver: 1 (default) runs the pipelined
 *                         row kernel where it applies (32-bit row offsets,
 *                         heavy threshold <= 2048, static tile order, no
 *                         perforation, staging or shared-memory copy of y):
 *                         a producer warp copies each tile's offsets, column
 *                         indices and per-row vectors into shared memory with
 *                         bulk asynchronous copies ahead of the gathering
 *                         warps.  0 = the row-by-row kernel that loads them
 *                         itself.  Same arithmetic either way.
 *   PR_OPT_TEST_WITHHOLD_COPY  test hook of the pipelined row kernel's
 *                         bounded waits: k > 0 makes block 0's producer announce
 *                         its k-th tile of each launch without copying it, so
 *                         the gathering warps' wait for that tile gives up after
 *                         about one second and the solve returns
 *                         PR_ERR_DEVICE_TIMEOUT (nothing faults; the graph and
 *                         the context stay usable).  0 (default) = off.
 *   PR_OPT_NB_FAIL_AFTER  barrier-free solver, for experiments: s > 0 makes
 *                         block 0 of the first persistent launch of each solve
 *                         stop after s sweeps -- the paper's failing thread
 *                         (Fig. 9) -- and take itself out of the other blocks'
 *                         stopping test.  The verifying synchronous update
 *                         then sees its stale rows and the solve resumes with
 *                         every block, so the result still meets tol (more
 *                         sweeps, two launches).  0 (default) = off.
 *   PR_OPT_LIGHT_LANES    lanes per row of the light-row tiles of every
 *                         solver: 1 (default) by the tile's row count, so that
 *                         a block covers a tile in one pass of two rows per
 *                         lane group where it can and each lane walks its
 *                         rows' edges four at a time; 0 by degree class
 *                         (2^min(k,5) lanes for degrees in [2^k, 2^(k+1))).
 *                         Changes the summation order only.
 *   PR_OPT_FUSED_SEGMENTS synchronous solver with the pipelined row kernel:
 *                         1 gathers the 2048-edge segments of the heavy rows
 *                         as tiles of that same kernel, interleaved with the
 *                         light-row tiles, one launch per iteration (the
 *                         block that gathers a heavy row's last segment
 *                         updates the row); 0 (default) runs them as a
 *                         separate kernel first.  On R-MAT-24 the fused form
 *                         measured 2.26 ms per iteration against 0.89: every
 *                         2048-edge segment then costs a whole block a
 *                         pipeline round trip.  Changes the summation order
 *                         of a segment only.
 *   PR_OPT_INDEX64        1: keep 64-bit row offsets on the device even when
 *                         the edge count fits 32 bits (thread-local default
 *                         for the next pr_create_graph, set with g = NULL;
 *                         0 restores the automatic choice).
 * Unknown keys or values out of range return PR_ERR_INVALID_ARG. */
#define PR_OPT_HEAVY_DEGREE 1
#define PR_OPT_USE_GRAPH 2
#define PR_OPT_CTAS_PER_SM 3
#define PR_OPT_INDEX64 4
#define PR_OPT_HOT_VERTICES 5
#define PR_OPT_HOT_CACHE 6
#define PR_OPT_STAGED_TILES 7
#define PR_OPT_NB_HUBS 8
#define PR_OPT_NB_L1_HUBS 9
#define PR_OPT_BATCH_BF16 10
#define PR_OPT_PERFORATION 11
#define PR_OPT_DYNAMIC_TILES 12
#define PR_OPT_DELAY_NS 13
#define PR_OPT_TMA_TILES 14
#define PR_OPT_TEST_WITHHOLD_COPY 15
#define PR_OPT_NB_FAIL_AFTER 16
#define PR_OPT_LIGHT_LANES 17
#define PR_OPT_BATCH_DC 18
#define PR_OPT_FUSED_SEGMENTS 19
#define PR_OPT_BATCH_ASYNC 20
#define PR_OPT_IMPLICIT_ZERO_ROWS 21
#define PR_OPT_SYNC_DC 22
#define PR_OPT_TMA_HOT_VERTICES 23
#define PR_OPT_NB_PIPELINE 24
PR_API pr_status pr_set_option(pr_graph* g, int key, int64_t value);

/* Batched personalised PageRank: k independent solves on one graph, one per
 * teleport vector (column), computed together as a sparse-times-dense
 * product (each gathered edge moves a whole row of k ranks).  Column j is the
 * fixed point of Eq. 1 with teleport t_j (the dangling mass of column j is
 * still spread uniformly, so sum(x_j) = sum(t_j)), iterated synchronously
 * (Alg. 1) until its L1 change is below tol; a converged column is frozen
 * (its residual mask bit cleared) while the others continue, and the loop
 * ends when every column is frozen or after max_iter iterations.  Each
 * column is finally rescaled to sum(t_j) in FP64.
 *   k              1 <= k <= 32 columns (rows are stored 32 wide on the
 *                  device whatever k is).
 *   teleport       host or device, n x k floats, row-major in the caller's
 *                  vertex order (row v holds t_0(v) .. t_{k-1}(v)), each
 *                  column non-negative with a positive sum; NULL = every
 *                  column uniform 1/n.  Only the nonzeros are kept on the
 *                  device.
 *   x_out          host or device, n x k floats, row-major, caller's order.
 *   col_residual   NULL or host array of k doubles: the last L1 change of
 *                  each column.
 *   col_iterations NULL or host array of k int32: iterations each column
 *                  ran before it was frozen (or max_iter).
 * info->iterations is the largest column count; info->converged is 1 only if
 * every column converged; info->residual_l1 is the largest column residual;
 * info->edge_visits counts edges x iterations (each visit moves k ranks).
 * Returns PR_NOT_CONVERGED (outputs still written) if a column did not
 * converge. */
PR_API pr_status pr_solve_batched(pr_graph* g, float damping, double tol, int32_t max_iter,
                                  int32_t k, const float* teleport, float* x_out,
                                  double* col_residual, int32_t* col_iterations, pr_info* info,
                                  void* stream);

/* Many independent graphs solved together.  Build one pr_graph from the
 * block-diagonal CSR of `count` graphs -- graph i owns the caller ids
 * [offsets[i], offsets[i+1]) and no edge joins two graphs -- then declare the
 * partition once:
 *   offsets    host, count+1 int64, offsets[0] = 0, strictly increasing,
 *              offsets[count] = n (every graph has at least one vertex).
 *   count      1 .. 2^20.
 * The partition is checked on the device: an edge between two graphs returns
 * PR_ERR_INVALID_GRAPH (and no partition is kept).  A new call replaces the
 * previous partition.  Synchronises `stream`. */
PR_API pr_status pr_graph_set_partition(pr_graph* g, int32_t count, const int64_t* offsets,
                                        void* stream);

/* PageRank of every graph of the partition (Eq. 1 per graph: teleport 1/n_i,
 * graph i's dangling mass spread over graph i only), by the synchronous
 * iteration of Alg. 1 run on all graphs at once -- each launch covers every
 * graph and the whole loop is one CUDA graph launch.  Graph i stops, and is
 * frozen, when its own L1 change falls below tol; the loop ends when all are
 * frozen or after max_iter iterations.  Each graph's ranks are rescaled to
 * sum 1 in FP64.
 *   x_out            host or device, n floats, caller's vertex order.
 *   graph_residual   NULL or host array of count doubles: last L1 change.
 *   graph_iterations NULL or host array of count int32: iterations run.
 * info->iterations is the largest count, info->converged is 1 only if every
 * graph converged, info->residual_l1 the largest residual, and
 * info->edge_visits = iterations x nnz (frozen graphs' rows are copied, not
 * gathered, after they stop).  Returns PR_NOT_CONVERGED (outputs written) if
 * some graph did not converge. */
PR_API pr_status pr_solve_set(pr_graph* g, float damping, double tol, int32_t max_iter, float* x_out,
                              double* graph_residual, int32_t* graph_iterations, pr_info* info,
                              void* stream);

/* Weighted graphs and the adjoint (gradients through the fixed point).
 *
 * Edge e = (u, v) carries a weight w(e) > 0; the transition probability is
 * P(u, v) = w(e) / W(u) with W(u) the sum of u's out-weights (the weights are
 * row-normalised), and a vertex without out-edges is dangling.  The forward
 * problem is Eq. 1 on P with teleport t: M x = (1-d) t, M = I - d P^T -
 * (d/n) 1 a^T.  For a loss L(x) with gradient c = dL/dx, implicit
 * differentiation of the fixed point gives M^T lambda = c and
 *   dL/dt(u)  = (1-d) lambda(u),
 *   dL/dw(e)  = d x(u) / W(u) * (lambda(v) - sum_v' P(u, v') lambda(v')).
 * The transposed system is solved by the synchronous iteration along the
 * out-edges (the forward "push"); the library keeps an out-edge CSR for it.
 * Vertices keep the caller's order (no relabelling).
 *
 * pr_create_wgraph: n, nnz as for pr_create_graph; rowptr int64 [n+1] and
 *   colidx int32 [nnz] (host or device) give the in-edge CSR, weights [nnz]
 *   (host or device) are aligned with colidx.  nnz < 2^31.  Validation is on
 *   the host (PR_ERR_INVALID_GRAPH); a weight that is not positive and finite
 *   returns PR_ERR_INVALID_ARG.  Synchronises `stream`. */
PR_API pr_status pr_create_wgraph(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                                  const float* weights, void* stream, pr_wgraph** out);
PR_API pr_status pr_destroy_wgraph(pr_wgraph* g);

/* Replace the edge weights (host or device, nnz floats aligned with colidx);
 * the structure is kept.  Synchronises `stream`. */
PR_API pr_status pr_wgraph_set_weights(pr_wgraph* g, const float* weights, void* stream);

/* The weighted PageRank vector: Alg. 1 on P from x0 = t until the L1 change
 * is below tol or max_iter, then rescaled to sum(t) in FP64 (so the result
 * is a linear function of t).  teleport: host or device, n floats, or NULL
 * for 1/n.  x_out: host or device, n floats.  Fills info like pr_solve. */
PR_API pr_status pr_solve_weighted(pr_wgraph* g, float damping, double tol, int32_t max_iter,
                                   const float* teleport, float* x_out, pr_info* info, void* stream);

/* Gradients of a loss L on the weighted PageRank vector x (the output of
 * pr_solve_weighted with the same damping):
 *   x, dL_dx         host or device, n floats;
 *   dL_dteleport     NULL or host or device, n floats;
 *   dL_dweights      NULL or host or device, nnz floats aligned with colidx.
 * lambda is iterated from c until its L1 change is below tol * ||c||_1 or
 * max_iter (PR_NOT_CONVERGED, outputs still written).  info->iterations are
 * the adjoint iterations, info->residual_l1 the last L1 change of lambda. */
PR_API pr_status pr_adjoint(pr_wgraph* g, float damping, double tol, int32_t max_iter, const float* x,
                            const float* dL_dx, float* dL_dteleport, float* dL_dweights, pr_info* info,
                            void* stream);

/* One synchronous PageRank update that allocates no memory -- for callers
 * that cannot call cudaMalloc (or anything that allocates) where they need an
 * update: code running inside a fixed memory pool or arena, under another
 * framework's allocator, or in a latency-bound loop where an allocation may
 * not happen.  The paper has no counterpart; it is a deployment convenience.
 *
 * It works directly on the caller's plain in-edge CSR (no pr_graph, no
 * relabelling) and computes
 *   x_out(v) = (1-d)/n + d * ( sum_{(u,v) in E} x_in(u) * inv_outdeg(u) + D/n )
 * with D the dangling mass of x_in (the vertices with inv_outdeg = 0).
 *   n            1 <= n <= 16,777,216 (the fixed scratch holds 8192 blocks of
 *                2048 rows); larger n returns PR_ERR_INVALID_ARG.
 *   rowptr       device, n+1 int32 offsets; colidx device, int32 sources.
 *   inv_outdeg   device, n floats: 1/outdeg(u), or 0 for dangling u.
 *   x_in, x_out  device, n floats each; the two ranges must not overlap
 *                (any shared element returns PR_ERR_INVALID_ARG).
 *   sums_out     device, 3 doubles: [0] dangling mass of x_in, [1] dangling
 *                mass of x_out, [2] ||x_out - x_in||_1.
 * The call is asynchronous on `stream` and does not validate the CSR.
 * Scratch lives in one fixed device array (about 128 KiB) that the library
 * keeps on every GPU that loads it, until the process exits; all calls share
 * it, so calls that overlap on the GPU race -- serialise them.  Every call
 * looks up that array's address on the current device (cudaGetSymbolAddress,
 * which allocates nothing), so a cudaDeviceReset between calls is safe; the
 * first call on a device, and the first after a reset, loads the module:
 * make it before any stream capture. */
PR_API pr_status pr_step_noalloc(int64_t n, const int32_t* rowptr, const int32_t* colidx,
                                 const float* inv_outdeg, float damping, const float* x_in,
                                 float* x_out, double* sums_out, void* stream);

/* ---- Diagnostics: the gather ceiling ---------------------------------------
 *
 * pr_measure_gather_rate times random 4-byte loads from a float vector, the
 * operation that dominates every pull gather of Eq. 1 (one load of
 * y(colidx[e]) per in-edge e), without a graph.  Warps stream random indices
 * in 16-byte vectors and keep 16 independent loads in flight per lane.  With
 * a vector that stays in L2 (n_values = 2^24, 64 MB) the result is the rate
 * at which the SMs can send L1 misses to L2, which bounds the iteration of
 * any pull-gather kernel on a graph whose quotient vector fits in L2.
 *   n_values       length of the gathered vector, in [1, 2^31 - 1].
 *   n_indices      random indices drawn on the device (SplitMix64 of
 *                  seed + i, modulo n_values); a multiple of 512 in
 *                  [1024, 2^31 - 1].  Warps wrap around them.
 *   cached         0: loads bypass L1 (ld.global.cg); 1: loads through L1
 *                  (ld.global.nc).
 *   blocks_per_sm  resident 256-thread blocks per SM, in [1, 8]; more than
 *                  fit on an SM returns PR_ERR_INVALID_ARG.
 *   chunks         512-index chunks each warp gathers in the timed launch, in
 *                  [1, 65536]; the launch makes
 *                  SMs x blocks_per_sm x 256 x 16 x chunks loads.
 *   out            host, 3 doubles: [0] loads per second, [1] milliseconds
 *                  of the timed launch (CUDA events on `stream`), [2] loads.
 * The call allocates its own device buffers (4 n_values + 4 n_indices bytes
 * and a small sink), runs one untimed warm-up launch, times one launch,
 * synchronises `stream` and frees the buffers.  Arguments are checked before
 * any CUDA call. */
PR_API pr_status pr_measure_gather_rate(int64_t n_values, int64_t n_indices, int cached,
                                        int blocks_per_sm, int32_t chunks, uint64_t seed,
                                        double* out, void* stream);

/* Static text for a status code. */
PR_API const char* pr_status_string(pr_status s);

/* Message of the last error raised on the calling thread ("" if none). */
PR_API const char* pr_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PAGERANK_GB300_H */
