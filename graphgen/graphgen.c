/*
 * graphgen.c -- seeded synthetic directed graphs, emitted as in-edge CSR.
 *
 * This module only builds inputs.  It holds none of the PageRank arithmetic:
 * no out-degrees, no ranks, no residuals.  Both the CUDA library and the CPU
 * oracle take its output (rowptr/colidx of in-edges: row v lists the sources u
 * of edges u -> v), so that the two sides can be fed the same graph.
 *
 * Generators
 *   - R-MAT (Chakrabarti, Zhan, Faloutsos 2004) with the Graph500 quadrant
 *     probabilities; the paper's synthetic datasets come from an R-MAT
 *     generator (Section 5.2, Datasets).  2^scale vertices, edge_factor*2^scale
 *     drawn edges, vertex ids relabelled by a seeded random permutation,
 *     self-loops and duplicate edges removed.
 *   - Erdos-Renyi style digraph with a fixed fraction of vertices forced to
 *     have no out-edges (dangling).  Every other vertex draws a Poisson
 *     out-degree and uniform destinations other than itself.
 *
 * Determinism: every random number is a pure function of (seed, stream,
 * counter) -- SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) evaluated at a
 * counter -- so the graph does not depend on the number of threads or on the
 * machine.  Each row's sources are sorted ascending, so the CSR is canonical.
 * Floating point is used only to turn probabilities into 32-bit integer
 * thresholds and for the Poisson draw; both use plain IEEE double operations
 * (compiled with -ffp-contract=off, no libm calls), so x86-64 and aarch64
 * produce the same graph.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <unistd.h>

#define GG_API __attribute__((visibility("default")))

/* ---------------------------------------------------------------- RNG ---- */

static const uint64_t GG_GAMMA = 0x9E3779B97F4A7C15ull;

static inline uint64_t gg_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* The i-th output of a SplitMix64 sequence whose state starts at `key`. */
static inline uint64_t gg_rand(uint64_t key, uint64_t i) {
    return gg_mix64(key + (i + 1) * GG_GAMMA);
}

/* Stream keys: one independent sequence per purpose. */
enum { GG_STREAM_RMAT = 1, GG_STREAM_PERM = 2, GG_STREAM_DANGLE = 3,
       GG_STREAM_DEG = 4, GG_STREAM_DST = 5, GG_STREAM_USER = 6 };

static inline uint64_t gg_key(uint64_t seed, uint64_t stream) {
    return gg_mix64(seed * 0xD1B54A32D192ED03ull + stream * GG_GAMMA + 0x8CB92BA72F3D8DD7ull);
}

/* Uniform integer in [0, m), m < 2^32, from the high 32 bits (Lemire's
 * multiply-shift without rejection; bias <= m / 2^32). */
static inline uint32_t gg_below(uint64_t r, uint32_t m) {
    return (uint32_t)(((r >> 32) * (uint64_t)m) >> 32);
}

/* Uniform double in (0, 1): 53 random bits, centred in their cell. */
static inline double gg_unit(uint64_t r) {
    return ((double)(r >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

GG_API uint64_t gg_random_u64(uint64_t seed, uint64_t stream, uint64_t i) {
    return gg_rand(gg_key(seed, stream), i);
}

/* Fill out[0..count) with uniform doubles in (0,1) from stream GG_STREAM_USER
 * shifted by `stream` -- used for seeded teleport vectors and test inputs. */
GG_API void gg_uniform(uint64_t seed, uint64_t stream, int64_t count, double* out) {
    uint64_t key = gg_key(seed, GG_STREAM_USER + 16 * stream);
    for (int64_t i = 0; i < count; ++i) out[i] = gg_unit(gg_rand(key, (uint64_t)i));
}

/* Fisher-Yates permutation of [0, n): perm[i] is the new label of vertex i. */
GG_API void gg_permutation(uint64_t seed, uint64_t stream, int64_t n, int32_t* perm) {
    uint64_t key = gg_key(seed, stream);
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        uint32_t j = gg_below(gg_rand(key, (uint64_t)i), (uint32_t)(i + 1));
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
}

/* ------------------------------------------------------------ threads ---- */

static int gg_threads(int want) {
    if (want > 0) return want > 256 ? 256 : want;
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    if (c < 1) c = 1;
    if (c > 64) c = 64;
    return (int)c;
}

typedef void (*gg_task_fn)(void* ctx, int64_t begin, int64_t end);

typedef struct {
    gg_task_fn fn;
    void* ctx;
    int64_t total;
    int64_t chunk;
    int64_t next;   /* shared cursor, advanced atomically */
} gg_pool_t;

static void* gg_worker(void* p) {
    gg_pool_t* pool = (gg_pool_t*)p;
    for (;;) {
        int64_t b = __atomic_fetch_add(&pool->next, pool->chunk, __ATOMIC_RELAXED);
        if (b >= pool->total) break;
        int64_t e = b + pool->chunk;
        if (e > pool->total) e = pool->total;
        pool->fn(pool->ctx, b, e);
    }
    return NULL;
}

/* Run fn over [0, total) in chunks on nthreads threads.  The result of every
 * task below is independent of which thread runs which chunk. */
static void gg_parallel(int nthreads, int64_t total, int64_t chunk, gg_task_fn fn, void* ctx) {
    gg_pool_t pool = { fn, ctx, total, chunk < 1 ? 1 : chunk, 0 };
    if (nthreads <= 1 || total <= chunk) { fn(ctx, 0, total); return; }
    pthread_t tid[256];
    int started = 0;
    for (int t = 0; t < nthreads - 1; ++t)
        if (pthread_create(&tid[started], NULL, gg_worker, &pool) == 0) ++started;
    gg_worker(&pool);
    for (int t = 0; t < started; ++t) pthread_join(tid[t], NULL);
}

/* ------------------------------------------------------ edge sources ---- */

#define GG_MAX_OUT 256

typedef struct {
    int kind;                 /* 0 = R-MAT, 1 = ER with dangling, 2 = R-MAT on n vertices */
    int64_t n;
    int64_t units;            /* R-MAT: edges; ER: source vertices */
    /* R-MAT */
    int scale;
    uint64_t key_rmat;
    uint64_t seed;            /* kind 2: keys of the retry streams */
    uint64_t t_a, t_ab, t_abc;
    const int32_t* perm;      /* NULL: no relabelling */
    /* ER */
    uint64_t key_deg, key_dst;
    const uint8_t* dangling;  /* 1 if the vertex has no out-edges */
    double exp_neg_lambda;
    /* driver state */
    uint32_t* count;          /* per-destination edge counts / cursors */
    int64_t* rowstart;        /* start of each row in tmp */
    int32_t* tmp;             /* unsorted sources, grouped by destination */
    int64_t* pre_edges;       /* per-chunk partial edge totals (pass 1) */
} gg_src_t;

/* One R-MAT draw (source s, destination d in [0, 2^scale)) from stream key. */
static void gg_rmat_pair(const gg_src_t* g, uint64_t key, int64_t unit, uint64_t* ps, uint64_t* pd) {
    uint64_t s = 0, d = 0;
    int nd = (g->scale + 1) / 2;
    for (int j = 0; j < nd; ++j) {
        uint64_t r = gg_rand(key, (uint64_t)unit * (uint64_t)nd + (uint64_t)j);
        for (int h = 0; h < 2; ++h) {
            int level = 2 * j + h;
            if (level >= g->scale) break;
            uint64_t u = h == 0 ? (r >> 32) : (r & 0xFFFFFFFFull);
            uint64_t sb, db;
            if (u < g->t_a)        { sb = 0; db = 0; }
            else if (u < g->t_ab)  { sb = 0; db = 1; }
            else if (u < g->t_abc) { sb = 1; db = 0; }
            else                   { sb = 1; db = 1; }
            s = (s << 1) | sb;
            d = (d << 1) | db;
        }
    }
    *ps = s;
    *pd = d;
}

/* Edges produced by one unit.  Returns how many were written to src/dst. */
static int gg_unit_edges(const gg_src_t* g, int64_t unit, int32_t* src, int32_t* dst) {
    if (g->kind == 2) {
        /* R-MAT on n vertices, 2^(scale-1) < n <= 2^scale: a draw outside
         * [0, n)^2 is redrawn from the next retry stream (up to 16 times). */
        for (int t = 0; t < 16; ++t) {
            uint64_t s, d;
            gg_rmat_pair(g, gg_key(g->seed, 7 + 16 * (uint64_t)t), unit, &s, &d);
            if ((int64_t)s >= g->n || (int64_t)d >= g->n) continue;
            if (s == d) return 0;
            if (g->perm) { s = (uint64_t)g->perm[s]; d = (uint64_t)g->perm[d]; }
            src[0] = (int32_t)s; dst[0] = (int32_t)d;
            return 1;
        }
        return 0;
    }
    if (g->kind == 0) {
        uint64_t s = 0, d = 0;
        int nd = (g->scale + 1) / 2;
        for (int j = 0; j < nd; ++j) {
            uint64_t r = gg_rand(g->key_rmat, (uint64_t)unit * (uint64_t)nd + (uint64_t)j);
            for (int h = 0; h < 2; ++h) {
                int level = 2 * j + h;
                if (level >= g->scale) break;
                uint64_t u = h == 0 ? (r >> 32) : (r & 0xFFFFFFFFull);
                uint64_t sb, db;
                if (u < g->t_a)        { sb = 0; db = 0; }
                else if (u < g->t_ab)  { sb = 0; db = 1; }
                else if (u < g->t_abc) { sb = 1; db = 0; }
                else                   { sb = 1; db = 1; }
                s = (s << 1) | sb;
                d = (d << 1) | db;
            }
        }
        if (s == d) return 0;                        /* self-loop dropped */
        if (g->perm) { s = (uint64_t)g->perm[s]; d = (uint64_t)g->perm[d]; }
        src[0] = (int32_t)s; dst[0] = (int32_t)d;
        return 1;
    }
    /* ER with dangling: unit = source vertex */
    if (g->dangling[unit]) return 0;
    /* Poisson(lambda) by multiplying uniforms until the product falls to
     * exp(-lambda) (Knuth, TAOCP vol. 2, 3.4.1). */
    int k = 0;
    double p = 1.0;
    for (;;) {
        p *= gg_unit(gg_rand(g->key_deg, ((uint64_t)unit << 8) | (uint64_t)(k & 255)));
        if (p <= g->exp_neg_lambda || k >= GG_MAX_OUT - 1) break;
        ++k;
    }
    for (int j = 0; j < k; ++j) {
        uint64_t r = gg_rand(g->key_dst, ((uint64_t)unit << 8) | (uint64_t)j);
        uint32_t v = gg_below(r, (uint32_t)(g->n - 1));
        if ((int64_t)v >= unit) v += 1;              /* never the source itself */
        src[j] = (int32_t)unit; dst[j] = (int32_t)v;
    }
    return k;
}

static void gg_pass_count(void* ctx, int64_t b, int64_t e) {
    gg_src_t* g = (gg_src_t*)ctx;
    int32_t s[GG_MAX_OUT], d[GG_MAX_OUT];
    int64_t total = 0;
    for (int64_t u = b; u < e; ++u) {
        int m = gg_unit_edges(g, u, s, d);
        for (int j = 0; j < m; ++j) __atomic_fetch_add(&g->count[d[j]], 1u, __ATOMIC_RELAXED);
        total += m;
    }
    __atomic_fetch_add(g->pre_edges, total, __ATOMIC_RELAXED);
}

/* Edge total only (sizing pass). */
static void gg_pass_total(void* ctx, int64_t b, int64_t e) {
    gg_src_t* g = (gg_src_t*)ctx;
    int32_t s[GG_MAX_OUT], d[GG_MAX_OUT];
    int64_t total = 0;
    for (int64_t u = b; u < e; ++u) total += gg_unit_edges(g, u, s, d);
    __atomic_fetch_add(g->pre_edges, total, __ATOMIC_RELAXED);
}

static void gg_pass_fill(void* ctx, int64_t b, int64_t e) {
    gg_src_t* g = (gg_src_t*)ctx;
    int32_t s[GG_MAX_OUT], d[GG_MAX_OUT];
    for (int64_t u = b; u < e; ++u) {
        int m = gg_unit_edges(g, u, s, d);
        for (int j = 0; j < m; ++j) {
            uint32_t slot = __atomic_fetch_add(&g->count[d[j]], 1u, __ATOMIC_RELAXED);
            g->tmp[g->rowstart[d[j]] + slot] = s[j];
        }
    }
}

static int gg_cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* Sort each row's sources and drop duplicates; count[v] := deduplicated length. */
static void gg_pass_sort(void* ctx, int64_t b, int64_t e) {
    gg_src_t* g = (gg_src_t*)ctx;
    for (int64_t v = b; v < e; ++v) {
        int32_t* row = g->tmp + g->rowstart[v];
        int64_t len = g->rowstart[v + 1] - g->rowstart[v];
        if (len > 1) {
            if (len <= 32) {
                for (int64_t i = 1; i < len; ++i) {
                    int32_t key = row[i];
                    int64_t j = i - 1;
                    while (j >= 0 && row[j] > key) { row[j + 1] = row[j]; --j; }
                    row[j + 1] = key;
                }
            } else {
                qsort(row, (size_t)len, sizeof(int32_t), gg_cmp_i32);
            }
        }
        int64_t w = 0;
        for (int64_t i = 0; i < len; ++i)
            if (w == 0 || row[i] != row[w - 1]) row[w++] = row[i];
        g->count[v] = (uint32_t)w;
    }
}

typedef struct { gg_src_t* g; const int64_t* rowptr; int32_t* colidx; } gg_copy_t;

static void gg_pass_copy(void* ctx, int64_t b, int64_t e) {
    gg_copy_t* c = (gg_copy_t*)ctx;
    for (int64_t v = b; v < e; ++v)
        memcpy(c->colidx + c->rowptr[v], c->g->tmp + c->g->rowstart[v],
               (size_t)(c->rowptr[v + 1] - c->rowptr[v]) * sizeof(int32_t));
}

/* Shared driver: count, fill, sort+dedup, compact.  Returns nnz, or
 * -1 (allocation failure) / -2 (colidx too small). */
static int64_t gg_build(gg_src_t* g, int nthreads, int64_t* rowptr, int32_t* colidx, int64_t cap) {
    int64_t n = g->n;
    int64_t pre = 0;
    g->count = (uint32_t*)calloc((size_t)n, sizeof(uint32_t));
    g->rowstart = (int64_t*)malloc((size_t)(n + 1) * sizeof(int64_t));
    if (!g->count || !g->rowstart) { free(g->count); free(g->rowstart); return -1; }
    g->pre_edges = &pre;
    int64_t chunk = g->kind != 1 ? (1 << 16) : (1 << 12);
    gg_parallel(nthreads, g->units, chunk, gg_pass_count, g);
    g->rowstart[0] = 0;
    for (int64_t v = 0; v < n; ++v) g->rowstart[v + 1] = g->rowstart[v] + g->count[v];
    g->tmp = (int32_t*)malloc((size_t)(pre > 0 ? pre : 1) * sizeof(int32_t));
    if (!g->tmp) { free(g->count); free(g->rowstart); return -1; }
    memset(g->count, 0, (size_t)n * sizeof(uint32_t));
    gg_parallel(nthreads, g->units, chunk, gg_pass_fill, g);
    gg_parallel(nthreads, n, 1 << 12, gg_pass_sort, g);
    rowptr[0] = 0;
    for (int64_t v = 0; v < n; ++v) rowptr[v + 1] = rowptr[v] + g->count[v];
    int64_t nnz = rowptr[n];
    if (nnz > cap) { free(g->tmp); free(g->count); free(g->rowstart); return -2; }
    gg_copy_t c = { g, rowptr, colidx };
    gg_parallel(nthreads, n, 1 << 12, gg_pass_copy, &c);
    free(g->tmp); free(g->count); free(g->rowstart);
    return nnz;
}

/* ------------------------------------------------------------- R-MAT ---- */

/* R-MAT digraph with 2^scale vertices and edge_factor * 2^scale drawn edges.
 * Quadrant probabilities a, b, c (d = 1 - a - b - c); a level picks the
 * source bit from the row and the destination bit from the column of the 2x2
 * matrix [[a, b], [c, d]].  With permute != 0 vertex ids are relabelled by a
 * seeded random permutation (the Graph500 convention).
 * rowptr: int64[2^scale + 1]; colidx: int32[cap].  colidx == NULL returns the
 * number of drawn edges (an upper bound on nnz) without building anything. */
GG_API int64_t gg_rmat(int scale, int edge_factor, double a, double b, double c,
                       uint64_t seed, int permute, int nthreads,
                       int64_t* rowptr, int32_t* colidx, int64_t cap) {
    if (scale < 1 || scale > 30 || edge_factor < 1) return -3;
    int64_t n = (int64_t)1 << scale;
    int64_t m = (int64_t)edge_factor << scale;
    if (!colidx) return m;
    if (!(a >= 0 && b >= 0 && c >= 0 && a + b + c <= 1.0)) return -3;
    gg_src_t g;
    memset(&g, 0, sizeof g);
    g.kind = 0; g.n = n; g.units = m; g.scale = scale;
    g.key_rmat = gg_key(seed, GG_STREAM_RMAT);
    g.t_a = (uint64_t)(a * 4294967296.0);
    g.t_ab = (uint64_t)((a + b) * 4294967296.0);
    g.t_abc = (uint64_t)((a + b + c) * 4294967296.0);
    int32_t* perm = NULL;
    if (permute) {
        perm = (int32_t*)malloc((size_t)n * sizeof(int32_t));
        if (!perm) return -1;
        gg_permutation(seed, GG_STREAM_PERM, n, perm);
        g.perm = perm;
    }
    int64_t nnz = gg_build(&g, gg_threads(nthreads), rowptr, colidx, cap);
    free(perm);
    return nnz;
}

/* R-MAT digraph on any n >= 2 vertices with edge_factor * n drawn edges: the
 * power-of-two generator above at scale = ceil(log2 n), a draw with an
 * endpoint >= n redrawn (at most 16 tries, then dropped), and a seeded
 * relabelling of range(n) when permute != 0.  Same buffers and return codes
 * as gg_rmat. */
GG_API int64_t gg_rmat_n(int64_t n, int edge_factor, double a, double b, double c,
                         uint64_t seed, int permute, int nthreads,
                         int64_t* rowptr, int32_t* colidx, int64_t cap) {
    if (n < 2 || n > ((int64_t)1 << 30) || edge_factor < 1) return -3;
    int scale = 0;
    while (((int64_t)1 << scale) < n) ++scale;
    int64_t m = (int64_t)edge_factor * n;
    if (!colidx) return m;
    if (!(a >= 0 && b >= 0 && c >= 0 && a + b + c <= 1.0)) return -3;
    gg_src_t g;
    memset(&g, 0, sizeof g);
    g.kind = 2; g.n = n; g.units = m; g.scale = scale; g.seed = seed;
    g.t_a = (uint64_t)(a * 4294967296.0);
    g.t_ab = (uint64_t)((a + b) * 4294967296.0);
    g.t_abc = (uint64_t)((a + b + c) * 4294967296.0);
    int32_t* perm = NULL;
    if (permute) {
        perm = (int32_t*)malloc((size_t)n * sizeof(int32_t));
        if (!perm) return -1;
        gg_permutation(seed, GG_STREAM_PERM, n, perm);
        g.perm = perm;
    }
    int64_t nnz = gg_build(&g, gg_threads(nthreads), rowptr, colidx, cap);
    free(perm);
    return nnz;
}

/* ---------------------------------------------------- ER + dangling ---- */

/* e^x for x >= 0 by its Taylor series in plain double arithmetic (no libm, so
 * every platform gets the same bits). */
static double gg_exp_pos(double x) {
    double sum = 1.0, term = 1.0;
    for (int k = 1; k < 400; ++k) {
        term = term * x / (double)k;
        sum += term;
        if (term < sum * 1e-18) break;
    }
    return sum;
}

/* Digraph on n vertices: round(frac_dangling * n) vertices, chosen by a seeded
 * permutation, get no out-edges; every other vertex u draws
 * k ~ Poisson(mean_deg / (1 - frac_dangling)) and k destinations uniform over
 * the vertices other than u.  Mean out-degree over all n is mean_deg before
 * duplicate removal.  colidx == NULL returns the drawn edge count (upper
 * bound on nnz). */
GG_API int64_t gg_er_dangling(int64_t n, double mean_deg, double frac_dangling, uint64_t seed,
                              int nthreads, int64_t* rowptr, int32_t* colidx, int64_t cap) {
    if (n < 2 || n > 0x7FFFFFFF || !(mean_deg > 0) || !(frac_dangling >= 0 && frac_dangling < 1))
        return -3;
    double lambda = mean_deg / (1.0 - frac_dangling);
    if (lambda > 100.0) return -3;
    gg_src_t g;
    memset(&g, 0, sizeof g);
    g.kind = 1; g.n = n; g.units = n;
    g.key_deg = gg_key(seed, GG_STREAM_DEG);
    g.key_dst = gg_key(seed, GG_STREAM_DST);
    g.exp_neg_lambda = 1.0 / gg_exp_pos(lambda);
    uint8_t* dangling = (uint8_t*)calloc((size_t)n, 1);
    int32_t* perm = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!dangling || !perm) { free(dangling); free(perm); return -1; }
    gg_permutation(seed, GG_STREAM_DANGLE, n, perm);
    int64_t nd = (int64_t)(frac_dangling * (double)n + 0.5);
    for (int64_t i = 0; i < nd; ++i) dangling[perm[i]] = 1;
    free(perm);
    g.dangling = dangling;
    int64_t result;
    if (!colidx) {
        int64_t total = 0;
        g.pre_edges = &total;
        gg_parallel(gg_threads(nthreads), n, 1 << 12, gg_pass_total, &g);
        result = total;
    } else {
        result = gg_build(&g, gg_threads(nthreads), rowptr, colidx, cap);
    }
    free(dangling);
    return result;
}
