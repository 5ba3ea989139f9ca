// pr_set.cu -- many independent graphs solved together (pr_solve_set).
//
// The caller builds one pr_graph from the block-diagonal CSR of `count`
// graphs (graph i owns the caller ids [offsets[i], offsets[i+1]) and no edge
// crosses two graphs) and declares the partition with pr_graph_set_partition.
// pr_solve_set then runs the synchronous iteration of Alg. 1 on every graph at
// once: each launch of the iteration kernels covers all graphs, the whole solve
// is one CUDA graph (a conditional while node over two iterations), and each
// graph keeps its own
//
//   teleport 1/n_i and dangling share D_i/n_i,   x'(v) = (1-d)/n_i + d (s(v) + D_i/n_i)
//   L1 change r_i, stopping test r_i < tol (a converged graph is frozen: its
//   rows are copied forward without gathering), and final rescaling to 1.
//
// Layout: the graph's degree binning is global, so rows of different graphs
// share degree classes; but within a class the binned order keeps the caller
// order, so each graph's rows of a class are contiguous.  The set's row tiles
// are the graph's tiles split at graph boundaries, each tagged with its graph:
// a tile belongs to one graph, and every tile's reductions are done per tile
// (a block reduction into a partial slot), then summed per graph over the
// graph's tiles in tile order -- deterministic, like the single-graph solve.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "pr_tile.cuh"

namespace prk {

struct SetState {
    double d;
    double tol;
    int32_t max_iter;
    int32_t iter;
    int32_t done;
    int32_t count;
    uint32_t ticket;
    uint32_t error;
    int32_t active_graphs;
    int32_t pad;
};

// Per-graph arrays of the set solver (device).
struct SetGraphs {
    double* inv_n;       // 1/n_i
    double* D;           // dangling mass of the current input
    double* resid;       // last L1 change
    double* sum_x;
    float* base;         // (1-d)/n_i + d D_i/n_i, read by the row kernel
    float* scale;        // 1/sum_x after the solve
    int32_t* active;     // 1 while graph i iterates
    int32_t* iters;      // iterations graph i ran
};

struct SetArgs {
    IterArgs it;                 // the graph's iteration arguments (rowptr, colidx, segments ...)
    const Tile* tiles;           // the set's tiles; Tile::pad = graph index
    int32_t n_tiles;
    int32_t count;
    const int32_t* gtile_ptr;    // tiles of graph i: gtiles[gtile_ptr[i] .. gtile_ptr[i+1])
    const int32_t* gtiles;
    double* tile_part;           // [n_tiles][2]
    SetState* state;
    SetGraphs gr;
    SolveState* single;          // the graph's own state: its done flag gates k_heavy_segments
    cudaGraphConditionalHandle cond;
    int32_t use_cond;
    int32_t pad;
};

__device__ __forceinline__ int32_t set_done(const SetState* st) {
    __shared__ int32_t done;
    if (threadIdx.x == 0) done = *(const volatile int32_t*)&st->done;
    __syncthreads();
    const int32_t v = done;
    __syncthreads();
    return v;
}

// Block reduction of the thread's (r, D) into the tile's partial slot.
__device__ __forceinline__ void tile_flush(Acc& acc, double* part) {
    double r = acc.resid(), m = acc.mass();
    block_sum2(r, m);
    if (threadIdx.x == 0) {
        part[0] = r;
        part[1] = m;
    }
    acc = Acc();
    __syncthreads();   // block_sum2's shared scratch is reused by the next tile
}

// One synchronous update of every active graph; frozen graphs copy forward.
template <typename IdxT>
__global__ void __launch_bounds__(kBlock) k_set_rows(SetArgs a, const float* __restrict__ x_in,
                                                     const float* __restrict__ y_in, float* __restrict__ x_out,
                                                     float* __restrict__ y_out) {
    if (set_done(a.state)) {
        if (a.use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(a.cond, 0);
        return;
    }
    const int tid = threadIdx.x;
    const float d = (float)a.state->d;
    RowCtx c{};
    c.d = d;
    c.one_m_d = 1.f - d;
    c.hot = a.it.hot;
    c.hot_n = 0;
    c.hot_sm = nullptr;
    c.lane_mode = a.it.lane_mode;
    Acc acc;
    for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        const Tile tile = a.tiles[t];
        const int gi = tile.pad;
        if (!a.gr.active[gi]) {
            for (int64_t r = tile.row_begin + tid; r < tile.row_end; r += kBlock) {
                x_out[r] = x_in[r];
                y_out[r] = y_in[r];
            }
            tile_flush(acc, a.tile_part + 2 * (size_t)t);
            continue;
        }
        c.base = a.gr.base[gi];
        c.d_share = 0.f;   // uniform teleport per graph: the base carries the share
        if (tile.kind >= 0) {
            process_light_tile<IdxT, true, false>(tile, a.it.rowptr, a.it.colidx, a.it.inv_out, nullptr,
                                                   x_in, y_in, x_out, y_out, c, acc, tid);
        } else if (tile.kind == kTileZero) {
            process_zero_tile<true, false>(tile, a.it.inv_out, nullptr, x_in, x_out, y_out, c, acc, tid);
        } else {   // heavy rows: sum of the segment partials
            for (int64_t r = tile.row_begin + tid; r < tile.row_end; r += kBlock) {
                const float xo = ld_stream(x_in + r);
                const float inv = ld_stream(a.it.inv_out + r);
                float s = 0.f;
                const int32_t j1 = a.it.seg_ptr[r + 1];
                for (int32_t j = a.it.seg_ptr[r]; j < j1; ++j) s += __ldcg(a.it.seg_sum + j);
                row_update<true, false>(r, s, xo, inv, 0.f, c, x_out, y_out, acc);
            }
        }
        tile_flush(acc, a.tile_part + 2 * (size_t)t);
    }
}

// Per-graph sums of the tile partials (block i sums graph i's tiles in tile
// order), the per-graph stopping test, and -- in the last block -- the loop
// condition.  mode 0: after an iteration; mode 1: after init (D only).
__global__ void __launch_bounds__(kBlock) k_set_reduce(SetArgs a, int mode) {
    SetState* st = a.state;
    if (mode == 0 && set_done(st)) return;
    __shared__ int last;
    __shared__ int32_t n_active;
    if (threadIdx.x == 0) n_active = 0;
    __syncthreads();
    for (int gi = blockIdx.x; gi < a.count; gi += gridDim.x) {
        double r = 0.0, m = 0.0;
        for (int32_t q = a.gtile_ptr[gi] + threadIdx.x; q < a.gtile_ptr[gi + 1]; q += blockDim.x) {
            const int32_t t = a.gtiles[q];
            r += __ldcg(a.tile_part + 2 * (size_t)t);
            m += __ldcg(a.tile_part + 2 * (size_t)t + 1);
        }
        block_sum2(r, m);
        if (threadIdx.x == 0) {
            const double d = st->d, inv_n = a.gr.inv_n[gi];
            const bool was = mode == 1 || a.gr.active[gi];
            if (mode == 1) {
                a.gr.D[gi] = m;
                a.gr.active[gi] = 1;
                a.gr.iters[gi] = 0;
                a.gr.resid[gi] = INFINITY;
                a.gr.base[gi] = (float)((1.0 - d) * inv_n + d * m * inv_n);
                ++n_active;
            } else if (was) {
                a.gr.D[gi] = m;
                a.gr.resid[gi] = r;
                a.gr.iters[gi] = st->iter + 1;
                a.gr.base[gi] = (float)((1.0 - d) * inv_n + d * m * inv_n);
                if (r < st->tol) a.gr.active[gi] = 0;
                else ++n_active;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (n_active) atomicAdd(&st->active_graphs, n_active);
        __threadfence();
        last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    const int32_t active = *(volatile int32_t*)&st->active_graphs;
    st->active_graphs = 0;
    st->ticket = 0;
    if (mode == 1) {
        st->iter = 0;
        st->done = 0;
        a.single->done = 0;
        return;
    }
    const int32_t it = st->iter + 1;
    st->iter = it;
    const int done = active == 0 || it >= st->max_iter;
    st->done = done;
    a.single->done = done;
    if (done && a.use_cond) cudaGraphSetConditional(a.cond, 0);
}

// x = 1/n_i, y = x/outdeg on every row; per-tile dangling partials.
__global__ void __launch_bounds__(kBlock) k_set_init(SetArgs a, float* __restrict__ x, float* __restrict__ y) {
    Acc acc;
    for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        const Tile tile = a.tiles[t];
        const float xv = (float)a.gr.inv_n[tile.pad];
        for (int64_t r = tile.row_begin + threadIdx.x; r < tile.row_end; r += kBlock) {
            const float inv = a.it.inv_out[r];
            x[r] = xv;
            y[r] = xv * inv;
            if (inv == 0.f) acc.kahan(xv);
        }
        tile_flush(acc, a.tile_part + 2 * (size_t)t);
    }
}

// Per-tile sums of the final vector (buffer iter & 1), as (sum, 0) partials.
__global__ void __launch_bounds__(kBlock) k_set_tile_sums(SetArgs a, const float* __restrict__ x0,
                                                          const float* __restrict__ x1) {
    const float* x = (a.state->iter & 1) ? x1 : x0;
    for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        const Tile tile = a.tiles[t];
        double s = 0.0, z = 0.0;
        for (int64_t r = tile.row_begin + threadIdx.x; r < tile.row_end; r += kBlock) s += (double)x[r];
        block_sum2(s, z);
        if (threadIdx.x == 0) {
            a.tile_part[2 * (size_t)t] = s;
            a.tile_part[2 * (size_t)t + 1] = 0.0;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kBlock) k_set_scale(SetArgs a) {
    for (int gi = blockIdx.x; gi < a.count; gi += gridDim.x) {
        double s = 0.0, z = 0.0;
        for (int32_t q = a.gtile_ptr[gi] + threadIdx.x; q < a.gtile_ptr[gi + 1]; q += blockDim.x)
            s += __ldcg(a.tile_part + 2 * (size_t)a.gtiles[q]);
        block_sum2(s, z);
        if (threadIdx.x == 0) {
            a.gr.sum_x[gi] = s;
            a.gr.scale[gi] = s > 0.0 ? (float)(1.0 / s) : 1.f;
        }
        __syncthreads();
    }
}

// out[v] = x[rank[v]] * scale of v's graph (caller order).
__global__ void k_set_unpermute(SetArgs a, const float* __restrict__ x0, const float* __restrict__ x1,
                                const int32_t* __restrict__ rank, const int32_t* __restrict__ gid_binned,
                                float* __restrict__ out) {
    const float* x = (a.state->iter & 1) ? x1 : x0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < a.it.n; v += stride) {
        const int32_t r = rank[v];
        out[v] = x[r] * a.gr.scale[gid_binned[r]];
    }
}

// Graph index of every binned row: the caller id order[i] located in offsets.
__global__ void k_set_gid(const int32_t* __restrict__ order, int64_t n, const int64_t* __restrict__ offsets,
                          int32_t count, int32_t* __restrict__ gid) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t v = order[i];
        int32_t lo = 0, hi = count;   // offsets[lo] <= v < offsets[hi]
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if (offsets[mid] <= v) lo = mid;
            else hi = mid;
        }
        gid[i] = lo;
    }
}

// Every edge stays inside one graph; a crossing edge sets *bad.
template <typename IdxT>
__global__ void k_set_check(const void* rowptr, const int32_t* __restrict__ colidx, int64_t n,
                            const int32_t* __restrict__ gid, unsigned int* bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        const int64_t e1 = row_at<IdxT>(rowptr, r + 1);
        const int32_t gr = gid[r];
        for (int64_t e = row_at<IdxT>(rowptr, r); e < e1; ++e)
            if (gid[colidx[e]] != gr) {
                atomicOr(bad, 1u);
                break;
            }
    }
}

// ------------------------------------------------------------------ host --

struct SetCtx {
    int32_t count = 0;
    std::vector<int64_t> offsets;
    int64_t* d_offsets = nullptr;
    int32_t* gid = nullptr;           // graph of each binned row
    Tile* tiles = nullptr;
    int32_t n_tiles = 0;
    int32_t* gtile_ptr = nullptr;
    int32_t* gtiles = nullptr;
    double* tile_part = nullptr;
    SetState* state = nullptr;
    SetState* host_state = nullptr;
    SetGraphs gr{};
    void* gr_block = nullptr;         // one allocation for the per-graph arrays
    cudaGraphExec_t loop_exec = nullptr;
};

namespace {

// Blocks per SM of the graph-set kernels: the row kernel uses 40 registers,
// so six 256-thread blocks fit (measured 0.46 -> 0.40 ms per iteration on the
// 64-graph set against four).
#ifndef PRK_SET_BLOCKS_PER_SM
#define PRK_SET_BLOCKS_PER_SM 6
#endif

int set_grid(const pr_graph* g, int64_t items) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)g->sm_count * PRK_SET_BLOCKS_PER_SM));
}

SetArgs set_args(const pr_graph* g, const SetCtx* sc) {
    SetArgs a{};
    a.it = make_args(g, true);
    a.tiles = sc->tiles;
    a.n_tiles = sc->n_tiles;
    a.count = sc->count;
    a.gtile_ptr = sc->gtile_ptr;
    a.gtiles = sc->gtiles;
    a.tile_part = sc->tile_part;
    a.state = sc->state;
    a.gr = sc->gr;
    a.single = g->state;
    return a;
}

cudaError_t enqueue_set_iteration(const pr_graph* g, const SetCtx* sc, const SetArgs& a, int src,
                                  cudaStream_t s) {
    int launches = 0;
    cudaError_t e = launch_segments(g, a.it, src, s, &launches);
    if (e != cudaSuccess) return e;
    const int grid = set_grid(g, sc->n_tiles);
    if (g->idx64)
        k_set_rows<int64_t><<<grid, kBlock, 0, s>>>(a, g->x[src], g->y[src], g->x[1 - src], g->y[1 - src]);
    else
        k_set_rows<int32_t><<<grid, kBlock, 0, s>>>(a, g->x[src], g->y[src], g->x[1 - src], g->y[1 - src]);
    k_set_reduce<<<set_grid(g, sc->count), kBlock, 0, s>>>(a, 0);
    return cudaGetLastError();
}

pr_status build_set_graph(pr_graph* g, SetCtx* sc) {
    cudaGraph_t graph = nullptr;
    PRK_CHECK(cudaGraphCreate(&graph, 0));
    struct Guard {
        cudaGraph_t gr;
        ~Guard() { if (gr) cudaGraphDestroy(gr); }
    } guard{graph};
    cudaGraphConditionalHandle handle;
    PRK_CHECK(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = handle;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    PRK_CHECK(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &p));
    cudaGraph_t body = p.conditional.phGraph_out[0];
    SetArgs a = set_args(g, sc);
    a.cond = handle;
    a.use_cond = 1;
    PRK_CHECK(cudaStreamBeginCaptureToGraph(g->capture_stream, body, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal));
    cudaError_t e1 = enqueue_set_iteration(g, sc, a, 0, g->capture_stream);
    cudaError_t e2 = cudaSuccess;
    if (e1 == cudaSuccess) e2 = enqueue_set_iteration(g, sc, a, 1, g->capture_stream);
    cudaGraph_t captured = nullptr;
    cudaError_t e3 = cudaStreamEndCapture(g->capture_stream, &captured);
    PRK_CHECK(e1);
    PRK_CHECK(e2);
    PRK_CHECK(e3);
    PRK_CHECK(cudaGraphInstantiate(&sc->loop_exec, graph, 0));
    return PR_OK;
}

}  // namespace

void drop_set_graph(pr_graph* g) {
    if (g->set && g->set->loop_exec) {
        cudaGraphExecDestroy(g->set->loop_exec);
        g->set->loop_exec = nullptr;
    }
}

void destroy_set(pr_graph* g) {
    SetCtx* sc = g->set;
    if (!sc) return;
    cudaDeviceSynchronize();   // earlier solves may still use the memory (cudaFree waited the same way)
    void* dev[] = {sc->d_offsets, sc->gid, sc->tiles, sc->gtile_ptr, sc->gtiles, sc->tile_part, sc->state,
                   sc->gr_block};
    for (void* p : dev)
        if (p) dev_free(p);
    if (sc->host_state) cudaFreeHost(sc->host_state);
    if (sc->loop_exec) cudaGraphExecDestroy(sc->loop_exec);
    delete sc;
    g->set = nullptr;
}

}  // namespace prk

using namespace prk;

extern "C" pr_status pr_graph_set_partition(pr_graph* g, int32_t count, const int64_t* offsets, void* stream) {
    if (!g) return fail(PR_ERR_INVALID_ARG, "pr_graph_set_partition: graph is NULL");
    if (count < 1 || count > (1 << 20)) return fail(PR_ERR_INVALID_ARG, "pr_graph_set_partition: count must be in [1, 2^20]");
    if (!offsets) return fail(PR_ERR_INVALID_ARG, "pr_graph_set_partition: offsets is NULL");
    if (is_device_pointer(offsets)) return fail(PR_ERR_INVALID_ARG, "pr_graph_set_partition: offsets must be host memory");
    if (offsets[0] != 0 || offsets[count] != g->n)
        return fail(PR_ERR_INVALID_ARG, "pr_graph_set_partition: offsets must start at 0 and end at n");
    for (int32_t i = 0; i < count; ++i)
        if (offsets[i + 1] <= offsets[i])
            return fail(PR_ERR_INVALID_ARG, "pr_graph_set_partition: every graph needs at least one vertex");
    cudaStream_t s = (cudaStream_t)stream;
    destroy_set(g);
    SetCtx* sc = new SetCtx();
    g->set = sc;
    sc->count = count;
    sc->offsets.assign(offsets, offsets + count + 1);
    const int64_t n = g->n;
    auto bail = [&](pr_status r) {
        destroy_set(g);
        return r;
    };
    if (dev_alloc(g, (void**)&sc->d_offsets, (size_t)(count + 1) * sizeof(int64_t)) != cudaSuccess ||
        dev_alloc(g, (void**)&sc->gid, (size_t)(n + kPad) * sizeof(int32_t)) != cudaSuccess)
        return bail(fail(PR_ERR_OOM, "pr_graph_set_partition: device allocation failed"));
    cudaError_t e = cudaMemcpyAsync(sc->d_offsets, offsets, (size_t)(count + 1) * sizeof(int64_t),
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return bail(cuda_fail(e, "pr_graph_set_partition: copy offsets"));
    k_set_gid<<<small_grid(g), kBlock, 0, s>>>(g->order, n, sc->d_offsets, count, sc->gid);
    unsigned int* bad = nullptr;
    if (cudaMalloc((void**)&bad, sizeof(unsigned int)) != cudaSuccess)
        return bail(fail(PR_ERR_OOM, "pr_graph_set_partition: device allocation failed"));
    cudaMemsetAsync(bad, 0, sizeof(unsigned int), s);
    if (g->idx64) k_set_check<int64_t><<<small_grid(g), kBlock, 0, s>>>(g->rowptr, g->colidx, n, sc->gid, bad);
    else k_set_check<int32_t><<<small_grid(g), kBlock, 0, s>>>(g->rowptr, g->colidx, n, sc->gid, bad);
    unsigned int hbad = 0;
    std::vector<int32_t> gid((size_t)n);
    e = cudaMemcpyAsync(&hbad, bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(gid.data(), sc->gid, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(bad);
    if (e != cudaSuccess) return bail(cuda_fail(e, "pr_graph_set_partition: partition check"));
    if (hbad) return bail(fail(PR_ERR_INVALID_GRAPH, "pr_graph_set_partition: an edge joins two graphs of the set"));

    // the graph's tiles split at graph boundaries, each tagged with its graph
    std::vector<Tile> tiles;
    for (const Tile& t : g->host_tiles) {
        int32_t r = t.row_begin;
        while (r < t.row_end) {
            int32_t q = r + 1;
            while (q < t.row_end && gid[q] == gid[r]) ++q;
            tiles.push_back(Tile{r, q, t.kind, gid[r]});
            r = q;
        }
    }
    sc->n_tiles = (int32_t)tiles.size();
    std::vector<int32_t> gptr((size_t)count + 1, 0), gt(tiles.size());
    for (const Tile& t : tiles) ++gptr[(size_t)t.pad + 1];
    for (int32_t i = 0; i < count; ++i) gptr[i + 1] += gptr[i];
    {
        std::vector<int32_t> cur(gptr.begin(), gptr.end() - 1);
        for (int32_t t = 0; t < sc->n_tiles; ++t) gt[cur[tiles[t].pad]++] = t;
    }
    std::vector<double> inv_n((size_t)count);
    for (int32_t i = 0; i < count; ++i) inv_n[i] = 1.0 / (double)(offsets[i + 1] - offsets[i]);
    // per-graph arrays in one block: 5 double arrays, 2 float arrays, 2 int arrays
    const size_t C = (size_t)count;
    const size_t bytes = C * (5 * sizeof(double) + 2 * sizeof(float) + 2 * sizeof(int32_t)) + 256;
    if (dev_alloc(g, (void**)&sc->tiles, (tiles.size() + 1) * sizeof(Tile)) != cudaSuccess ||
        dev_alloc(g, (void**)&sc->gtile_ptr, (C + 1) * sizeof(int32_t)) != cudaSuccess ||
        dev_alloc(g, (void**)&sc->gtiles, (tiles.size() + 1) * sizeof(int32_t)) != cudaSuccess ||
        dev_alloc(g, (void**)&sc->tile_part, (tiles.size() + 1) * 2 * sizeof(double)) != cudaSuccess ||
        dev_alloc(g, (void**)&sc->state, sizeof(SetState)) != cudaSuccess ||
        dev_alloc(g, &sc->gr_block, bytes) != cudaSuccess ||
        cudaMallocHost((void**)&sc->host_state, sizeof(SetState)) != cudaSuccess)
        return bail(fail(PR_ERR_OOM, "pr_graph_set_partition: allocation failed"));
    char* p = (char*)sc->gr_block;
    sc->gr.inv_n = (double*)p; p += C * sizeof(double);
    sc->gr.D = (double*)p; p += C * sizeof(double);
    sc->gr.resid = (double*)p; p += C * sizeof(double);
    sc->gr.sum_x = (double*)p; p += C * sizeof(double);
    p += C * sizeof(double);   // spare
    sc->gr.base = (float*)p; p += C * sizeof(float);
    sc->gr.scale = (float*)p; p += C * sizeof(float);
    sc->gr.active = (int32_t*)p; p += C * sizeof(int32_t);
    sc->gr.iters = (int32_t*)p;
    e = cudaMemcpyAsync(sc->tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sc->gtile_ptr, gptr.data(), gptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sc->gtiles, gt.data(), gt.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sc->gr.inv_n, inv_n.data(), C * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bail(cuda_fail(e, "pr_graph_set_partition: upload"));
    return PR_OK;
}

extern "C" pr_status pr_solve_set(pr_graph* g, float damping, double tol, int32_t max_iter, float* x_out,
                                  double* graph_residual, int32_t* graph_iterations, pr_info* info,
                                  void* stream) {
    if (!g) return fail(PR_ERR_INVALID_ARG, "pr_solve_set: graph is NULL");
    if (!g->set) return fail(PR_ERR_INVALID_ARG, "pr_solve_set: no partition (call pr_graph_set_partition)");
    if (!(damping >= 0.0f && damping < 1.0f)) return fail(PR_ERR_INVALID_ARG, "damping must be in [0, 1)");
    if (!(tol > 0.0) || !std::isfinite(tol)) return fail(PR_ERR_INVALID_ARG, "tol must be a positive finite number");
    if (max_iter < 1) return fail(PR_ERR_INVALID_ARG, "max_iter must be >= 1");
    if (!x_out) return fail(PR_ERR_INVALID_ARG, "x_out is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    SetCtx* sc = g->set;
    pr_status rc = ensure_stage(g);
    if (rc != PR_OK) return rc;
    const bool out_dev = is_device_pointer(x_out);
    float* out = out_dev ? x_out : g->stage + (size_t)2 * (size_t)(g->n + kPad);

    SetState* hs = sc->host_state;
    memset(hs, 0, sizeof(SetState));
    hs->d = (double)damping;
    hs->tol = tol;
    hs->max_iter = max_iter;
    hs->count = sc->count;
    PRK_CHECK(cudaEventRecord(g->ev_start, s));
    PRK_CHECK(cudaMemcpyAsync(sc->state, hs, sizeof(SetState), cudaMemcpyHostToDevice, s));
    SetArgs a = set_args(g, sc);
    int launches = 0;
    k_set_init<<<set_grid(g, sc->n_tiles), kBlock, 0, s>>>(a, g->x[0], g->y[0]);
    k_set_reduce<<<set_grid(g, sc->count), kBlock, 0, s>>>(a, 1);
    launches += 2;
    PRK_CHECK(cudaGetLastError());
    PRK_CHECK(cudaEventRecord(g->ev_loop0, s));
    if (g->use_graph) {
        if (!sc->loop_exec && (rc = build_set_graph(g, sc)) != PR_OK) return rc;
        PRK_CHECK(cudaGraphLaunch(sc->loop_exec, s));
        ++launches;
    } else {
        for (int32_t it = 0; it < max_iter;) {
            const int c = std::min<int32_t>(8, max_iter - it);
            for (int i = 0; i < c; ++i) {
                PRK_CHECK(enqueue_set_iteration(g, sc, a, (it + i) & 1, s));
                launches += g->n_seg > 0 ? 3 : 2;
            }
            it += c;
            PRK_CHECK(cudaMemcpyAsync(hs, sc->state, sizeof(SetState), cudaMemcpyDeviceToHost, s));
            PRK_CHECK(cudaStreamSynchronize(s));
            if (hs->done) break;
        }
    }
    PRK_CHECK(cudaEventRecord(g->ev_loop1, s));
    k_set_tile_sums<<<set_grid(g, sc->n_tiles), kBlock, 0, s>>>(a, g->x[0], g->x[1]);
    k_set_scale<<<set_grid(g, sc->count), kBlock, 0, s>>>(a);
    k_set_unpermute<<<small_grid(g), kBlock, 0, s>>>(a, g->x[0], g->x[1], g->rank, sc->gid, out);
    launches += 3;
    PRK_CHECK(cudaGetLastError());
    PRK_CHECK(cudaEventRecord(g->ev_stop, s));
    if (!out_dev) PRK_CHECK(cudaMemcpyAsync(x_out, out, (size_t)g->n * sizeof(float), cudaMemcpyDeviceToHost, s));
    PRK_CHECK(cudaMemcpyAsync(hs, sc->state, sizeof(SetState), cudaMemcpyDeviceToHost, s));
    const size_t C = (size_t)sc->count;
    std::vector<double> res(C), sums(C), dang(C);
    std::vector<int32_t> its(C);
    PRK_CHECK(cudaMemcpyAsync(res.data(), sc->gr.resid, C * sizeof(double), cudaMemcpyDeviceToHost, s));
    PRK_CHECK(cudaMemcpyAsync(sums.data(), sc->gr.sum_x, C * sizeof(double), cudaMemcpyDeviceToHost, s));
    PRK_CHECK(cudaMemcpyAsync(dang.data(), sc->gr.D, C * sizeof(double), cudaMemcpyDeviceToHost, s));
    PRK_CHECK(cudaMemcpyAsync(its.data(), sc->gr.iters, C * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PRK_CHECK(cudaStreamSynchronize(s));
    float ms = 0.f, ms_loop = 0.f;
    PRK_CHECK(cudaEventElapsedTime(&ms, g->ev_start, g->ev_stop));
    PRK_CHECK(cudaEventElapsedTime(&ms_loop, g->ev_loop0, g->ev_loop1));
    int conv = 1;
    double worst = 0.0, sx = 0.0, dm = 0.0;
    for (size_t i = 0; i < C; ++i) {
        if (!(res[i] < tol)) conv = 0;
        worst = std::max(worst, res[i]);
        sx += sums[i];
        dm += dang[i];
        if (graph_residual) graph_residual[i] = res[i];
        if (graph_iterations) graph_iterations[i] = its[i];
    }
    if (info) {
        info->iterations = hs->iter;
        info->converged = conv;
        info->residual_l1 = worst;
        info->sum_x = sx;
        info->dangling_mass = dm;
        info->edge_visits = (double)hs->iter * (double)g->nnz;
        info->ms_device = ms;
        info->launches = launches;
        info->loop_edge_visits = info->edge_visits;
        info->ms_loop = ms_loop;
        info->frozen_rows = 0;
    }
    return conv ? PR_OK : PR_NOT_CONVERGED;
}
