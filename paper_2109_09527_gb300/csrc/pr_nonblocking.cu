// pr_nonblocking.cu -- barrier-free, in-place PageRank: the GPU form of No-Sync (Alg. 3).
//
// One persistent launch.  Each block owns a fixed set of work items -- row
// tiles and segments of heavy rows, dealt round-robin so that every block gets
// the same mix (static allocation, as the paper's threads own fixed
// partitions) -- and sweeps it repeatedly:
//
//   for each owned row v:  x(v) <- (1-d) t(v) + d (sum_{u->v} y(u) + share)
//                          y(v) <- x(v) / outdeg(v)        (in place, no copy)
//
// reading whatever y values the other blocks have written so far (Eqs. 4 and 7:
// a row may combine in-neighbours from different sweeps).  There is no
// grid-wide synchronisation and no block ever waits for another: y is read and
// written with relaxed gpu-scope atomics (the read-write races of Alg. 3 made
// well-defined), and the only shared bookkeeping is
//
//   S     the running rank mass of vertices with out-edges, updated with one
//         FP64 atomic add of each block's change per sweep.  The dangling
//         share is share = (T - S)/n with T = sum(t): equal to D/n at the fixed
//         point, and, unlike a running dangling mass, it puts back the rank
//         mass that in-place updates gain or lose, which keeps in-place sweeps
//         converging faster than synchronous iterations;
//   slot  each block's L1 change of its latest sweep.  After every sweep a
//         block sums all slots (slots start at +inf, so no block stops before
//         every block has published) and stops once the sum is below the
//         internal tolerance -- thread-level convergence (Section 4.3) -- or
//         when it has made max_sweeps sweeps.  Nothing spins.
//
// The result is then checked with one synchronous update (the Jacobi kernels);
// its L1 change is the residual reported.  If it is not below tol the
// persistent kernel runs again from the current vector with a tighter
// internal tolerance, within the sweep budget.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "pr_tile.cuh"

namespace prk {

// Work item of a heavy row (Tile fields reused): row_begin = the row,
// row_end = a segment id (kSegEdges edges of the row), pad = 1 when the
// segment is the row's last one, whose item also updates the row.
constexpr int kItemSegment = -3;

// Items a block processes between two publications of its mass change.
constexpr int kPublishEvery = 4;

struct NbArgs {
    const void* rowptr;
    const int32_t* colidx;
    const float* inv_out;
    const float* teleport;
    const Tile* items;
    int32_t n_items;
    const int32_t* seg_ptr;      // first segment of each heavy row
    float* seg_sum;              // latest partial sum of each segment
    double* slots;               // [grid]
    double* scalars;             // [0] running non-dangling mass S
    int32_t* block_sweeps;       // [grid] sweeps made by each block
    int32_t* sweeps_max;
    SolveState* state;
    float* x;
    float* y;
    double tol_int;
    int32_t max_sweeps;
    int32_t pad;
    long long* trace;            // NULL, or 8 values per block (see k_nonblocking)
    float* history;              // NULL, or the L1 change of block 0's first 256 sweeps
    int32_t dangling_form;       // 1: share = (T - S)/n (default); 0: running dangling mass
    int32_t pad2;
};

// One segment of a heavy row, gathered by the whole block (at most three
// 16-byte colidx loads and twelve gathers per thread, all issued before use).
// The partial sum is published with a relaxed store; the row's last segment
// then sums the latest partials of all the row's segments -- some may be a
// sweep old, which an asynchronous iteration allows -- and updates the row.
template <typename IdxT, bool kUniform>
__device__ __forceinline__ void heavy_segment(const Tile& item, const NbArgs& a, const RowCtx& c, Acc& acc) {
    const int64_t r = item.row_begin;
    const int32_t sid = item.row_end;
    const int32_t s0 = a.seg_ptr[r], s1 = a.seg_ptr[r + 1];
    const int64_t rb = row_at<IdxT>(a.rowptr, r), re = row_at<IdxT>(a.rowptr, r + 1);
    const int64_t e0 = rb + (int64_t)(sid - s0) * kSegEdges;
    const int64_t e1 = min(e0 + (int64_t)kSegEdges, re);
    const int64_t a0 = e0 & ~(int64_t)3;
    int4 cv[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int64_t p = a0 + 4 * (int64_t)threadIdx.x + (int64_t)j * 4 * kBlock;
        cv[j] = p < e1 ? ld_stream4(a.colidx + p) : make_int4(0, 0, 0, 0);
    }
    float g[12];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int64_t p = a0 + 4 * (int64_t)threadIdx.x + (int64_t)j * 4 * kBlock;
        g[4 * j + 0] = (p + 0 >= e0 && p + 0 < e1) ? ld_relaxed(a.y + cv[j].x) : 0.f;
        g[4 * j + 1] = (p + 1 >= e0 && p + 1 < e1) ? ld_relaxed(a.y + cv[j].y) : 0.f;
        g[4 * j + 2] = (p + 2 >= e0 && p + 2 < e1) ? ld_relaxed(a.y + cv[j].z) : 0.f;
        g[4 * j + 3] = (p + 3 >= e0 && p + 3 < e1) ? ld_relaxed(a.y + cv[j].w) : 0.f;
    }
    float v = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) +
              ((g[8] + g[9]) + (g[10] + g[11]));
    v = block_sum(v);
    if (threadIdx.x == 0) st_relaxed(a.seg_sum + sid, v);
    if (item.pad) {
        float p = 0.f;
        for (int32_t j = s0 + threadIdx.x; j < s1; j += kBlock) p += (j == sid) ? v : ld_relaxed(a.seg_sum + j);
        p = block_sum(p);
        if (threadIdx.x == 0) {
            const float tv = kUniform ? 0.f : ld_stream(a.teleport + r);
            row_update<kUniform, true>(r, p, Mem<true>::load_x(a.x + r), ld_stream(a.inv_out + r), tv, c,
                                       a.x, a.y, acc);
        }
    }
}

template <typename IdxT, bool kUniform>
__global__ void __launch_bounds__(kBlock) k_nonblocking(NbArgs a) {
    const SolveState* st = a.state;
    const double d = st->d, inv_n = st->inv_n, T = st->t_sum;
    // Static, interleaved ownership: block b owns items b, b + G, b + 2G, ...
    const int32_t i0 = blockIdx.x, i1 = a.n_items, istep = gridDim.x;
    int32_t sweeps = 0;
    long long t_start = 0;
    if (a.trace && threadIdx.x == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_start));
    double last_R = 0.0, last_est = 0.0;
    Acc acc;
    while (sweeps < a.max_sweeps) {
        RowCtx c;
        c.d = (float)d;
        c.one_m_d = (float)(1.0 - d);
        c.hot = 0;
        c.hot_n = 0;
        c.hot_sm = nullptr;
        float r_sweep = 0.f;
        int since = kPublishEvery;
        for (int32_t it = i0; it < i1 || since > 0; it += istep) {
            if (since == kPublishEvery || it >= i1) {
                // Publish the mass change of the items done since the last
                // publication and re-read the running mass, so that the share
                // used next matches the ranks the other blocks can already see.
                double dS = acc.mass(), dD = (double)acc.dd;
                block_sum2(dS, dD);
                if (threadIdx.x == 0) {
                    if (dS != 0.0) atomicAdd(a.scalars, dS);
                    if (!a.dangling_form && dD != 0.0) atomicAdd(a.scalars + 1, dD);
                }
                r_sweep += acc.r;
                acc = Acc();
                if (it >= i1) break;
                const double share = a.dangling_form ? (T - ld_relaxed(a.scalars)) * inv_n
                                                     : ld_relaxed(a.scalars + 1) * inv_n;
                c.d_share = (float)(d * share);
                c.base = (float)((1.0 - d) * inv_n + d * share);
                since = 0;
            }
            const Tile item = a.items[it];
            if (item.kind >= 0)
                process_light_tile<IdxT, kUniform, true>(item, a.rowptr, a.colidx, a.inv_out, a.teleport,
                                                          a.x, a.y, a.x, a.y, c, acc, threadIdx.x);
            else if (item.kind == kTileZero)
                process_zero_tile<kUniform, true>(item, a.inv_out, a.teleport, a.x, a.x, a.y, c, acc, threadIdx.x);
            else
                heavy_segment<IdxT, kUniform>(item, a, c, acc);
            ++since;
        }
        ++sweeps;
        double R = (double)r_sweep, unused1 = 0.0;
        block_sum2(R, unused1);
        if (threadIdx.x == 0) {
            st_relaxed(a.slots + blockIdx.x, R);
            if (a.history && blockIdx.x == 0 && sweeps <= 256) a.history[sweeps - 1] = (float)R;
        }
        double est = 0.0, unused = 0.0;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += kBlock) est += ld_relaxed(a.slots + i);
        block_sum2(est, unused);
        last_R = R;
        last_est = est;
        if (est < a.tol_int) break;
    }
    if (a.trace && threadIdx.x == 0) {
        // per block: sweeps, start/end (ns, %globaltimer), last sweep change, last estimate,
        // first item, item count
        long long t_end;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
        long long* tr = a.trace + 8 * blockIdx.x;
        tr[0] = sweeps;
        tr[1] = t_start;
        tr[2] = t_end;
        tr[3] = __double_as_longlong(last_R);
        tr[4] = __double_as_longlong(last_est);
        tr[5] = i0;
        tr[6] = (i1 - i0 + istep - 1) / istep;
        tr[7] = 0;
    }
    if (threadIdx.x == 0) {
        a.block_sweeps[blockIdx.x] = sweeps;
        atomicMax(a.sweeps_max, sweeps);
    }
}

// Mass of x split by dangling status: writes S (non-dangling) to scalars[0],
// and D (dangling) to the solve state, and resets the iteration counters for
// the synchronous update that follows.
__global__ void __launch_bounds__(kBlock) k_mass_split(IterArgs a, const float* __restrict__ x,
                                                       double* scalars) {
    SolveState* st = a.state;
    double s_nd = 0.0, s_d = 0.0;
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < a.n; i += stride) {
        const float v = x[i];
        if (a.inv_out[i] == 0.f) s_d += (double)v;
        else s_nd += (double)v;
    }
    double S, D;
    if (block_pair_to_grid(s_nd, s_d, a.slots, &st->ticket, &S, &D) && threadIdx.x == 0) {
        scalars[0] = S;
        scalars[1] = D;
        st->D = D;
        st->iter = 0;
        st->done = 0;
        st->resid = INFINITY;
        st->ticket = 0;
    }
}

template <typename IdxT>
__global__ void k_item_edges(const void* rowptr, const int32_t* seg_ptr, const Tile* items,
                             int64_t count, int64_t* edges) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        const Tile t = items[i];
        if (t.kind == kItemSegment) {
            const int64_t rb = row_at<IdxT>(rowptr, t.row_begin), re = row_at<IdxT>(rowptr, t.row_begin + 1);
            const int64_t e0 = rb + (int64_t)(t.row_end - seg_ptr[t.row_begin]) * kSegEdges;
            edges[i] = min(e0 + (int64_t)kSegEdges, re) - e0;
        } else {
            edges[i] = row_at<IdxT>(rowptr, t.row_end) - row_at<IdxT>(rowptr, t.row_begin);
        }
    }
}

namespace {

int g_occ_nb = 0;


template <typename IdxT, bool kUniform>
void* nb_kernel() {
    return (void*)k_nonblocking<IdxT, kUniform>;
}

void* pick_kernel(const pr_graph* g, bool uniform) {
    if (g->idx64) return uniform ? nb_kernel<int64_t, true>() : nb_kernel<int64_t, false>();
    return uniform ? nb_kernel<int32_t, true>() : nb_kernel<int32_t, false>();
}

// Work items and the per-block partition, built on first use.
pr_status build_items(pr_graph* g, cudaStream_t s) {
    if (g->nb_items) return PR_OK;
    if (g_occ_nb == 0) {
        int occ = 1 << 30;
        int o = 0;
        PRK_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_nonblocking<int32_t, true>, kBlock, 0));
        occ = std::min(occ, o);
        PRK_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_nonblocking<int32_t, false>, kBlock, 0));
        occ = std::min(occ, o);
        PRK_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_nonblocking<int64_t, true>, kBlock, 0));
        occ = std::min(occ, o);
        PRK_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_nonblocking<int64_t, false>, kBlock, 0));
        occ = std::min(occ, o);
        g_occ_nb = std::max(1, occ);
    }
    // heavy rows [0, n_heavy): one item per segment (the Jacobi segments)
    std::vector<int32_t> seg_ptr((size_t)g->n_heavy + 1, 0);
    if (g->n_heavy > 0)
        PRK_CHECK(cudaMemcpy(seg_ptr.data(), g->seg_ptr, seg_ptr.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    std::vector<Tile> items;
    for (int64_t r = 0; r < g->n_heavy; ++r)
        for (int32_t sgi = seg_ptr[r]; sgi < seg_ptr[r + 1]; ++sgi)
            items.push_back(Tile{(int32_t)r, sgi, kItemSegment, sgi + 1 == seg_ptr[r + 1] ? 1 : 0});
    for (const Tile& t : g->host_tiles)
        if (t.kind != kTileHeavy) items.push_back(t);
    const int64_t count = (int64_t)items.size();

    // edges per item, then a balanced contiguous partition
    Tile* d_items = nullptr;
    int64_t* d_edges = nullptr;
    PRK_CHECK(dev_alloc(g, (void**)&d_items, (size_t)(count + 1) * sizeof(Tile)));
    g->nb_items = (int32_t*)d_items;
    g->nb_items_count = count;
    PRK_CHECK(cudaMemcpyAsync(d_items, items.data(), (size_t)count * sizeof(Tile), cudaMemcpyHostToDevice, s));
    PRK_CHECK(cudaMalloc((void**)&d_edges, (size_t)(count + 1) * sizeof(int64_t)));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((count + kBlock - 1) / kBlock, 4096));
    if (g->idx64) k_item_edges<int64_t><<<grid, kBlock, 0, s>>>(g->rowptr, g->seg_ptr, d_items, count, d_edges);
    else k_item_edges<int32_t><<<grid, kBlock, 0, s>>>(g->rowptr, g->seg_ptr, d_items, count, d_edges);
    std::vector<int64_t> edges((size_t)count);
    cudaError_t e = cudaMemcpyAsync(edges.data(), d_edges, (size_t)count * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_edges);
    PRK_CHECK(e);

    const int per_sm = g->ctas_per_sm > 0 ? std::min(g->ctas_per_sm, g_occ_nb) : g_occ_nb;
    const int G = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)g->sm_count * per_sm, count));
    // Items are dealt to blocks round-robin, so every block owns the same mix
    // of heavy-row segments, light tiles and rows without in-edges.
    g->nb_cta_edges.assign((size_t)G, 0);
    for (int64_t i = 0; i < count; ++i) g->nb_cta_edges[i % G] += edges[i];
    g->nb_grid = G;
    PRK_CHECK(dev_alloc(g, (void**)&g->nb_slots, (size_t)G * sizeof(double)));
    PRK_CHECK(dev_alloc(g, (void**)&g->nb_scalars, 8 * sizeof(double)));
    PRK_CHECK(dev_alloc(g, (void**)&g->nb_block_sweeps, (size_t)G * sizeof(int32_t) + 256 * sizeof(float)));
    PRK_CHECK(cudaStreamSynchronize(s));
    return PR_OK;
}

}  // namespace

pr_status solve_nonblocking(pr_graph* g, float damping, double tol, int32_t max_iter,
                            const float* teleport, const float* x0, float* x_out, pr_info* info,
                            cudaStream_t s) {
    pr_status rc = build_items(g, s);
    if (rc != PR_OK) return rc;
    if ((rc = ensure_stage(g)) != PR_OK) return rc;
    const float* t_dev = nullptr;
    const float* x0_dev = nullptr;
    if ((rc = stage_input(g, teleport, 0, s, &t_dev)) != PR_OK) return rc;
    if ((rc = stage_input(g, x0, 1, s, &x0_dev)) != PR_OK) return rc;
    const bool uniform = teleport == nullptr;
    if (!uniform && (rc = ensure_teleport(g)) != PR_OK) return rc;
    const bool out_dev = is_device_pointer(x_out);
    float* out = out_dev ? x_out : g->stage + (size_t)2 * (size_t)(g->n + kPad);
    const int G = g->nb_grid;

    SolveState* hs = g->host_state;
    memset(hs, 0, sizeof(SolveState));
    hs->d = (double)damping;
    hs->tol = tol;
    hs->inv_n = 1.0 / (double)g->n;
    hs->t_sum = 1.0;
    hs->max_iter = 1;  // the verifying synchronous update
    hs->uniform_t = uniform ? 1 : 0;
    PRK_CHECK(cudaEventRecord(g->ev_start, s));
    PRK_CHECK(cudaMemcpyAsync(g->state, hs, sizeof(SolveState), cudaMemcpyHostToDevice, s));
    IterArgs a = make_args(g, uniform);
    int launches = 0;
    launch_init(g, a, t_dev, x0_dev, s);
    ++launches;
    PRK_CHECK(cudaGetLastError());

    // +inf slot pattern and zeroed counters, staged in pinned memory
    std::vector<double> inf_slots((size_t)G, INFINITY);
    double* h_inf = nullptr;
    PRK_CHECK(cudaMallocHost((void**)&h_inf, (size_t)G * sizeof(double) + 64));
    struct PinnedGuard {
        double* p;
        ~PinnedGuard() { if (p) cudaFreeHost(p); }
    } guard{h_inf};
    memcpy(h_inf, inf_slots.data(), (size_t)G * sizeof(double));
    unsigned long long* h_counts = (unsigned long long*)(h_inf + G);  // pinned scratch for counters
    std::vector<int32_t> h_sweeps((size_t)G, 0);

    NbArgs na{};
    na.rowptr = g->rowptr;
    na.colidx = g->colidx;
    na.inv_out = g->inv_out;
    na.teleport = uniform ? nullptr : g->teleport;
    na.items = (const Tile*)g->nb_items;
    na.n_items = (int32_t)g->nb_items_count;
    na.seg_ptr = g->seg_ptr;
    na.seg_sum = g->seg_sum;
    na.slots = g->nb_slots;
    na.scalars = g->nb_scalars;
    na.block_sweeps = g->nb_block_sweeps;
    na.sweeps_max = (int32_t*)(g->nb_scalars + 3);
    const char* form_env = getenv("PR_NB_DANGLING_FORM");
    na.dangling_form = (form_env && form_env[0] == '0') ? 0 : 1;
    na.state = g->state;
    na.x = g->x[0];
    na.y = g->y[0];
    void* kernel = pick_kernel(g, uniform);
    // Opt-in diagnostics: PR_TRACE_NB=<file> appends one CSV line per block and launch.
    const char* trace_path = getenv("PR_TRACE_NB");
    long long* d_trace = nullptr;
    if (trace_path && *trace_path) {
        PRK_CHECK(cudaMalloc((void**)&d_trace, (size_t)G * 8 * sizeof(long long)));
        PRK_CHECK(cudaMemsetAsync(d_trace, 0, (size_t)G * 8 * sizeof(long long), s));
    }
    struct TraceGuard {
        long long* p;
        ~TraceGuard() { if (p) cudaFree(p); }
    } trace_guard{d_trace};
    na.trace = d_trace;
    na.history = d_trace ? (float*)(g->nb_block_sweeps + G) : nullptr;
    int launch_no = 0;

    int32_t used = 0;
    int32_t iterations = 0;
    double visits = 0.0;
    double tol_int = tol;
    bool converged = false;
    while (true) {
        PRK_CHECK(cudaMemcpyAsync(g->nb_slots, h_inf, (size_t)G * sizeof(double), cudaMemcpyHostToDevice, s));
        PRK_CHECK(cudaMemsetAsync(g->nb_scalars + 2, 0, 2 * sizeof(double), s));
        k_mass_split<<<small_grid(g), kBlock, 0, s>>>(a, g->x[0], g->nb_scalars);
        ++launches;
        // segment partials of the current vector, read by the first sweep
        PRK_CHECK(launch_segments(g, a, 0, s, &launches));
        na.tol_int = tol_int;
        na.max_sweeps = std::max(1, max_iter - used);
        void* args[] = {&na};
        PRK_CHECK(cudaLaunchCooperativeKernel(kernel, dim3(G), dim3(kBlock), args, 0, s));
        ++launches;
        // verify with one synchronous update x[0] -> x[1]
        k_mass_split<<<small_grid(g), kBlock, 0, s>>>(a, g->x[0], g->nb_scalars + 4);
        ++launches;
        PRK_CHECK(cudaGetLastError());
        PRK_CHECK(enqueue_iteration(g, a, 0, uniform, s, &launches));
        PRK_CHECK(cudaMemcpyAsync(h_counts, g->nb_scalars + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        PRK_CHECK(cudaMemcpyAsync(h_sweeps.data(), g->nb_block_sweeps, (size_t)G * sizeof(int32_t),
                                  cudaMemcpyDeviceToHost, s));
        PRK_CHECK(cudaMemcpyAsync(hs, g->state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        PRK_CHECK(cudaStreamSynchronize(s));
        if (d_trace) {
            std::vector<long long> tr((size_t)G * 8);
            PRK_CHECK(cudaMemcpy(tr.data(), d_trace, tr.size() * sizeof(long long), cudaMemcpyDeviceToHost));
            if (FILE* f = fopen(trace_path, "a")) {
                long long t0 = tr[1];
                for (int c = 0; c < G; ++c) t0 = std::min(t0, tr[8 * c + 1]);
                for (int c = 0; c < G; ++c) {
                    double lr, le;
                    memcpy(&lr, &tr[8 * c + 3], sizeof(double));
                    memcpy(&le, &tr[8 * c + 4], sizeof(double));
                    fprintf(f, "%d,%d,%lld,%lld,%lld,%.6e,%.6e,%lld,%lld,%lld\n", launch_no, c, tr[8 * c],
                            tr[8 * c + 1] - t0, tr[8 * c + 2] - t0, lr, le, tr[8 * c + 5], tr[8 * c + 6],
                            (long long)g->nb_cta_edges[c]);
                }
                fclose(f);
            }
        }
        ++launch_no;
        const int32_t sweeps = (int32_t)(((const int32_t*)(h_counts + 1))[0]);
        used += std::max(1, sweeps);
        iterations += sweeps + 1;
        for (int c = 0; c < G; ++c) visits += (double)h_sweeps[c] * (double)g->nb_cta_edges[c];
        visits += (double)g->nnz;   // the verifying synchronous update
        if (d_trace) {
            float hist[256];
            PRK_CHECK(cudaMemcpy(hist, na.history, sizeof(hist), cudaMemcpyDeviceToHost));
            if (FILE* f = fopen(trace_path, "a")) {
                fprintf(f, "# block0 history");
                for (int k = 0; k < std::min(256, std::max(1, h_sweeps[0])); ++k) fprintf(f, " %.3e", hist[k]);
                fprintf(f, "\n");
                fclose(f);
            }
        }
        if (hs->resid < tol) { converged = true; break; }
        if (used >= max_iter) break;
        tol_int *= 0.25;
    }
    launch_finalize(g, a, out, true, s, &launches);
    PRK_CHECK(cudaGetLastError());
    PRK_CHECK(cudaEventRecord(g->ev_stop, s));
    if (!out_dev)
        PRK_CHECK(cudaMemcpyAsync(x_out, out, (size_t)g->n * sizeof(float), cudaMemcpyDeviceToHost, s));
    PRK_CHECK(cudaMemcpyAsync(hs, g->state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    PRK_CHECK(cudaStreamSynchronize(s));
    float ms = 0.f;
    PRK_CHECK(cudaEventElapsedTime(&ms, g->ev_start, g->ev_stop));
    if (hs->error)
        return fail(PR_ERR_CUDA, "internal error: a row tile exceeded its shared-memory staging area");
    if (info) {
        info->iterations = iterations;
        info->converged = converged ? 1 : 0;
        info->residual_l1 = hs->resid;
        info->sum_x = hs->sum_x;
        info->dangling_mass = hs->D;
        info->edge_visits = visits;
        info->ms_device = ms;
        info->launches = launches;
    }
    return converged ? PR_OK : PR_NOT_CONVERGED;
}

}  // namespace prk
