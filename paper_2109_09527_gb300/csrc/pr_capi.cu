// pr_capi.cu -- error reporting, options, statistics and teardown of the C ABI.
#include <cstring>
#include <mutex>
#include <string>

#include "pr_common.cuh"

namespace prk {

namespace {
thread_local std::string t_last_error;
thread_local int t_heavy_degree = kDefaultHeavy;
thread_local bool t_force_index64 = false;
}  // namespace

void set_error(const std::string& msg) { t_last_error = msg; }

pr_status fail(pr_status s, const std::string& msg) {
    set_error(msg);
    return s;
}

pr_status cuda_fail(cudaError_t e, const char* what) {
    std::string msg = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    set_error(msg);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();  // clear the sticky-free allocation error
        return PR_ERR_OOM;
    }
    return PR_ERR_CUDA;
}

// ---- device memory of graphs: one stream-ordered pool per device ----------
//
// Graph objects and their set-up scratch take memory from a pool the library
// creates per device (cudaMemPoolCreate), with a release threshold that keeps
// freed memory in the pool: a graph created after another was destroyed
// reuses its memory instead of mapping new pages (which, for the gigabytes a
// large graph holds, costs milliseconds per allocation).  The pool keeps at
// most what the library held at its peak; pr_trim_memory returns it to the
// system.  Allocation runs on a library stream that has no other work, and
// that stream is synchronised before the memory is handed out, so any stream
// may use it at once.
#if PRK_POOL
namespace {
constexpr int kPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kPoolDevices] = {};
cudaStream_t g_pool_stream[kPoolDevices] = {};
}  // namespace

cudaError_t lib_pool(cudaMemPool_t* pool, cudaStream_t* stream) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kPoolDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t mp = nullptr;
        if ((e = cudaMemPoolCreate(&mp, &props)) != cudaSuccess) return e;
        uint64_t keep = ~0ull;
        if ((e = cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&g_pool_stream[dev], cudaStreamNonBlocking)) != cudaSuccess) {
            cudaMemPoolDestroy(mp);
            return e;
        }
        g_pool[dev] = mp;
    }
    *pool = g_pool[dev];
    *stream = g_pool_stream[dev];
    return cudaSuccess;
}

cudaError_t pool_alloc(void** p, size_t bytes) {
    *p = nullptr;
    cudaMemPool_t pool;
    cudaStream_t ps;
    cudaError_t e = lib_pool(&pool, &ps);
    if (e != cudaSuccess) return e;
    e = cudaMallocFromPoolAsync(p, bytes ? bytes : 16, pool, ps);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ps);
    if (e != cudaSuccess) *p = nullptr;
    return e;
}

cudaError_t pool_free(void* p, cudaStream_t stream) {
    if (!p) return cudaSuccess;
    if (stream) return cudaFreeAsync(p, stream);
    cudaMemPool_t pool;
    cudaStream_t ps;
    cudaError_t e = lib_pool(&pool, &ps);
    if (e != cudaSuccess) return e;
    return cudaFreeAsync(p, ps);
}

// Blocks last used by work on `stream` go back to the pool on the pool's own
// stream, which first waits for `stream` to reach this point.  Freed there,
// they are reusable in stream order by the next allocation (which runs on
// the pool stream), so a set-up that frees its scratch and then allocates
// does not make the pool grow while the scratch's kernels are still queued.
cudaError_t pool_free_after(void* const* ptrs, size_t count, cudaStream_t stream) {
    if (count == 0) return cudaSuccess;
    cudaMemPool_t pool;
    cudaStream_t ps;
    cudaError_t e = lib_pool(&pool, &ps);
    cudaEvent_t ev = nullptr;
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ps, ev, 0);
    if (ev) cudaEventDestroy(ev);   // released once the wait has been satisfied
    cudaError_t first = e;
    for (size_t i = 0; i < count; ++i)
        if (ptrs[i]) {
            const cudaError_t f = e == cudaSuccess ? cudaFreeAsync(ptrs[i], ps) : cudaFreeAsync(ptrs[i], stream);
            if (first == cudaSuccess) first = f;
        }
    return first;
}
#else
cudaError_t pool_alloc(void** p, size_t bytes) { return cudaMalloc(p, bytes ? bytes : 16); }
cudaError_t pool_free(void* p, cudaStream_t) { return p ? cudaFree(p) : cudaSuccess; }
cudaError_t pool_free_after(void* const* ptrs, size_t count, cudaStream_t) {
    cudaError_t first = cudaSuccess;
    for (size_t i = 0; i < count; ++i)
        if (ptrs[i]) {
            const cudaError_t f = cudaFree(ptrs[i]);
            if (first == cudaSuccess) first = f;
        }
    return first;
}
#endif

cudaError_t dev_alloc(pr_graph* g, void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = pool_alloc(p, bytes);
    if (e == cudaSuccess) g->device_bytes += (int64_t)bytes;
    else *p = nullptr;
    return e;
}

// Memory of a graph object: every kernel that may use it has finished (the
// caller destroys a graph after its last call; the device is synchronised
// first, as cudaFree would).
cudaError_t dev_free(void* p) { return pool_free(p, nullptr); }

bool is_device_pointer(const void* p) {
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int thread_heavy_degree() { return t_heavy_degree; }

void set_thread_heavy_degree(int v) { t_heavy_degree = v; }

bool thread_force_index64() { return t_force_index64; }

}  // namespace prk

using namespace prk;

extern "C" pr_status pr_destroy_graph(pr_graph* g) {
    if (!g) return PR_OK;
    // every kernel that may still use the graph's memory finishes first (what
    // cudaFree did implicitly; the memory goes back to the pool stream-ordered)
    cudaError_t sync = cudaDeviceSynchronize();
    destroy_batch(g);
    destroy_set(g);
    void* dev[] = {g->rowptr, g->colidx, g->inv_out, g->order, g->rank, g->x[0], g->x[1],
                   g->y[0], g->y[1], g->teleport, g->stage, g->seg_row, g->seg_ptr, g->seg_sum,
                   g->tiles, g->tma_tiles, g->tma_fused, g->tma_fused_e1, g->row_cnt, g->hr_part,
                   g->out_src, g->out_pos, g->contrib, g->state, g->slots,
                   g->nb_items, g->nb_slots, g->nbp_items, g->nbp_e1,
                   g->nb_scalars, g->nb_block_sweeps, g->frozen,
                   g->dc_r, g->dc_delta, g->dc_q[0], g->dc_q[1]};
    cudaError_t first = cudaSuccess;
    if (sync != cudaSuccess) first = sync;
    for (void* p : dev)
        if (p) {
            cudaError_t e = dev_free(p);
            if (first == cudaSuccess) first = e;
        }
    for (auto& ex : g->loop_exec)
        if (ex) cudaGraphExecDestroy(ex);
    if (g->host_state) cudaFreeHost(g->host_state);
    if (g->host_flag) cudaFreeHost(g->host_flag);
    if (g->capture_stream) cudaStreamDestroy(g->capture_stream);
    if (g->ev_start) cudaEventDestroy(g->ev_start);
    if (g->ev_stop) cudaEventDestroy(g->ev_stop);
    if (g->ev_loop0) cudaEventDestroy(g->ev_loop0);
    if (g->ev_loop1) cudaEventDestroy(g->ev_loop1);
    delete g;
    if (first != cudaSuccess) return cuda_fail(first, "pr_destroy_graph: freeing device memory");
    return PR_OK;
}

extern "C" pr_status pr_trim_memory(void) {
#if PRK_POOL
    cudaMemPool_t pool;
    cudaStream_t ps;
    cudaError_t e = lib_pool(&pool, &ps);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ps);
    if (e == cudaSuccess) e = cudaMemPoolTrimTo(pool, 0);
    if (e != cudaSuccess) return cuda_fail(e, "pr_trim_memory");
#endif
    return PR_OK;
}

extern "C" pr_status pr_graph_get_stats(const pr_graph* g, pr_graph_stats* s) {
    if (!g || !s) return fail(PR_ERR_INVALID_ARG, "pr_graph_get_stats: NULL argument");
    memset(s, 0, sizeof(*s));
    s->n = g->n;
    s->nnz = g->nnz;
    s->n_dangling = g->n_dangling;
    s->n_zero_indeg = g->n_zero_indeg;
    s->n_heavy = g->n_heavy;
    s->n_segments = g->n_seg;
    s->n_tiles = g->n_tiles;
    s->max_indeg = g->max_indeg;
    s->rowptr_bytes = g->idx64 ? 8 : 4;
    s->sm_count = g->sm_count;
    s->device_bytes = g->device_bytes;
    s->setup_ms = g->setup_ms;
    s->n_tma_tiles = g->n_tma_tiles;
    s->hub_prefix_edges = g->hub_prefix_edges;
    s->n_isolated = g->n_isolated;
    return PR_OK;
}

namespace {

void drop_loop_graphs(pr_graph* g) {
    for (auto& ex : g->loop_exec)
        if (ex) {
            cudaGraphExecDestroy(ex);
            ex = nullptr;
        }
    drop_batch_graph(g);
    drop_set_graph(g);
}

}  // namespace

static pr_status set_option_impl(pr_graph* g, int key, int64_t value) {
    switch (key) {
        case PR_OPT_HEAVY_DEGREE:
            if (g) return fail(PR_ERR_INVALID_ARG, "PR_OPT_HEAVY_DEGREE is set with g = NULL (it applies to the next pr_create_graph)");
            if (value < 64 || value > 4096 || (value & (value - 1)))
                return fail(PR_ERR_INVALID_ARG, "PR_OPT_HEAVY_DEGREE must be a power of two in [64, 4096]");
            set_thread_heavy_degree((int)value);
            return PR_OK;
        case PR_OPT_USE_GRAPH:
            if (!g) return fail(PR_ERR_INVALID_ARG, "PR_OPT_USE_GRAPH needs a graph");
            if (value != 0 && value != 1) return fail(PR_ERR_INVALID_ARG, "PR_OPT_USE_GRAPH is 0 or 1");
            g->use_graph = value == 1;
            return PR_OK;
        case PR_OPT_CTAS_PER_SM:
            if (!g) return fail(PR_ERR_INVALID_ARG, "PR_OPT_CTAS_PER_SM needs a graph");
            if (value < 0 || value > 8) return fail(PR_ERR_INVALID_ARG, "PR_OPT_CTAS_PER_SM is 0 (automatic) to 8");
            g->ctas_per_sm = (int)value;
            return PR_OK;
        case PR_OPT_HOT_VERTICES:
            if (!g) return fail(PR_ERR_INVALID_ARG, "PR_OPT_HOT_VERTICES needs a graph");
            if (value < 0 || value > 0x7fffffffLL) return fail(PR_ERR_INVALID_ARG, "PR_OPT_HOT_VERTICES out of range");
            if ((value >> 28) > 4) return fail(PR_ERR_INVALID_ARG, "PR_OPT_HOT_VERTICES: policy (bits 28..31) must be 0..4");
            g->hot_vertices = value;
            return PR_OK;
        case PR_OPT_TMA_HOT_VERTICES:
            if (!g) return fail(PR_ERR_INVALID_ARG, "PR_OPT_TMA_HOT_VERTICES needs a graph");
            if (value < 0 || value > 0x0fffffffLL)
                return fail(PR_ERR_INVALID_ARG, "PR_OPT_TMA_HOT_VERTICES must be in [0, 2^28)");
            g->tma_hot = value;
            return PR_OK;
        case PR_OPT_HOT_CACHE:
            if (!g) return fail(PR_ERR_INVALID_ARG, "PR_OPT_HOT_CACHE needs a graph");
            if (value < 0 || value > kHotCacheMax)
                return fail(PR_ERR_INVALID_ARG, "PR_OPT_HOT_CACHE must be in [0, 40960]");
            g->hot_cache = value;
            return PR_OK;
        case PR_OPT_STAGED_TILES:
            if (!g) return fail(PR_ERR_INVALID_ARG, "PR_OPT_STAGED_TILES needs a graph");
            if (value < 0 || value > 3)
                return fail(PR_ERR_INVALID_ARG, "PR_OPT_STAGED_TILES must be in [0, 3]");
            g->staged_tiles = (int)value;
            return PR_OK;
        case PR_OPT_NB_HUBS:
            if (!g) return fail(PR_ERR_INVALID_ARG, "PR_OPT_NB_HUBS needs a graph");
            if (value < 0 || value > kNbHubsMax)
                return fail(PR_ERR_INVALID_ARG, "PR_OPT_NB_HUBS must be in [0, 8192]");
            g->nb_hubs = value;
            return PR_OK;
        case PR_OPT_NB_L1_HUBS:
            if (!g) return fail(PR_ERR_INVALID_ARG, "PR_OPT_NB_L1_HUBS needs a graph");
            if (value < 0 || value > 0x7fffffffLL)
                return fail(PR_ERR_INVALID_ARG, "PR_OPT_NB_L1_HUBS must be in [0, 2^31-1]");
            g->nb_l1_hubs = value;
            return PR_OK;
        case PR_OPT_BATCH_BF16:
            if (!g) return fail(PR_ERR_INVALID_ARG, "PR_OPT_BATCH_BF16 needs a graph");
            if (value < 0 || value > 8) return fail(PR_ERR_INVALID_ARG, "PR_OPT_BATCH_BF16 must be in [0, 8]");
            g->batch_bf16 = (int)value;
            return PR_OK;
        case PR_OPT_PERFORATION:
            if (!g) return fail(PR_ERR_INVALID_ARG, "PR_OPT_PERFORATION needs a graph");
            if (value < 0 || value > 30) return fail(PR_ERR_INVALID_ARG, "PR_OPT_PERFORATION must be in [0, 30]");
            if (value > 0 && !g->frozen) {
                cudaError_t e = dev_alloc(g, (void**)&g->frozen, (size_t)(g->n + kPad));
                if (e != cudaSuccess) return cuda_fail(e, "PR_OPT_PERFORATION: allocation");
            }
            g->perforation = (int)value;
            return PR_OK;
        case PR_OPT_DYNAMIC_TILES:
            if (!g) return fail(PR_ERR_INVALID_ARG, "PR_OPT_DYNAMIC_TILES needs a graph");
            if (value != 0 && value != 1) return fail(PR_ERR_INVALID_ARG, "PR_OPT_DYNAMIC_TILES is 0 or 1");
            g->dynamic_tiles = (int)value;
            return PR_OK;
        case PR_OPT_DELAY_NS:
            if (!g) return fail(PR_ERR_INVALID_ARG, "PR_OPT_DELAY_NS needs a graph");
            if (value < 0 || value > 1000000) return fail(PR_ERR_INVALID_ARG, "PR_OPT_DELAY_NS must be in [0, 1e6]");
            g->delay_ns = (int)value;
            return PR_OK;
        case PR_OPT_TMA_TILES:
            if (!g) return fail(PR_ERR_INVALID_ARG, "PR_OPT_TMA_TILES needs a graph");
            if (value != 0 && value != 1) return fail(PR_ERR_INVALID_ARG, "PR_OPT_TMA_TILES is 0 or 1");
            g->use_tma = (int)value;
            return PR_OK;
        case PR_OPT_TEST_WITHHOLD_COPY:
            if (!g) return fail(PR_ERR_INVALID_ARG, "PR_OPT_TEST_WITHHOLD_COPY needs a graph");
            if (value < 0 || value > 1000000)
                return fail(PR_ERR_INVALID_ARG, "PR_OPT_TEST_WITHHOLD_COPY must be in [0, 1e6]");
            g->test_withhold = (int)value;
            return PR_OK;
        case PR_OPT_NB_FAIL_AFTER:
            if (!g) return fail(PR_ERR_INVALID_ARG, "PR_OPT_NB_FAIL_AFTER needs a graph");
            if (value < 0 || value > 1000000)
                return fail(PR_ERR_INVALID_ARG, "PR_OPT_NB_FAIL_AFTER must be in [0, 1e6]");
            g->nb_fail_after = (int)value;
            return PR_OK;
        case PR_OPT_BATCH_DC:
            if (!g) return fail(PR_ERR_INVALID_ARG, "PR_OPT_BATCH_DC needs a graph");
            if (value < 0 || value > 32) return fail(PR_ERR_INVALID_ARG, "PR_OPT_BATCH_DC must be in [0, 32]");
            g->batch_dc = (int)value;
            return PR_OK;
        case PR_OPT_BATCH_ASYNC:
            if (!g) return fail(PR_ERR_INVALID_ARG, "PR_OPT_BATCH_ASYNC needs a graph");
            if (value != 0 && value != 1) return fail(PR_ERR_INVALID_ARG, "PR_OPT_BATCH_ASYNC is 0 or 1");
            g->batch_async = (int)value;
            return PR_OK;
        case PR_OPT_NB_PIPELINE:
            if (!g) return fail(PR_ERR_INVALID_ARG, "PR_OPT_NB_PIPELINE needs a graph");
            if (value != 0 && value != 1) return fail(PR_ERR_INVALID_ARG, "PR_OPT_NB_PIPELINE is 0 or 1");
            g->nb_pipeline = (int)value;
            return PR_OK;
        case PR_OPT_SYNC_DC:
            if (!g) return fail(PR_ERR_INVALID_ARG, "PR_OPT_SYNC_DC needs a graph");
            if (value < 0 || value > 32) return fail(PR_ERR_INVALID_ARG, "PR_OPT_SYNC_DC must be in [0, 32]");
            g->sync_dc = (int)value;
            return PR_OK;
        case PR_OPT_IMPLICIT_ZERO_ROWS:
            if (!g) return fail(PR_ERR_INVALID_ARG, "PR_OPT_IMPLICIT_ZERO_ROWS needs a graph");
            if (value != 0 && value != 1) return fail(PR_ERR_INVALID_ARG, "PR_OPT_IMPLICIT_ZERO_ROWS is 0 or 1");
            g->implicit_zero = (int)value;
            return PR_OK;
        case PR_OPT_FUSED_SEGMENTS:
            if (!g) return fail(PR_ERR_INVALID_ARG, "PR_OPT_FUSED_SEGMENTS needs a graph");
            if (value != 0 && value != 1) return fail(PR_ERR_INVALID_ARG, "PR_OPT_FUSED_SEGMENTS is 0 or 1");
            g->fuse_segments = (int)value;
            return PR_OK;
        case PR_OPT_LIGHT_LANES:
            if (!g) return fail(PR_ERR_INVALID_ARG, "PR_OPT_LIGHT_LANES needs a graph");
            if (value != 0 && value != 1) return fail(PR_ERR_INVALID_ARG, "PR_OPT_LIGHT_LANES is 0 or 1");
            g->lane_mode = (int)value;
            return PR_OK;
        case PR_OPT_INDEX64:
            if (g) return fail(PR_ERR_INVALID_ARG, "PR_OPT_INDEX64 is set with g = NULL (it applies to the next pr_create_graph)");
            if (value != 0 && value != 1) return fail(PR_ERR_INVALID_ARG, "PR_OPT_INDEX64 is 0 or 1");
            t_force_index64 = value == 1;
            return PR_OK;
        default:
            return fail(PR_ERR_INVALID_ARG, "unknown option key");
    }
}

extern "C" pr_status pr_set_option(pr_graph* g, int key, int64_t value) {
    pr_status rc = set_option_impl(g, key, value);
    // captured loop graphs bake the options in: rebuild them on next use
    if (rc == PR_OK && g) drop_loop_graphs(g);
    return rc;
}


extern "C" const char* pr_status_string(pr_status s) {
    switch (s) {
        case PR_OK: return "PR_OK";
        case PR_ERR_INVALID_ARG: return "PR_ERR_INVALID_ARG";
        case PR_ERR_CUDA: return "PR_ERR_CUDA";
        case PR_ERR_OOM: return "PR_ERR_OOM";
        case PR_NOT_CONVERGED: return "PR_NOT_CONVERGED";
        case PR_ERR_UNSUPPORTED: return "PR_ERR_UNSUPPORTED";
        case PR_ERR_INVALID_GRAPH: return "PR_ERR_INVALID_GRAPH";
        case PR_ERR_DEVICE_TIMEOUT: return "PR_ERR_DEVICE_TIMEOUT";
        default: return "PR_UNKNOWN_STATUS";
    }
}

extern "C" const char* pr_last_error(void) { return prk::t_last_error.c_str(); }
