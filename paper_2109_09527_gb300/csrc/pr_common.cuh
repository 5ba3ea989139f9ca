// pr_common.cuh -- internal definitions shared by the library's CUDA sources.
//
// Device data layout of a graph (all in HBM, owned by pr_graph):
//   Vertices are relabelled at set-up so that rows with similar in-degree are
//   contiguous: first the heavy rows (in-degree >= heavy threshold, gathered in
//   fixed-size edge segments), then the light rows in bins of decreasing
//   power-of-two in-degree class, then the rows without in-edges.  Every
//   per-vertex vector below is in this "binned" order; order[i] is the caller's
//   id of binned vertex i and rank[v] the binned id of caller vertex v.
//
//   rowptr   IdxT[n+1]   in-edge offsets (IdxT = int32 when nnz < 2^31)
//   colidx   int32[nnz]  binned source ids, each row in the caller's order
//   inv_out  float[n]    1/outdeg, 0 for dangling vertices
//   x[2], y[2] float[n]  rank and rank/outdeg (the quotient vector the gather
//                        reads), double-buffered for the synchronous update
//   seg_*                segments of heavy rows and their partial sums
//   tiles               row ranges of the per-iteration row kernel
//
// Every array is allocated with kPad spare elements so that 16-byte vector
// loads that start inside the array never leave the allocation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "pagerank.h"

namespace prk {

struct BatchCtx;   // buffers of the batched solver (pr_batched.cu)
struct SetCtx;     // partition and buffers of the graph-set solver (pr_set.cu)

constexpr int kBlock = 256;              // threads of a tile group (and of the small kernels)
constexpr int kWarps = kBlock / 32;
constexpr int kIterBlock = 256;          // threads per block of the Jacobi iteration kernels
// Blocks per SM the gather kernels are compiled for (__launch_bounds__): with
// 256 threads, 4 blocks allow 64 registers a thread, 6 allow 40, 8 allow 32.
#ifndef PRK_GATHER_MIN_BLOCKS
#define PRK_GATHER_MIN_BLOCKS 4
#endif
constexpr int kGatherMinBlocks = PRK_GATHER_MIN_BLOCKS;
// The barrier-free kernel is latency-bound.  With two edges of each row in
// flight per lane, six blocks per SM (40 registers a thread, a few spilled)
// measured faster than four (ER-24: 2.15 -> 1.77 ms per sweep-equivalent).
// With the next step's column indices loaded while a step's gathers are in
// flight, four blocks of four edges per row and lane (61 registers) measured
// best (R-MAT-24 + ER-24 solves: 24.05 ms, against 24.18 at five blocks of
// four edges, 24.42 at five of two, 24.98 at six of two).
#ifndef PRK_NB_MIN_BLOCKS
#define PRK_NB_MIN_BLOCKS 4
#endif
// Edges of each of its two rows a lane of the barrier-free kernel gathers per step.
#ifndef PRK_NB_UNROLL
#define PRK_NB_UNROLL 4
#endif
constexpr int kNbMinBlocks = PRK_NB_MIN_BLOCKS;
constexpr int kHotCacheMax = 40960;      // largest shared-memory copy of y's hot prefix (160 KB)
constexpr int kTileEdgesMax = 6144;      // edges of a light tile
constexpr int kTileRowsMax = 2048;       // rows of a light tile
constexpr int kSegEdges = 2048;          // edges per segment of a heavy row
constexpr int kDefaultHeavy = 256;       // default heavy in-degree threshold
constexpr int kNbSegDegree = 1024;       // rows the barrier-free kernel gathers in segments (see build_items)
constexpr int kPad = 64;                 // spare elements after every device array
constexpr int kTileHeavy = -1;           // tile kind: epilogue of heavy rows
constexpr int kTileZero = -2;            // tile kind: rows without in-edges
constexpr int kTileSeg = -3;             // tile kind (fused pipelined kernel): one 2048-edge segment of a
                                         // heavy row; row_begin = the row, row_end = the segment's index
constexpr int kMaxBins = 43;
// 1: graph memory and set-up scratch come from the library's stream-ordered
// pool (pool_alloc); 0: plain cudaMalloc / cudaFree.
#ifndef PRK_POOL
#define PRK_POOL 1
#endif
// Lanes per row of light tiles (PR_OPT_LIGHT_LANES): 0 by degree class, 1 by
// the tile's row count (see light_lanes_log2).
#ifndef PRK_DEFAULT_LANE_MODE
#define PRK_DEFAULT_LANE_MODE 1
#endif
constexpr int kDefaultLaneMode = PRK_DEFAULT_LANE_MODE;
#ifndef PRK_DEFAULT_BATCH_ASYNC
#define PRK_DEFAULT_BATCH_ASYNC 1
#endif
constexpr int kDefaultBatchAsync = PRK_DEFAULT_BATCH_ASYNC;

// Pipelined synchronous row kernel (k_rows_tma): a producer warp copies each
// tile's offsets, column indices and per-row vectors into shared memory with
// bulk asynchronous copies, kTmaStages tiles deep, for 8 consumer warps.  Its
// tiles are the same bins cut to at most kTmaEdges edges and kTmaRows rows.
#ifndef PRK_TMA_STAGES
#define PRK_TMA_STAGES 2
#endif
#ifndef PRK_TMA_EDGES
#define PRK_TMA_EDGES 3072
#endif
#ifndef PRK_TMA_ROWS
#define PRK_TMA_ROWS 512
#endif
#ifndef PRK_TMA_MIN_BLOCKS
#define PRK_TMA_MIN_BLOCKS 3
#endif
constexpr int kTmaStages = PRK_TMA_STAGES;
constexpr int kTmaEdges = PRK_TMA_EDGES;
constexpr int kTmaRows = PRK_TMA_ROWS;
constexpr int kTmaMinBlocks = PRK_TMA_MIN_BLOCKS;
constexpr int kTmaColWords = kTmaEdges + 8;    // a copy starts up to 3 words early and ends up to 3 late
constexpr int kTmaRowWords = kTmaRows + 8;     // rows + 1 offsets, same slack
constexpr int kTmaStageWords = kTmaColWords + 4 * kTmaRowWords;   // colidx, rowptr, x, 1/outdeg, teleport
constexpr int kTmaThreads = kBlock + 32;       // 8 consumer warps + 1 producer warp
constexpr size_t kTmaSmemBytes = 2 * kTmaStages * sizeof(uint64_t) + (size_t)kTmaStages * kTmaStageWords * 4;
#ifndef PRK_DEFAULT_STAGED
#define PRK_DEFAULT_STAGED 0
#endif
constexpr int kDefaultStaged = PRK_DEFAULT_STAGED;
constexpr int kNbHubsMax = 8192;         // largest hub snapshot of the barrier-free kernel (32 KB)
#ifndef PRK_DEFAULT_NB_HUBS
#define PRK_DEFAULT_NB_HUBS 0
#endif
constexpr int kDefaultNbHubs = PRK_DEFAULT_NB_HUBS;
constexpr int64_t kDefaultNbL1Hubs = 49152;   // barrier-free hub gathers through L1  // light-tile mode per variant (PR_OPT_STAGED_TILES)
constexpr int64_t kDefaultTmaHot = 16384;  // the pipelined row kernel's hub count (its L1 is smaller)
constexpr int64_t kDefaultHot = (4LL << 28) | 49152;  // gather L1 policy 4, 48K hot ids (see ld_gather)   // degree bins: 40 power-of-two classes + zero + spare

// A tile of the row kernel: rows [row_begin, row_end) of one bin.  kind >= 0
// is log2 of the lanes that gather one row together.
struct Tile {
    int32_t row_begin;
    int32_t row_end;
    int32_t kind;
    int32_t pad;
};

// Per-solve device state.  Parameters are written by the host before a solve;
// the running fields are written by the last block of each kernel that
// reduces (see the "last block" pattern in pr_jacobi.cu).
struct SolveState {
    double d;          // damping
    double tol;        // stop when the L1 change of an iteration is below this
    double inv_n;      // 1/n
    double t_sum;      // sum of the teleport vector (1 when uniform)
    int32_t max_iter;
    int32_t uniform_t;
    double D;          // dangling mass of the current input vector
    double resid;      // L1 change of the last iteration
    double sum_x;      // sum of the final vector (finalise)
    double scale;      // t_sum / sum_x (finalise)
    double edge_visits;
    int32_t iter;      // iterations completed
    int32_t done;      // stopping test met or budget spent
    uint32_t ticket;   // arrival counter of the last-block reductions
    uint32_t error;    // device-side error bits
    int32_t sweeps_max;
    uint32_t tile_next;  // next tile to hand out (dynamic tile assignment)
    uint32_t frozen;     // rows frozen by loop perforation (counted after the solve)
    int32_t implicit;    // 1: ranks of rows without in-edges implicit after the first update
    double Dz;           // implicit rows: the dangling mass their current ranks use
    double t_iso;        // implicit rows: teleport sum over the isolated vertices
    double Ldc;          // correction sweeps: mass the BF16 quotients of delta do not pass on
};

// Arguments of the per-iteration kernels (passed by value).
struct IterArgs {
    const void* rowptr;          // IdxT*
    const int32_t* colidx;
    const float* inv_out;
    const float* teleport;       // binned order, NULL when uniform
    const int32_t* seg_row;      // heavy row of each segment
    const int32_t* seg_ptr;      // first segment of each heavy row, [n_heavy+1]
    float* seg_sum;              // partial gather sum of each segment
    const Tile* tiles;
    int64_t n;
    int32_t n_seg;
    int32_t n_tiles;
    SolveState* state;
    double* slots;               // two doubles per block of the row kernel
    cudaGraphConditionalHandle cond;
    int32_t use_cond;            // 1: the kernel runs inside the while-graph
    int32_t hot;                 // L1 policy of the global gathers (ld_gather)
    int32_t hot_n;               // ids [0, hot_n) of y are cached in shared memory
    int32_t staged;              // 1: light tiles gathered edge-parallel (process_staged_tile)
    uint8_t* frozen;             // loop perforation: frozen rows (NULL = off)
    float perf_eps;
    int32_t dynamic;             // 1: blocks take tiles from a shared counter (helping)
    int32_t delay_ns;            // > 0: block 0 sleeps this long per tile (slow-processor model)
    int32_t withhold;            // > 0: test hook of the pipelined kernel (PR_OPT_TEST_WITHHOLD_COPY)
    int64_t nnz;
    int32_t edge;                // 1: the edge-centric iteration (Alg. 2, pr_edge.cu)
    int32_t lane_mode;           // lanes per light row (PR_OPT_LIGHT_LANES)
    const int32_t* out_src;      // edge-centric form: source of each out-edge, in out-edge order
    const int32_t* out_pos;      // edge-centric form: in-edge slot of each out-edge
    const int32_t* tile_e1;      // fused pipelined kernel: one past the last edge of each tile
    int32_t* row_cnt;            // fused: segments of each heavy row gathered so far this iteration
    float2* hr_part;             // fused: (L1 change, dangling mass) of each heavy row's update
    int32_t fused;               // 1: heavy-row segments are tiles of the pipelined kernel
    int32_t n_heavy;             // rows [0, n_heavy) are gathered in segments
    int32_t n_tiles_live;        // pipelined kernel: tiles before those of the isolated vertices
    int32_t hot_tma;             // pipelined kernel: L1 policy and hub count of its gathers (as hot)
    int64_t zero_start;          // rows [zero_start, n) have no in-edges
    int64_t iso_start;           // rows [iso_start, n) have no in- and no out-edges
};

}  // namespace prk

// The opaque graph object of the C ABI.
struct pr_graph {
    int device = 0;
    int sm_count = 0;
    int64_t n = 0;
    int64_t nnz = 0;
    bool idx64 = false;          // rowptr kept as int64
    bool out_layout = false;     // created from an out-edge CSR (PR_OUT_CSR), transposed at set-up
    int heavy_degree = prk::kDefaultHeavy;
    int ctas_per_sm = 0;         // 0 = from occupancy
    bool use_graph = true;
    int64_t hot_vertices = prk::kDefaultHot;  // see ld_gather
    int64_t tma_hot = prk::kDefaultTmaHot;    // hub count of the pipelined row kernel (PR_OPT_TMA_HOT_VERTICES)
    int64_t hot_cache = 0;                    // size of the shared-memory copy of y's prefix (off)
    int64_t nb_hubs = prk::kDefaultNbHubs;    // hub snapshot of the barrier-free kernel (PR_OPT_NB_HUBS)
    int64_t nb_l1_hubs = prk::kDefaultNbL1Hubs;  // weak L1-cached hub gathers (PR_OPT_NB_L1_HUBS)
    int batch_bf16 = 0;                       // batched solver: BF16 Y until changes < 10^-value (0 = off)
    int batch_dc = 0;                         // batched solver: BF16 correction sweeps per FP32 step (0 = off)
    int batch_async = prk::kDefaultBatchAsync; // batched gathers with asynchronous copies (PR_OPT_BATCH_ASYNC)
    int implicit_zero = 1;                    // ranks of rows without in-edges kept implicit in the
                                              // batched solver and the pipelined synchronous iteration
                                              // (PR_OPT_IMPLICIT_ZERO_ROWS)
    int perforation = 0;                      // loop perforation eps = 10^-value (0 = off)
    int dynamic_tiles = 0;                    // PR_OPT_DYNAMIC_TILES
    int delay_ns = 0;                         // PR_OPT_DELAY_NS
    uint8_t* frozen = nullptr;                // frozen rows of the perforated synchronous solve
    int staged_tiles = prk::kDefaultStaged;   // bit 0: Jacobi, bit 1: barrier-free (see PR_OPT_STAGED_TILES)
    int use_tma = 1;                          // PR_OPT_TMA_TILES: pipelined synchronous row kernel
    int lane_mode = prk::kDefaultLaneMode;    // PR_OPT_LIGHT_LANES: lanes per light row
    int test_withhold = 0;                    // PR_OPT_TEST_WITHHOLD_COPY (test hook, 0 = off)
    int nb_fail_after = 0;                    // PR_OPT_NB_FAIL_AFTER (0 = off)

    void* rowptr = nullptr;
    int32_t* colidx = nullptr;
    float* inv_out = nullptr;
    int32_t* order = nullptr;    // binned -> caller id
    int32_t* rank = nullptr;     // caller -> binned id
    float* x[2] = {nullptr, nullptr};
    float* y[2] = {nullptr, nullptr};
    float* teleport = nullptr;   // binned teleport (allocated on first use)
    int sync_dc = 0;             // BF16 correction sweeps per FP32 step of the synchronous solver (PR_OPT_SYNC_DC)
    float* dc_r = nullptr;       // correction sweeps: residual F(x) - x of the FP32 step
    float* dc_delta = nullptr;   // correction sweeps: the latest correction (FP32)
    void* dc_q[2] = {nullptr, nullptr};   // correction sweeps: BF16 quotients delta / outdeg
    float* stage = nullptr;      // staging for host inputs/outputs (first use)
    int32_t* seg_row = nullptr;
    int32_t* seg_ptr = nullptr;
    float* seg_sum = nullptr;
    prk::Tile* tiles = nullptr;
    prk::Tile* tma_tiles = nullptr;  // tiles of k_rows_tma (pad = first edge), + a sentinel at n
    int32_t* out_src = nullptr;      // edge-centric form (first use): out-edge sources and in-edge slots,
    int32_t* out_pos = nullptr;      // and the per-edge contribution array
    float* contrib = nullptr;
    int64_t n_tma_tiles = 0;         // 0: the layout cannot use k_rows_tma
    int64_t hub_prefix_edges = 0;    // edges whose source is among the default L1 hub prefix
    prk::Tile* tma_fused = nullptr;  // fused tile list: light and empty-row tiles with every heavy-row
                                     // segment as a tile of its own, interleaved (pad = first edge)
    int32_t* tma_fused_e1 = nullptr; // one past the last edge of each fused tile
    int64_t n_tma_fused = 0;         // 0: no fused list (no heavy rows, or the kernel does not apply)
    int32_t* row_cnt = nullptr;      // per heavy row: its segments gathered so far in an iteration
    float2* hr_part = nullptr;       // per heavy row: (L1 change, dangling mass) of its update
    int fuse_segments = 0;           // PR_OPT_FUSED_SEGMENTS (off: measured 2.5x slower, see the option)
    prk::SolveState* state = nullptr;
    double* slots = nullptr;
    int slot_capacity = 0;       // blocks the slot array can serve
    prk::SolveState* host_state = nullptr;  // pinned mirror
    int32_t* host_flag = nullptr;           // pinned: done flag of the host-driven loop

    // barrier-free solver (built on first use)
    int32_t* nb_items = nullptr;     // Tile[]: work items of the persistent kernel
    double* nb_slots = nullptr;      // latest sweep residual of each block
    double* nb_scalars = nullptr;    // running non-dangling mass, counters
    int32_t* nb_block_sweeps = nullptr;  // sweeps per block of the last launch (+ diagnostics)
    int nb_grid = 0;
    int64_t nb_items_count = 0;
    int64_t nb_n_seg = 0;                // segments the barrier-free kernel gathers (the first ones)
    std::vector<int64_t> nb_cta_edges;  // edges owned by each block (items dealt round-robin)
    std::vector<int64_t> nb_item_edges; // edges of each work item
    std::vector<int64_t> nb_seg_edges;  // edges of each heavy-row segment
    int32_t* nbp_items = nullptr;       // Tile[]: light and empty-row tiles of the pipelined kernel (pad = first edge)
    int32_t* nbp_e1 = nullptr;          // one past the last edge of each of those tiles
    int64_t nbp_items_count = 0;
    std::vector<int64_t> nbp_item_edges;
    int nb_pipeline = 0;                // PR_OPT_NB_PIPELINE (measured slower: off)
    std::vector<int64_t> bin_start;     // first binned row of each degree bin (+ n)
    std::vector<prk::Tile> host_tiles;  // copy of tiles

    int64_t n_heavy = 0;
    int64_t n_seg = 0;
    int64_t n_tiles = 0;
    int64_t n_dangling = 0;
    int64_t n_zero_indeg = 0;
    int64_t n_isolated = 0;             // no in- and no out-edges: the last rows of the binned order
    int64_t n_tma_live = 0;             // pipelined-kernel tiles before those of the isolated vertices
    int64_t max_indeg = 0;
    int64_t device_bytes = 0;
    float setup_ms = 0.f;

    // while-graph of the Jacobi loop, one per teleport kind (uniform / given)
    cudaGraphExec_t loop_exec[2] = {nullptr, nullptr};
    cudaStream_t capture_stream = nullptr;
    cudaEvent_t ev_start = nullptr;
    cudaEvent_t ev_stop = nullptr;
    cudaEvent_t ev_loop0 = nullptr;  // around the iteration loop alone
    cudaEvent_t ev_loop1 = nullptr;

    prk::BatchCtx* batch = nullptr;  // batched solver (built on first use)
    prk::SetCtx* set = nullptr;      // graph-set partition (pr_graph_set_partition)
};

namespace prk {

// Thread-local error message of the C ABI.
void set_error(const std::string& msg);
pr_status fail(pr_status s, const std::string& msg);
pr_status cuda_fail(cudaError_t e, const char* what);

// Grid size of the persistent per-iteration kernels for graph g.
int row_grid(const pr_graph* g, bool staged);
int seg_grid(const pr_graph* g);

// Device allocation recorded in g->device_bytes.
cudaError_t dev_alloc(pr_graph* g, void** p, size_t bytes);
cudaError_t dev_free(void* p);
// Memory from the library's pool on the current device (see pr_capi.cu):
// pool_free with a stream frees in that stream's order, without a stream on
// the library's own stream (the caller has made sure nothing still uses it).
cudaError_t pool_alloc(void** p, size_t bytes);
cudaError_t pool_free(void* p, cudaStream_t stream);

bool is_device_pointer(const void* p);

// Heavy in-degree threshold that the next pr_create_graph of this thread uses.
int thread_heavy_degree();
void set_thread_heavy_degree(int v);
bool thread_force_index64();

// Allocate the solver's vectors, state and slots once the layout exists.
pr_status alloc_solver(pr_graph* g);

// Solver pieces shared by the synchronous and the barrier-free drivers.
IterArgs make_args(const pr_graph* g, bool uniform);
int small_grid(const pr_graph* g);
cudaError_t enqueue_iteration(const pr_graph* g, const IterArgs& a, int src, bool uniform,
                              cudaStream_t s, int* launches);
cudaError_t launch_segments(const pr_graph* g, const IterArgs& a, int src, cudaStream_t s, int* launches);
// Edge-centric iteration (Alg. 2): its out-edge list, built on first use, and
// one iteration reading buffer src.
pr_status ensure_edge(pr_graph* g, cudaStream_t s);
cudaError_t enqueue_edge_iteration(const pr_graph* g, const IterArgs& a, int src, bool uniform, cudaStream_t s,
                                   int* launches);
// Tile list of the layout for another heavy threshold (>= the layout's own),
// and the number of rows at or above it.
std::vector<Tile> tiles_with_threshold(const pr_graph* g, int heavy_degree, int64_t* heavy_rows,
                                       int64_t max_edges = kTileEdgesMax, int64_t max_rows = kTileRowsMax);
// Set pad = offset of the first edge for tiles[0..count] (the last one a
// sentinel at row n), 32-bit offsets.
cudaError_t fill_tile_edges(Tile* tiles, int64_t count, const int32_t* rowptr, cudaStream_t s);
pr_status stage_input(pr_graph* g, const float* src, int slot, cudaStream_t s, const float** out);
pr_status ensure_stage(pr_graph* g);
pr_status ensure_teleport(pr_graph* g);
void launch_init(const pr_graph* g, const IterArgs& a, const float* t_dev, const float* x0_dev,
                 cudaStream_t s);
// Edge ranges (pad, e1) and segment rows of the fused tile list of k_rows_tma.
cudaError_t fill_fused_tiles(Tile* tiles, int32_t* e1, int64_t count, const int32_t* rowptr, const int32_t* seg_row,
                             const int32_t* seg_ptr, cudaStream_t s);
// Count the frozen rows of a perforated solve into SolveState::frozen.
cudaError_t launch_count_frozen(const pr_graph* g, cudaStream_t s);
void launch_finalize(const pr_graph* g, const IterArgs& a, float* out, bool renormalise,
                     cudaStream_t s, int* launches, bool implicit = false);
// Defect correction with BF16 quotients after the FP32 step x[src] -> x[1-src]
// of the synchronous solver (PR_OPT_SYNC_DC, pr_dc.cu).
pr_status ensure_sync_dc(pr_graph* g);
cudaError_t enqueue_sync_dc(const pr_graph* g, const IterArgs& a, int src, int sweeps, cudaStream_t s,
                            int* launches);

// Exclusive scan of count int64 values into int32 offsets[count + 1] (device
// arrays); synchronises the stream before its temporaries are freed.
cudaError_t scan_counts_i32(const int64_t* counts, int64_t count, int32_t* offsets, cudaStream_t st);

// Free the batched / graph-set solvers' buffers (nothing if never used), or
// only their captured loop graphs.
void destroy_batch(pr_graph* g);
void destroy_set(pr_graph* g);
void drop_batch_graph(pr_graph* g);
void drop_set_graph(pr_graph* g);

pr_status solve_nonblocking(pr_graph* g, float damping, double tol, int32_t max_iter,
                            const float* teleport, const float* x0, float* x_out, pr_info* info,
                            cudaStream_t s);

}  // namespace prk

#define PRK_CHECK(call)                                                     \
    do {                                                                    \
        cudaError_t prk_e_ = (call);                                        \
        if (prk_e_ != cudaSuccess) return prk::cuda_fail(prk_e_, #call);    \
    } while (0)
