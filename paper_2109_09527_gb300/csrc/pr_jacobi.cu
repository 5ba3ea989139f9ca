// pr_jacobi.cu -- the synchronous (Jacobi) PageRank iteration on the device.
//
// One iteration k (Alg. 1, loop body) computes, from x = x_k and its quotient
// vector y = x / outdeg (0 for dangling vertices):
//
//   s(v)   = sum_{e in row v} y[colidx[e]]                      (gather)
//   x'(v)  = (1-d) t(v) + d (s(v) + D/n)                        (Eq. 1 + dangling share)
//   y'(v)  = x'(v) / outdeg(v)                                  (next quotient)
//   D'     = sum_{outdeg(v)=0} x'(v)                            (next dangling mass)
//   r      = sum_v |x'(v) - x(v)|                               (L1 change)
//
// Two launches per iteration:
//   k_heavy_segments  a warp per 2048-edge segment of every heavy row: streams
//                     colidx with 16-byte loads, gathers y, writes the
//                     segment's partial sum;
//   k_rows_tma        (default) persistent blocks walk the row tiles
//                     round-robin, a producer warp staging each tile's
//                     offsets, column indices and per-row vectors in shared
//                     memory ahead of 8 gathering warps (see below):
//                     heavy-row epilogues (sum of the segment partials),
//                     light rows gathered by groups of 1..32 lanes sized to
//                     the bin's degree class, rows without in-edges; the
//                     epilogue writes x' and y' and accumulates r and D'.
//                     The last block to finish (arrival ticket) reduces the
//                     per-block partials in a fixed order, so D' and r are
//                     bitwise reproducible, and applies the stopping test;
//   k_rows            the same without staging (64-bit offsets, long light
//                     rows, and the staged, perforated and dynamic modes).
//
// The solve loop is a CUDA graph with a conditional while node whose body
// holds two iterations (x0 -> x1, x1 -> x0); the last block clears the
// condition when r < tol or the budget is spent.
#include <algorithm>
#include <cmath>
#include <vector>

#include <cstring>

#include "pr_tile.cuh"
#include "pr_tma.cuh"

namespace prk {

// 1: the segment kernel loads the next 256-edge chunk's indices while the
// current chunk's gathers are in flight; 0: 512-edge chunks, loads then gathers.
#ifndef PRK_SEG_PIPE
#define PRK_SEG_PIPE 0
#endif

// --------------------------------------------------------- iteration kernels --

// Copy y[0, hot_n) -- the sources of most edges in a power-law graph, which
// the degree binning puts first -- into shared memory with 16-byte loads.
__device__ __forceinline__ void load_hot(const float* __restrict__ y, int32_t hot_n, float* sm) {
    const float4* src = reinterpret_cast<const float4*>(y);
    float4* dst = reinterpret_cast<float4*>(sm);
    for (int i = threadIdx.x; i < (hot_n >> 2); i += blockDim.x) dst[i] = __ldg(src + i);
    __syncthreads();
}

// YT: FP32 quotients, or BF16 ones (the correction sweeps of PR_OPT_SYNC_DC,
// no shared-memory hub copy).
template <typename IdxT, typename YT = float>
__global__ void __launch_bounds__(kIterBlock, kGatherMinBlocks) k_heavy_segments(IterArgs a, const YT* __restrict__ y) {
    extern __shared__ __align__(16) float hot_sm[];
    if (block_state(a.state).done) return;
    if constexpr (std::is_same<YT, float>::value) load_hot(y, a.hot_n, hot_sm);
    RowCtx c{};
    c.hot = a.hot;
    c.hot_n = a.hot_n;
    c.hot_sm = hot_sm;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s = warp; s < a.n_seg; s += nwarp) {
        const int32_t h = a.seg_row[s];
        const int64_t re = row_at<IdxT>(a.rowptr, h + 1);
        const int64_t e0 = row_at<IdxT>(a.rowptr, h) + (s - a.seg_ptr[h]) * (int64_t)kSegEdges;
        const int64_t e1 = min(e0 + (int64_t)kSegEdges, re);
        const int64_t a0 = e0 & ~(int64_t)3;   // 16-byte aligned start
        float acc = 0.f;
#if PRK_SEG_PIPE
        // 256-edge chunks, the next chunk's indices loaded while this chunk's
        // gathers are in flight
        int4 cv[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int64_t p = a0 + 128 * j + 4 * lane;
            cv[j] = p < e1 ? ld_stream4(a.colidx + p) : make_int4(0, 0, 0, 0);
        }
        for (int64_t base = a0; base < e1; base += 256) {
            int4 nx[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int64_t p = base + 256 + 128 * j + 4 * lane;
                nx[j] = p < e1 ? ld_stream4(a.colidx + p) : make_int4(0, 0, 0, 0);
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int64_t p = base + 128 * j + 4 * lane;
                const float v0 = (p + 0 >= e0 && p + 0 < e1) ? Mem<false>::gather(y, cv[j].x, c) : 0.f;
                const float v1 = (p + 1 >= e0 && p + 1 < e1) ? Mem<false>::gather(y, cv[j].y, c) : 0.f;
                const float v2 = (p + 2 >= e0 && p + 2 < e1) ? Mem<false>::gather(y, cv[j].z, c) : 0.f;
                const float v3 = (p + 3 >= e0 && p + 3 < e1) ? Mem<false>::gather(y, cv[j].w, c) : 0.f;
                acc += (v0 + v1) + (v2 + v3);
            }
            cv[0] = nx[0];
            cv[1] = nx[1];
        }
#else
        for (int64_t base = a0; base < e1; base += 512) {
            int4 cv[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t p = base + 128 * j + 4 * lane;
                cv[j] = p < e1 ? ld_stream4(a.colidx + p) : make_int4(0, 0, 0, 0);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t p = base + 128 * j + 4 * lane;
                const float v0 = (p + 0 >= e0 && p + 0 < e1) ? Mem<false>::gather(y, cv[j].x, c) : 0.f;
                const float v1 = (p + 1 >= e0 && p + 1 < e1) ? Mem<false>::gather(y, cv[j].y, c) : 0.f;
                const float v2 = (p + 2 >= e0 && p + 2 < e1) ? Mem<false>::gather(y, cv[j].z, c) : 0.f;
                const float v3 = (p + 3 >= e0 && p + 3 < e1) ? Mem<false>::gather(y, cv[j].w, c) : 0.f;
                acc += (v0 + v1) + (v2 + v3);
            }
        }
#endif
        acc = warp_sum(acc);
        if (lane == 0) a.seg_sum[s] = acc;
    }
}

// One block of kIterBlock threads per SM; each 256-thread group walks its own
// tiles (round-robin over all groups of the grid) and shares the block's copy
// of the hot prefix of y.
template <typename IdxT, bool kUniform, bool kStaged, bool kPerf>
__global__ void __launch_bounds__(kIterBlock, kGatherMinBlocks) k_rows(IterArgs a, const float* __restrict__ x_in,
                                                     const float* __restrict__ y_in,
                                                     float* __restrict__ x_out, float* __restrict__ y_out) {
    extern __shared__ __align__(16) float hot_sm[];
    SolveState* st = a.state;
    const StateView sv = block_state(st);
    if (sv.done) {
        // A skipped iteration inside the while-graph keeps the loop closed.
        if (a.use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(a.cond, 0);
        return;
    }
    load_hot(y_in, a.hot_n, hot_sm);
    const double d = sv.d;
    const double share = sv.D * sv.inv_n;   // D/n
    RowCtx c;
    c.d = (float)d;
    c.one_m_d = (float)(1.0 - d);
    c.d_share = (float)(d * share);
    c.base = (float)((1.0 - d) * sv.inv_n + d * share);
    c.hot = a.hot;
    c.hot_n = a.hot_n;
    c.hot_sm = hot_sm;
    c.lane_mode = a.lane_mode;
    const Perf pf{a.frozen, a.perf_eps};
    Acc acc;
    const int groups = blockDim.x / kBlock;
    const int tid = threadIdx.x & (kBlock - 1);
    const int group = blockIdx.x * groups + threadIdx.x / kBlock;

    // Static assignment: tiles group, group + #groups, ...  Dynamic (the GPU
    // form of Barrier-Helper, Alg. 6): a block takes the next unclaimed tile
    // from a shared counter, so blocks that finish early take over the work of
    // slow ones and no block waits on another's share.
    // A slowed block 0 (PR_OPT_DELAY_NS) sleeps before taking each tile.
    __shared__ int s_tile;
    auto next_tile = [&](int prev) -> int {
        if (a.delay_ns > 0 && blockIdx.x == 0) {
            if (threadIdx.x == 0) __nanosleep((unsigned)a.delay_ns);
            __syncthreads();
        }
        if (!a.dynamic) return prev < 0 ? group : prev + (int)gridDim.x * groups;
        __syncthreads();
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(&st->tile_next, 1u);
        __syncthreads();
        return s_tile;
    };
    for (int t = next_tile(-1); t < a.n_tiles; t = next_tile(t)) {
        const Tile tile = a.tiles[t];
        if (tile.kind >= 0) {
            if (kStaged) {
                if (!process_staged_tile<IdxT, kUniform, false>(tile, a.rowptr, a.colidx, a.inv_out,
                                                                a.teleport, x_in, y_in, x_out, y_out, c,
                                                                acc, tid, hot_sm + a.hot_n) &&
                    threadIdx.x == 0)
                    atomicOr(&st->error, 1u);
            } else if (kPerf) {
                perf_light_tile<IdxT, kUniform>(tile, a.rowptr, a.colidx, a.inv_out, a.teleport, x_in, y_in,
                                                x_out, y_out, c, pf, acc, tid);
            } else {
                process_light_tile<IdxT, kUniform, false>(tile, a.rowptr, a.colidx, a.inv_out, a.teleport,
                                                           x_in, y_in, x_out, y_out, c, acc, tid);
            }
        } else if (tile.kind == kTileZero) {
            if (kPerf)
                perf_zero_tile<kUniform>(tile, a.inv_out, a.teleport, x_in, y_in, x_out, y_out, c, pf, acc, tid);
            else
                process_zero_tile<kUniform, false>(tile, a.inv_out, a.teleport, x_in, x_out, y_out, c, acc, tid);
        } else {  // heavy rows: sum of the segment partials
            for (int64_t r = tile.row_begin + tid; r < tile.row_end; r += kBlock) {
                const float xo = ld_stream(x_in + r);
                const float inv = ld_stream(a.inv_out + r);
                if (kPerf && pf.frozen[r]) {
                    perf_copy(r, xo, ld_stream(y_in + r), inv, x_out, y_out, acc);
                    continue;
                }
                const float tv = kUniform ? 0.f : ld_stream(a.teleport + r);
                float s = 0.f;
                const int32_t j1 = a.seg_ptr[r + 1];
                for (int32_t j = a.seg_ptr[r]; j < j1; ++j) s += __ldcg(a.seg_sum + j);
                if (kPerf) perf_update<kUniform>(r, s, xo, inv, tv, c, pf, x_out, y_out, acc);
                else row_update<kUniform, false>(r, s, xo, inv, tv, c, x_out, y_out, acc);
            }
        }
    }

    double R, Dn;
    if (block_pair_to_grid(acc.resid(), acc.mass(), a.slots, &st->ticket, &R, &Dn) &&
        threadIdx.x == 0) {
        st->resid = R;
        st->D = Dn;
        st->iter += 1;
        const int done = (R < st->tol) || (st->iter >= st->max_iter);
        st->done = done;
        st->ticket = 0;
        st->tile_next = 0;
        if (done && a.use_cond) cudaGraphSetConditional(a.cond, 0);
    }
}

// ------------------------------------------------ pipelined row kernel --
//
// k_rows_tma computes exactly what k_rows computes, for the configuration
// the solver runs by default (32-bit offsets, tiles in a fixed round-robin
// order, no perforation, no shared-memory copy of y), except that by default
// (PR_OPT_IMPLICIT_ZERO_ROWS) it keeps the ranks of rows without in-edges
// implicit after the first update: the same iterates, with the dangling mass
// and the L1 change of those rows summed in FP64.  In k_rows a row group
// waits on three memory latencies per pair of rows: the row offsets, then the
// column indices, then the gathers.  Here a producer warp moves every tile's
// offsets, column indices and per-row vectors (x, 1/outdeg, teleport) into
// shared memory with bulk asynchronous copies (cp.async.bulk, completion
// counted in bytes on an mbarrier), kTmaStages tiles ahead of the 8 consumer
// warps, so that the only latency a row group still waits on is its gathers.
// Each stage has a "full" barrier (the producer's expect-tx arrival + the
// copies' bytes) and an "empty" barrier (one arrival per consumer warp when it
// is done with the stage).  Every wait is bounded: a wait that runs out sets
// error bit 2 and the solve reports PR_ERR_DEVICE_TIMEOUT.

// Shared-memory stage of one tile: colidx, then rowptr, x, 1/outdeg and
// teleport, each copied from its 16-byte aligned start at or before the
// tile's first element.
struct TmaStage {
    int32_t* col;
    int32_t* rp;
    float* x;
    float* inv;
    float* tel;
    __device__ __forceinline__ TmaStage(uint32_t* base, int s) {
        uint32_t* p = base + (size_t)s * kTmaStageWords;
        col = (int32_t*)p;
        rp = (int32_t*)(p + kTmaColWords);
        x = (float*)(p + kTmaColWords + kTmaRowWords);
        inv = (float*)(p + kTmaColWords + 2 * kTmaRowWords);
        tel = (float*)(p + kTmaColWords + 3 * kTmaRowWords);
    }
};

// Producer side: copies of tile `t` into stage st, arrival with the bytes.
template <bool kUniform>
__device__ __forceinline__ void tma_issue(const IterArgs& a, const Tile& tile, int64_t e0, int64_t e1,
                                          const float* x_in, TmaStage st, uint64_t* full) {
    if (tile.kind == kTileSeg) {
        // a heavy-row segment: its column indices only
        const int64_t c0 = e0 & ~(int64_t)3;
        const uint32_t col_bytes = (uint32_t)((((e1 + 3) & ~(int64_t)3) - c0) * 4);
        if (col_bytes > kTmaColWords * 4u) {
            atomicOr(&a.state->error, 4u);
            mbar_arrive_expect_tx(full, 0);
            return;
        }
        mbar_arrive_expect_tx(full, col_bytes);
        if (col_bytes) bulk_copy_g2s(st.col, a.colidx + c0, col_bytes, full);
        return;
    }
    const int64_t r0 = tile.row_begin & ~3, r1 = (tile.row_end + 3) & ~3;
    const uint32_t vec_bytes = (uint32_t)(r1 - r0) * 4u;
    uint32_t bytes = (kUniform ? 2u : 3u) * vec_bytes;
    int64_t c0 = 0, p1 = 0;
    uint32_t col_bytes = 0, rp_bytes = 0;
    if (tile.kind >= 0) {
        c0 = e0 & ~(int64_t)3;
        col_bytes = (uint32_t)((((e1 + 3) & ~(int64_t)3) - c0) * 4);
        p1 = (tile.row_end + 1 + 3) & ~3;
        rp_bytes = (uint32_t)(p1 - r0) * 4u;
        bytes += col_bytes + rp_bytes;
    }
    if (vec_bytes > kTmaRowWords * 4u || col_bytes > kTmaColWords * 4u || rp_bytes > kTmaRowWords * 4u) {
        // a tile larger than a stage (the tiling at set-up rules this out):
        // copy nothing, complete the phase, flag the solve
        atomicOr(&a.state->error, 4u);
        mbar_arrive_expect_tx(full, 0);
        return;
    }
    mbar_arrive_expect_tx(full, bytes);
    bulk_copy_g2s(st.x, x_in + r0, vec_bytes, full);
    bulk_copy_g2s(st.inv, a.inv_out + r0, vec_bytes, full);
    if (!kUniform) bulk_copy_g2s(st.tel, a.teleport + r0, vec_bytes, full);
    if (tile.kind >= 0) {
        if (col_bytes) bulk_copy_g2s(st.col, a.colidx + c0, col_bytes, full);
        bulk_copy_g2s(st.rp, (const int32_t*)a.rowptr + r0, rp_bytes, full);
    }
}

// Consumer side: one light tile from its stage (same groups, passes and
// update as process_light_tile).
template <bool kUniform>
__device__ __forceinline__ void tma_light_tile(const Tile& tile, const TmaStage& st, const float* y_in,
                                               float* x_out, float* y_out, const RowCtx& c, Acc& acc, int tid) {
    const int lg = light_lanes_log2(tile, c.lane_mode);
    const int g = 1 << lg;
    const int rpp = kBlock >> lg;
    const int grp = tid >> lg;
    const int gl = tid & (g - 1);
    const int o = tile.row_begin & 3;                  // row i of the tile is element o + i
    const int32_t* rp = st.rp + o;
    const int32_t base = rp[0] & ~3;                  // st.col[e - base] = colidx[e]
    const int nrows = tile.row_end - tile.row_begin;
    for (int i0 = 0; i0 < nrows; i0 += 2 * rpp) {
        int ii[2];
        bool act[2];
        int32_t b[2], e[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            ii[q] = i0 + q * rpp + grp;
            act[q] = ii[q] < nrows;
            b[q] = act[q] ? rp[ii[q]] - base : 0;
            e[q] = act[q] ? rp[ii[q] + 1] - base : 0;
        }
        float s[2] = {0.f, 0.f};
        const int32_t* col = st.col;
        gather_row_pair<false>([col](int32_t p) { return col[p]; }, b[0] + gl, e[0], b[1] + gl, e[1], g, y_in, c,
                               s[0], s[1]);
#pragma unroll
        for (int m = 1; m < 32; m <<= 1)
            if (m < g) {
                s[0] += __shfl_xor_sync(0xffffffffu, s[0], m);
                s[1] += __shfl_xor_sync(0xffffffffu, s[1], m);
            }
        if (gl == 0) {
#pragma unroll
            for (int q = 0; q < 2; ++q)
                if (act[q]) {
                    const int i = o + ii[q];
                    row_update<kUniform, false>(tile.row_begin + ii[q], s[q], st.x[i], st.inv[i],
                                                kUniform ? 0.f : st.tel[i], c, x_out, y_out, acc);
                }
        }
    }
}

// Consumer side of a heavy-row segment (fused list): the 256 consumer threads
// gather the segment's edges from the stage (thread i takes edges e0 + i,
// e0 + i + 256, ..., four in flight), each warp sums its share, and the
// warp that finishes last (a shared-memory counter per stage; no block
// barrier, so a consumer warp whose bounded wait ran out cannot hold the
// others) adds the eight warp sums in warp order and publishes the
// segment's partial sum.  The block that publishes a heavy row's last
// segment sums the row's partials in segment order and updates the row;
// its L1 change and dangling mass go to hr_part, which the grid's last
// block adds in row order, so the iteration stays deterministic.
struct SegRed {
    float part[kTmaStages][kWarps];
    int32_t cnt[kTmaStages];
};

template <bool kUniform>
__device__ __forceinline__ void tma_segment_tile(const IterArgs& a, const Tile& tile, int32_t e1, const TmaStage& st,
                                                 int stage, SegRed& red, const float* x_in, const float* y_in,
                                                 float* x_out, float* y_out, const RowCtx& c, int tid) {
    const int32_t e0 = tile.pad;
    const int32_t base = e0 & ~3;   // st.col[e - base] = colidx[e]
    const int32_t* col = st.col;
    float v = 0.f;
    for (int32_t p = e0 + tid; p < e1; p += 4 * kBlock) {
        float g[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int32_t q = p + j * kBlock;
            g[j] = q < e1 ? Mem<false>::gather(y_in, col[q - base], c) : 0.f;
        }
        v += (g[0] + g[1]) + (g[2] + g[3]);
    }
    v = warp_sum(v);
    if ((tid & 31) != 0) return;
    red.part[stage][tid >> 5] = v;
    __threadfence_block();
    if (atomicAdd(&red.cnt[stage], 1) != kWarps - 1) return;
    __threadfence_block();
    red.cnt[stage] = 0;
    float sum = 0.f;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) sum += red.part[stage][w];
    const int32_t h = tile.row_begin;
    a.seg_sum[tile.row_end] = sum;
    __threadfence();
    const int32_t j0 = a.seg_ptr[h], j1 = a.seg_ptr[h + 1];
    if (atomicAdd(a.row_cnt + h, 1) != j1 - j0 - 1) return;
    __threadfence();
    a.row_cnt[h] = 0;   // ready for the next iteration
    float rs = 0.f;
    for (int32_t j = j0; j < j1; ++j) rs += __ldcg(a.seg_sum + j);
    const float xo = ld_stream(x_in + h);
    const float inv = ld_stream(a.inv_out + h);
    const float tv = kUniform ? 0.f : ld_stream(a.teleport + h);
    const float b = kUniform ? c.base : fmaf(c.one_m_d, tv, c.d_share);
    const float xn = fmaf(c.d, rs, b);
    st_stream(x_out + h, xn);
    st_y(y_out + h, xn * inv);
    a.hr_part[h] = make_float2(fabsf(xn - xo), inv == 0.f ? xn : 0.f);
}

template <bool kUniform>
__global__ void __launch_bounds__(kTmaThreads, kTmaMinBlocks) k_rows_tma(IterArgs a, const float* __restrict__ x_in,
                                                                      const float* __restrict__ y_in,
                                                                      float* __restrict__ x_out,
                                                                      float* __restrict__ y_out) {
    extern __shared__ __align__(128) uint64_t tma_smem[];
    uint64_t* full = tma_smem;
    uint64_t* empty = tma_smem + kTmaStages;
    uint32_t* stages = (uint32_t*)(tma_smem + 2 * kTmaStages);
    SolveState* st = a.state;
    const StateView sv = block_state(st);
    if (sv.done) {
        if (a.use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(a.cond, 0);
        return;
    }
    __shared__ SegRed seg_red;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kTmaStages; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, kWarps);
            seg_red.cnt[s] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const double d = sv.d;
    const double share = sv.D * sv.inv_n;
    RowCtx c;
    c.d = (float)d;
    c.one_m_d = (float)(1.0 - d);
    c.d_share = (float)(d * share);
    c.base = (float)((1.0 - d) * sv.inv_n + d * share);
    c.hot = a.hot_tma;
    c.hot_n = 0;
    c.hot_sm = nullptr;
    c.lane_mode = a.lane_mode;
    Acc acc;
    // Rows without in-edges gather nothing: by Eq. 1 their rank is
    // (1-d) t_v + d D/n.  After the first update (implicit) their ranks are
    // neither read nor written: the tiles of isolated vertices are skipped and
    // the other such rows store their quotient only; the last block adds their
    // L1 change and the isolated vertices' dangling mass, and k_zero_fill
    // writes the ranks after the loop.
    const bool implicit = sv.implicit && sv.iter > 0 && !a.fused;
    const int n_tiles = implicit ? a.n_tiles_live : a.n_tiles;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    bool timed_out = false;
    if (warp == kWarps) {
        // producer: lane 0 issues the copies of the block's tiles in order
        if (lane == 0) {
            int k = 0;
            for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++k) {
                const int s = k % kTmaStages;
                const int use = k / kTmaStages;
                if (use > 0 && !mbar_wait(empty + s, (uint32_t)(use - 1) & 1u)) {
                    timed_out = true;
                    break;
                }
                const Tile tile = a.tiles[t];
                if (a.withhold > 0 && blockIdx.x == 0 && k + 1 == a.withhold) {
                    // test hook: announce a copy that never comes, so that the
                    // consumers' bounded wait for this stage runs out
                    mbar_arrive_expect_tx(full + s, 16);
                    continue;
                }
                tma_issue<kUniform>(a, tile, tile.pad, a.fused ? a.tile_e1[t] : a.tiles[t + 1].pad, x_in,
                                    TmaStage(stages, s), full + s);
            }
            // let every copy land before the block can exit
            const int issued = k;
            for (int s = 0; s < kTmaStages && s < issued; ++s) {
                const int last = (issued - 1 - s) / kTmaStages;   // last use of stage s
                if (!mbar_wait(full + s, (uint32_t)last & 1u)) timed_out = true;
            }
        }
    } else {
        const int tid = threadIdx.x;
        int k = 0;
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++k) {
            const int s = k % kTmaStages;
            if (!mbar_wait(full + s, (uint32_t)(k / kTmaStages) & 1u)) {
                timed_out = true;
                break;
            }
            const Tile tile = a.tiles[t];
            const TmaStage stg(stages, s);
            if (tile.kind >= 0) {
                tma_light_tile<kUniform>(tile, stg, y_in, x_out, y_out, c, acc, tid);
            } else if (tile.kind == kTileSeg) {
                tma_segment_tile<kUniform>(a, tile, a.tile_e1[t], stg, s, seg_red, x_in, y_in, x_out, y_out, c, tid);
            } else if (implicit && tile.kind == kTileZero) {
                // the quotient of the implicit rank (what row_update stores for s = 0)
                const int o = tile.row_begin & 3;
                for (int i = tid; i < tile.row_end - tile.row_begin; i += kBlock) {
                    const float b = kUniform ? c.base : fmaf(c.one_m_d, stg.tel[o + i], c.d_share);
                    st_y(y_out + tile.row_begin + i, b * stg.inv[o + i]);
                }
            } else {
                const int o = tile.row_begin & 3;
                for (int i = tid; i < tile.row_end - tile.row_begin; i += kBlock) {
                    const int64_t r = tile.row_begin + i;
                    float sum = 0.f;
                    if (tile.kind == kTileHeavy) {
                        const int32_t j1 = a.seg_ptr[r + 1];
                        for (int32_t j = a.seg_ptr[r]; j < j1; ++j) sum += __ldcg(a.seg_sum + j);
                    }
                    row_update<kUniform, false>(r, sum, stg.x[o + i], stg.inv[o + i],
                                                kUniform ? 0.f : stg.tel[o + i], c, x_out, y_out, acc);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(empty + s);
        }
    }
    if (timed_out) atomicOr(&st->error, 2u);

    double R, Dn;
    const bool last_block = block_pair_to_grid(acc.resid(), acc.mass(), a.slots, &st->ticket, &R, &Dn);
    if (last_block && a.fused) {
        // the heavy rows' updates, in row order
        double hr = 0.0, hd = 0.0;
        for (int32_t h = threadIdx.x; h < a.n_heavy; h += blockDim.x) {
            const float2 p = __ldcg(a.hr_part + h);
            hr += (double)p.x;
            hd += (double)p.y;
        }
        block_sum2(hr, hd);
        R += hr;
        Dn += hd;
    }
    if (last_block && threadIdx.x == 0) {
        if (implicit) {
            // every row without in-edges changed by d |D - Dz| / n; the
            // isolated ones are dangling: (1-d) t_iso + n_iso d D / n
            R += (double)(a.n - a.zero_start) * d * fabs(sv.D - st->Dz) * sv.inv_n;
            Dn += (1.0 - d) * st->t_iso + (double)(a.n - a.iso_start) * d * sv.D * sv.inv_n;
        }
        st->Dz = sv.D;
        st->resid = R;
        st->D = Dn;
        st->iter += 1;
        const int done = (R < st->tol) || (st->iter >= st->max_iter) || st->error != 0;
        st->done = done;
        st->ticket = 0;
        st->tile_next = 0;
        if (done && a.use_cond) cudaGraphSetConditional(a.cond, 0);
    }
}

// Teleport sum over the isolated vertices (binned rows [iso_start, n)).
__global__ void __launch_bounds__(kBlock) k_t_iso(IterArgs a, const float* __restrict__ t_bin) {
    SolveState* st = a.state;
    KahanF s;
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t i = a.iso_start + (int64_t)blockIdx.x * kBlock + threadIdx.x; i < a.n; i += stride) s.add(t_bin[i]);
    double T, unused;
    if (block_pair_to_grid(s.value(), 0.0, a.slots, &st->ticket, &T, &unused) && threadIdx.x == 0) {
        st->t_iso = T;
        st->ticket = 0;
    }
}

// The ranks of the rows without in-edges after a loop that kept them implicit
// (k_rows_tma): (1-d) t_v + d Dz/n, in the arithmetic of the row kernel.
__global__ void __launch_bounds__(kBlock) k_zero_fill(IterArgs a, float* __restrict__ x0, float* __restrict__ x1) {
    const SolveState* st = a.state;
    if (!st->implicit || st->iter < 2) return;   // after one update the rows were written in full
    float* x = (st->iter & 1) ? x1 : x0;
    const double d = st->d;
    const double share = st->Dz * st->inv_n;
    const float base = (float)((1.0 - d) * st->inv_n + d * share);
    const float one_m_d = (float)(1.0 - d), d_share = (float)(d * share);
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t i = a.zero_start + (int64_t)blockIdx.x * kBlock + threadIdx.x; i < a.n; i += stride)
        x[i] = a.teleport ? fmaf(one_m_d, a.teleport[i], d_share) : base;
}

// Rows frozen by loop perforation, added into the solve state.
__global__ void __launch_bounds__(kBlock) k_count_frozen(const uint8_t* __restrict__ frozen, int64_t n,
                                                         SolveState* st) {
    uint32_t c = 0;
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n; i += stride) c += frozen[i] != 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&st->frozen, c);
}

// The fused list's edge ranges: light and empty-row tiles [rowptr[row_begin],
// rowptr[row_end]); a segment tile (row_end = its index s) the row of s and
// its 2048-edge range within that row.
__global__ void k_fused_tile_edges(Tile* tiles, int32_t* e1, int64_t count, const int32_t* __restrict__ rowptr,
                                   const int32_t* __restrict__ seg_row, const int32_t* __restrict__ seg_ptr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        Tile t = tiles[i];
        if (t.kind == kTileSeg) {
            const int32_t h = seg_row[t.row_end];
            const int32_t b = rowptr[h] + (t.row_end - seg_ptr[h]) * kSegEdges;
            t.row_begin = h;
            t.pad = b;
            e1[i] = min(b + kSegEdges, rowptr[h + 1]);
        } else {
            t.pad = rowptr[t.row_begin];
            e1[i] = rowptr[t.row_end];
        }
        tiles[i] = t;
    }
}

cudaError_t fill_fused_tiles(Tile* tiles, int32_t* e1, int64_t count, const int32_t* rowptr, const int32_t* seg_row,
                             const int32_t* seg_ptr, cudaStream_t s) {
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((count + kBlock - 1) / kBlock, 1024));
    k_fused_tile_edges<<<grid, kBlock, 0, s>>>(tiles, e1, count, rowptr, seg_row, seg_ptr);
    return cudaGetLastError();
}

// pad of every tile of the pipelined kernel (and of the sentinel after the
// last) = offset of the tile's first edge.
__global__ void k_tile_edges(Tile* tiles, int64_t count, const int32_t* __restrict__ rowptr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= count; i += stride)
        tiles[i].pad = rowptr[tiles[i].row_begin];
}

// x = t or x0 (both in the caller's order), y = x/outdeg, D = dangling mass of
// x, sum(t); resets the running state.
__global__ void __launch_bounds__(kBlock) k_init(IterArgs a, const float* __restrict__ t_src,
                                                 const float* __restrict__ x0_src,
                                                 const int32_t* __restrict__ order,
                                                 float* __restrict__ t_bin, float* __restrict__ x,
                                                 float* __restrict__ y) {
    SolveState* st = a.state;
    const float tu = (float)block_state(st).inv_n;
    KahanF dsum, tsum;
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < a.n; i += stride) {
        const int32_t o = order[i];
        const float tv = t_src ? t_src[o] : tu;
        if (t_src) t_bin[i] = tv;
        const float xv = x0_src ? x0_src[o] : tv;
        const float inv = a.inv_out[i];
        x[i] = xv;
        y[i] = xv * inv;
        if (inv == 0.f) dsum.add(xv);
        tsum.add(tv);
    }
    double D, T;
    if (block_pair_to_grid(dsum.value(), tsum.value(), a.slots, &st->ticket, &D, &T) && threadIdx.x == 0) {
        st->D = D;
        st->t_sum = t_src ? T : 1.0;
        st->iter = 0;
        st->done = 0;
        st->resid = INFINITY;
        st->error = 0;
        st->ticket = 0;
        st->tile_next = 0;
    }
}

// Sum of the final vector (buffer x[iter & 1]) and the renormalising scale.
__global__ void __launch_bounds__(kBlock) k_sum_x(IterArgs a, const float* __restrict__ x0,
                                                  const float* __restrict__ x1) {
    SolveState* st = a.state;
    const float* x = (block_state(st).iter & 1) ? x1 : x0;
    KahanF s;
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < a.n; i += stride) s.add(x[i]);
    double S, unused;
    if (block_pair_to_grid(s.value(), 0.0, a.slots, &st->ticket, &S, &unused) && threadIdx.x == 0) {
        st->sum_x = S;
        st->scale = S > 0.0 ? st->t_sum / S : 1.0;
        st->ticket = 0;
    }
}

// out[v] = x[rank[v]] (* scale): back to the caller's vertex order.
__global__ void __launch_bounds__(kBlock) k_unpermute(IterArgs a, const float* __restrict__ x0,
                                                      const float* __restrict__ x1,
                                                      const int32_t* __restrict__ rank,
                                                      float* __restrict__ out, int apply_scale) {
    const StateView sv = block_state(a.state);
    const float* x = (sv.iter & 1) ? x1 : x0;
    const float sc = apply_scale ? (float)sv.scale : 1.0f;
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t v = (int64_t)blockIdx.x * kBlock + threadIdx.x; v < a.n; v += stride)
        out[v] = x[rank[v]] * sc;
}

// ------------------------------------------------------------------ host --

namespace {
int g_occ_rows = 0;
int g_occ_rows_staged = 0;
int g_occ_seg = 0;
int g_occ_tma = 0;
}  // namespace

cudaError_t fill_tile_edges(Tile* tiles, int64_t count, const int32_t* rowptr, cudaStream_t s) {
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((count + kBlock) / kBlock, 1024));
    k_tile_edges<<<grid, kBlock, 0, s>>>(tiles, count, rowptr);
    return cudaGetLastError();
}

// The pipelined row kernel applies to this graph and these options.
static bool tma_applies(const pr_graph* g, const IterArgs& a) {
    return g->use_tma && g->n_tma_tiles > 0 && !g->idx64 && !a.frozen && !a.staged && a.hot_n == 0 &&
           !a.dynamic && a.delay_ns == 0;
}

static int tma_grid(const pr_graph* g) {
    int per_sm = g->ctas_per_sm > 0 ? std::min(g->ctas_per_sm, g_occ_tma) : g_occ_tma;
    int64_t blocks = (int64_t)g->sm_count * std::max(1, per_sm);
    blocks = std::min<int64_t>(blocks, std::max<int64_t>(1, std::max(g->n_tma_tiles, g->n_tma_fused)));
    return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)g->slot_capacity));
}

IterArgs make_args(const pr_graph* g, bool uniform) {
    IterArgs a{};
    a.rowptr = g->rowptr;
    a.colidx = g->colidx;
    a.inv_out = g->inv_out;
    a.teleport = uniform ? nullptr : g->teleport;
    a.seg_row = g->seg_row;
    a.seg_ptr = g->seg_ptr;
    a.seg_sum = g->seg_sum;
    a.tiles = g->tiles;
    a.n = g->n;
    a.n_seg = (int32_t)g->n_seg;
    a.n_tiles = (int32_t)g->n_tiles;
    a.state = g->state;
    a.slots = g->slots;
    a.cond = 0;
    a.use_cond = 0;
    a.hot = (int32_t)(((g->hot_vertices >> 28) << 28) |
                      std::min<int64_t>(g->hot_vertices & 0x0fffffff, g->n));
    a.hot_n = (int32_t)(std::min<int64_t>(g->hot_cache, g->n) & ~(int64_t)3);
    a.staged = g->staged_tiles & 1;
    a.frozen = g->perforation > 0 ? g->frozen : nullptr;
    a.perf_eps = g->perforation > 0 ? (float)std::pow(10.0, -(double)g->perforation) : 0.f;
    a.dynamic = g->dynamic_tiles;
    a.delay_ns = g->delay_ns;
    a.withhold = g->test_withhold;
    a.nnz = g->nnz;
    a.lane_mode = g->lane_mode;
    a.n_tiles_live = (int32_t)g->n_tma_live;
    {
        const int32_t count = a.hot & 0x0fffffff;
        const int32_t cap = g->tma_hot > 0 ? (int32_t)std::min<int64_t>(g->tma_hot, count) : count;
        a.hot_tma = (int32_t)(((uint32_t)a.hot & 0xf0000000u) | (uint32_t)cap);
    }
    a.zero_start = g->n - g->n_zero_indeg;
    a.iso_start = g->n - g->n_isolated;
    return a;
}

int small_grid(const pr_graph* g) {
    int64_t blocks = (g->n + kBlock - 1) / kBlock;
    return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)g->slot_capacity));
}

cudaError_t launch_count_frozen(const pr_graph* g, cudaStream_t s) {
    if (g->perforation <= 0 || !g->frozen) return cudaSuccess;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((g->n + kBlock - 1) / kBlock, 4096));
    k_count_frozen<<<grid, kBlock, 0, s>>>(g->frozen, g->n, g->state);
    return cudaGetLastError();
}

// Enqueue one iteration reading buffer `src` and writing buffer 1-src.
template <typename IdxT>
cudaError_t enqueue_iteration_t(const pr_graph* g, const IterArgs& a, int src, bool uniform,
                                cudaStream_t s, int* launches) {
    if (a.edge) return enqueue_edge_iteration(g, a, src, uniform, s, launches);
    const size_t hot = (size_t)a.hot_n * sizeof(float);
    const size_t rows_smem = hot + (a.staged ? (size_t)kStageFloats * sizeof(float) : 0);
    // the pipelined kernel with the heavy-row segments as tiles of its own
    const bool fused = sizeof(IdxT) == 4 && tma_applies(g, a) && g->fuse_segments && g->n_tma_fused > 0;
    if (g->n_seg > 0 && !fused) {
        k_heavy_segments<IdxT><<<seg_grid(g), kIterBlock, hot, s>>>(a, g->y[src]);
        ++*launches;
    }
    const int grid = row_grid(g, a.staged != 0 && !a.frozen);
    const float* xi = g->x[src];
    const float* yi = g->y[src];
    float* xo = g->x[1 - src];
    float* yo = g->y[1 - src];
    if (sizeof(IdxT) == 4 && tma_applies(g, a)) {
        IterArgs at = a;
        at.tiles = fused ? g->tma_fused : g->tma_tiles;
        at.n_tiles = (int32_t)(fused ? g->n_tma_fused : g->n_tma_tiles);
        at.fused = fused ? 1 : 0;
        at.tile_e1 = g->tma_fused_e1;
        at.row_cnt = g->row_cnt;
        at.hr_part = g->hr_part;
        at.n_heavy = (int32_t)g->n_heavy;
        const int tg = tma_grid(g);
        if (uniform) k_rows_tma<true><<<tg, kTmaThreads, kTmaSmemBytes, s>>>(at, xi, yi, xo, yo);
        else k_rows_tma<false><<<tg, kTmaThreads, kTmaSmemBytes, s>>>(at, xi, yi, xo, yo);
    } else if (a.frozen) {   // loop perforation (row-by-row tiles only)
        if (uniform) k_rows<IdxT, true, false, true><<<grid, kIterBlock, hot, s>>>(a, xi, yi, xo, yo);
        else k_rows<IdxT, false, false, true><<<grid, kIterBlock, hot, s>>>(a, xi, yi, xo, yo);
    } else if (a.staged) {
        if (uniform) k_rows<IdxT, true, true, false><<<grid, kIterBlock, rows_smem, s>>>(a, xi, yi, xo, yo);
        else k_rows<IdxT, false, true, false><<<grid, kIterBlock, rows_smem, s>>>(a, xi, yi, xo, yo);
    } else {
        if (uniform) k_rows<IdxT, true, false, false><<<grid, kIterBlock, rows_smem, s>>>(a, xi, yi, xo, yo);
        else k_rows<IdxT, false, false, false><<<grid, kIterBlock, rows_smem, s>>>(a, xi, yi, xo, yo);
    }
    ++*launches;
    return cudaGetLastError();
}

// k_heavy_segments over BF16 quotients (the correction sweeps of PR_OPT_SYNC_DC).
cudaError_t launch_segments_q16(const pr_graph* g, const IterArgs& a, const __nv_bfloat16* q, cudaStream_t s,
                                int* launches) {
    if (a.n_seg == 0) return cudaSuccess;
    IterArgs b = a;
    b.hot_n = 0;
    if (g->idx64) k_heavy_segments<int64_t, __nv_bfloat16><<<seg_grid(g), kIterBlock, 0, s>>>(b, q);
    else k_heavy_segments<int32_t, __nv_bfloat16><<<seg_grid(g), kIterBlock, 0, s>>>(b, q);
    ++*launches;
    return cudaGetLastError();
}

// k_heavy_segments over segments [0, a.n_seg) alone.
cudaError_t launch_segments(const pr_graph* g, const IterArgs& a, int src, cudaStream_t s, int* launches) {
    if (a.n_seg == 0) return cudaSuccess;
    const size_t smem = (size_t)a.hot_n * sizeof(float);
    if (g->idx64) k_heavy_segments<int64_t><<<seg_grid(g), kIterBlock, smem, s>>>(a, g->y[src]);
    else k_heavy_segments<int32_t><<<seg_grid(g), kIterBlock, smem, s>>>(a, g->y[src]);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t enqueue_iteration(const pr_graph* g, const IterArgs& a, int src, bool uniform,
                              cudaStream_t s, int* launches) {
    return g->idx64 ? enqueue_iteration_t<int64_t>(g, a, src, uniform, s, launches)
                    : enqueue_iteration_t<int32_t>(g, a, src, uniform, s, launches);
}

// The while-graph: body = two iterations, x0 -> x1 and x1 -> x0.
pr_status build_loop_graph(pr_graph* g, bool uniform) {
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
    IterArgs a = make_args(g, uniform);
    a.cond = handle;
    a.use_cond = 1;
    PRK_CHECK(cudaStreamBeginCaptureToGraph(g->capture_stream, body, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal));
    int launches = 0;
    cudaError_t e1 = enqueue_iteration(g, a, 0, uniform, g->capture_stream, &launches);
    cudaError_t e2 = cudaSuccess;
    if (e1 == cudaSuccess) e2 = enqueue_iteration(g, a, 1, uniform, g->capture_stream, &launches);
    cudaGraph_t captured = nullptr;
    cudaError_t e3 = cudaStreamEndCapture(g->capture_stream, &captured);
    PRK_CHECK(e1);
    PRK_CHECK(e2);
    PRK_CHECK(e3);
    cudaGraphExec_t exec = nullptr;
    PRK_CHECK(cudaGraphInstantiate(&exec, graph, 0));
    g->loop_exec[uniform ? 0 : 1] = exec;
    return PR_OK;
}

// Input vector from the caller: device pointers are used in place, host
// memory is staged through g->stage + offset.
pr_status stage_input(pr_graph* g, const float* src, int slot, cudaStream_t s, const float** out) {
    *out = nullptr;
    if (!src) return PR_OK;
    if (is_device_pointer(src)) {
        *out = src;
        return PR_OK;
    }
    float* dst = g->stage + (size_t)slot * (size_t)(g->n + kPad);
    PRK_CHECK(cudaMemcpyAsync(dst, src, (size_t)g->n * sizeof(float), cudaMemcpyHostToDevice, s));
    *out = dst;
    return PR_OK;
}

pr_status ensure_stage(pr_graph* g) {
    if (g->stage) return PR_OK;
    PRK_CHECK(dev_alloc(g, (void**)&g->stage, (size_t)3 * (size_t)(g->n + kPad) * sizeof(float)));
    return PR_OK;
}

pr_status ensure_teleport(pr_graph* g) {
    if (g->teleport) return PR_OK;
    PRK_CHECK(dev_alloc(g, (void**)&g->teleport, (size_t)(g->n + kPad) * sizeof(float)));
    return PR_OK;
}

void launch_init(const pr_graph* g, const IterArgs& a, const float* t_dev, const float* x0_dev,
                 cudaStream_t s) {
    // the fused kernel's per-row segment counters return to 0 after every
    // iteration; an iteration cut short (a wait that ran out) may leave some set
    if (g->row_cnt) cudaMemsetAsync(g->row_cnt, 0, (size_t)g->n_heavy * sizeof(int32_t), s);
    k_init<<<small_grid(g), kBlock, 0, s>>>(a, t_dev, x0_dev, g->order, g->teleport, g->x[0], g->y[0]);
}

void launch_finalize(const pr_graph* g, const IterArgs& a, float* out, bool renormalise, cudaStream_t s,
                     int* launches, bool implicit) {
    if (implicit && a.zero_start < a.n) {
        k_zero_fill<<<small_grid(g), kBlock, 0, s>>>(a, g->x[0], g->x[1]);
        ++*launches;
    }
    if (renormalise) {
        k_sum_x<<<small_grid(g), kBlock, 0, s>>>(a, g->x[0], g->x[1]);
        ++*launches;
    }
    k_unpermute<<<small_grid(g), kBlock, 0, s>>>(a, g->x[0], g->x[1], g->rank, out, renormalise ? 1 : 0);
    ++*launches;
}

int row_grid(const pr_graph* g, bool staged) {
    const int occ = staged ? g_occ_rows_staged : g_occ_rows;
    int per_sm = g->ctas_per_sm > 0 ? std::min(g->ctas_per_sm, occ) : occ;
    int64_t blocks = (int64_t)g->sm_count * per_sm;
    blocks = std::min<int64_t>(blocks, std::max<int64_t>(1, g->n_tiles));
    return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)g->slot_capacity));
}

int seg_grid(const pr_graph* g) {
    int64_t blocks = (g->n_seg + (kIterBlock / 32) - 1) / (kIterBlock / 32);
    int64_t cap = (int64_t)g->sm_count * g_occ_seg;
    return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, cap));
}

pr_status alloc_solver(pr_graph* g) {
    const size_t vec = (size_t)(g->n + kPad) * sizeof(float);
    for (int i = 0; i < 2; ++i) {
        PRK_CHECK(dev_alloc(g, (void**)&g->x[i], vec));
        PRK_CHECK(dev_alloc(g, (void**)&g->y[i], vec));
        PRK_CHECK(cudaMemset(g->x[i], 0, vec));
        PRK_CHECK(cudaMemset(g->y[i], 0, vec));
    }
    PRK_CHECK(dev_alloc(g, (void**)&g->state, sizeof(SolveState)));
    PRK_CHECK(cudaMemset(g->state, 0, sizeof(SolveState)));
    g->slot_capacity = g->sm_count * 8;   // also bounds every grid that reduces through slots
    PRK_CHECK(dev_alloc(g, (void**)&g->slots, (size_t)g->slot_capacity * 2 * sizeof(double)));
    PRK_CHECK(cudaMallocHost((void**)&g->host_state, sizeof(SolveState)));
    memset(g->host_state, 0, sizeof(SolveState));
    PRK_CHECK(cudaMallocHost((void**)&g->host_flag, 4 * sizeof(int32_t)));
    memset(g->host_flag, 0, 4 * sizeof(int32_t));
    PRK_CHECK(cudaStreamCreateWithFlags(&g->capture_stream, cudaStreamNonBlocking));
    if (g_occ_rows == 0) {
        const int hot = (int)(kHotCacheMax * sizeof(float));
        const int rows = (int)((kHotCacheMax + kStageFloats) * sizeof(float));
        const void* row_kernels[] = {
            (const void*)k_rows<int32_t, true, false, false>, (const void*)k_rows<int32_t, false, false, false>,
            (const void*)k_rows<int64_t, true, false, false>, (const void*)k_rows<int64_t, false, false, false>,
            (const void*)k_rows<int32_t, true, true, false>,  (const void*)k_rows<int32_t, false, true, false>,
            (const void*)k_rows<int64_t, true, true, false>,  (const void*)k_rows<int64_t, false, true, false>,
            (const void*)k_rows<int32_t, true, false, true>,  (const void*)k_rows<int32_t, false, false, true>,
            (const void*)k_rows<int64_t, true, false, true>,  (const void*)k_rows<int64_t, false, false, true>};
        const void* seg_kernels[] = {(const void*)k_heavy_segments<int32_t, float>,
                                     (const void*)k_heavy_segments<int64_t, float>,
                                     (const void*)k_heavy_segments<int32_t, __nv_bfloat16>,
                                     (const void*)k_heavy_segments<int64_t, __nv_bfloat16>};
        // These kernels need little shared memory: the preferred carveout 0
        // gives the rest of the SRAM to L1, which caches the hub ranks.
        // The staged kernels (entries 4..7) hold a 24.6 KB staging area per
        // block: carve out enough shared memory for four blocks per SM.
        for (int i = 0; i < 12; ++i) {
            const bool staged = i >= 4 && i < 8;
            PRK_CHECK(cudaFuncSetAttribute(row_kernels[i], cudaFuncAttributeMaxDynamicSharedMemorySize, rows));
            PRK_CHECK(cudaFuncSetAttribute(row_kernels[i], cudaFuncAttributePreferredSharedMemoryCarveout,
                                           staged ? 50 : 0));
        }
        for (const void* k : seg_kernels) {
            PRK_CHECK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, hot));
            PRK_CHECK(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 0));
        }
        int occ = 0;
        PRK_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_rows<int32_t, false, true, false>, kIterBlock,
                                                                 kStageFloats * sizeof(float)));
        g_occ_rows_staged = std::max(1, occ);
        PRK_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_rows<int32_t, false, false, false>, kIterBlock, 0));
        // the pipelined kernel: shared memory for kTmaMinBlocks blocks of
        // kTmaSmemBytes each (plus the 1 KB the CUDA driver reserves per block),
        // the rest of the SRAM to L1
        const void* tma_kernels[] = {(const void*)k_rows_tma<true>, (const void*)k_rows_tma<false>};
        const int carve = (int)std::min<int64_t>(
            100, (int64_t)(kTmaMinBlocks * (kTmaSmemBytes + 1024) * 100 + 228 * 1024 - 1) / (228 * 1024));
        for (const void* k : tma_kernels) {
            PRK_CHECK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTmaSmemBytes));
            PRK_CHECK(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, carve));
        }
        int occ_tma = 0;
        PRK_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_tma, k_rows_tma<false>, kTmaThreads, kTmaSmemBytes));
        g_occ_tma = std::max(1, occ_tma);
        int occ_seg = 0;
        PRK_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_seg, k_heavy_segments<int32_t, float>, kIterBlock, 0));
        g_occ_seg = std::max(1, occ_seg);
        g_occ_rows = std::max(1, occ);   // last: marks the block as done
    }
    return PR_OK;
}

}  // namespace prk

using namespace prk;

namespace {

pr_status check_solve_args(pr_graph* g, float damping, double tol, int32_t max_iter, float* x_out) {
    if (!g) return fail(PR_ERR_INVALID_ARG, "graph is NULL");
    if (!(damping >= 0.0f && damping < 1.0f)) return fail(PR_ERR_INVALID_ARG, "damping must be in [0, 1)");
    if (!(tol > 0.0) || !std::isfinite(tol)) return fail(PR_ERR_INVALID_ARG, "tol must be a positive finite number");
    if (max_iter < 1) return fail(PR_ERR_INVALID_ARG, "max_iter must be >= 1");
    if (!x_out) return fail(PR_ERR_INVALID_ARG, "x_out is NULL");
    return PR_OK;
}

// Shared body of pr_solve (Jacobi) and pr_iterate.
// edge: the edge-centric form of the iteration (Alg. 2, pr_edge.cu), run by
// the host-driven loop.
pr_status run_jacobi(pr_graph* g, float damping, double tol, int32_t max_iter, const float* teleport,
                     const float* x0, float* x_out, bool renormalise, bool allow_graph, pr_info* info,
                     cudaStream_t s, bool edge = false) {
    pr_status rc = ensure_stage(g);
    if (rc != PR_OK) return rc;
    if (edge && (rc = ensure_edge(g, s)) != PR_OK) return rc;
    if (edge) allow_graph = false;
    const float* t_dev = nullptr;
    const float* x0_dev = nullptr;
    if ((rc = stage_input(g, teleport, 0, s, &t_dev)) != PR_OK) return rc;
    if ((rc = stage_input(g, x0, 1, s, &x0_dev)) != PR_OK) return rc;
    const bool uniform = teleport == nullptr;
    if (!uniform && (rc = ensure_teleport(g)) != PR_OK) return rc;
    const bool out_dev = is_device_pointer(x_out);
    float* out = out_dev ? x_out : g->stage + (size_t)2 * (size_t)(g->n + kPad);

    SolveState* hs = g->host_state;
    memset(hs, 0, sizeof(SolveState));
    hs->d = (double)damping;
    hs->tol = tol;
    hs->inv_n = 1.0 / (double)g->n;
    hs->t_sum = 1.0;
    hs->max_iter = max_iter;
    hs->uniform_t = uniform ? 1 : 0;
    IterArgs a = make_args(g, uniform);
    if (edge) {
        a.edge = 1;
        a.out_src = g->out_src;
        a.out_pos = g->out_pos;
    }
    // BF16 correction sweeps after each FP32 step (PR_OPT_SYNC_DC; the solve only)
    const bool dc = g->sync_dc > 0 && renormalise && !edge && !a.frozen;
    if (dc && (rc = ensure_sync_dc(g)) != PR_OK) return rc;
    // implicit ranks of rows without in-edges: the pipelined kernel with the
    // heavy-row segments in a kernel of their own
    const bool tma = !edge && !g->idx64 && tma_applies(g, a);
    const bool implicit = !dc && g->implicit_zero && tma && !(g->fuse_segments && g->n_tma_fused > 0);
    hs->implicit = implicit ? 1 : 0;
    hs->t_iso = (double)g->n_isolated * hs->inv_n;   // uniform teleport; else summed on the device
    PRK_CHECK(cudaEventRecord(g->ev_start, s));
    PRK_CHECK(cudaMemcpyAsync(g->state, hs, sizeof(SolveState), cudaMemcpyHostToDevice, s));

    int launches = 0;
    launch_init(g, a, t_dev, x0_dev, s);
    ++launches;
    if (implicit && !uniform) {
        k_t_iso<<<small_grid(g), kBlock, 0, s>>>(a, g->teleport);
        ++launches;
    }
    PRK_CHECK(cudaGetLastError());
    if (a.frozen) PRK_CHECK(cudaMemsetAsync(g->frozen, 0, (size_t)g->n, s));   // nothing frozen yet
    PRK_CHECK(cudaEventRecord(g->ev_loop0, s));

    if (dc) {
        // host-driven outer steps: the FP32 step, then (unless it met the
        // stopping test) the correction; the done flag read after each step
        for (int32_t it = 0; it < max_iter; ++it) {
            const int src = it & 1;
            cudaError_t e = enqueue_iteration(g, a, src, uniform, s, &launches);
            if (e == cudaSuccess) e = enqueue_sync_dc(g, a, src, g->sync_dc, s, &launches);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(&g->host_flag[0], &g->state->done, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_fail(e, "correction step");
            if (*(volatile int32_t*)&g->host_flag[0]) break;
        }
    } else if (allow_graph && g->use_graph) {
        const int kind = uniform ? 0 : 1;
        if (!g->loop_exec[kind] && (rc = build_loop_graph(g, uniform)) != PR_OK) return rc;
        PRK_CHECK(cudaGraphLaunch(g->loop_exec[kind], s));
        ++launches;
    } else {
        // Host-driven loop: enqueue chunks of iterations and read the done
        // flag of the chunk before last, so the device is never idle.
        const int chunk = 8;
        int32_t launched = 0;
        cudaEvent_t ev[2];
        PRK_CHECK(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
        PRK_CHECK(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
        int pending = -1;
        pr_status loop_rc = PR_OK;
        while (launched < max_iter) {
            const int c = std::min<int32_t>(chunk, max_iter - launched);
            for (int i = 0; i < c && loop_rc == PR_OK; ++i) {
                cudaError_t e = enqueue_iteration(g, a, (launched + i) & 1, uniform, s, &launches);
                if (e != cudaSuccess) loop_rc = cuda_fail(e, "iteration launch");
            }
            launched += c;
            if (loop_rc != PR_OK) break;
            const int slot = (launched / chunk) & 1;
            cudaError_t e = cudaMemcpyAsync(&g->host_flag[slot], &g->state->done, sizeof(int32_t),
                                            cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaEventRecord(ev[slot], s);
            if (e != cudaSuccess) { loop_rc = cuda_fail(e, "loop bookkeeping"); break; }
            if (pending >= 0) {
                e = cudaEventSynchronize(ev[pending]);
                if (e != cudaSuccess) { loop_rc = cuda_fail(e, "cudaEventSynchronize"); break; }
                if (*(volatile int32_t*)&g->host_flag[pending]) break;
            }
            pending = slot;
        }
        cudaEventSynchronize(ev[0]);
        cudaEventSynchronize(ev[1]);
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
        if (loop_rc != PR_OK) return loop_rc;
    }
    PRK_CHECK(cudaEventRecord(g->ev_loop1, s));

    launch_finalize(g, a, out, renormalise, s, &launches, implicit);
    PRK_CHECK(cudaGetLastError());
    if (a.frozen) {
        PRK_CHECK(launch_count_frozen(g, s));
        ++launches;
    }
    PRK_CHECK(cudaEventRecord(g->ev_stop, s));
    if (!out_dev)
        PRK_CHECK(cudaMemcpyAsync(x_out, out, (size_t)g->n * sizeof(float), cudaMemcpyDeviceToHost, s));
    PRK_CHECK(cudaMemcpyAsync(hs, g->state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    PRK_CHECK(cudaStreamSynchronize(s));
    if (hs->error & 2u)
        return fail(PR_ERR_DEVICE_TIMEOUT, "a bounded device-side wait for a tile copy gave up");
    if (hs->error)
        return fail(PR_ERR_CUDA, "internal error: a row tile exceeded its shared-memory staging area");
    float ms = 0.f, ms_loop = 0.f;
    PRK_CHECK(cudaEventElapsedTime(&ms, g->ev_start, g->ev_stop));
    PRK_CHECK(cudaEventElapsedTime(&ms_loop, g->ev_loop0, g->ev_loop1));
    const bool converged = hs->resid < tol;
    if (info) {
        info->iterations = hs->iter;
        info->converged = converged ? 1 : 0;
        info->residual_l1 = hs->resid;
        info->sum_x = renormalise ? hs->sum_x : 0.0;
        info->dangling_mass = hs->D;
        // correction sweeps ran after every FP32 step but the last
        const double sweeps = dc ? (double)g->sync_dc * (double)std::max(0, hs->iter - 1) : 0.0;
        info->edge_visits = ((double)hs->iter + sweeps) * (double)g->nnz;
        info->ms_device = ms;
        info->launches = launches;
        info->loop_edge_visits = info->edge_visits;
        info->ms_loop = ms_loop;
        info->frozen_rows = a.frozen ? (int32_t)hs->frozen : 0;
    }
    return converged ? PR_OK : PR_NOT_CONVERGED;
}

}  // namespace

extern "C" pr_status pr_solve(pr_graph* g, float damping, double tol, int32_t max_iter, int variant,
                              const float* teleport, const float* x0, float* x_out, pr_info* info,
                              void* stream) {
    pr_status rc = check_solve_args(g, damping, tol, max_iter, x_out);
    if (rc != PR_OK) return rc;
    if (variant == PR_JACOBI)
        return run_jacobi(g, damping, tol, max_iter, teleport, x0, x_out, true, true, info,
                          (cudaStream_t)stream);
    if (variant == PR_NONBLOCKING)
        return solve_nonblocking(g, damping, tol, max_iter, teleport, x0, x_out, info,
                                 (cudaStream_t)stream);
    if (variant == PR_EDGE)
        return run_jacobi(g, damping, tol, max_iter, teleport, x0, x_out, true, false, info,
                          (cudaStream_t)stream, true);
    return fail(PR_ERR_INVALID_ARG, "variant must be PR_JACOBI, PR_NONBLOCKING or PR_EDGE");
}

extern "C" pr_status pr_iterate(pr_graph* g, float damping, const float* teleport, const float* x_in,
                                int32_t n_iter, float* x_out, pr_info* info, void* stream) {
    if (!x_in) return fail(PR_ERR_INVALID_ARG, "x_in is NULL");
    pr_status rc = check_solve_args(g, damping, 1.0, n_iter, x_out);
    if (rc != PR_OK) return rc;
    // tol 0 is never met: exactly n_iter updates, no early stop
    rc = run_jacobi(g, damping, 0.0, n_iter, teleport, x_in, x_out, false, false, info,
                    (cudaStream_t)stream);
    return rc == PR_NOT_CONVERGED ? PR_OK : rc;
}
