// pr_batched.cu -- batched personalised PageRank: k <= 32 teleport vectors
// solved together on one graph (pr_solve_batched).
//
// Column j of the n x 32 rank matrix X is the PageRank vector of teleport t_j
// (Eq. 1 with (1-d) t_j(v) in place of (1-d)/n; the dangling mass of column j
// is still spread uniformly).  One synchronous iteration (Alg. 1, all
// columns at once) is the sparse-times-dense product
//
//   S(v, :)  = sum_{e in row v} Y(colidx[e], :)          Y = X / outdeg (row-wise)
//   X'(v, j) = (1-d) t_j(v) + d (S(v, j) + D_j / n)      for active columns j
//   Y'(v, :) = X'(v, :) / outdeg(v)
//   D'_j     = sum_{outdeg(v)=0} X'(v, j),  r_j = sum_v |X'(v, j) - X(v, j)|
//
// so every gathered edge moves one 128-byte row of Y (one coalesced load per
// warp, lane j = column j) instead of one 4-byte value: the irregular access
// of the single-vector solve is paid once for 32 solves.  A column whose L1
// change r_j falls below tol is frozen (its bit in the active mask clears, its
// ranks are copied forward unchanged) and the loop ends when no column is
// active or after max_iter iterations.
//
// Three kernels per iteration, captured twice (ping-pong buffers) in a CUDA
// graph under a conditional while node, like the single-vector solve:
//   k_b_segments  heavy rows: a warp per 2048-edge segment sums 32 rows of Y
//                 per step (32 independent 128-byte loads in flight per
//                 warp) into a partial row P(segment, :);
//   k_b_light     light rows: a warp per task (rows of one degree class, at
//                 most kBTaskEdges edges) walks the task's edges in windows
//                 of 16 (one colidx load, then 16 independent row loads),
//                 closing a row of S at each row end;
//   k_b_update    four rows per warp over the n x 32 matrix: the update, the
//                 quotient, and per-column Kahan dangling mass and L1 change,
//                 reduced in a fixed block order by the last block, which
//                 also clears converged columns and the loop condition.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "pr_tile.cuh"

namespace prk {

constexpr int kBK = 32;              // row width of the batched matrices (floats)
// Edges of a light-row task of k_b_light: a warp walks its task's rows one
// after the other, so the row kernel's 6144-edge tiles would leave the
// launch waiting on the warps that drew the largest ones.
#ifndef PRK_BATCH_TASK_EDGES
#define PRK_BATCH_TASK_EDGES 512
#endif
constexpr int kBTaskEdges = PRK_BATCH_TASK_EDGES;
constexpr int kBUpdateBlocksPerSM = 4;
// Rows a warp of the update kernels has in flight per pass (each lane loads
// its column of S or the segment partials, and of X).  The update streams
// 4 n k floats per iteration and is latency-bound: at 4 rows a warp it ran at
// about half the DRAM bandwidth.
#ifndef PRK_BATCH_UPDATE_ROWS
#define PRK_BATCH_UPDATE_ROWS 4
#endif
constexpr int kBUpdateRows = PRK_BATCH_UPDATE_ROWS;
// Quads of four rows a warp of k_b_update has in flight (each lane one float4
// of S or the segment partials, and of X, per quad).
#ifndef PRK_BATCH_UPDATE_QUADS
#define PRK_BATCH_UPDATE_QUADS 4
#endif
constexpr int kBUpdateQuads = PRK_BATCH_UPDATE_QUADS;

// Device state of a batched solve.
struct BatchState {
    double d;
    double inv_n;
    double tol;
    int32_t max_iter;
    int32_t iter;
    int32_t done;
    int32_t k;
    uint32_t ticket;
    uint32_t active;                 // bit j: column j still iterating
    uint32_t error;                  // bit 0: a column with a non-positive or negative teleport
    int32_t uniform;                 // 1: every column's teleport is 1/n
    int32_t bf16;                    // 1 while the gathers read the BF16 copy of Y
    int32_t pad0;
    double bf16_switch;              // leave BF16 once every active column's change is below this
    const int32_t* tptr;             // teleport nonzeros of each binned row (CSR), when !uniform
    const int32_t* tcol;
    const float* tval;
    int32_t dc_sweeps;               // defect correction: BF16 correction sweeps made
    int32_t implicit_zero;           // 1: rows without in-edges implicit after the first update
    double Ddc[kBK];                 // defect correction: dangling mass of each column of delta
    double Dz[kBK];                  // implicit rows: dangling mass of each column's latest update
    double Tiso[kBK];                // teleport sum of each column over the isolated vertices
    double D[kBK];                   // dangling mass of each column of the current input
    double T[kBK];                   // teleport sum of each column
    double resid[kBK];               // last L1 change of each column
    double sum_x[kBK];
    double scale[kBK];
    int32_t col_iter[kBK];
};

struct BatchArgs {
    const void* rowptr;
    const int32_t* colidx;
    const float* inv_out;
    const int32_t* seg_row;
    const int32_t* seg_ptr;
    const Tile* tiles;
    int64_t n;
    int64_t n_heavy;                 // rows [0, n_heavy) are gathered in segments
    int64_t zero_start;              // rows [zero_start, n) have no in-edges
    int64_t iso_start;               // rows [iso_start, n) have no in- and no out-edges
    int32_t n_seg;
    int32_t n_tiles;
    BatchState* state;
    double* slots;                   // [grid][kBK][2] per-block column partials
    float* P;                        // [n_seg][kBK] segment partial rows
    float* S;                        // [n][kBK] gathered row sums of the light rows
    cudaGraphConditionalHandle cond;
    int32_t use_cond;
    int32_t pad;
};

// A quotient of Y as float, from FP32 or BF16 storage.
__device__ __forceinline__ float ld_q(const float* Y, int64_t i) { return __ldg(Y + i); }
__device__ __forceinline__ float ld_q(const __nv_bfloat16* Y, int64_t i) {
    return __bfloat162float(__ldg(Y + i));
}

template <typename T>
constexpr int kIsBf16 = 0;
template <>
constexpr int kIsBf16<__nv_bfloat16> = 1;

// True if this launch has nothing to do: the solve is done, or the gathers
// read the other storage type of Y in this phase.
template <typename T>
__device__ __forceinline__ bool batch_skip(const BatchState* st) {
    __shared__ int32_t skip;
    if (threadIdx.x == 0) {
        const int32_t done = *(const volatile int32_t*)&st->done;
        const int32_t bf = *(const volatile int32_t*)&st->bf16;
        skip = done || (bf != kIsBf16<T>);
    }
    __syncthreads();
    const bool v = skip;
    __syncthreads();
    return v;
}

// done flag of the solve, read once per block.
__device__ __forceinline__ int32_t batch_done(const BatchState* st) {
    __shared__ int32_t done;
    if (threadIdx.x == 0) done = *(const volatile int32_t*)&st->done;
    __syncthreads();
    const int32_t v = done;
    __syncthreads();
    return v;
}

// Heavy rows: one warp per segment; lane j accumulates column j.
template <typename IdxT, typename T>
__global__ void __launch_bounds__(kBlock) k_b_segments(BatchArgs a, const T* __restrict__ Y) {
    if (batch_skip<T>(a.state)) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s = warp; s < a.n_seg; s += nwarp) {
        const int32_t h = a.seg_row[s];
        const int64_t re = row_at<IdxT>(a.rowptr, h + 1);
        const int64_t e0 = row_at<IdxT>(a.rowptr, h) + (s - a.seg_ptr[h]) * (int64_t)kSegEdges;
        const int64_t e1 = min(e0 + (int64_t)kSegEdges, re);
        float acc = 0.f;
        for (int64_t wb = e0; wb < e1; wb += 32) {
            const int32_t c = wb + lane < e1 ? ld_stream(a.colidx + wb + lane) : -1;
            float v[32];
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                const int32_t u = __shfl_sync(0xffffffffu, c, e);
                v[e] = u >= 0 ? ld_q(Y, (int64_t)u * kBK + lane) : 0.f;
            }
#pragma unroll
            for (int e = 0; e < 32; ++e) acc += v[e];
        }
        a.P[s * kBK + lane] = acc;
    }
}

// Light rows: one warp per tile of rows with at least one in-edge each.  The
// tile's edges are walked in windows of kBW = 16: lane e loads colidx of edge
// wb + e, every lane then loads its column of the 16 source rows (16
// independent 128-byte row loads per warp), and the sums are closed at the
// row ends.  The lanes hold the end offsets of 32 rows starting at rbase; a
// window closes at most 16 rows, so while row - rbase < 16 every end inside
// the window is described, and one warp-wide OR of (1 << position of a row's
// last edge in the window) gives all of them as a bit mask.
constexpr int kBW = 16;

template <typename IdxT, typename T>
__global__ void __launch_bounds__(kBlock, 4) k_b_light(BatchArgs a, const T* __restrict__ Y) {
    if (batch_skip<T>(a.state)) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = warp; t < a.n_tiles; t += nwarp) {
        const Tile tile = a.tiles[t];
        if (tile.kind < 0) continue;    // heavy epilogue and empty rows: not gathered here
        const int64_t r1 = tile.row_end;
        const int64_t eend = row_at<IdxT>(a.rowptr, r1);
        int64_t row = tile.row_begin;   // row being summed
        int64_t rbase = row;            // first row whose end offset the lanes hold
        int64_t rend = rbase + 1 + lane <= r1 ? row_at<IdxT>(a.rowptr, rbase + 1 + lane) : INT64_MAX;
        float acc = 0.f;
        for (int64_t wb = row_at<IdxT>(a.rowptr, row); wb < eend; wb += kBW) {
            const int32_t c = (lane < kBW && wb + lane < eend) ? ld_stream(a.colidx + wb + lane) : -1;
            float v[kBW];
#pragma unroll
            for (int e = 0; e < kBW; ++e) {
                const int32_t u = __shfl_sync(0xffffffffu, c, e);
                v[e] = u >= 0 ? ld_q(Y, (int64_t)u * kBK + lane) : 0.f;
            }
            const int64_t pos = rend - 1 - wb;
            const unsigned ends = __reduce_or_sync(0xffffffffu, (pos >= 0 && pos < kBW) ? (1u << pos) : 0u);
#pragma unroll
            for (int e = 0; e < kBW; ++e) {
                acc += v[e];   // v[e] = 0 past the tile's last edge
                if ((ends >> e) & 1u) {
                    a.S[row * kBK + lane] = acc;
                    acc = 0.f;
                    ++row;
                }
            }
            if (row - rbase >= kBW && row < r1) {
                rbase = row;
                rend = rbase + 1 + lane <= r1 ? row_at<IdxT>(a.rowptr, rbase + 1 + lane) : INT64_MAX;
            }
        }
    }
}

// ---- gathers with asynchronous copies (PR_OPT_BATCH_ASYNC) ----------------
//
// The gathers above hold each row they load in registers until it is summed,
// which caps a warp at 16 (light) or 32 (segments) rows in flight and makes
// them latency-bound (ncu: L1->L2 request path 14-15% busy, DRAM 12-13%).
// These copy the rows of a 32-edge window into a per-warp shared-memory
// buffer with cp.async (16-byte pieces, no register dependency) while the
// previous window is summed from the other buffer, so each warp keeps 64
// rows in flight and needs few registers.  Lane j still sums column j.
constexpr int kAW = 32;   // edges per window

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// This lane's column index of the window of edges [wb, min(wb + kAW, ee))
// (-1 past ee): loaded a window ahead of its copies, so that issuing them
// does not wait on it.
__device__ __forceinline__ int32_t window_col(const int32_t* __restrict__ colidx, int64_t wb, int64_t ee, int lane) {
    return wb + lane < ee ? __ldg(colidx + wb + lane) : -1;
}

// Copy the source rows of a window (lane l holds the column index u_l of its
// edge l, -1 for none) into buf (row e of the window at buf + e * kBK
// elements).
template <typename T>
__device__ __forceinline__ void issue_window(int32_t u_l, const T* __restrict__ Y, T* buf, int lane) {
    constexpr int kPieces = kBK * (int)sizeof(T) / 16;   // 16-byte pieces of a row: 8 (FP32) or 4 (BF16)
#pragma unroll
    for (int k = 0; k < kPieces; ++k) {
        const int c = lane + 32 * k;          // piece c: row c / kPieces, part c % kPieces
        const int r = c / kPieces, part = c % kPieces;
        const int32_t u = __shfl_sync(0xffffffffu, u_l, r);
        if (u >= 0)
            cp_async16(reinterpret_cast<char*>(buf + (size_t)r * kBK) + 16 * part,
                       reinterpret_cast<const char*>(Y + (size_t)u * kBK) + 16 * part);
    }
    cp_async_commit();
}

__device__ __forceinline__ float ld_sm(const float* p) { return *p; }
__device__ __forceinline__ float ld_sm(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// Heavy rows: a warp per segment, windows double-buffered in shared memory.
template <typename IdxT, typename T>
__global__ void __launch_bounds__(kBlock) k_b_segments_async(BatchArgs a, const T* __restrict__ Y) {
    extern __shared__ __align__(16) unsigned char b_smem[];
    if (batch_skip<T>(a.state)) return;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    T* buf0 = reinterpret_cast<T*>(b_smem) + (size_t)wib * 2 * kAW * kBK;
    T* buf1 = buf0 + kAW * kBK;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s = warp; s < a.n_seg; s += nwarp) {
        const int32_t h = a.seg_row[s];
        const int64_t re = row_at<IdxT>(a.rowptr, h + 1);
        const int64_t e0 = row_at<IdxT>(a.rowptr, h) + (s - a.seg_ptr[h]) * (int64_t)kSegEdges;
        const int64_t e1 = min(e0 + (int64_t)kSegEdges, re);
        float acc = 0.f;
        issue_window<T>(window_col(a.colidx, e0, e1, lane), Y, buf0, lane);
        int32_t u_next = window_col(a.colidx, e0 + kAW, e1, lane);
        int w = 0;
        for (int64_t wb = e0; wb < e1; wb += kAW, ++w) {
            T* cur = (w & 1) ? buf1 : buf0;
            T* nxt = (w & 1) ? buf0 : buf1;
            if (wb + kAW < e1) issue_window<T>(u_next, Y, nxt, lane);
            else cp_async_commit();   // an empty group keeps the count of groups in flight fixed
            u_next = window_col(a.colidx, wb + 2 * kAW, e1, lane);
            cp_async_wait<1>();
            __syncwarp();
            const int cnt = (int)min((int64_t)kAW, e1 - wb);
            if (cnt == kAW) {
                // a full window: straight-line loads and adds, edge order
#pragma unroll
                for (int e = 0; e < kAW; ++e) acc += ld_sm(cur + e * kBK + lane);
            } else {
                for (int e = 0; e < cnt; ++e) acc += ld_sm(cur + e * kBK + lane);
            }
            __syncwarp();   // the buffer is refilled two windows on
        }
        cp_async_wait<0>();
        __syncwarp();
        a.P[s * kBK + lane] = acc;
    }
}

// Light rows: a warp per task, windows double-buffered in shared memory, the
// row ends of a window from one warp-wide OR (the lanes hold the end offsets
// of the 32 rows from the first row the window touches).
template <typename IdxT, typename T>
__global__ void __launch_bounds__(kBlock) k_b_light_async(BatchArgs a, const T* __restrict__ Y) {
    extern __shared__ __align__(16) unsigned char b_smem[];
    if (batch_skip<T>(a.state)) return;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    T* buf0 = reinterpret_cast<T*>(b_smem) + (size_t)wib * 2 * kAW * kBK;
    T* buf1 = buf0 + kAW * kBK;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = warp; t < a.n_tiles; t += nwarp) {
        const Tile tile = a.tiles[t];
        if (tile.kind < 0) continue;
        const int64_t r1 = tile.row_end;
        const int64_t eb = row_at<IdxT>(a.rowptr, tile.row_begin), eend = row_at<IdxT>(a.rowptr, r1);
        int64_t row = tile.row_begin;
        float acc = 0.f;
        issue_window<T>(window_col(a.colidx, eb, eend, lane), Y, buf0, lane);
        int32_t u_next = window_col(a.colidx, eb + kAW, eend, lane);
        // the lanes hold the end offsets of rows rbase + 1 .. rbase + 32; a
        // window closes at most 32 rows from `row`, so they are reloaded only
        // when a row has closed since (rows longer than a window skip it)
        int64_t rbase = row;
        int64_t rend = rbase + 1 + lane <= r1 ? row_at<IdxT>(a.rowptr, rbase + 1 + lane) : INT64_MAX;
        int w = 0;
        for (int64_t wb = eb; wb < eend; wb += kAW, ++w) {
            T* cur = (w & 1) ? buf1 : buf0;
            T* nxt = (w & 1) ? buf0 : buf1;
            if (wb + kAW < eend) issue_window<T>(u_next, Y, nxt, lane);
            else cp_async_commit();
            u_next = window_col(a.colidx, wb + 2 * kAW, eend, lane);
            if (row != rbase) {
                rbase = row;
                rend = rbase + 1 + lane <= r1 ? row_at<IdxT>(a.rowptr, rbase + 1 + lane) : INT64_MAX;
            }
            const int64_t pos = rend - 1 - wb;
            const unsigned ends = __reduce_or_sync(0xffffffffu, (pos >= 0 && pos < kAW) ? (1u << pos) : 0u);
            const int cnt = (int)min((int64_t)kAW, eend - wb);
            cp_async_wait<1>();
            __syncwarp();
            if (ends == 0u && cnt == kAW) {
                // no row ends in a full window: straight-line loads and adds
#pragma unroll
                for (int e = 0; e < kAW; ++e) acc += ld_sm(cur + e * kBK + lane);
            } else {
                // the edges up to each row end (bit k: a row ends at edge k), then
                // the rest; the same order of adds as edge by edge
                int e = 0;
                for (unsigned m = ends; m != 0u; m &= m - 1u) {
                    const int k = __ffs((int)m) - 1;
                    for (; e <= k; ++e) acc += ld_sm(cur + e * kBK + lane);
                    a.S[row * kBK + lane] = acc;
                    acc = 0.f;
                    ++row;
                }
                for (; e < cnt; ++e) acc += ld_sm(cur + e * kBK + lane);
            }
            __syncwarp();
        }
        cp_async_wait<0>();
        __syncwarp();
    }
}

// Per-column block partials of N values -> slots (N doubles per block and
// column; the buffer holds kSlotValues); the last block gets the grid totals
// of its own column in every lane-j thread of warp 0 (fixed order).
constexpr int kSlotValues = 3;
template <int N>
__device__ __forceinline__ bool batch_columns_to_grid_n(const double (&v)[N], double* slots, uint32_t* ticket,
                                                        double (&t)[N]) {
    static_assert(N <= kSlotValues, "slot values");
    __shared__ double sv[N][kBlock / 32][32];
    __shared__ int last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < N; ++i) sv[i][warp][lane] = v[i];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            double A = 0.0;
            for (int w = 0; w < kBlock / 32; ++w) A += sv[i][w][lane];
            slots[((size_t)blockIdx.x * kBK + lane) * N + i] = A;
        }
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return false;
    __threadfence();
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) t[i] = 0.0;
        for (unsigned blk = 0; blk < gridDim.x; ++blk)
#pragma unroll
            for (int i = 0; i < N; ++i) t[i] += __ldcg(slots + ((size_t)blk * kBK + lane) * N + i);
    }
    return true;
}

__device__ __forceinline__ bool batch_columns_to_grid(double a, double b, double* slots, uint32_t* ticket,
                                                      double* ta, double* tb) {
    const double v[2] = {a, b};
    double t[2] = {0.0, 0.0};
    const bool last = batch_columns_to_grid_n<2>(v, slots, ticket, t);
    *ta = t[0];
    *tb = t[1];
    return last;
}

// X' from S / P, per-column dangling mass and L1 change; lane j = column j.
//
// Rows without in-edges (binned rows [zero_start, n)) gather nothing, so by
// Eq. 1 a column's rank there is (1-d) t_v + d D/n, D its dangling mass.
// With implicit_zero, after the first update such a row's rank is not read
// or written: the update writes only the quotient of those with out-edges
// (rows up to iso_start) and nothing for the isolated vertices after them;
// for each active column the rows' L1 change, n_z d |D - Dz| / n with Dz
// the dangling mass of the column's previous update, and the isolated
// vertices' ranks, (1-d) Tiso + n_iso d D / n, as part of the next dangling
// mass, are added in FP64 by the last block.  k_b_zero_fill writes the ranks
// after the loop.  The quotients are those the full update would store.
__global__ void __launch_bounds__(kBlock) k_b_update(BatchArgs a, const float* __restrict__ Xin,
                                                     float* __restrict__ Xout, float* __restrict__ Yout,
                                                     __nv_bfloat16* __restrict__ Yout16) {
    __shared__ int32_t s_implicit;
    __shared__ int32_t s_bf16;
    __shared__ float s_dshare[kBK];
    __shared__ float s_base[kBK];
    __shared__ uint32_t s_active;
    __shared__ const int32_t* s_tptr;
    __shared__ const int32_t* s_tcol;
    __shared__ const float* s_tval;
    __shared__ int32_t s_done;
    __shared__ float s_d, s_omd;
    BatchState* st = a.state;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        const double d = st->d;
        s_dshare[lane] = (float)(d * st->D[lane] * st->inv_n);
        s_base[lane] = (float)((1.0 - d) * st->inv_n + d * st->D[lane] * st->inv_n);
        if (lane == 0) {
            s_active = st->active;
            s_bf16 = st->bf16;
            s_implicit = st->implicit_zero && st->iter > 0;
            s_done = *(const volatile int32_t*)&st->done;
            s_tptr = st->uniform ? nullptr : st->tptr;
            s_tcol = st->tcol;
            s_tval = st->tval;
            s_d = (float)d;
            s_omd = (float)(1.0 - d);
        }
    }
    __syncthreads();
    if (s_done) {
        if (a.use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(a.cond, 0);
        return;
    }
    // Rows in quads of four consecutive rows: lane l holds columns c0 .. c0+3
    // (c0 = 4 (l % 8)) of row l / 8 of the quad, so every load of S, P, X and
    // every store of X', Y' is one float4 per lane and a warp instruction moves
    // 512 contiguous bytes; kQuads quads (4 kQuads rows) per warp in flight.
    const int c0 = (lane & 7) * 4;
    const int sub = lane >> 3;
    float dsh[4], bas[4];
    bool act[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        dsh[k] = s_dshare[c0 + k];
        bas[k] = s_base[c0 + k];
        act[k] = (s_active >> (c0 + k)) & 1u;
    }
    const float d = s_d, omd = s_omd;
    const int32_t* tptr = s_tptr;
    // this lane's four teleport values of row v (the CSR of the nonzeros)
    auto teleports = [&](int64_t v, float (&tv)[4]) {
#pragma unroll
        for (int k = 0; k < 4; ++k) tv[k] = 0.f;
        const int32_t p1 = tptr[v + 1];
        for (int32_t p = tptr[v]; p < p1; ++p) {
            const int j = s_tcol[p] - c0;
            const float val = s_tval[p];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (j == k) tv[k] = val;
        }
    };
    Acc acc[4];
    constexpr int kQuads = kBUpdateQuads;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t step = (((int64_t)gridDim.x * blockDim.x) >> 5) * kQuads * 4;
    const bool implicit = s_implicit != 0;
    const int64_t hi = implicit ? a.zero_start : a.n;   // rows updated in full
    for (int64_t q0 = warp * kQuads * 4; q0 < hi; q0 += step) {
        float4 sv[kQuads], xo[kQuads];
        float inv[kQuads];
#pragma unroll
        for (int q = 0; q < kQuads; ++q) {
            const int64_t v = q0 + 4 * q + sub;
            sv[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            xo[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            inv[q] = 0.f;
            if (v < hi) {
                if (v < a.n_heavy) {
                    const int32_t j1 = a.seg_ptr[v + 1];
                    for (int32_t j = a.seg_ptr[v]; j < j1; ++j) {
                        const float4 p = __ldcg(reinterpret_cast<const float4*>(a.P + (size_t)j * kBK + c0));
                        sv[q].x += p.x;
                        sv[q].y += p.y;
                        sv[q].z += p.z;
                        sv[q].w += p.w;
                    }
                } else if (v < a.zero_start) {
                    sv[q] = __ldcs(reinterpret_cast<const float4*>(a.S + (size_t)v * kBK + c0));
                }
                xo[q] = __ldcs(reinterpret_cast<const float4*>(Xin + (size_t)v * kBK + c0));
                inv[q] = __ldg(a.inv_out + v);
            }
        }
#pragma unroll
        for (int q = 0; q < kQuads; ++q) {
            const int64_t v = q0 + 4 * q + sub;
            if (v >= hi) continue;
            const float s4[4] = {sv[q].x, sv[q].y, sv[q].z, sv[q].w};
            const float x4[4] = {xo[q].x, xo[q].y, xo[q].z, xo[q].w};
            float tv[4] = {0.f, 0.f, 0.f, 0.f};
            if (tptr) teleports(v, tv);
            float xn[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                xn[k] = x4[k];
                if (act[k]) xn[k] = tptr ? fmaf(d, s4[k], fmaf(omd, tv[k], dsh[k])) : fmaf(d, s4[k], bas[k]);
            }
            const float iv = inv[q];
            __stcs(reinterpret_cast<float4*>(Xout + (size_t)v * kBK + c0), make_float4(xn[0], xn[1], xn[2], xn[3]));
            __stcs(reinterpret_cast<float4*>(Yout + (size_t)v * kBK + c0),
                   make_float4(xn[0] * iv, xn[1] * iv, xn[2] * iv, xn[3] * iv));
            if (s_bf16) {
                __nv_bfloat162* y16 = reinterpret_cast<__nv_bfloat162*>(Yout16 + (size_t)v * kBK + c0);
                y16[0] = __floats2bfloat162_rn(xn[0] * iv, xn[1] * iv);
                y16[1] = __floats2bfloat162_rn(xn[2] * iv, xn[3] * iv);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                acc[k].add_r(fabsf(xn[k] - x4[k]));
                if (iv == 0.f) acc[k].kahan(xn[k]);
            }
        }
    }
    if (implicit) {
        // rows without in-edges that have out-edges: the quotient only (the
        // same value as the full update's, which adds d * 0)
        for (int64_t q0 = a.zero_start + warp * kQuads * 4; q0 < a.iso_start; q0 += step) {
            float inv[kQuads];
#pragma unroll
            for (int q = 0; q < kQuads; ++q) {
                const int64_t v = q0 + 4 * q + sub;
                inv[q] = v < a.iso_start ? __ldg(a.inv_out + v) : 0.f;
            }
#pragma unroll
            for (int q = 0; q < kQuads; ++q) {
                const int64_t v = q0 + 4 * q + sub;
                if (v >= a.iso_start) continue;
                float xn[4];
                float tv[4] = {0.f, 0.f, 0.f, 0.f};
                if (tptr) teleports(v, tv);
#pragma unroll
                for (int k = 0; k < 4; ++k) xn[k] = tptr ? fmaf(omd, tv[k], dsh[k]) : bas[k];
                const float iv = inv[q];
                __stcs(reinterpret_cast<float4*>(Yout + (size_t)v * kBK + c0),
                       make_float4(xn[0] * iv, xn[1] * iv, xn[2] * iv, xn[3] * iv));
            }
        }
    }
    // the warp's per-column totals in lane order: the lanes with the same c0
    // hold the same columns; lane j then takes column j = c0 + k of lane j / 4
    double rj = 0.0, mj = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double rk = acc[k].resid(), mk = acc[k].mass();
#pragma unroll
        for (int o = 8; o < 32; o <<= 1) {
            rk += __shfl_xor_sync(0xffffffffu, rk, o);
            mk += __shfl_xor_sync(0xffffffffu, mk, o);
        }
        rk = __shfl_sync(0xffffffffu, rk, lane >> 2);
        mk = __shfl_sync(0xffffffffu, mk, lane >> 2);
        if ((lane & 3) == k) {
            rj = rk;
            mj = mk;
        }
    }
    double R, Dn;
    if (batch_columns_to_grid(rj, mj, a.slots, &st->ticket, &R, &Dn) && threadIdx.x < 32) {
        const bool was_active = (s_active >> lane) & 1u;
        const double prev = st->resid[lane];
        if (implicit) {
            const double dd = st->d, Du = st->D[lane], Dz = st->Dz[lane];
            if (was_active) R += (double)(a.n - a.zero_start) * dd * fabs(Du - Dz) * st->inv_n;
            Dn += (1.0 - dd) * st->Tiso[lane] + (double)(a.n - a.iso_start) * dd * (was_active ? Du : Dz) * st->inv_n;
        }
        if (was_active) st->Dz[lane] = st->D[lane];   // the mass this update's zero-row ranks use
        st->D[lane] = Dn;
        const int32_t it = st->iter + 1;
        if (was_active) {
            st->resid[lane] = R;
            st->col_iter[lane] = it;
        }
        // A column converges only on FP32 iterates: in the BF16 phase the
        // iteration contracts towards the fixed point of the rounded map, whose
        // changes can fall below tol away from the true fixed point.
        const bool bf = st->bf16 != 0;
        const bool stays = was_active && (bf || !(R < st->tol));
        const uint32_t mask = __ballot_sync(0xffffffffu, stays);
        // BF16 phase: leave it once no active column both changes by
        // max(bf16_switch, tol) or more and still shrinks its change by 10% an
        // iteration (past that, BF16 rounding, not the iteration, sets the change)
        const double sw = fmax(st->bf16_switch, st->tol);
        const uint32_t big = __ballot_sync(0xffffffffu, was_active && !(R < sw) && R < 0.9 * prev);
        if (lane == 0) {
            if (bf && big == 0u) st->bf16 = 0;
            st->active = mask;
            st->iter = it;
            const int done = mask == 0u || it >= st->max_iter;
            st->done = done;
            st->ticket = 0;
            if (done && a.use_cond) cudaGraphSetConditional(a.cond, 0);
        }
    }
}

// ---- BF16 storage by defect correction (PR_OPT_BATCH_DC) -------------------
//
// The iteration x <- F(x) = b + A x of Eq. 1 (A = d (P^T + 1 a^T / n)) is
// split into an outer FP32 step and an inner correction solve.  From the
// current X, the FP32 step gives X' = F(X) and r = X' - X (its L1 norm per
// column is the usual stopping test, on FP32 iterates).  The error e = x* - X
// solves e = r + A e, which M sweeps approximate from delta_0 = r:
//   delta_{m+1} = r + A delta_m,
// gathering delta / outdeg from a BF16 copy (64-byte rows, FP32 sums).  Then
// X <- X + delta_M.  BF16 rounds delta, not x, so its error shrinks with the
// residual and the outer steps reach the FP32 tolerance.

// Rounding a quotient delta(u)/outdeg(u) to BF16 changes the mass the
// gathers pass on by outdeg(u) times the rounding error -- for a hub, ten
// thousand times a 2^-9 relative error.  Left alone this mass error is what
// the corrections stall on (an FP32 emulation of R-MAT-16 with 8 seed-set
// columns: 10 outer steps instead of 4, the iterates' mass 1e-3 off).  So the
// mass each row loses to rounding, delta(u) - outdeg(u) bf16(delta(u)/outdeg(u)),
// is summed per column and spread uniformly with the dangling mass: every
// sweep then conserves mass exactly (up to FP32 rounding).
__device__ __forceinline__ __nv_bfloat16 dc_quotient(float dv, float inv, KahanF& dm) {
    const __nv_bfloat16 q = __float2bfloat16_rn(dv * inv);
    if (inv == 0.f) dm.add(dv);                                   // dangling: all of it
    else dm.add(dv - __bfloat162float(q) / inv);                 // what rounding lost
    return q;
}

// R = X' - X and delta_0 = R for the active columns (0 for the others), the
// BF16 quotient of delta_0 and the mass it does not pass on per column (its
// dangling mass and the rounding loss); the gathers that follow read BF16.
__global__ void __launch_bounds__(kBlock) k_b_dc_prep(BatchArgs a, const float* __restrict__ Xprev,
                                                      const float* __restrict__ Xcur, float* __restrict__ R,
                                                      __nv_bfloat16* __restrict__ Yd16) {
    BatchState* st = a.state;
    if (batch_done(st)) return;
    const int lane = threadIdx.x & 31;
    const bool active = (st->active >> lane) & 1u;
    KahanF dm;
    const int64_t rows_per_pass = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < a.n; v += rows_per_pass) {
        const size_t i = (size_t)v * kBK + lane;
        const float r = active ? __ldcs(Xcur + i) - __ldcs(Xprev + i) : 0.f;
        const float inv = __ldg(a.inv_out + v);
        R[i] = r;
        Yd16[i] = dc_quotient(r, inv, dm);
    }
    double Dd, unused;
    if (batch_columns_to_grid(dm.value(), 0.0, a.slots, &st->ticket, &Dd, &unused) && threadIdx.x < 32) {
        st->Ddc[lane] = Dd;
        if (lane == 0) {
            st->bf16 = 1;
            st->ticket = 0;
        }
    }
}

// One correction sweep: delta'(v, j) = R(v, j) + d (S(v, j) + Ddc_j / n) from
// the gathered sums of the BF16 quotient of delta, Ddc the mass those sums do
// not carry (dangling mass and rounding loss); writes delta' (FP32) and its
// BF16 quotient, and the new Ddc.
__global__ void __launch_bounds__(kBlock) k_b_dc_update(BatchArgs a, const float* __restrict__ R,
                                                        float* __restrict__ Dl, __nv_bfloat16* __restrict__ Yd16) {
    BatchState* st = a.state;
    if (batch_done(st)) return;
    const int lane = threadIdx.x & 31;
    const float d = (float)st->d;
    const float share = (float)(st->Ddc[lane] * st->inv_n);   // Ddc / n; d multiplies the sum below
    KahanF dm;
    constexpr int kRows = kBUpdateRows;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t step = (((int64_t)gridDim.x * blockDim.x) >> 5) * kRows;
    for (int64_t v0 = warp * kRows; v0 < a.n; v0 += step) {
        float sv[kRows], rv[kRows], inv[kRows];
#pragma unroll
        for (int q = 0; q < kRows; ++q) {
            const int64_t v = v0 + q;
            sv[q] = rv[q] = inv[q] = 0.f;
            if (v < a.n) {
                if (v < a.n_heavy) {
                    const int32_t q1 = a.seg_ptr[v + 1];
                    for (int32_t j = a.seg_ptr[v]; j < q1; ++j) sv[q] += __ldcg(a.P + (size_t)j * kBK + lane);
                } else if (v < a.zero_start) {
                    sv[q] = __ldcs(a.S + (size_t)v * kBK + lane);
                }
                rv[q] = __ldcs(R + (size_t)v * kBK + lane);
                inv[q] = __ldg(a.inv_out + v);
            }
        }
#pragma unroll
        for (int q = 0; q < kRows; ++q) {
            const int64_t v = v0 + q;
            if (v >= a.n) break;
            const float dn = rv[q] + d * (sv[q] + share);   // 0 for inactive columns (R = 0, S = 0)
            Dl[(size_t)v * kBK + lane] = dn;
            Yd16[(size_t)v * kBK + lane] = dc_quotient(dn, inv[q], dm);
        }
    }
    double Dd, unused;
    if (batch_columns_to_grid(dm.value(), 0.0, a.slots, &st->ticket, &Dd, &unused) && threadIdx.x < 32) {
        st->Ddc[lane] = Dd;
        if (lane == 0) {
            st->dc_sweeps += 1;
            st->ticket = 0;
        }
    }
}

// X <- Xprev + delta for the active columns (the others keep the FP32 step's
// copy), Y = X / outdeg, the dangling mass of every column; the gathers that
// follow read FP32 again.
__global__ void __launch_bounds__(kBlock) k_b_dc_apply(BatchArgs a, const float* __restrict__ Xprev,
                                                       float* __restrict__ Xcur, const float* __restrict__ Dl,
                                                       float* __restrict__ Ycur) {
    BatchState* st = a.state;
    if (batch_done(st)) return;
    const int lane = threadIdx.x & 31;
    const bool active = (st->active >> lane) & 1u;
    KahanF dm;
    const int64_t rows_per_pass = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < a.n; v += rows_per_pass) {
        const size_t i = (size_t)v * kBK + lane;
        const float inv = __ldg(a.inv_out + v);
        float x = __ldcs(Xcur + i);
        if (active) {
            x = __ldcs(Xprev + i) + __ldcs(Dl + i);
            Xcur[i] = x;
            Ycur[i] = x * inv;
        }
        if (inv == 0.f) dm.add(x);
    }
    double Dn, unused;
    if (batch_columns_to_grid(dm.value(), 0.0, a.slots, &st->ticket, &Dn, &unused) && threadIdx.x < 32) {
        st->D[lane] = Dn;
        if (lane == 0) {
            st->bf16 = 0;
            st->ticket = 0;
        }
    }
}

// X = T (binned order, 32 wide), Y = X / outdeg, per-column D and T; resets
// the loop state.  t_dense: caller order, n x k, or NULL for uniform.
__global__ void __launch_bounds__(kBlock) k_b_init(BatchArgs a, const float* __restrict__ t_dense,
                                                   const int32_t* __restrict__ order, float* __restrict__ X,
                                                   float* __restrict__ Y, __nv_bfloat16* __restrict__ Y16) {
    BatchState* st = a.state;
    const int lane = threadIdx.x & 31;
    const int k = st->k;
    const float tu = (float)st->inv_n;
    double dsum = 0.0, tsum = 0.0, tiso = 0.0;
    bool bad = false;
    const int64_t rows_per_pass = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < a.n; v += rows_per_pass) {
        float tv = 0.f;
        if (lane < k) {
            tv = t_dense ? t_dense[(size_t)order[v] * k + lane] : tu;
            if (!(tv >= 0.f)) bad = true;   // negative or NaN
        }
        const float inv = a.inv_out[v];
        X[(size_t)v * kBK + lane] = tv;
        Y[(size_t)v * kBK + lane] = tv * inv;
        if (Y16) Y16[(size_t)v * kBK + lane] = __float2bfloat16_rn(tv * inv);
        if (inv == 0.f) dsum += (double)tv;
        if (v >= a.iso_start) tiso += (double)tv;
        tsum += (double)tv;
    }
    if (bad) atomicOr(&st->error, 1u);
    const double part[3] = {dsum, tsum, tiso};
    double tot[3];
    if (batch_columns_to_grid_n<3>(part, a.slots, &st->ticket, tot) && threadIdx.x < 32) {
        const double D = tot[0], T = tot[1];
        st->D[lane] = D;
        st->T[lane] = T;
        st->Tiso[lane] = tot[2];
        st->resid[lane] = INFINITY;
        st->col_iter[lane] = 0;
        if (lane < k && !(T > 0.0)) atomicOr(&st->error, 1u);
        if (lane == 0) {
            st->iter = 0;
            st->done = 0;
            st->active = k == 32 ? 0xffffffffu : ((1u << k) - 1u);
            st->ticket = 0;
        }
    }
}

// The ranks of the rows without in-edges after a loop that kept them implicit
// (k_b_update): (1-d) t_v + d Dz/n for each of the k columns, Dz the dangling
// mass of the column's last update, in the same FP32 arithmetic as the update.
__global__ void __launch_bounds__(kBlock) k_b_zero_fill(BatchArgs a, float* __restrict__ X0, float* __restrict__ X1) {
    const BatchState* st = a.state;
    if (!st->implicit_zero || st->iter < 2) return;   // after one update the rows were written in full
    float* X = (st->iter & 1) ? X1 : X0;
    const int lane = threadIdx.x & 31;
    if (lane >= st->k) return;
    const double d = st->d;
    const float omd = (float)(1.0 - d);
    const float dshare = (float)(d * st->Dz[lane] * st->inv_n);
    const float base = (float)((1.0 - d) * st->inv_n + d * st->Dz[lane] * st->inv_n);
    const int32_t* tptr = st->uniform ? nullptr : st->tptr;
    const int32_t* tcol = st->tcol;
    const float* tval = st->tval;
    const int64_t rows_per_pass = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = a.zero_start + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); v < a.n;
         v += rows_per_pass) {
        float xn = base;
        if (tptr) {
            float tv = 0.f;
            const int32_t p1 = tptr[v + 1];
            for (int32_t p = tptr[v]; p < p1; ++p)
                if (tcol[p] == lane) tv = tval[p];
            xn = fmaf(omd, tv, dshare);
        }
        X[(size_t)v * kBK + lane] = xn;
    }
}

// Nonzeros of each binned row of the caller's teleport matrix.
__global__ void k_b_tcount(const float* __restrict__ t_dense, const int32_t* __restrict__ order, int64_t n,
                           int k, int64_t* __restrict__ counts) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const float* row = t_dense + (size_t)order[v] * k;
        int64_t c = 0;
        for (int j = 0; j < k; ++j) c += row[j] != 0.f;
        counts[v] = c;
    }
}

__global__ void k_b_tfill(const float* __restrict__ t_dense, const int32_t* __restrict__ order, int64_t n, int k,
                          const int32_t* __restrict__ tptr, int32_t* __restrict__ tcol, float* __restrict__ tval) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const float* row = t_dense + (size_t)order[v] * k;
        int32_t p = tptr[v];
        for (int j = 0; j < k; ++j)
            if (row[j] != 0.f) {
                tcol[p] = j;
                tval[p] = row[j];
                ++p;
            }
    }
}

// Per-column sum of the final X (buffer iter & 1) and the rescaling factors.
__global__ void __launch_bounds__(kBlock) k_b_sum(BatchArgs a, const float* __restrict__ X0,
                                                  const float* __restrict__ X1) {
    BatchState* st = a.state;
    const float* X = (st->iter & 1) ? X1 : X0;
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    const int64_t rows_per_pass = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < a.n; v += rows_per_pass)
        s += (double)X[(size_t)v * kBK + lane];
    double S, unused;
    if (batch_columns_to_grid(s, 0.0, a.slots, &st->ticket, &S, &unused) && threadIdx.x < 32) {
        st->sum_x[lane] = S;
        st->scale[lane] = S > 0.0 ? st->T[lane] / S : 1.0;
        if (lane == 0) st->ticket = 0;
    }
}

// out[v][j] = X[rank[v]][j] * scale_j, caller order, k columns.
__global__ void k_b_unpermute(BatchArgs a, const float* __restrict__ X0, const float* __restrict__ X1,
                              const int32_t* __restrict__ rank, float* __restrict__ out, int k) {
    const BatchState* st = a.state;
    const float* X = (st->iter & 1) ? X1 : X0;
    const int64_t total = a.n * (int64_t)k;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const int64_t v = i / k;
        const int j = (int)(i - v * k);
        out[i] = X[(size_t)rank[v] * kBK + j] * (float)st->scale[j];
    }
}

// ------------------------------------------------------------------ host --

// Buffers of the batched solver, allocated on the first batched call.
struct BatchCtx {
    float* X[2] = {nullptr, nullptr};
    float* Y[2] = {nullptr, nullptr};
    __nv_bfloat16* Y16[2] = {nullptr, nullptr};   // BF16 copies of Y (first BF16 solve)
    int graph_bf16 = -1;             // storage mode the captured loop graph was built for
    float* S = nullptr;
    float* P = nullptr;
    float* R = nullptr;              // defect correction: residual X' - X of the FP32 step
    float* Dl = nullptr;             // defect correction: latest correction delta (FP32)
    int32_t* tptr = nullptr;
    int32_t* tcol = nullptr;
    float* tval = nullptr;
    int64_t t_cap = 0;
    int64_t* tcount = nullptr;
    float* t_stage = nullptr;        // host teleports copied here
    float* out_stage = nullptr;      // host outputs staged here
    BatchState* state = nullptr;
    BatchState* host_state = nullptr;
    double* slots = nullptr;
    int slot_blocks = 0;
    int64_t zero_start = 0;
    Tile* tasks = nullptr;           // light-row tasks of k_b_light (rows of one degree class)
    int64_t n_tasks = 0;
    cudaGraphExec_t loop_exec = nullptr;
};

namespace {

int g_occ_bseg = 0, g_occ_blight = 0;

int batch_grid(const pr_graph* g, int64_t warps, int occ) {
    const int64_t blocks = (warps + kWarps - 1) / kWarps;
    return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)g->sm_count * occ));
}

BatchArgs batch_args(const pr_graph* g, const BatchCtx* b) {
    BatchArgs a{};
    a.rowptr = g->rowptr;
    a.colidx = g->colidx;
    a.inv_out = g->inv_out;
    a.seg_row = g->seg_row;
    a.seg_ptr = g->seg_ptr;
    a.tiles = b->tasks;
    a.n = g->n;
    a.n_heavy = g->n_heavy;
    a.zero_start = b->zero_start;
    a.iso_start = g->n - g->n_isolated;
    a.n_seg = (int32_t)g->n_seg;
    a.n_tiles = (int32_t)b->n_tasks;
    a.state = b->state;
    a.slots = b->slots;
    a.P = b->P;
    a.S = b->S;
    return a;
}

int update_grid(const pr_graph* g, const BatchCtx* b) {
    const int64_t want = (g->n * 32 + kBlock - 1) / kBlock;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)b->slot_blocks));
}

// Dynamic shared memory of the asynchronous gathers: two windows per warp.
template <typename T>
constexpr size_t async_smem() {
    return (size_t)kWarps * 2 * kAW * kBK * sizeof(T);
}

// Blocks per SM of an asynchronous gather kernel (shared memory bounds it),
// set up once per kernel.
template <typename K>
int async_occupancy(K kernel, size_t smem) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kernel, kBlock, smem) != cudaSuccess) {
        cudaGetLastError();
        o = 1;
    }
    return std::max(1, o);
}

// The segment and light-row gathers of one sweep over the quotient matrix Y
// (FP32 or BF16), with register loads or, with PR_OPT_BATCH_ASYNC, with
// asynchronous copies into shared memory.  Returns the kernels launched.
// Blocks per SM of the asynchronous gathers, [segments, light][IdxT 32/64][FP32, BF16];
// set by ensure_batch (outside any stream capture).
int g_occ_async[2][2][2] = {};

template <typename IdxT, typename T>
void init_async_occupancy() {
    const int i = sizeof(IdxT) == 8 ? 1 : 0, j = sizeof(T) == 2 ? 1 : 0;
    g_occ_async[0][i][j] = async_occupancy(k_b_segments_async<IdxT, T>, async_smem<T>());
    g_occ_async[1][i][j] = async_occupancy(k_b_light_async<IdxT, T>, async_smem<T>());
}

template <typename IdxT, typename T>
int launch_gathers(const pr_graph* g, const BatchCtx* b, const BatchArgs& a, const T* Y, cudaStream_t s) {
    int n = 0;
    if (g->batch_async) {
        const int i = sizeof(IdxT) == 8 ? 1 : 0, j = sizeof(T) == 2 ? 1 : 0;
        const int occ_s = g_occ_async[0][i][j], occ_l = g_occ_async[1][i][j];
        if (g->n_seg > 0) {
            k_b_segments_async<IdxT, T><<<batch_grid(g, g->n_seg, occ_s), kBlock, async_smem<T>(), s>>>(a, Y);
            ++n;
        }
        k_b_light_async<IdxT, T><<<batch_grid(g, b->n_tasks, occ_l), kBlock, async_smem<T>(), s>>>(a, Y);
        return n + 1;
    }
    if (g->n_seg > 0) {
        k_b_segments<IdxT, T><<<batch_grid(g, g->n_seg, g_occ_bseg), kBlock, 0, s>>>(a, Y);
        ++n;
    }
    k_b_light<IdxT, T><<<batch_grid(g, b->n_tasks, g_occ_blight), kBlock, 0, s>>>(a, Y);
    return n + 1;
}

// One iteration.  With BF16 storage both gather versions are enqueued and the
// one that does not match the current phase returns at once.
template <typename IdxT>
cudaError_t enqueue_batch_iteration(const pr_graph* g, const BatchCtx* b, const BatchArgs& a, int src,
                                    bool bf16, cudaStream_t s) {
    if (bf16) launch_gathers<IdxT, __nv_bfloat16>(g, b, a, b->Y16[src], s);
    launch_gathers<IdxT, float>(g, b, a, b->Y[src], s);
    k_b_update<<<update_grid(g, b), kBlock, 0, s>>>(a, b->X[src], b->X[1 - src], b->Y[1 - src],
                                                   bf16 ? b->Y16[1 - src] : nullptr);
    return cudaGetLastError();
}

cudaError_t enqueue_batch(const pr_graph* g, const BatchCtx* b, const BatchArgs& a, int src, bool bf16,
                          cudaStream_t s) {
    return g->idx64 ? enqueue_batch_iteration<int64_t>(g, b, a, src, bf16, s)
                    : enqueue_batch_iteration<int32_t>(g, b, a, src, bf16, s);
}

// One outer step of the defect-correction form: the FP32 step X[src] ->
// X[1-src], the residual, `sweeps` BF16 correction sweeps, the correction
// applied to X[1-src].  Returns the kernels launched.
template <typename IdxT>
cudaError_t enqueue_dc_step(const pr_graph* g, const BatchCtx* b, const BatchArgs& a, int src, int sweeps,
                            cudaStream_t s, int* launches) {
    cudaError_t e = enqueue_batch_iteration<IdxT>(g, b, a, src, false, s);
    if (e != cudaSuccess) return e;
    *launches += g->n_seg > 0 ? 3 : 2;
    const int ug = update_grid(g, b);
    k_b_dc_prep<<<ug, kBlock, 0, s>>>(a, b->X[src], b->X[1 - src], b->R, b->Y16[0]);
    ++*launches;
    for (int m = 0; m < sweeps; ++m) {
        *launches += launch_gathers<IdxT, __nv_bfloat16>(g, b, a, b->Y16[m & 1], s);
        k_b_dc_update<<<ug, kBlock, 0, s>>>(a, b->R, b->Dl, b->Y16[(m + 1) & 1]);
        ++*launches;
    }
    k_b_dc_apply<<<ug, kBlock, 0, s>>>(a, b->X[src], b->X[1 - src], b->Dl, b->Y[1 - src]);
    ++*launches;
    return cudaGetLastError();
}

pr_status ensure_batch(pr_graph* g) {
    if (g->batch) return PR_OK;
    BatchCtx* b = new BatchCtx();
    g->batch = b;
    const size_t mat = (size_t)(g->n + kPad) * kBK * sizeof(float);
    for (int i = 0; i < 2; ++i) {
        PRK_CHECK(dev_alloc(g, (void**)&b->X[i], mat));
        PRK_CHECK(dev_alloc(g, (void**)&b->Y[i], mat));
    }
    PRK_CHECK(dev_alloc(g, (void**)&b->S, mat));
    PRK_CHECK(dev_alloc(g, (void**)&b->P, (size_t)(g->n_seg + 1) * kBK * sizeof(float)));
    PRK_CHECK(dev_alloc(g, (void**)&b->tptr, (size_t)(g->n + 1) * sizeof(int32_t)));
    PRK_CHECK(dev_alloc(g, (void**)&b->tcount, (size_t)(g->n + 1) * sizeof(int64_t)));
    PRK_CHECK(dev_alloc(g, (void**)&b->state, sizeof(BatchState)));
    PRK_CHECK(cudaMallocHost((void**)&b->host_state, sizeof(BatchState)));
    b->slot_blocks = g->sm_count * kBUpdateBlocksPerSM;
    PRK_CHECK(dev_alloc(g, (void**)&b->slots, (size_t)b->slot_blocks * kBK * kSlotValues * sizeof(double)));
    b->zero_start = g->n;
    for (const Tile& t : g->host_tiles)
        if (t.kind == kTileZero) {
            b->zero_start = std::min<int64_t>(b->zero_start, t.row_begin);
        }
    {
        int64_t heavy_rows = 0;
        std::vector<Tile> tasks;
        for (const Tile& t : tiles_with_threshold(g, g->heavy_degree, &heavy_rows, kBTaskEdges, kTileRowsMax))
            if (t.kind >= 0) tasks.push_back(t);
        b->n_tasks = (int64_t)tasks.size();
        PRK_CHECK(dev_alloc(g, (void**)&b->tasks, (tasks.size() + 1) * sizeof(Tile)));
        if (!tasks.empty())
            PRK_CHECK(cudaMemcpy(b->tasks, tasks.data(), tasks.size() * sizeof(Tile), cudaMemcpyHostToDevice));
    }
    if (g_occ_async[1][0][0] == 0) {
        init_async_occupancy<int32_t, float>();
        init_async_occupancy<int32_t, __nv_bfloat16>();
        init_async_occupancy<int64_t, float>();
        init_async_occupancy<int64_t, __nv_bfloat16>();
    }
    if (g_occ_bseg == 0) {
        int o = 0;
        PRK_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_b_segments<int32_t, float>, kBlock, 0));
        g_occ_bseg = std::max(1, o);
        PRK_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_b_light<int32_t, float>, kBlock, 0));
        g_occ_blight = std::max(1, o);
    }
    return PR_OK;
}

pr_status build_batch_graph(pr_graph* g, BatchCtx* b, bool bf16) {
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
    BatchArgs a = batch_args(g, b);
    a.cond = handle;
    a.use_cond = 1;
    PRK_CHECK(cudaStreamBeginCaptureToGraph(g->capture_stream, body, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal));
    cudaError_t e1 = enqueue_batch(g, b, a, 0, bf16, g->capture_stream);
    cudaError_t e2 = cudaSuccess;
    if (e1 == cudaSuccess) e2 = enqueue_batch(g, b, a, 1, bf16, g->capture_stream);
    cudaGraph_t captured = nullptr;
    cudaError_t e3 = cudaStreamEndCapture(g->capture_stream, &captured);
    PRK_CHECK(e1);
    PRK_CHECK(e2);
    PRK_CHECK(e3);
    PRK_CHECK(cudaGraphInstantiate(&b->loop_exec, graph, 0));
    b->graph_bf16 = bf16 ? 1 : 0;
    return PR_OK;
}

// The caller's teleport matrix as a CSR of its nonzeros over binned rows.
pr_status build_teleport_csr(pr_graph* g, BatchCtx* b, const float* t_dev, int k, cudaStream_t s) {
    const int grid = small_grid(g);
    k_b_tcount<<<grid, kBlock, 0, s>>>(t_dev, g->order, g->n, k, b->tcount);
    PRK_CHECK(cudaGetLastError());
    PRK_CHECK(scan_counts_i32(b->tcount, g->n, b->tptr, s));
    int32_t nnz = 0;
    PRK_CHECK(cudaMemcpyAsync(&nnz, b->tptr + g->n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PRK_CHECK(cudaStreamSynchronize(s));
    if (nnz > b->t_cap) {
        PRK_CHECK(cudaStreamSynchronize(s));   // earlier solves on this stream are done with them
        if (b->tcol) dev_free(b->tcol);
        if (b->tval) dev_free(b->tval);
        b->tcol = nullptr;
        b->tval = nullptr;
        b->t_cap = 0;
        PRK_CHECK(dev_alloc(g, (void**)&b->tcol, (size_t)nnz * sizeof(int32_t)));
        PRK_CHECK(dev_alloc(g, (void**)&b->tval, (size_t)nnz * sizeof(float)));
        b->t_cap = nnz;
    }
    k_b_tfill<<<grid, kBlock, 0, s>>>(t_dev, g->order, g->n, k, b->tptr, b->tcol, b->tval);
    PRK_CHECK(cudaGetLastError());
    return PR_OK;
}

}  // namespace

void drop_batch_graph(pr_graph* g) {
    if (g->batch && g->batch->loop_exec) {
        cudaGraphExecDestroy(g->batch->loop_exec);
        g->batch->loop_exec = nullptr;
    }
}

void destroy_batch(pr_graph* g) {
    BatchCtx* b = g->batch;
    if (!b) return;
    cudaDeviceSynchronize();   // earlier solves may still use the memory (cudaFree waited the same way)
    void* dev[] = {b->X[0], b->X[1], b->Y[0], b->Y[1], b->Y16[0], b->Y16[1], b->S, b->P, b->R, b->Dl, b->tptr,
                   b->tcol, b->tval, b->tcount, b->t_stage, b->out_stage, b->state, b->slots, b->tasks};
    for (void* p : dev)
        if (p) dev_free(p);
    if (b->host_state) cudaFreeHost(b->host_state);
    if (b->loop_exec) cudaGraphExecDestroy(b->loop_exec);
    delete b;
    g->batch = nullptr;
}

}  // namespace prk

using namespace prk;

extern "C" pr_status pr_solve_batched(pr_graph* g, float damping, double tol, int32_t max_iter, int32_t k,
                                      const float* teleport, float* x_out, double* col_residual,
                                      int32_t* col_iterations, pr_info* info, void* stream) {
    if (!g) return fail(PR_ERR_INVALID_ARG, "pr_solve_batched: graph is NULL");
    if (!(damping >= 0.0f && damping < 1.0f)) return fail(PR_ERR_INVALID_ARG, "damping must be in [0, 1)");
    if (!(tol > 0.0) || !std::isfinite(tol)) return fail(PR_ERR_INVALID_ARG, "tol must be a positive finite number");
    if (max_iter < 1) return fail(PR_ERR_INVALID_ARG, "max_iter must be >= 1");
    if (k < 1 || k > kBK) return fail(PR_ERR_INVALID_ARG, "k must be in [1, 32]");
    if (!x_out) return fail(PR_ERR_INVALID_ARG, "x_out is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    pr_status rc = ensure_batch(g);
    if (rc != PR_OK) return rc;
    BatchCtx* b = g->batch;
    const size_t nk = (size_t)g->n * (size_t)k;

    // teleport: device pointer in place, host memory staged
    const float* t_dev = nullptr;
    if (teleport) {
        if (is_device_pointer(teleport)) {
            t_dev = teleport;
        } else {
            if (!b->t_stage) PRK_CHECK(dev_alloc(g, (void**)&b->t_stage, (size_t)(g->n + kPad) * kBK * sizeof(float)));
            PRK_CHECK(cudaMemcpyAsync(b->t_stage, teleport, nk * sizeof(float), cudaMemcpyHostToDevice, s));
            t_dev = b->t_stage;
        }
        if ((rc = build_teleport_csr(g, b, t_dev, k, s)) != PR_OK) return rc;
    }
    const bool out_dev = is_device_pointer(x_out);
    float* out = x_out;
    if (!out_dev) {
        if (!b->out_stage) PRK_CHECK(dev_alloc(g, (void**)&b->out_stage, (size_t)(g->n + kPad) * kBK * sizeof(float)));
        out = b->out_stage;
    }

    const bool dc = g->batch_dc > 0;                 // defect-correction form
    const bool bf16 = !dc && g->batch_bf16 > 0;      // plain BF16 phase
    if ((bf16 || dc) && !b->Y16[0]) {
        const size_t m16 = (size_t)(g->n + kPad) * kBK * sizeof(__nv_bfloat16);
        PRK_CHECK(dev_alloc(g, (void**)&b->Y16[0], m16));
        PRK_CHECK(dev_alloc(g, (void**)&b->Y16[1], m16));
    }
    if (dc && !b->R) {
        const size_t mat = (size_t)(g->n + kPad) * kBK * sizeof(float);
        PRK_CHECK(dev_alloc(g, (void**)&b->R, mat));
        PRK_CHECK(dev_alloc(g, (void**)&b->Dl, mat));
    }
    BatchState* hs = b->host_state;
    memset(hs, 0, sizeof(BatchState));
    hs->bf16 = bf16 ? 1 : 0;
    hs->bf16_switch = bf16 ? std::pow(10.0, -(double)g->batch_bf16) : 0.0;
    hs->d = (double)damping;
    hs->inv_n = 1.0 / (double)g->n;
    hs->tol = tol;
    hs->max_iter = max_iter;
    hs->k = k;
    hs->uniform = teleport ? 0 : 1;
    hs->tptr = b->tptr;
    hs->tcol = b->tcol;
    hs->tval = b->tval;
    hs->implicit_zero = (!dc && !bf16 && g->implicit_zero) ? 1 : 0;
    PRK_CHECK(cudaEventRecord(g->ev_start, s));
    PRK_CHECK(cudaMemcpyAsync(b->state, hs, sizeof(BatchState), cudaMemcpyHostToDevice, s));
    BatchArgs a = batch_args(g, b);
    int launches = 0;
    k_b_init<<<update_grid(g, b), kBlock, 0, s>>>(a, t_dev, g->order, b->X[0], b->Y[0],
                                                 bf16 ? b->Y16[0] : nullptr);
    ++launches;
    PRK_CHECK(cudaGetLastError());
    PRK_CHECK(cudaEventRecord(g->ev_loop0, s));
    if (dc) {
        // host-driven outer steps (one FP32 step + the correction sweeps
        // each), the done flag read after every step
        for (int32_t it = 0, src = 0; it < max_iter; ++it, src = 1 - src) {
            PRK_CHECK(g->idx64 ? enqueue_dc_step<int64_t>(g, b, a, src, g->batch_dc, s, &launches)
                               : enqueue_dc_step<int32_t>(g, b, a, src, g->batch_dc, s, &launches));
            PRK_CHECK(cudaMemcpyAsync(hs, b->state, sizeof(BatchState), cudaMemcpyDeviceToHost, s));
            PRK_CHECK(cudaStreamSynchronize(s));
            if (hs->done) break;
        }
    } else if (g->use_graph) {
        if (b->loop_exec && b->graph_bf16 != (bf16 ? 1 : 0)) drop_batch_graph(g);
        if (!b->loop_exec && (rc = build_batch_graph(g, b, bf16)) != PR_OK) return rc;
        PRK_CHECK(cudaGraphLaunch(b->loop_exec, s));
        ++launches;
    } else {
        // host-driven: iterations in chunks of 8 (the kernels return at once
        // when the state says done), then read the flag
        for (int32_t it = 0; it < max_iter;) {
            const int c = std::min<int32_t>(8, max_iter - it);
            for (int i = 0; i < c; ++i) {
                PRK_CHECK(enqueue_batch(g, b, a, (it + i) & 1, bf16, s));
                launches += (g->n_seg > 0 ? 3 : 2) + (bf16 ? (g->n_seg > 0 ? 2 : 1) : 0);
            }
            it += c;
            PRK_CHECK(cudaMemcpyAsync(hs, b->state, sizeof(BatchState), cudaMemcpyDeviceToHost, s));
            PRK_CHECK(cudaStreamSynchronize(s));
            if (hs->done) break;
        }
    }
    PRK_CHECK(cudaEventRecord(g->ev_loop1, s));
    k_b_zero_fill<<<update_grid(g, b), kBlock, 0, s>>>(a, b->X[0], b->X[1]);
    k_b_sum<<<update_grid(g, b), kBlock, 0, s>>>(a, b->X[0], b->X[1]);
    k_b_unpermute<<<small_grid(g), kBlock, 0, s>>>(a, b->X[0], b->X[1], g->rank, out, k);
    launches += 3;
    PRK_CHECK(cudaGetLastError());
    PRK_CHECK(cudaEventRecord(g->ev_stop, s));
    if (!out_dev) PRK_CHECK(cudaMemcpyAsync(x_out, out, nk * sizeof(float), cudaMemcpyDeviceToHost, s));
    PRK_CHECK(cudaMemcpyAsync(hs, b->state, sizeof(BatchState), cudaMemcpyDeviceToHost, s));
    PRK_CHECK(cudaStreamSynchronize(s));
    if (hs->error)
        return fail(PR_ERR_INVALID_ARG, "pr_solve_batched: a teleport column has a negative entry or a zero sum");
    float ms = 0.f, ms_loop = 0.f;
    PRK_CHECK(cudaEventElapsedTime(&ms, g->ev_start, g->ev_stop));
    PRK_CHECK(cudaEventElapsedTime(&ms_loop, g->ev_loop0, g->ev_loop1));
    double worst = 0.0;
    int conv = 1;
    for (int j = 0; j < k; ++j) {
        worst = std::max(worst, hs->resid[j]);
        if (!(hs->resid[j] < tol)) conv = 0;
        if (col_residual) col_residual[j] = hs->resid[j];
        if (col_iterations) col_iterations[j] = hs->col_iter[j];
    }
    if (info) {
        info->iterations = hs->iter;
        info->converged = conv;
        info->residual_l1 = worst;
        double sx = 0.0;
        for (int j = 0; j < k; ++j) sx += hs->sum_x[j];
        info->sum_x = sx;
        double dm = 0.0;
        for (int j = 0; j < k; ++j) dm += hs->D[j];
        info->dangling_mass = dm;
        info->edge_visits = (double)(hs->iter + hs->dc_sweeps) * (double)g->nnz;
        info->ms_device = ms;
        info->launches = launches;
        info->loop_edge_visits = info->edge_visits;
        info->ms_loop = ms_loop;
        info->frozen_rows = 0;
    }
    return conv ? PR_OK : PR_NOT_CONVERGED;
}
