// pr_edge.cu -- the edge-centric synchronous iteration (Barriers-Edge, Alg. 2),
// kept for comparison with the vertex-centric pull of pr_jacobi.cu.
//
// Alg. 2 splits an update into two phases separated by a barrier:
//   phase I   every source u with out-edges writes its contribution
//             y(u) = x(u) / outdeg(u) into the slot of each of its out-edges
//             in a per-edge array (contrib, one slot per edge, laid out in the
//             in-edge order of the targets);
//   phase II  every target v sums the contiguous slots of its in-edges and
//             updates x'(v), y'(v), with the dangling mass and L1 change
//             reduced as in the vertex form.
// On the GPU phase I is a push over the out-edge list (edge-parallel: the
// source of out-edge k and the in-edge slot it fills, both in out-edge order,
// so consecutive threads read the same source's contribution), and phase II a
// streaming row sum over the degree-binned tiles -- no irregular load, but
// one irregular 4-byte store per edge in phase I and 8 more bytes per edge
// (the slot written, then read back).  The out-edge list (sources and slots)
// is built on first use by a counting sort of the in-edges by source; the
// order of one source's out-edges does not matter (they all receive the same
// value), so the results are deterministic.
#include <algorithm>
#include <vector>

#include "pr_tile.cuh"

namespace prk {

// out-degree histogram of the binned sources
__global__ void k_edge_count(const int32_t* __restrict__ colidx, int64_t nnz, int64_t* __restrict__ counts) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride)
        atomicAdd((unsigned long long*)(counts + colidx[e]), 1ull);
}

// place every in-edge e = (u -> v) into u's out-edge range: its source and slot
__global__ void k_edge_fill(const int32_t* __restrict__ colidx, int64_t nnz, int32_t* __restrict__ cursor,
                            int32_t* __restrict__ out_src, int32_t* __restrict__ out_pos) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
        const int32_t u = colidx[e];
        const int32_t k = atomicAdd(cursor + u, 1);
        out_src[k] = u;
        out_pos[k] = (int32_t)e;
    }
}

// phase I: contrib[slot of out-edge k] = y(source of k)
__global__ void __launch_bounds__(kBlock) k_edge_scatter(IterArgs a, const float* __restrict__ y,
                                                         float* __restrict__ contrib) {
    if (block_state(a.state).done) return;
    const int64_t nnz = a.nnz;
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t k = (int64_t)blockIdx.x * kBlock + threadIdx.x; k < nnz; k += stride)
        contrib[ld_stream(a.out_pos + k)] = __ldg(y + ld_stream(a.out_src + k));
}

// phase II: row sums of contrib over the degree-binned tiles (light rows by
// groups of 2^kind lanes, one row per group at a time; rows of the heavy
// tiles a warp each; rows without in-edges a thread each; each lane's share
// summed with compensation, since a row's slots are read in a plain stride),
// the update, and the reductions, with the same last-block stopping test as
// k_rows.
template <typename IdxT, bool kUniform>
__global__ void __launch_bounds__(kBlock, 4) k_edge_rows(IterArgs a, const float* __restrict__ x_in,
                                                         const float* __restrict__ contrib,
                                                         float* __restrict__ x_out, float* __restrict__ y_out) {
    SolveState* st = a.state;
    const StateView sv = block_state(st);
    if (sv.done) return;
    const double d = sv.d;
    const double share = sv.D * sv.inv_n;
    RowCtx c{};
    c.d = (float)d;
    c.one_m_d = (float)(1.0 - d);
    c.d_share = (float)(d * share);
    c.base = (float)((1.0 - d) * sv.inv_n + d * share);
    Acc acc;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        const Tile tile = a.tiles[t];
        if (tile.kind >= 0) {
            const int lg = tile.kind, g = 1 << lg, rpp = kBlock >> lg;
            const int grp = tid >> lg, gl = tid & (g - 1);
            for (int64_t r0 = tile.row_begin; r0 < tile.row_end; r0 += rpp) {   // uniform per block
                const int64_t r = r0 + grp;
                const bool act = r < tile.row_end;
                KahanF ks;
                if (act) {
                    const int64_t b = row_at<IdxT>(a.rowptr, r), e = row_at<IdxT>(a.rowptr, r + 1);
                    for (int64_t k = b + gl; k < e; k += g) ks.add(ld_stream(contrib + k));
                }
                float s = (float)ks.value();
#pragma unroll
                for (int o = 1; o < 32; o <<= 1)
                    if (o < g) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (act && gl == 0) {
                    const float tv = kUniform ? 0.f : ld_stream(a.teleport + r);
                    row_update<kUniform, false>(r, s, ld_stream(x_in + r), ld_stream(a.inv_out + r), tv, c, x_out,
                                                y_out, acc);
                }
            }
        } else if (tile.kind == kTileHeavy) {
            for (int64_t r = tile.row_begin + warp; r < tile.row_end; r += kWarps) {
                const int64_t b = row_at<IdxT>(a.rowptr, r), e = row_at<IdxT>(a.rowptr, r + 1);
                KahanF ks;
                for (int64_t k = b + lane; k < e; k += 32) ks.add(ld_stream(contrib + k));
                const float s = warp_sum((float)ks.value());
                if (lane == 0) {
                    const float tv = kUniform ? 0.f : ld_stream(a.teleport + r);
                    row_update<kUniform, false>(r, s, ld_stream(x_in + r), ld_stream(a.inv_out + r), tv, c, x_out,
                                                y_out, acc);
                }
            }
        } else {
            process_zero_tile<kUniform, false>(tile, a.inv_out, a.teleport, x_in, x_out, y_out, c, acc, tid);
        }
    }
    double R, Dn;
    if (block_pair_to_grid(acc.resid(), acc.mass(), a.slots, &st->ticket, &R, &Dn) && threadIdx.x == 0) {
        st->resid = R;
        st->D = Dn;
        st->iter += 1;
        st->done = (R < st->tol) || (st->iter >= st->max_iter);
        st->ticket = 0;
    }
}

namespace {
int g_occ_edge = 0;
}  // namespace

pr_status ensure_edge(pr_graph* g, cudaStream_t s) {
    if (g->out_src) return PR_OK;
    if (g->idx64) return fail(PR_ERR_UNSUPPORTED, "the edge-centric variant needs 32-bit row offsets");
    const int64_t n = g->n, nnz = g->nnz;
    int64_t* counts = nullptr;
    int32_t* cursor = nullptr;
    struct Free {
        void* p[2];
        ~Free() {
            for (void* q : p)
                if (q) cudaFree(q);
        }
    } tmp{{nullptr, nullptr}};
    PRK_CHECK(cudaMalloc((void**)&counts, (size_t)(n + 1) * sizeof(int64_t)));
    tmp.p[0] = counts;
    PRK_CHECK(cudaMalloc((void**)&cursor, (size_t)(n + 1) * sizeof(int32_t)));
    tmp.p[1] = cursor;
    PRK_CHECK(dev_alloc(g, (void**)&g->out_src, (size_t)(nnz + kPad) * sizeof(int32_t)));
    PRK_CHECK(dev_alloc(g, (void**)&g->out_pos, (size_t)(nnz + kPad) * sizeof(int32_t)));
    PRK_CHECK(dev_alloc(g, (void**)&g->contrib, (size_t)(nnz + kPad) * sizeof(float)));
    PRK_CHECK(cudaMemsetAsync(counts, 0, (size_t)(n + 1) * sizeof(int64_t), s));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((nnz + kBlock - 1) / kBlock, (int64_t)g->sm_count * 8));
    if (nnz > 0) k_edge_count<<<grid, kBlock, 0, s>>>(g->colidx, nnz, counts);
    PRK_CHECK(cudaGetLastError());
    PRK_CHECK(scan_counts_i32(counts, n, cursor, s));   // cursor[u] = first out-edge of u (synchronises s)
    if (nnz > 0) k_edge_fill<<<grid, kBlock, 0, s>>>(g->colidx, nnz, cursor, g->out_src, g->out_pos);
    PRK_CHECK(cudaGetLastError());
    PRK_CHECK(cudaStreamSynchronize(s));
    if (g_occ_edge == 0) {
        int o = 0;
        PRK_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_edge_rows<int32_t, false>, kBlock, 0));
        g_occ_edge = std::max(1, o);
    }
    return PR_OK;
}

cudaError_t enqueue_edge_iteration(const pr_graph* g, const IterArgs& a, int src, bool uniform, cudaStream_t s,
                                   int* launches) {
    const int grid_e = (int)std::max<int64_t>(
        1, std::min<int64_t>((g->nnz + kBlock - 1) / kBlock, (int64_t)g->sm_count * 8));
    k_edge_scatter<<<grid_e, kBlock, 0, s>>>(a, g->y[src], g->contrib);
    int64_t blocks = (int64_t)g->sm_count * std::max(1, g_occ_edge);
    blocks = std::min<int64_t>(blocks, std::max<int64_t>(1, g->n_tiles));
    const int grid_r = (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)g->slot_capacity));
    if (uniform)
        k_edge_rows<int32_t, true><<<grid_r, kBlock, 0, s>>>(a, g->x[src], g->contrib, g->x[1 - src], g->y[1 - src]);
    else
        k_edge_rows<int32_t, false><<<grid_r, kBlock, 0, s>>>(a, g->x[src], g->contrib, g->x[1 - src], g->y[1 - src]);
    *launches += 2;
    return cudaGetLastError();
}

}  // namespace prk
