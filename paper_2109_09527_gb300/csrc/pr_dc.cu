// BF16 storage of the quotient vector in the synchronous solver, by defect
// correction (PR_OPT_SYNC_DC).
//
// The iteration of Eq. 1 is x <- F(x) = b + A x with A = d (P^T + 1 a^T / n)
// (a: the dangling indicator).  After an FP32 step x' = F(x) -- whose L1
// change is the solver's stopping test, so the returned vector is always an
// FP32 iterate -- the error e = x* - x solves e = r + A e with r = x' - x.
// M sweeps approximate it from delta_0 = r:
//     delta_{m+1} = r + d (P^T q_m + L_m / n),   q_m = bf16(delta_m / outdeg),
// gathering the 2-byte quotients q_m with FP32 sums, and x <- x + delta_M.
// L_m is the mass q_m does not pass on: delta_m(u) of a dangling row and
// delta_m(u) - outdeg(u) q_m(u) (the rounding loss) of the others, so every
// sweep conserves mass exactly as A does.  BF16 rounds the correction, not
// x, so its error shrinks with the residual and the FP32 steps still reach
// the FP32 tolerance.
//
// Kernels: k_dc_prep (r, delta_0's quotients and L_0), then per sweep the
// segment kernel over BF16 quotients (heavy rows) and k_dc_rows (light, heavy
// and empty rows, the tiles of the row kernel), then k_dc_apply (x + delta,
// its quotients y and dangling mass for the next FP32 step).

#include "pr_tile.cuh"

namespace prk {

cudaError_t launch_segments_q16(const pr_graph* g, const IterArgs& a, const __nv_bfloat16* q, cudaStream_t s,
                                int* launches);

namespace {

// BF16 quotient of a correction value; adds the mass it does not pass on.
__device__ __forceinline__ __nv_bfloat16 dc_quotient(float dv, float inv, KahanF& lost) {
    const __nv_bfloat16 q = __float2bfloat16_rn(dv * inv);
    if (inv == 0.f) lost.add(dv);
    else lost.add(dv - __bfloat162float(q) / inv);
    return q;
}

// The last block stores the grid total of `lost` as the next sweep's L.
__device__ __forceinline__ void store_lost(const IterArgs& a, const KahanF& lost) {
    SolveState* st = a.state;
    double L, unused;
    if (block_pair_to_grid(lost.value(), 0.0, a.slots, &st->ticket, &L, &unused) && threadIdx.x == 0) {
        st->Ldc = L;
        st->ticket = 0;
    }
}

// r = x' - x, delta_0 = r: its quotients and L_0.
__global__ void __launch_bounds__(kBlock) k_dc_prep(IterArgs a, const float* __restrict__ x_prev,
                                                    const float* __restrict__ x_new, float* __restrict__ r,
                                                    __nv_bfloat16* __restrict__ q) {
    if (block_state(a.state).done) return;
    KahanF lost;
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t v = (int64_t)blockIdx.x * kBlock + threadIdx.x; v < a.n; v += stride) {
        const float rv = x_new[v] - x_prev[v];
        r[v] = rv;
        q[v] = dc_quotient(rv, a.inv_out[v], lost);
    }
    store_lost(a, lost);
}

// One correction sweep over the row tiles: delta' = r + d (s + L/n), s the
// gathered quotients of the row's in-neighbours (segment partials for heavy
// rows, nothing for rows without in-edges).
template <typename IdxT>
__global__ void __launch_bounds__(kBlock) k_dc_rows(IterArgs a, const float* __restrict__ r,
                                                    const __nv_bfloat16* __restrict__ q_in,
                                                    float* __restrict__ delta, __nv_bfloat16* __restrict__ q_out) {
    SolveState* st = a.state;
    const StateView sv = block_state(st);
    if (sv.done) return;
    __shared__ double s_L;
    if (threadIdx.x == 0) s_L = st->Ldc;
    __syncthreads();
    const float d = (float)sv.d;
    const float dshare = (float)(sv.d * s_L * sv.inv_n);
    RowCtx c{};
    c.hot = a.hot;
    c.hot_n = 0;
    c.lane_mode = a.lane_mode;
    KahanF lost;
    const int tid = threadIdx.x;
    auto update = [&](int64_t v, float s) {
        const float dv = fmaf(d, s, r[v] + dshare);
        delta[v] = dv;
        q_out[v] = dc_quotient(dv, a.inv_out[v], lost);
    };
    for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        const Tile tile = a.tiles[t];
        if (tile.kind >= 0) {
            // light rows: as process_light_tile, two rows per lane group
            const int lg = light_lanes_log2(tile, c.lane_mode);
            const int g = 1 << lg;
            const int rpp = kBlock >> lg;
            const int grp = tid >> lg;
            const int gl = tid & (g - 1);
            for (int64_t r0 = tile.row_begin; r0 < tile.row_end; r0 += 2 * rpp) {
                int64_t rr[2], b[2], e[2];
                bool act[2];
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    rr[k] = r0 + k * rpp + grp;
                    act[k] = rr[k] < tile.row_end;
                    b[k] = act[k] ? row_at<IdxT>(a.rowptr, rr[k]) : 0;
                    e[k] = act[k] ? row_at<IdxT>(a.rowptr, rr[k] + 1) : 0;
                }
                float s[2] = {0.f, 0.f};
                const int32_t* colidx = a.colidx;
                gather_row_pair<false, 4, true>([&](int64_t p) { return ld_col<PRK_SYNC_COL_L1>(colidx + p); }, b[0] + gl, e[0],
                                          b[1] + gl, e[1], g, q_in, c, s[0], s[1]);
#pragma unroll
                for (int o = 1; o < 32; o <<= 1)
                    if (o < g) {
                        s[0] += __shfl_xor_sync(0xffffffffu, s[0], o);
                        s[1] += __shfl_xor_sync(0xffffffffu, s[1], o);
                    }
                if (gl == 0) {
#pragma unroll
                    for (int k = 0; k < 2; ++k)
                        if (act[k]) update(rr[k], s[k]);
                }
            }
        } else {
            for (int64_t v = tile.row_begin + tid; v < tile.row_end; v += kBlock) {
                float s = 0.f;
                if (tile.kind == kTileHeavy) {
                    const int32_t j1 = a.seg_ptr[v + 1];
                    for (int32_t j = a.seg_ptr[v]; j < j1; ++j) s += __ldcg(a.seg_sum + j);
                }
                update(v, s);
            }
        }
    }
    store_lost(a, lost);
}

// x <- x + delta_M, with the quotients y and the dangling mass D of the new x
// (the input of the next FP32 step).
__global__ void __launch_bounds__(kBlock) k_dc_apply(IterArgs a, const float* __restrict__ x_prev,
                                                     const float* __restrict__ delta, float* __restrict__ x_out,
                                                     float* __restrict__ y_out) {
    SolveState* st = a.state;
    if (block_state(st).done) return;
    KahanF dm;
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t v = (int64_t)blockIdx.x * kBlock + threadIdx.x; v < a.n; v += stride) {
        const float xn = x_prev[v] + delta[v];
        const float inv = a.inv_out[v];
        x_out[v] = xn;
        y_out[v] = xn * inv;
        if (inv == 0.f) dm.add(xn);
    }
    double D, unused;
    if (block_pair_to_grid(dm.value(), 0.0, a.slots, &st->ticket, &D, &unused) && threadIdx.x == 0) {
        st->D = D;
        st->ticket = 0;
    }
}

int dc_row_grid(const pr_graph* g) {
    const int64_t blocks = std::min<int64_t>((int64_t)g->sm_count * 4, std::max<int64_t>(1, g->n_tiles));
    return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)g->slot_capacity));
}

}  // namespace

pr_status ensure_sync_dc(pr_graph* g) {
    if (g->dc_r) return PR_OK;
    const size_t vec = (size_t)(g->n + kPad) * sizeof(float);
    const size_t half = (size_t)(g->n + kPad) * sizeof(__nv_bfloat16);
    PRK_CHECK(dev_alloc(g, (void**)&g->dc_r, vec));
    PRK_CHECK(dev_alloc(g, (void**)&g->dc_delta, vec));
    PRK_CHECK(dev_alloc(g, &g->dc_q[0], half));
    PRK_CHECK(dev_alloc(g, &g->dc_q[1], half));
    return PR_OK;
}

cudaError_t enqueue_sync_dc(const pr_graph* g, const IterArgs& a, int src, int sweeps, cudaStream_t s,
                            int* launches) {
    __nv_bfloat16* q[2] = {(__nv_bfloat16*)g->dc_q[0], (__nv_bfloat16*)g->dc_q[1]};
    const int vg = small_grid(g);
    k_dc_prep<<<vg, kBlock, 0, s>>>(a, g->x[src], g->x[1 - src], g->dc_r, q[0]);
    ++*launches;
    const int rg = dc_row_grid(g);
    for (int m = 0; m < sweeps; ++m) {
        cudaError_t e = launch_segments_q16(g, a, q[m & 1], s, launches);
        if (e != cudaSuccess) return e;
        if (g->idx64) k_dc_rows<int64_t><<<rg, kBlock, 0, s>>>(a, g->dc_r, q[m & 1], g->dc_delta, q[(m + 1) & 1]);
        else k_dc_rows<int32_t><<<rg, kBlock, 0, s>>>(a, g->dc_r, q[m & 1], g->dc_delta, q[(m + 1) & 1]);
        ++*launches;
    }
    k_dc_apply<<<vg, kBlock, 0, s>>>(a, g->x[src], g->dc_delta, g->x[1 - src], g->y[1 - src]);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace prk
