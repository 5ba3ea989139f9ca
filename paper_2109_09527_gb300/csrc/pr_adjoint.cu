// pr_adjoint.cu -- weighted PageRank and its adjoint (gradients of a loss on
// the ranks with respect to the teleport vector and the edge weights).
//
// Weighted graph: edge e = (u, v) has weight w(e) > 0 and transition
// probability P(u, v) = w(e) / W(u), W(u) = sum of u's out-weights; a vertex
// without out-edges is dangling and its rank is spread uniformly.  The fixed
// point x of Eq. 1 on P solves
//
//   M x = (1-d) t,       M = I - d P^T - (d/n) 1 a^T      (a = dangling indicator)
//
// and for a loss L(x) with gradient c = dL/dx, implicit differentiation gives
//
//   M^T lambda = c,      dL/dt = (1-d) lambda,
//   dL/dw(e) = d x(u) / W(u) * (lambda(v) - mu(u)),   mu(u) = sum_v' P(u,v') lambda(v'),
//
// (the second line from dM = -d dP^T and the quotient rule on w(e)/W(u)).  The
// transposed system is solved by the same synchronous iteration run backwards
// along the edges:  lambda'(u) = c(u) + d (mu(u) + a(u) sum(lambda)/n),  a
// gather over u's OUT-edges -- so the graph keeps both an in-edge CSR (the
// forward pull) and an out-edge CSR (the adjoint pull, i.e. the forward
// push), each with its edges' transition probabilities.
//
// Vertices stay in the caller's order (no relabelling): rows with 32 or more
// edges are gathered a warp each, the others by groups of 8 lanes, from a row
// list sorted into those two classes.  The out-edge CSR is built on the host by a stable counting
// sort of the in-edges by source, so each out-row lists its edges in in-edge
// order and every sum has a fixed order (bitwise reproducible results).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "pr_tile.cuh"

namespace prk {

struct WState {
    double d;
    double tol;             // forward: L1 change; adjoint: L1 change / ||c||_1
    double inv_n;
    double t_sum;
    double D;               // forward: dangling mass of the current x
    double L;               // adjoint: sum(lambda) of the current lambda
    double c_norm;          // adjoint: ||c||_1
    double resid;
    double sum_x;
    double scale;
    int32_t max_iter;
    int32_t iter;
    int32_t done;
    uint32_t ticket;
    uint32_t error;
    int32_t pad;
};

// Ends of the row classes in a class order (rows listed class by class, in
// caller order within a class): [0, giant) rows with >= kWGiantEdges edges,
// [giant, heavy) those with >= 32, [heavy, mid) 8..31 edges, [mid, small)
// 1..7 edges, [small, n) rows without edges.
struct WClasses {
    int64_t giant;
    int64_t heavy;
    int64_t mid;
    int64_t small;
};

struct WArgs {
    int64_t n;
    int64_t nnz;
    const int64_t* rowptr;      // in-edge CSR (rows = targets)
    const int32_t* colidx;
    const float* in_p;          // P(u, v) of each in-edge
    const int64_t* out_rowptr;  // out-edge CSR (rows = sources)
    const int32_t* out_dst;
    const float* out_p;         // P(u, v) of each out-edge
    const float* inv_w;         // 1/W(u), 0 for dangling u
    const int32_t* in_order;    // rows by in-degree class (WClasses)
    WClasses in_cls;
    const int32_t* out_order;   // the same classes by out-degree
    WClasses out_cls;
    WState* state;
    double* slots;
};

// Rows are visited class by class: rows with at least kWGiantEdges edges a
// block each (a power-law hub has tens of thousands: one warp walking it
// would set the length of the whole launch), rows with at least 32 edges a
// warp each, rows of 8..31 edges by groups of 8 lanes and rows of 1..7 by
// groups of 4 (four or eight rows per warp at a time), rows without edges a
// thread each.  The row body gather(row, lane_in_group, group_size) returns
// this lane's share of the row's sum; the group's total reaches the group's
// first thread, where `epilogue(row, sum)` runs (with sum 0 for a row without
// edges).  With PRK_W_CLASSES = 0 the set-up lists every row below 32 edges in
// one class of 8-lane groups.
#ifndef PRK_W_CLASSES
#define PRK_W_CLASSES 1
#endif
constexpr int kWLightLanes = 8;
constexpr int kWSmallLanes = 4;
constexpr int kWSmallEdges = 8;
#ifndef PRK_W_GIANT_EDGES
#define PRK_W_GIANT_EDGES 2048
#endif
constexpr int64_t kWGiantEdges = PRK_W_GIANT_EDGES;

// Rows [begin, end) of the order by groups of G lanes; the loop bound is
// uniform per warp, so every lane reaches the shuffles.
template <int G, typename Gather, typename Epilogue>
__device__ __forceinline__ void w_groups(const int32_t* order, int64_t begin, int64_t end, int64_t warp,
                                         int64_t nwarp, int lane, Gather& gather, Epilogue& epilogue) {
    constexpr int per = 32 / G;
    const int sub = lane / G, sl = lane % G;
    for (int64_t i0 = begin + warp * per; i0 < end; i0 += nwarp * per) {
        const int64_t i = i0 + sub;
        const bool act = i < end;
        const int32_t r = act ? order[i] : 0;
        float s = act ? gather(r, sl, G) : 0.f;
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (act && sl == 0) epilogue(r, s);
    }
}

template <typename Gather, typename Epilogue>
__device__ __forceinline__ void w_rows(const int32_t* order, int64_t n, const WClasses& cls, Gather gather,
                                       Epilogue epilogue) {
    const int lane = threadIdx.x & 31;
    for (int64_t i = blockIdx.x; i < cls.giant; i += gridDim.x) {   // uniform per block
        const int32_t r = order[i];
        const float s = block_sum(gather(r, (int)threadIdx.x, (int)blockDim.x));
        if (threadIdx.x == 0) epilogue(r, s);
    }
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = cls.giant + warp; i < cls.heavy; i += nwarp) {
        const int32_t r = order[i];
        float s = warp_sum(gather(r, lane, 32));
        if (lane == 0) epilogue(r, s);
    }
    w_groups<kWLightLanes>(order, cls.heavy, cls.mid, warp, nwarp, lane, gather, epilogue);
    w_groups<kWSmallLanes>(order, cls.mid, cls.small, warp, nwarp, lane, gather, epilogue);
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = cls.small + tid; i < n; i += nthreads) epilogue(order[i], 0.f);
}

// sum over the edges k of row r of p[k] * vec[idx[k]], this lane's share
// (edges l, l+g, ...), accumulated in edge order with one FMA per edge; the
// loads of four edges are issued before their products are added.
__device__ __forceinline__ float w_gather(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ idx,
                                          const float* __restrict__ p, const float* __restrict__ vec, int32_t r,
                                          int l, int g) {
    const int64_t e = __ldg(rowptr + r + 1);
    int64_t k = __ldg(rowptr + r) + l;
    float s = 0.f;
    for (; k + 3 * g < e; k += 4 * g) {
        const int32_t c0 = __ldg(idx + k), c1 = __ldg(idx + k + g), c2 = __ldg(idx + k + 2 * g),
                      c3 = __ldg(idx + k + 3 * g);
        const float p0 = __ldg(p + k), p1 = __ldg(p + k + g), p2 = __ldg(p + k + 2 * g), p3 = __ldg(p + k + 3 * g);
        const float v0 = __ldg(vec + c0), v1 = __ldg(vec + c1), v2 = __ldg(vec + c2), v3 = __ldg(vec + c3);
        s = fmaf(p0, v0, s);
        s = fmaf(p1, v1, s);
        s = fmaf(p2, v2, s);
        s = fmaf(p3, v3, s);
    }
    for (; k < e; k += g) s = fmaf(__ldg(p + k), __ldg(vec + __ldg(idx + k)), s);
    return s;
}

// ------------------------------------------------------------------ kernels --

// x' = (1-d) t + d (sum_e P(e) x(u_e) + D/n), with D' and the L1 change.
__global__ void __launch_bounds__(kBlock) k_w_forward(WArgs a, const float* __restrict__ t, const float* __restrict__ x,
                                                      float* __restrict__ xo) {
    WState* st = a.state;
    __shared__ double s_d, s_D, s_inv_n;
    __shared__ int32_t s_done;
    if (threadIdx.x == 0) {
        s_done = *(volatile int32_t*)&st->done;
        s_d = st->d;
        s_D = st->D;
        s_inv_n = st->inv_n;
    }
    __syncthreads();
    if (s_done) return;
    const float d = (float)s_d;
    const float share = (float)(s_D * s_inv_n);
    const float tu = (float)s_inv_n;
    Acc acc;
    w_rows(a.in_order, a.n, a.in_cls,
           [&](int32_t v, int l, int g) { return w_gather(a.rowptr, a.colidx, a.in_p, x, v, l, g); },
           [&](int32_t v, float s) {
               const float tv = t ? t[v] : tu;
               const float xn = fmaf(1.f - d, tv, d * (s + share));
               xo[v] = xn;
               acc.add_r(fabsf(xn - x[v]));
               if (a.inv_w[v] == 0.f) acc.kahan(xn);
           });
    double R, Dn;
    if (block_pair_to_grid(acc.resid(), acc.mass(), a.slots, &st->ticket, &R, &Dn) && threadIdx.x == 0) {
        st->resid = R;
        st->D = Dn;
        st->iter += 1;
        st->done = (R < st->tol) || (st->iter >= st->max_iter);
        st->ticket = 0;
    }
}

// lambda'(u) = c(u) + d (mu(u) + a(u) L/n), mu(u) = sum over u's out-edges of
// P(e) lambda(v_e); with sum(lambda') and the L1 change.  With final != 0 it
// only stores mu of the current lambda (no update, no state change).
__global__ void __launch_bounds__(kBlock) k_w_adjoint(WArgs a, const float* __restrict__ c, const float* __restrict__ lam,
                                                      float* __restrict__ lo, float* __restrict__ mu, int final) {
    WState* st = a.state;
    __shared__ double s_d, s_L, s_inv_n;
    __shared__ int32_t s_done;
    if (threadIdx.x == 0) {
        s_done = *(volatile int32_t*)&st->done;
        s_d = st->d;
        s_L = st->L;
        s_inv_n = st->inv_n;
    }
    __syncthreads();
    if (s_done && !final) return;
    const float d = (float)s_d;
    const float lshare = (float)(s_L * s_inv_n);
    double r = 0.0, L = 0.0;
    w_rows(a.out_order, a.n, a.out_cls,
           [&](int32_t u, int l, int g) { return w_gather(a.out_rowptr, a.out_dst, a.out_p, lam, u, l, g); },
           [&](int32_t u, float m) {
               if (final) {
                   mu[u] = m;
               } else {
                   const float ln = c[u] + d * (m + (a.inv_w[u] == 0.f ? lshare : 0.f));
                   lo[u] = ln;
                   r += fabs((double)ln - (double)lam[u]);
                   L += (double)ln;
               }
           });
    if (final) return;
    double R, Ln;
    if (block_pair_to_grid(r, L, a.slots, &st->ticket, &R, &Ln) && threadIdx.x == 0) {
        st->resid = R;
        st->L = Ln;
        st->iter += 1;
        st->done = (R < st->tol * st->c_norm) || (st->iter >= st->max_iter);
        st->ticket = 0;
    }
}

// dL/dw for every in-edge e = (u, v): d x(u) / W(u) * (lambda(v) - mu(u)); and
// dL/dt = (1-d) lambda.
__global__ void __launch_bounds__(kBlock) k_w_grads(WArgs a, const float* __restrict__ x, const float* __restrict__ lam,
                                                    const float* __restrict__ mu, float* __restrict__ grad_t,
                                                    float* __restrict__ grad_w) {
    const float d = (float)a.state->d;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < a.n; u += stride)
        if (grad_t) grad_t[u] = (1.f - d) * lam[u];
    if (!grad_w) return;
    w_rows(a.in_order, a.n, a.in_cls,
           [&](int32_t v, int l, int g) {
               const float lv = lam[v];
               for (int64_t e = a.rowptr[v] + l; e < a.rowptr[v + 1]; e += g) {
                   const int32_t u = a.colidx[e];
                   grad_w[e] = d * x[u] * a.inv_w[u] * (lv - mu[u]);
               }
               return 0.f;
           },
           [&](int32_t, float) {});
}

// Sums for the forward init (D of x0, sum t) or the adjoint init (sum c, ||c||_1).
__global__ void __launch_bounds__(kBlock) k_w_init(WArgs a, const float* __restrict__ t, float* __restrict__ x,
                                                   const float* __restrict__ c, float* __restrict__ lam) {
    WState* st = a.state;
    const float tu = (float)st->inv_n;
    double s1 = 0.0, s2 = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += stride) {
        if (c) {
            const float cv = c[v];
            lam[v] = cv;
            s1 += (double)cv;
            s2 += fabs((double)cv);
        } else {
            const float tv = t ? t[v] : tu;
            if (!(tv >= 0.f)) atomicOr(&st->error, 1u);
            x[v] = tv;
            if (a.inv_w[v] == 0.f) s1 += (double)tv;
            s2 += (double)tv;
        }
    }
    double A, B;
    if (block_pair_to_grid(s1, s2, a.slots, &st->ticket, &A, &B) && threadIdx.x == 0) {
        if (c) {
            st->L = A;
            st->c_norm = B;
        } else {
            st->D = A;
            st->t_sum = B;
            if (!(B > 0.0)) st->error |= 1u;
        }
        st->iter = 0;
        st->done = 0;
        st->resid = INFINITY;
        st->ticket = 0;
    }
}

__global__ void __launch_bounds__(kBlock) k_w_sum(WArgs a, const float* __restrict__ x) {
    WState* st = a.state;
    double s = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += stride) s += (double)x[v];
    double S, unused;
    if (block_pair_to_grid(s, 0.0, a.slots, &st->ticket, &S, &unused) && threadIdx.x == 0) {
        st->sum_x = S;
        st->scale = S > 0.0 ? st->t_sum / S : 1.0;
        st->ticket = 0;
    }
}

__global__ void k_w_scale(WArgs a, const float* __restrict__ x, float* __restrict__ out) {
    const float sc = (float)a.state->scale;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += stride) out[v] = x[v] * sc;
}

// P of every edge from the weights: W(u) in FP64 (atomics; the sum of FP32
// weights within a 2^29 range of one another and fewer than 2^24 of them per
// vertex is exact in FP64, hence independent of the order), then 1/W, the
// in-edge and out-edge probabilities.  A non-positive weight sets *bad.
__global__ void k_w_outweight(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colidx, int64_t n,
                              const float* __restrict__ w, double* __restrict__ W, unsigned int* bad) {
    const int64_t nnz = rowptr[n];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
        const float we = w[e];
        if (!(we > 0.f) || !isfinite(we)) atomicOr(bad, 1u);
        atomicAdd(W + colidx[e], (double)we);
    }
}

__global__ void k_w_probs(int64_t n, int64_t nnz, const int32_t* __restrict__ colidx, const float* __restrict__ w,
                          const double* __restrict__ W, const int64_t* __restrict__ out_eid, float* __restrict__ inv_w,
                          float* __restrict__ in_p, float* __restrict__ out_p) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride)
        inv_w[u] = W[u] > 0.0 ? (float)(1.0 / W[u]) : 0.f;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
        in_p[e] = (float)((double)w[e] / W[colidx[e]]);
        const int64_t ie = out_eid[e];
        out_p[e] = (float)((double)w[ie] / W[colidx[ie]]);
    }
}

}  // namespace prk

// -------------------------------------------------------------------- host --

struct pr_wgraph {
    int device = 0;
    int sm_count = 0;
    int64_t n = 0;
    int64_t nnz = 0;
    int64_t* rowptr = nullptr;
    int32_t* colidx = nullptr;
    float* w = nullptr;
    float* in_p = nullptr;
    int64_t* out_rowptr = nullptr;
    int32_t* out_dst = nullptr;
    int64_t* out_eid = nullptr;
    float* out_p = nullptr;
    float* inv_w = nullptr;
    double* W = nullptr;
    int32_t* in_order = nullptr;
    int32_t* out_order = nullptr;
    prk::WClasses in_cls{};
    prk::WClasses out_cls{};
    float* vec[4] = {nullptr, nullptr, nullptr, nullptr};   // iterate buffers, mu
    float* stage = nullptr;                                 // host inputs / outputs
    prk::WState* state = nullptr;
    prk::WState* host_state = nullptr;
    double* slots = nullptr;
    unsigned int* bad = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

using namespace prk;

namespace {

// Blocks per SM of every weighted kernel (256 threads, 40 registers: six fit);
// the reduction slots are allocated for exactly this grid.
constexpr int kWBlocksPerSm = 6;

int w_grid(const pr_wgraph* g) { return g->sm_count * kWBlocksPerSm; }

WArgs w_args(const pr_wgraph* g) {
    WArgs a{};
    a.n = g->n;
    a.nnz = g->nnz;
    a.rowptr = g->rowptr;
    a.colidx = g->colidx;
    a.in_p = g->in_p;
    a.out_rowptr = g->out_rowptr;
    a.out_dst = g->out_dst;
    a.out_p = g->out_p;
    a.inv_w = g->inv_w;
    a.in_order = g->in_order;
    a.in_cls = g->in_cls;
    a.out_order = g->out_order;
    a.out_cls = g->out_cls;
    a.state = g->state;
    a.slots = g->slots;
    return a;
}

// A caller vector: device pointers in place, host memory staged in slot k.
pr_status w_input(pr_wgraph* g, const float* src, int k, cudaStream_t s, const float** out) {
    *out = nullptr;
    if (!src) return PR_OK;
    if (is_device_pointer(src)) {
        *out = src;
        return PR_OK;
    }
    float* dst = g->stage + (size_t)k * (size_t)(g->n + kPad);
    PRK_CHECK(cudaMemcpyAsync(dst, src, (size_t)g->n * sizeof(float), cudaMemcpyHostToDevice, s));
    *out = dst;
    return PR_OK;
}

pr_status w_set_weights(pr_wgraph* g, const float* weights, cudaStream_t s) {
    if (is_device_pointer(weights)) {
        PRK_CHECK(cudaMemcpyAsync(g->w, weights, (size_t)g->nnz * sizeof(float), cudaMemcpyDeviceToDevice, s));
    } else {
        PRK_CHECK(cudaMemcpyAsync(g->w, weights, (size_t)g->nnz * sizeof(float), cudaMemcpyHostToDevice, s));
    }
    PRK_CHECK(cudaMemsetAsync(g->W, 0, (size_t)g->n * sizeof(double), s));
    PRK_CHECK(cudaMemsetAsync(g->bad, 0, sizeof(unsigned int), s));
    const int grid = w_grid(g);
    if (g->nnz > 0) k_w_outweight<<<grid, kBlock, 0, s>>>(g->rowptr, g->colidx, g->n, g->w, g->W, g->bad);
    k_w_probs<<<grid, kBlock, 0, s>>>(g->n, g->nnz, g->colidx, g->w, g->W, g->out_eid, g->inv_w, g->in_p, g->out_p);
    PRK_CHECK(cudaGetLastError());
    unsigned int bad = 0;
    PRK_CHECK(cudaMemcpyAsync(&bad, g->bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    PRK_CHECK(cudaStreamSynchronize(s));
    if (bad) return fail(PR_ERR_INVALID_ARG, "edge weights must be positive and finite");
    return PR_OK;
}

// Host-driven loop: chunks of 8 kernels, then the done flag.
template <typename Enqueue>
pr_status w_loop(pr_wgraph* g, int32_t max_iter, cudaStream_t s, int* launches, Enqueue enqueue) {
    for (int32_t it = 0; it < max_iter;) {
        const int c = std::min<int32_t>(8, max_iter - it);
        for (int i = 0; i < c; ++i) {
            enqueue(it + i);
            ++*launches;
        }
        it += c;
        PRK_CHECK(cudaGetLastError());
        PRK_CHECK(cudaMemcpyAsync(g->host_state, g->state, sizeof(WState), cudaMemcpyDeviceToHost, s));
        PRK_CHECK(cudaStreamSynchronize(s));
        if (g->host_state->done) break;
    }
    return PR_OK;
}

}  // namespace

extern "C" pr_status pr_destroy_wgraph(pr_wgraph* g) {
    if (!g) return PR_OK;
    void* dev[] = {g->rowptr, g->colidx, g->w, g->in_p, g->out_rowptr, g->out_dst, g->out_eid, g->out_p,
                   g->inv_w, g->W, g->vec[0], g->vec[1], g->vec[2], g->vec[3], g->stage, g->state, g->slots,
                   g->bad, g->in_order, g->out_order};
    for (void* p : dev)
        if (p) cudaFree(p);
    if (g->host_state) cudaFreeHost(g->host_state);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    delete g;
    return PR_OK;
}

extern "C" pr_status pr_create_wgraph(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                                      const float* weights, void* stream, pr_wgraph** out) {
    if (!out) return fail(PR_ERR_INVALID_ARG, "pr_create_wgraph: out is NULL");
    *out = nullptr;
    if (n < 1 || n > 0x7fffffffLL) return fail(PR_ERR_INVALID_ARG, "pr_create_wgraph: n must be in [1, 2^31-1]");
    if (nnz < 0 || nnz > 0x7fffffffLL) return fail(PR_ERR_INVALID_ARG, "pr_create_wgraph: nnz must be in [0, 2^31-1]");
    if (!rowptr || (nnz > 0 && (!colidx || !weights)))
        return fail(PR_ERR_INVALID_ARG, "pr_create_wgraph: NULL rowptr, colidx or weights");
    cudaStream_t s = (cudaStream_t)stream;
    // the CSR on the host: validation and the stable out-edge sort
    std::vector<int64_t> rp((size_t)n + 1);
    std::vector<int32_t> ci((size_t)std::max<int64_t>(nnz, 1));
    cudaError_t e = cudaMemcpy(rp.data(), rowptr, rp.size() * sizeof(int64_t), cudaMemcpyDefault);
    if (e == cudaSuccess && nnz > 0) e = cudaMemcpy(ci.data(), colidx, (size_t)nnz * sizeof(int32_t), cudaMemcpyDefault);
    if (e != cudaSuccess) return cuda_fail(e, "pr_create_wgraph: copy of the CSR");
    if (rp[0] != 0 || rp[n] != nnz) return fail(PR_ERR_INVALID_GRAPH, "pr_create_wgraph: rowptr[0] != 0 or rowptr[n] != nnz");
    for (int64_t v = 0; v < n; ++v)
        if (rp[v + 1] < rp[v]) return fail(PR_ERR_INVALID_GRAPH, "pr_create_wgraph: rowptr decreases");
    std::vector<int64_t> orp((size_t)n + 1, 0);
    for (int64_t k = 0; k < nnz; ++k) {
        if (ci[k] < 0 || ci[k] >= n) return fail(PR_ERR_INVALID_GRAPH, "pr_create_wgraph: colidx out of range");
        ++orp[(size_t)ci[k] + 1];
    }
    for (int64_t u = 0; u < n; ++u) orp[u + 1] += orp[u];
    std::vector<int32_t> odst((size_t)std::max<int64_t>(nnz, 1));
    std::vector<int64_t> oeid((size_t)std::max<int64_t>(nnz, 1));
    {
        std::vector<int64_t> cur(orp.begin(), orp.end() - 1);
        for (int64_t v = 0; v < n; ++v)
            for (int64_t k = rp[v]; k < rp[v + 1]; ++k) {
                const int64_t slot = cur[ci[k]]++;
                odst[slot] = (int32_t)v;
                oeid[slot] = k;
            }
    }
    // the row classes of w_rows, each in caller order
    auto split = [&](const std::vector<int64_t>& ptr, std::vector<int32_t>& order, WClasses& cls) {
        order.clear();
        order.reserve((size_t)n);
        auto take = [&](int64_t lo, int64_t hi) {   // rows with lo <= edges < hi
            for (int64_t v = 0; v < n; ++v) {
                const int64_t dv = ptr[v + 1] - ptr[v];
                if (dv >= lo && dv < hi) order.push_back((int32_t)v);
            }
            return (int64_t)order.size();
        };
        cls.giant = take(kWGiantEdges, INT64_MAX);
        cls.heavy = take(32, kWGiantEdges);
        if (PRK_W_CLASSES) {
            cls.mid = take(kWSmallEdges, 32);
            cls.small = take(1, kWSmallEdges);
            take(0, 1);
        } else {
            cls.mid = cls.small = take(0, 32);
        }
    };
    std::vector<int32_t> in_order, out_order;
    WClasses in_cls{}, out_cls{};
    split(rp, in_order, in_cls);
    split(orp, out_order, out_cls);
    pr_wgraph* g = new (std::nothrow) pr_wgraph();
    if (!g) return fail(PR_ERR_OOM, "pr_create_wgraph: host allocation failed");
    g->in_cls = in_cls;
    g->out_cls = out_cls;
    g->n = n;
    g->nnz = nnz;
    pr_status rc = PR_OK;
    do {
        if ((e = cudaGetDevice(&g->device)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device)) != cudaSuccess) {
            rc = cuda_fail(e, "pr_create_wgraph: device query");
            break;
        }
        const size_t E = (size_t)std::max<int64_t>(nnz, 1) + kPad, N = (size_t)n + kPad;
        bool ok = cudaMalloc((void**)&g->rowptr, N * sizeof(int64_t)) == cudaSuccess &&
                  cudaMalloc((void**)&g->colidx, E * sizeof(int32_t)) == cudaSuccess &&
                  cudaMalloc((void**)&g->w, E * sizeof(float)) == cudaSuccess &&
                  cudaMalloc((void**)&g->in_p, E * sizeof(float)) == cudaSuccess &&
                  cudaMalloc((void**)&g->out_rowptr, N * sizeof(int64_t)) == cudaSuccess &&
                  cudaMalloc((void**)&g->out_dst, E * sizeof(int32_t)) == cudaSuccess &&
                  cudaMalloc((void**)&g->out_eid, E * sizeof(int64_t)) == cudaSuccess &&
                  cudaMalloc((void**)&g->out_p, E * sizeof(float)) == cudaSuccess &&
                  cudaMalloc((void**)&g->inv_w, N * sizeof(float)) == cudaSuccess &&
                  cudaMalloc((void**)&g->W, N * sizeof(double)) == cudaSuccess &&
                  cudaMalloc((void**)&g->stage, 3 * N * sizeof(float)) == cudaSuccess &&
                  cudaMalloc((void**)&g->state, sizeof(WState)) == cudaSuccess &&
                  cudaMalloc((void**)&g->slots, (size_t)w_grid(g) * 2 * sizeof(double)) == cudaSuccess &&
                  cudaMalloc((void**)&g->bad, sizeof(unsigned int)) == cudaSuccess &&
                  cudaMalloc((void**)&g->in_order, N * sizeof(int32_t)) == cudaSuccess &&
                  cudaMalloc((void**)&g->out_order, N * sizeof(int32_t)) == cudaSuccess &&
                  cudaMallocHost((void**)&g->host_state, sizeof(WState)) == cudaSuccess &&
                  cudaEventCreate(&g->ev0) == cudaSuccess && cudaEventCreate(&g->ev1) == cudaSuccess;
        for (int i = 0; ok && i < 4; ++i) ok = cudaMalloc((void**)&g->vec[i], N * sizeof(float)) == cudaSuccess;
        if (!ok) {
            rc = fail(PR_ERR_OOM, "pr_create_wgraph: device allocation failed");
            break;
        }
        e = cudaMemcpyAsync(g->rowptr, rp.data(), rp.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g->colidx, ci.data(), ci.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g->out_rowptr, orp.data(), orp.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g->out_dst, odst.data(), odst.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g->out_eid, oeid.data(), oeid.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g->in_order, in_order.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g->out_order, out_order.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "pr_create_wgraph: upload");
            break;
        }
        rc = nnz > 0 ? w_set_weights(g, weights, s) : PR_OK;
        if (nnz == 0) {
            if ((e = cudaMemsetAsync(g->inv_w, 0, (size_t)n * sizeof(float), s)) != cudaSuccess ||
                (e = cudaStreamSynchronize(s)) != cudaSuccess)
                rc = cuda_fail(e, "pr_create_wgraph: init");
        }
    } while (0);
    if (rc != PR_OK) {
        pr_destroy_wgraph(g);
        return rc;
    }
    *out = g;
    return PR_OK;
}

extern "C" pr_status pr_wgraph_set_weights(pr_wgraph* g, const float* weights, void* stream) {
    if (!g || (g->nnz > 0 && !weights)) return fail(PR_ERR_INVALID_ARG, "pr_wgraph_set_weights: NULL argument");
    if (g->nnz == 0) return PR_OK;
    return w_set_weights(g, weights, (cudaStream_t)stream);
}

extern "C" pr_status pr_solve_weighted(pr_wgraph* g, float damping, double tol, int32_t max_iter,
                                       const float* teleport, float* x_out, pr_info* info, void* stream) {
    if (!g || !x_out) return fail(PR_ERR_INVALID_ARG, "pr_solve_weighted: NULL graph or x_out");
    if (!(damping >= 0.0f && damping < 1.0f)) return fail(PR_ERR_INVALID_ARG, "damping must be in [0, 1)");
    if (!(tol > 0.0) || !std::isfinite(tol)) return fail(PR_ERR_INVALID_ARG, "tol must be a positive finite number");
    if (max_iter < 1) return fail(PR_ERR_INVALID_ARG, "max_iter must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    const float* t = nullptr;
    pr_status rc = w_input(g, teleport, 0, s, &t);
    if (rc != PR_OK) return rc;
    WState* hs = g->host_state;
    memset(hs, 0, sizeof(WState));
    hs->d = damping;
    hs->tol = tol;
    hs->inv_n = 1.0 / (double)g->n;
    hs->max_iter = max_iter;
    PRK_CHECK(cudaEventRecord(g->ev0, s));
    PRK_CHECK(cudaMemcpyAsync(g->state, hs, sizeof(WState), cudaMemcpyHostToDevice, s));
    WArgs a = w_args(g);
    int launches = 0;
    k_w_init<<<w_grid(g), kBlock, 0, s>>>(a, t, g->vec[0], nullptr, nullptr);
    ++launches;
    float* xv[2] = {g->vec[0], g->vec[1]};
    rc = w_loop(g, max_iter, s, &launches, [&](int it) {
        k_w_forward<<<w_grid(g), kBlock, 0, s>>>(a, t, xv[it & 1], xv[1 - (it & 1)]);
    });
    if (rc != PR_OK) return rc;
    const bool out_dev = is_device_pointer(x_out);
    float* out = out_dev ? x_out : g->stage + (size_t)2 * (size_t)(g->n + kPad);
    const float* xfin = xv[hs->iter & 1];
    k_w_sum<<<w_grid(g), kBlock, 0, s>>>(a, xfin);
    k_w_scale<<<w_grid(g), kBlock, 0, s>>>(a, xfin, out);
    launches += 2;
    PRK_CHECK(cudaGetLastError());
    PRK_CHECK(cudaEventRecord(g->ev1, s));
    if (!out_dev) PRK_CHECK(cudaMemcpyAsync(x_out, out, (size_t)g->n * sizeof(float), cudaMemcpyDeviceToHost, s));
    PRK_CHECK(cudaMemcpyAsync(hs, g->state, sizeof(WState), cudaMemcpyDeviceToHost, s));
    PRK_CHECK(cudaStreamSynchronize(s));
    if (hs->error) return fail(PR_ERR_INVALID_ARG, "pr_solve_weighted: teleport has a negative entry or a zero sum");
    float ms = 0.f;
    PRK_CHECK(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
    const bool conv = hs->resid < tol;
    if (info) {
        memset(info, 0, sizeof(*info));
        info->iterations = hs->iter;
        info->converged = conv ? 1 : 0;
        info->residual_l1 = hs->resid;
        info->sum_x = hs->sum_x;
        info->dangling_mass = hs->D;
        info->edge_visits = (double)hs->iter * (double)g->nnz;
        info->ms_device = ms;
        info->launches = launches;
        info->loop_edge_visits = info->edge_visits;
        info->ms_loop = ms;
    }
    return conv ? PR_OK : PR_NOT_CONVERGED;
}

extern "C" pr_status pr_adjoint(pr_wgraph* g, float damping, double tol, int32_t max_iter, const float* x,
                                const float* dL_dx, float* dL_dteleport, float* dL_dweights, pr_info* info,
                                void* stream) {
    if (!g || !x || !dL_dx) return fail(PR_ERR_INVALID_ARG, "pr_adjoint: NULL graph, x or dL_dx");
    if (!dL_dteleport && !dL_dweights) return fail(PR_ERR_INVALID_ARG, "pr_adjoint: no output requested");
    if (!(damping >= 0.0f && damping < 1.0f)) return fail(PR_ERR_INVALID_ARG, "damping must be in [0, 1)");
    if (!(tol > 0.0) || !std::isfinite(tol)) return fail(PR_ERR_INVALID_ARG, "tol must be a positive finite number");
    if (max_iter < 1) return fail(PR_ERR_INVALID_ARG, "max_iter must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    const float* xd = nullptr;
    const float* c = nullptr;
    pr_status rc = w_input(g, x, 0, s, &xd);
    if (rc == PR_OK) rc = w_input(g, dL_dx, 1, s, &c);
    if (rc != PR_OK) return rc;
    // device outputs in place; host outputs through device buffers
    const bool gt_dev = dL_dteleport && is_device_pointer(dL_dteleport);
    const bool gw_dev = dL_dweights && is_device_pointer(dL_dweights);
    float* gt = dL_dteleport ? (gt_dev ? dL_dteleport : g->stage + (size_t)2 * (size_t)(g->n + kPad)) : nullptr;
    float* gw = gw_dev ? dL_dweights : nullptr;
    float* gw_tmp = nullptr;
    if (dL_dweights && !gw_dev) {
        PRK_CHECK(cudaMalloc((void**)&gw_tmp, (size_t)std::max<int64_t>(g->nnz, 1) * sizeof(float)));
        gw = gw_tmp;
    }
    struct TmpGuard {
        float* p;
        ~TmpGuard() { if (p) cudaFree(p); }
    } guard{gw_tmp};
    WState* hs = g->host_state;
    memset(hs, 0, sizeof(WState));
    hs->d = damping;
    hs->tol = tol;
    hs->inv_n = 1.0 / (double)g->n;
    hs->max_iter = max_iter;
    PRK_CHECK(cudaEventRecord(g->ev0, s));
    PRK_CHECK(cudaMemcpyAsync(g->state, hs, sizeof(WState), cudaMemcpyHostToDevice, s));
    WArgs a = w_args(g);
    int launches = 0;
    float* lv[2] = {g->vec[0], g->vec[1]};
    float* mu = g->vec[2];
    k_w_init<<<w_grid(g), kBlock, 0, s>>>(a, nullptr, nullptr, c, lv[0]);
    ++launches;
    rc = w_loop(g, max_iter, s, &launches, [&](int it) {
        k_w_adjoint<<<w_grid(g), kBlock, 0, s>>>(a, c, lv[it & 1], lv[1 - (it & 1)], mu, 0);
    });
    if (rc != PR_OK) return rc;
    const float* lam = lv[hs->iter & 1];
    k_w_adjoint<<<w_grid(g), kBlock, 0, s>>>(a, c, lam, nullptr, mu, 1);
    k_w_grads<<<w_grid(g), kBlock, 0, s>>>(a, xd, lam, mu, gt, gw);
    launches += 2;
    PRK_CHECK(cudaGetLastError());
    PRK_CHECK(cudaEventRecord(g->ev1, s));
    if (dL_dteleport && !gt_dev)
        PRK_CHECK(cudaMemcpyAsync(dL_dteleport, gt, (size_t)g->n * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (dL_dweights && !gw_dev)
        PRK_CHECK(cudaMemcpyAsync(dL_dweights, gw, (size_t)g->nnz * sizeof(float), cudaMemcpyDeviceToHost, s));
    PRK_CHECK(cudaMemcpyAsync(hs, g->state, sizeof(WState), cudaMemcpyDeviceToHost, s));
    PRK_CHECK(cudaStreamSynchronize(s));
    float ms = 0.f;
    PRK_CHECK(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
    const bool conv = hs->resid < tol * hs->c_norm;
    if (info) {
        memset(info, 0, sizeof(*info));
        info->iterations = hs->iter;
        info->converged = conv ? 1 : 0;
        info->residual_l1 = hs->resid;
        info->sum_x = hs->L;
        info->edge_visits = (double)(hs->iter + 2) * (double)g->nnz;
        info->ms_device = ms;
        info->launches = launches;
        info->loop_edge_visits = (double)hs->iter * (double)g->nnz;
        info->ms_loop = ms;
    }
    return conv ? PR_OK : PR_NOT_CONVERGED;
}
