// pr_setup.cu -- pr_create_graph: copy, validate and lay out a graph in HBM.
//
// Steps (all on the device, enqueued on the caller's stream):
//   1. copy rowptr/colidx in (H2D or D2D) and validate them;
//   2. out-degree histogram from colidx (the "outDeg(v)" of Alg. 1 and the
//      divisor of the contribution in Alg. 2, computed once per graph);
//   3. bin every row by in-degree -- heavy rows, power-of-two classes, rows
//      without in-edges -- and relabel vertices with a stable counting sort
//      so that each bin is a contiguous id range;
//   4. build the binned CSR (rowptr by an exclusive scan of the binned
//      degrees, colidx copied row by row through the relabelling), the
//      inverse out-degrees, the segments of heavy rows and the row tiles.
#include <algorithm>
#include <cmath>
#include <vector>

#include "pr_common.cuh"

namespace prk {

// pool_free of every pointer once `stream` has reached this point, returned
// on the pool's own stream (reusable in stream order by the next pool_alloc);
// defined beside the pool in pr_capi.cu.
cudaError_t pool_free_after(void* const* ptrs, size_t count, cudaStream_t stream);

namespace {

constexpr int kChunk = 4096;  // elements per block in the scan and sort kernels (256 x 16)
constexpr int kPer = kChunk / kBlock;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Exclusive scan across the 256 threads of a block; returns the thread's
// exclusive prefix and, if total is not NULL, stores the block total there
// (every thread sees it).
__device__ int64_t block_excl_scan(int64_t v, int64_t* total) {
    __shared__ int64_t warp_pre[kWarps];
    __shared__ int64_t block_total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = warp_incl_scan(v);
    if (lane == 31) warp_pre[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < kWarps ? warp_pre[lane] : 0;
        int64_t wi = warp_incl_scan(w);
        if (lane < kWarps) warp_pre[lane] = wi - w;
        if (lane == kWarps - 1) block_total = wi;
    }
    __syncthreads();
    int64_t r = incl - v + warp_pre[warp];
    if (total) *total = block_total;
    __syncthreads();
    return r;
}

// ---- 3-phase exclusive scan of int64 values into OutT[count+1] ----

__global__ void k_scan_sums(const int64_t* __restrict__ in, int64_t count, int64_t* __restrict__ sums) {
    const int64_t base = (int64_t)blockIdx.x * kChunk + (int64_t)threadIdx.x * kPer;
    int64_t s = 0;
    for (int j = 0; j < kPer; ++j)
        if (base + j < count) s += in[base + j];
    int64_t total;
    block_excl_scan(s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// One block scans the nb block sums in place (exclusive) and writes the grand total.
__global__ void k_scan_block_sums(int64_t* sums, int64_t nb, int64_t* grand) {
    const int64_t per = (nb + kBlock - 1) / kBlock;
    const int64_t b0 = (int64_t)threadIdx.x * per;
    int64_t s = 0;
    for (int64_t j = 0; j < per; ++j)
        if (b0 + j < nb) s += sums[b0 + j];
    int64_t total;
    int64_t pre = block_excl_scan(s, &total);
    for (int64_t j = 0; j < per; ++j)
        if (b0 + j < nb) {
            int64_t v = sums[b0 + j];
            sums[b0 + j] = pre;
            pre += v;
        }
    if (threadIdx.x == 0) *grand = total;
}

template <typename OutT>
__global__ void k_scan_apply(const int64_t* __restrict__ in, int64_t count,
                             const int64_t* __restrict__ sums, const int64_t* __restrict__ grand,
                             OutT* __restrict__ out) {
    const int64_t base = (int64_t)blockIdx.x * kChunk + (int64_t)threadIdx.x * kPer;
    int64_t v[kPer];
    int64_t s = 0;
    for (int j = 0; j < kPer; ++j) {
        v[j] = base + j < count ? in[base + j] : 0;
        s += v[j];
    }
    int64_t pre = block_excl_scan(s, nullptr) + sums[blockIdx.x];
    for (int j = 0; j < kPer; ++j)
        if (base + j < count) {
            out[base + j] = (OutT)pre;
            pre += v[j];
        }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[count] = (OutT)*grand;
}

// ---- validation, degrees, bins ----

template <typename RP>
__global__ void k_validate(const RP* __restrict__ rp, int64_t n, int64_t nnz,
                           const int32_t* __restrict__ ci, uint32_t* err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    uint32_t e = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += stride) {
        int64_t a = (int64_t)rp[v];
        if (v == 0 && a != 0) e |= 1u;
        if (v == n && a != nnz) e |= 2u;
        if (v < n && (int64_t)rp[v + 1] < a) e |= 4u;
    }
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += stride) {
        int32_t c = ci[k];
        if (c < 0 || (int64_t)c >= n) e |= 8u;
    }
    if (e) atomicOr(err, e);
}

__global__ void k_outdeg(const int32_t* __restrict__ ci, int64_t nnz, uint32_t* __restrict__ outdeg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += stride)
        atomicAdd(&outdeg[ci[k]], 1u);
}

// Bin of a row by in-degree: bin 40 - floor(log2 deg) for deg >= 1 (so bins
// 1..40 hold decreasing power-of-two degree classes), bin kZeroBin for rows
// without in-edges that have out-edges, and bin kIsoBin, the last, for
// isolated vertices (no in- and no out-edges).  With a power-of-two heavy
// threshold the heavy rows are the prefix of bins up to 40 - log2(heavy).
constexpr int kTopClass = 40;
constexpr int kZeroBin = kTopClass + 1;
constexpr int kIsoBin = kTopClass + 2;
constexpr int kNumBins = kTopClass + 3;
static_assert(kNumBins <= kMaxBins, "bin count");

template <typename RP>
__global__ void k_bins(const RP* __restrict__ rp, int64_t n, const uint32_t* __restrict__ outdeg,
                       uint8_t* __restrict__ bin, int64_t* __restrict__ deg_out, unsigned long long* max_deg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long mx = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        int64_t deg = (int64_t)rp[v + 1] - (int64_t)rp[v];
        int b = deg != 0 ? kTopClass - (63 - __clzll((unsigned long long)deg))
                         : (outdeg[v] == 0 ? kIsoBin : kZeroBin);
        bin[v] = (uint8_t)b;
        deg_out[v] = deg;
        if ((unsigned long long)deg > mx) mx = (unsigned long long)deg;
    }
    atomicMax(max_deg, mx);
}

// counts[b * nblk + blk] = elements of chunk blk in bin b
__global__ void k_bin_count(const uint8_t* __restrict__ bin, int64_t n, int nbins, int64_t nblk,
                            int64_t* __restrict__ counts) {
    __shared__ unsigned int c[kNumBins];
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) c[b] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kChunk + (int64_t)threadIdx.x * kPer;
    for (int j = 0; j < kPer; ++j)
        if (base + j < n) atomicAdd(&c[bin[base + j]], 1u);
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) counts[(int64_t)b * nblk + blockIdx.x] = c[b];
}

// Stable scatter: position = start of (bin, chunk) + earlier elements of the same
// bin in the chunk (threads own contiguous runs, so thread order = element order).
__global__ void k_bin_scatter(const uint8_t* __restrict__ bin, int64_t n, int nbins, int64_t nblk,
                              const int64_t* __restrict__ offsets, int32_t* __restrict__ order,
                              int32_t* __restrict__ rank) {
    extern __shared__ int32_t cnt[];  // [nbins][kBlock]
    for (int b = 0; b < nbins; ++b) cnt[b * kBlock + threadIdx.x] = 0;
    const int64_t base = (int64_t)blockIdx.x * kChunk + (int64_t)threadIdx.x * kPer;
    for (int j = 0; j < kPer; ++j)
        if (base + j < n) cnt[bin[base + j] * kBlock + threadIdx.x] += 1;
    __syncthreads();
    for (int b = 0; b < nbins; ++b) {
        int64_t v = cnt[b * kBlock + threadIdx.x];
        int64_t ex = block_excl_scan(v, nullptr);
        cnt[b * kBlock + threadIdx.x] = (int32_t)ex;
        __syncthreads();
    }
    for (int j = 0; j < kPer; ++j) {
        int64_t v = base + j;
        if (v < n) {
            int b = bin[v];
            int64_t pos = offsets[(int64_t)b * nblk + blockIdx.x] + cnt[b * kBlock + threadIdx.x];
            cnt[b * kBlock + threadIdx.x] += 1;
            order[pos] = (int32_t)v;
            rank[v] = (int32_t)pos;
        }
    }
}

__global__ void k_gather_deg(const int32_t* __restrict__ order, const int64_t* __restrict__ deg,
                             int64_t n, int64_t* __restrict__ ndeg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        ndeg[i] = deg[order[i]];
}

// Copy the sources of binned row i (caller row order[i]) through rank[].
// Warp per row for rows [row_lo, row_hi).
template <typename RP, typename IdxT>
__global__ void k_relabel_warp(const RP* __restrict__ rp, const int32_t* __restrict__ ci,
                               const IdxT* __restrict__ nrp, int32_t* __restrict__ nci,
                               const int32_t* __restrict__ order, const int32_t* __restrict__ rank,
                               int64_t row_lo, int64_t row_hi) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = row_lo + wid; i < row_hi; i += nw) {
        const int64_t src = (int64_t)rp[order[i]];
        const int64_t deg = (int64_t)rp[order[i] + 1] - src;
        const int64_t dst = (int64_t)nrp[i];
        for (int64_t k = lane; k < deg; k += 32) nci[dst + k] = rank[ci[src + k]];
    }
}

// Block per row for the heavy rows [0, row_hi).
template <typename RP, typename IdxT>
__global__ void k_relabel_block(const RP* __restrict__ rp, const int32_t* __restrict__ ci,
                                const IdxT* __restrict__ nrp, int32_t* __restrict__ nci,
                                const int32_t* __restrict__ order, const int32_t* __restrict__ rank,
                                int64_t row_hi) {
    for (int64_t i = blockIdx.x; i < row_hi; i += gridDim.x) {
        const int64_t src = (int64_t)rp[order[i]];
        const int64_t deg = (int64_t)rp[order[i] + 1] - src;
        const int64_t dst = (int64_t)nrp[i];
        for (int64_t k = threadIdx.x; k < deg; k += blockDim.x) nci[dst + k] = rank[ci[src + k]];
    }
}

// Edges whose (binned) source id is below `limit`.
__global__ void k_count_below(const int32_t* __restrict__ ci, int64_t nnz, int32_t limit,
                              unsigned long long* __restrict__ count) {
    unsigned long long c = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += stride) c += ci[k] < limit;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

__global__ void k_inv_outdeg(const uint32_t* __restrict__ outdeg, const int32_t* __restrict__ order,
                             int64_t n, float* __restrict__ inv, unsigned long long* n_dangling) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uint32_t od = outdeg[order[i]];
        inv[i] = od ? 1.0f / (float)od : 0.0f;
        c += od == 0;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(n_dangling, c);
}

__global__ void k_seg_counts(const int64_t* __restrict__ ndeg, int64_t n_heavy, int64_t* __restrict__ nseg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < n_heavy; h += stride)
        nseg[h] = (ndeg[h] + kSegEdges - 1) / kSegEdges;
}

__global__ void k_seg_rows(const int32_t* __restrict__ seg_ptr, int64_t n_heavy, int32_t* __restrict__ seg_row) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < n_heavy; h += stride)
        for (int32_t s = seg_ptr[h]; s < seg_ptr[h + 1]; ++s) seg_row[s] = (int32_t)h;
}

int grid_for(int64_t work, int sm_count) {
    int64_t b = (work + kBlock - 1) / kBlock;
    int64_t cap = (int64_t)sm_count * 16;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}

// Scratch allocations freed when set-up returns.
// With a stream, the scratch goes back to the pool once that stream has
// reached the end of the set-up kernels that use it (pool_free_after),
// without a device-wide wait.
struct Scratch {
    std::vector<void*> ptrs;
    cudaStream_t stream = nullptr;
    Scratch() = default;
    explicit Scratch(cudaStream_t s) : stream(s) {}
    ~Scratch() {
        if (stream) {
            pool_free_after(ptrs.data(), ptrs.size(), stream);
            return;
        }
        for (void* p : ptrs) {
            cudaDeviceSynchronize();
            pool_free(p, nullptr);
        }
    }
    cudaError_t alloc(void** p, size_t bytes) {
        cudaError_t e = pool_alloc(p, bytes ? bytes : 16);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
};

template <typename OutT>
cudaError_t exclusive_scan(Scratch& s, const int64_t* in, int64_t count, OutT* out, cudaStream_t st) {
    int64_t nb = (count + kChunk - 1) / kChunk;
    if (nb < 1) nb = 1;
    int64_t* sums = nullptr;
    int64_t* grand = nullptr;
    cudaError_t e = s.alloc((void**)&sums, (size_t)nb * sizeof(int64_t));
    if (e != cudaSuccess) return e;
    e = s.alloc((void**)&grand, sizeof(int64_t));
    if (e != cudaSuccess) return e;
    k_scan_sums<<<(unsigned)nb, kBlock, 0, st>>>(in, count, sums);
    k_scan_block_sums<<<1, kBlock, 0, st>>>(sums, nb, grand);
    k_scan_apply<OutT><<<(unsigned)nb, kBlock, 0, st>>>(in, count, sums, grand, out);
    return cudaGetLastError();
}

// Host-side tile list from the bin boundaries (bin b holds binned rows
// [bin_start[b], bin_start[b+1])); lh = log2 of the heavy threshold.  A light
// tile holds at most max_rows rows and (by its degree class) max_edges edges;
// heavy-row and empty-row tiles hold heavy_rows and zero_rows rows.
std::vector<Tile> make_tiles(const std::vector<int64_t>& bin_start, int lh, int64_t max_edges = kTileEdgesMax,
                             int64_t max_rows = kTileRowsMax, int64_t heavy_rows = 4 * kBlock,
                             int64_t zero_rows = 16 * kBlock) {
    std::vector<Tile> tiles;
    auto add = [&](int64_t lo, int64_t hi, int64_t rows, int kind) {
        for (int64_t r = lo; r < hi; r += rows)
            tiles.push_back(Tile{(int32_t)r, (int32_t)std::min(hi, r + rows), kind, 0});
    };
    const int first_light = kTopClass + 1 - lh;   // bin of degree class lh-1
    add(0, bin_start[first_light], heavy_rows, kTileHeavy);
    for (int b = first_light; b <= kTopClass; ++b) {
        const int k = kTopClass - b;             // degree class [2^k, 2^(k+1))
        const int lg = std::min(k, 5);           // lanes per row = 2^lg
        // every row of the class has at most 2^(k+1)-1 edges, so this many rows
        // always fit the shared-memory staging area of a tile
        const int64_t rows = std::max<int64_t>(1, std::min<int64_t>(max_rows, max_edges / ((1LL << (k + 1)) - 1)));
        add(bin_start[b], bin_start[b + 1], rows, lg);
    }
    add(bin_start[kZeroBin], bin_start[kIsoBin], zero_rows, kTileZero);
    add(bin_start[kIsoBin], bin_start[kNumBins], zero_rows, kTileZero);   // isolated vertices: the last tiles
    return tiles;
}

template <typename RP, typename IdxT>
pr_status build_layout(pr_graph* g, const RP* rp, const int32_t* ci, cudaStream_t st, Scratch& s) {
    const int64_t n = g->n, nnz = g->nnz;
    const int sm = g->sm_count;

    // out-degrees
    uint32_t* outdeg = nullptr;
    PRK_CHECK(s.alloc((void**)&outdeg, (size_t)n * sizeof(uint32_t)));
    PRK_CHECK(cudaMemsetAsync(outdeg, 0, (size_t)n * sizeof(uint32_t), st));
    if (nnz > 0) k_outdeg<<<grid_for(nnz, sm), kBlock, 0, st>>>(ci, nnz, outdeg);

    // bins
    int lh = 0;
    while ((1LL << lh) < (int64_t)g->heavy_degree) ++lh;  // heavy = 2^lh
    const int nbins = kNumBins;
    uint8_t* bin = nullptr;
    int64_t* deg = nullptr;
    unsigned long long* dmax = nullptr;
    PRK_CHECK(s.alloc((void**)&bin, (size_t)n));
    PRK_CHECK(s.alloc((void**)&deg, (size_t)n * sizeof(int64_t)));
    PRK_CHECK(s.alloc((void**)&dmax, 2 * sizeof(unsigned long long)));
    PRK_CHECK(cudaMemsetAsync(dmax, 0, 2 * sizeof(unsigned long long), st));
    k_bins<RP><<<grid_for(n, sm), kBlock, 0, st>>>(rp, n, outdeg, bin, deg, dmax);

    // stable counting sort by bin
    const int64_t nblk = (n + kChunk - 1) / kChunk;
    int64_t* counts = nullptr;
    int64_t* offsets = nullptr;
    PRK_CHECK(s.alloc((void**)&counts, (size_t)(nbins * nblk) * sizeof(int64_t)));
    PRK_CHECK(s.alloc((void**)&offsets, (size_t)(nbins * nblk + 1) * sizeof(int64_t)));
    k_bin_count<<<(unsigned)nblk, kBlock, 0, st>>>(bin, n, nbins, nblk, counts);
    PRK_CHECK(exclusive_scan<int64_t>(s, counts, nbins * nblk, offsets, st));
    PRK_CHECK(dev_alloc(g, (void**)&g->order, (size_t)(n + kPad) * sizeof(int32_t)));
    PRK_CHECK(dev_alloc(g, (void**)&g->rank, (size_t)(n + kPad) * sizeof(int32_t)));
    k_bin_scatter<<<(unsigned)nblk, kBlock, (size_t)nbins * kBlock * sizeof(int32_t), st>>>(
        bin, n, nbins, nblk, offsets, g->order, g->rank);

    // binned rowptr
    int64_t* ndeg = nullptr;
    PRK_CHECK(s.alloc((void**)&ndeg, (size_t)n * sizeof(int64_t)));
    k_gather_deg<<<grid_for(n, sm), kBlock, 0, st>>>(g->order, deg, n, ndeg);
    PRK_CHECK(dev_alloc(g, &g->rowptr, (size_t)(n + 1 + kPad) * sizeof(IdxT)));
    PRK_CHECK(exclusive_scan<IdxT>(s, ndeg, n, (IdxT*)g->rowptr, st));

    // bin boundaries to the host
    std::vector<int64_t> bin_start(nbins + 1);
    for (int b = 0; b < nbins; ++b)
        PRK_CHECK(cudaMemcpyAsync(&bin_start[b], offsets + (int64_t)b * nblk, sizeof(int64_t),
                                  cudaMemcpyDeviceToHost, st));
    unsigned long long hmax = 0;
    PRK_CHECK(cudaMemcpyAsync(&hmax, dmax, sizeof(hmax), cudaMemcpyDeviceToHost, st));
    PRK_CHECK(cudaStreamSynchronize(st));
    bin_start[nbins] = n;
    g->max_indeg = (int64_t)hmax;
    g->n_heavy = bin_start[kTopClass + 1 - lh];
    g->n_zero_indeg = n - bin_start[kZeroBin];
    g->n_isolated = n - bin_start[kIsoBin];
    g->bin_start = bin_start;

    // binned colidx
    PRK_CHECK(dev_alloc(g, (void**)&g->colidx, (size_t)(nnz + kPad) * sizeof(int32_t)));
    PRK_CHECK(cudaMemsetAsync(g->colidx, 0, (size_t)(nnz + kPad) * sizeof(int32_t), st));
    if (nnz > 0) {
        if (g->n_heavy > 0)
            k_relabel_block<RP, IdxT><<<(unsigned)std::min<int64_t>(g->n_heavy, sm * 8), kBlock, 0, st>>>(
                rp, ci, (const IdxT*)g->rowptr, g->colidx, g->order, g->rank, g->n_heavy);
        const int64_t light_hi = bin_start[kZeroBin];
        if (light_hi > g->n_heavy)
            k_relabel_warp<RP, IdxT><<<grid_for((light_hi - g->n_heavy) * 32, sm), kBlock, 0, st>>>(
                rp, ci, (const IdxT*)g->rowptr, g->colidx, g->order, g->rank, g->n_heavy, light_hi);
    }

    // inverse out-degrees in binned order
    PRK_CHECK(dev_alloc(g, (void**)&g->inv_out, (size_t)(n + kPad) * sizeof(float)));
    PRK_CHECK(cudaMemsetAsync(g->inv_out, 0, (size_t)(n + kPad) * sizeof(float), st));
    k_inv_outdeg<<<grid_for(n, sm), kBlock, 0, st>>>(outdeg, g->order, n, g->inv_out, dmax + 1);

    // heavy-row segments
    int32_t n_seg = 0;
    const int64_t H = g->n_heavy;
    PRK_CHECK(dev_alloc(g, (void**)&g->seg_ptr, (size_t)(H + 1 + kPad) * sizeof(int32_t)));
    if (H > 0) {
        int64_t* nseg = nullptr;
        PRK_CHECK(s.alloc((void**)&nseg, (size_t)H * sizeof(int64_t)));
        k_seg_counts<<<grid_for(H, sm), kBlock, 0, st>>>(ndeg, H, nseg);
        PRK_CHECK(exclusive_scan<int32_t>(s, nseg, H, g->seg_ptr, st));
        PRK_CHECK(cudaMemcpyAsync(&n_seg, g->seg_ptr + H, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        PRK_CHECK(cudaStreamSynchronize(st));
    } else {
        PRK_CHECK(cudaMemsetAsync(g->seg_ptr, 0, sizeof(int32_t), st));
    }
    g->n_seg = n_seg;
    PRK_CHECK(dev_alloc(g, (void**)&g->seg_row, (size_t)(n_seg + kPad) * sizeof(int32_t)));
    PRK_CHECK(dev_alloc(g, (void**)&g->seg_sum, (size_t)(n_seg + kPad) * sizeof(float)));
    if (n_seg > 0) k_seg_rows<<<grid_for(H, sm), kBlock, 0, st>>>(g->seg_ptr, H, g->seg_row);

    // tiles
    std::vector<Tile> tiles = make_tiles(bin_start, lh);
    g->n_tiles = (int64_t)tiles.size();
    g->host_tiles = tiles;
    PRK_CHECK(dev_alloc(g, (void**)&g->tiles, (tiles.size() + 1) * sizeof(Tile)));
    PRK_CHECK(cudaMemcpyAsync(g->tiles, tiles.data(), tiles.size() * sizeof(Tile),
                              cudaMemcpyHostToDevice, st));

    // tiles of the pipelined row kernel: 32-bit offsets, and every light row
    // short enough for a shared-memory stage (heavy threshold <= kTmaEdges + 1)
    g->n_tma_tiles = 0;
    if (sizeof(IdxT) == 4 && (1LL << lh) <= (int64_t)kTmaEdges + 1) {
        std::vector<Tile> tt = make_tiles(bin_start, lh, kTmaEdges, kTmaRows, kTmaRows, kTmaRows);
        tt.push_back(Tile{(int32_t)n, (int32_t)n, kTileZero, 0});   // sentinel: its pad is nnz
        PRK_CHECK(dev_alloc(g, (void**)&g->tma_tiles, tt.size() * sizeof(Tile)));
        PRK_CHECK(cudaMemcpyAsync(g->tma_tiles, tt.data(), tt.size() * sizeof(Tile), cudaMemcpyHostToDevice, st));
        PRK_CHECK(fill_tile_edges(g->tma_tiles, (int64_t)tt.size() - 1, (const int32_t*)g->rowptr, st));
        g->n_tma_tiles = (int64_t)tt.size() - 1;
        g->n_tma_live = 0;
        while (g->n_tma_live < g->n_tma_tiles && tt[(size_t)g->n_tma_live].row_begin < bin_start[kIsoBin])
            ++g->n_tma_live;

        // The fused list: the light and empty-row tiles in the same order, with
        // every heavy-row segment a tile of its own, spread evenly among them,
        // so that each block's round-robin share mixes the two kinds of work.
        if (g->n_seg > 0 && kTmaEdges >= kSegEdges) {
            std::vector<Tile> lt;
            for (size_t i = 0; i + 1 < tt.size(); ++i)
                if (tt[i].kind != kTileHeavy) lt.push_back(tt[i]);
            const int64_t L = (int64_t)lt.size(), S = g->n_seg;
            std::vector<Tile> ft;
            ft.reserve((size_t)(L + S));
            for (int64_t li = 0, si = 0; li < L || si < S;) {
                if (si < S && (li >= L || si * L <= li * S)) ft.push_back(Tile{0, (int32_t)si++, kTileSeg, 0});
                else ft.push_back(lt[(size_t)li++]);
            }
            PRK_CHECK(dev_alloc(g, (void**)&g->tma_fused, ft.size() * sizeof(Tile)));
            PRK_CHECK(dev_alloc(g, (void**)&g->tma_fused_e1, ft.size() * sizeof(int32_t)));
            PRK_CHECK(cudaMemcpyAsync(g->tma_fused, ft.data(), ft.size() * sizeof(Tile), cudaMemcpyHostToDevice, st));
            PRK_CHECK(fill_fused_tiles(g->tma_fused, g->tma_fused_e1, (int64_t)ft.size(), (const int32_t*)g->rowptr,
                                       g->seg_row, g->seg_ptr, st));
            PRK_CHECK(dev_alloc(g, (void**)&g->row_cnt, (size_t)g->n_heavy * sizeof(int32_t)));
            PRK_CHECK(cudaMemsetAsync(g->row_cnt, 0, (size_t)g->n_heavy * sizeof(int32_t), st));
            PRK_CHECK(dev_alloc(g, (void**)&g->hr_part, (size_t)g->n_heavy * sizeof(float2)));
            g->n_tma_fused = (int64_t)ft.size();
        }
    }

    // edges whose source is in the hub prefix the gathers read through L1
    unsigned long long* hub_edges = nullptr;
    PRK_CHECK(s.alloc((void**)&hub_edges, sizeof(unsigned long long)));
    PRK_CHECK(cudaMemsetAsync(hub_edges, 0, sizeof(unsigned long long), st));
    if (nnz > 0)
        k_count_below<<<grid_for(nnz, sm), kBlock, 0, st>>>(g->colidx, nnz, (int32_t)(kDefaultHot & 0x0fffffff),
                                                             hub_edges);
    unsigned long long ndang = 0, nhub = 0;
    PRK_CHECK(cudaMemcpyAsync(&ndang, dmax + 1, sizeof(ndang), cudaMemcpyDeviceToHost, st));
    PRK_CHECK(cudaMemcpyAsync(&nhub, hub_edges, sizeof(nhub), cudaMemcpyDeviceToHost, st));
    PRK_CHECK(cudaStreamSynchronize(st));
    g->n_dangling = (int64_t)ndang;
    g->hub_prefix_edges = (int64_t)nhub;
    return PR_OK;
}

// ---- PR_OUT_CSR: the in-edge CSR from an out-edge CSR, on the device ------
//
// The out-edge CSR lists the edges grouped by source in increasing source
// order.  Sorting them by target with a stable sort keeps that order within
// every target, so each in-row lists its sources in increasing order, the
// same for every run.  The sort is an LSD radix sort of edge positions on the
// target id, four bits per pass, each pass the stable counting sort of the
// binning step (k_bin_count, k_bin_scatter) on a 16-bucket digit.

// src[e] = source u of edge e (warp per row of the out-edge CSR)
template <typename RP>
__global__ void k_edge_sources(const RP* __restrict__ rp, int64_t n, int32_t* __restrict__ src) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
        const int64_t e1 = (int64_t)rp[u + 1];
        for (int64_t e = (int64_t)rp[u] + lane; e < e1; e += 32) src[e] = (int32_t)u;
    }
}

__global__ void k_iota(int32_t* __restrict__ p, int64_t count) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) p[i] = (int32_t)i;
}

// digit of the target of the edge at sorted position i
__global__ void k_target_digit(const int32_t* __restrict__ dst, const int32_t* __restrict__ perm, int64_t count,
                               int shift, uint8_t* __restrict__ digit) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
        digit[i] = (uint8_t)((dst[perm[i]] >> shift) & 15);
}

// out[i] = in[order[i]]
__global__ void k_permute_i32(const int32_t* __restrict__ in, const int32_t* __restrict__ order, int64_t count,
                              int32_t* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) out[i] = in[order[i]];
}

// in-degree of every target, 64-bit counts for the scan
__global__ void k_target_counts(const int32_t* __restrict__ dst, int64_t nnz, unsigned long long* __restrict__ cnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride)
        atomicAdd(cnt + dst[e], 1ull);
}

// The in-edge CSR (rp_in[n+1], ci_in[nnz], scratch-owned) of a validated
// out-edge CSR (rp, ci); nnz < 2^31.
template <typename RP>
cudaError_t transpose_to_in_csr(const pr_graph* g, const RP* rp, const int32_t* ci, Scratch& s, cudaStream_t st,
                                RP** rp_in, int32_t** ci_in) {
    const int64_t n = g->n, nnz = g->nnz;
    const int sm = g->sm_count;
    unsigned long long* cnt = nullptr;
    cudaError_t e = s.alloc((void**)&cnt, (size_t)n * sizeof(unsigned long long));
    if (e == cudaSuccess) e = s.alloc((void**)rp_in, (size_t)(n + 1) * sizeof(RP));
    if (e == cudaSuccess) e = s.alloc((void**)ci_in, (size_t)(nnz + kPad) * sizeof(int32_t));
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(cnt, 0, (size_t)n * sizeof(unsigned long long), st)) != cudaSuccess) return e;
    if (nnz > 0) k_target_counts<<<grid_for(nnz, sm), kBlock, 0, st>>>(ci, nnz, cnt);
    if ((e = exclusive_scan<RP>(s, (const int64_t*)cnt, n, *rp_in, st)) != cudaSuccess) return e;
    if (nnz == 0) return cudaGetLastError();
    int32_t *src = nullptr, *perm = nullptr, *order = nullptr, *rank = nullptr, *next = nullptr;
    uint8_t* digit = nullptr;
    const int64_t nblk = (nnz + kChunk - 1) / kChunk;
    int64_t *counts = nullptr, *offsets = nullptr;
    for (auto pp : {&src, &perm, &order, &rank, &next})
        if ((e = s.alloc((void**)pp, (size_t)nnz * sizeof(int32_t))) != cudaSuccess) return e;
    if ((e = s.alloc((void**)&digit, (size_t)nnz)) != cudaSuccess) return e;
    if ((e = s.alloc((void**)&counts, (size_t)(16 * nblk) * sizeof(int64_t))) != cudaSuccess) return e;
    if ((e = s.alloc((void**)&offsets, (size_t)(16 * nblk + 1) * sizeof(int64_t))) != cudaSuccess) return e;
    k_edge_sources<RP><<<grid_for(n * 32, sm), kBlock, 0, st>>>(rp, n, src);
    k_iota<<<grid_for(nnz, sm), kBlock, 0, st>>>(perm, nnz);
    int bits = 1;
    while (bits < 31 && (1LL << bits) < n) ++bits;
    for (int shift = 0; shift < bits; shift += 4) {
        k_target_digit<<<grid_for(nnz, sm), kBlock, 0, st>>>(ci, perm, nnz, shift, digit);
        k_bin_count<<<(unsigned)nblk, kBlock, 0, st>>>(digit, nnz, 16, nblk, counts);
        if ((e = exclusive_scan<int64_t>(s, counts, 16 * nblk, offsets, st)) != cudaSuccess) return e;
        k_bin_scatter<<<(unsigned)nblk, kBlock, (size_t)16 * kBlock * sizeof(int32_t), st>>>(digit, nnz, 16, nblk,
                                                                                           offsets, order, rank);
        k_permute_i32<<<grid_for(nnz, sm), kBlock, 0, st>>>(perm, order, nnz, next);
        std::swap(perm, next);
    }
    k_permute_i32<<<grid_for(nnz, sm), kBlock, 0, st>>>(src, perm, nnz, *ci_in);
    return cudaGetLastError();
}

template <typename RP>
pr_status create_typed(pr_graph* g, const void* rowptr, const int32_t* colidx, cudaStream_t st) {
    const int64_t n = g->n, nnz = g->nnz;
    Scratch s(st);
    RP* rp = nullptr;
    int32_t* ci = nullptr;
    PRK_CHECK(s.alloc((void**)&rp, (size_t)(n + 1) * sizeof(RP)));
    PRK_CHECK(s.alloc((void**)&ci, (size_t)(nnz + kPad) * sizeof(int32_t)));
    PRK_CHECK(cudaMemcpyAsync(rp, rowptr, (size_t)(n + 1) * sizeof(RP), cudaMemcpyDefault, st));
    if (nnz > 0)
        PRK_CHECK(cudaMemcpyAsync(ci, colidx, (size_t)nnz * sizeof(int32_t), cudaMemcpyDefault, st));

    uint32_t* err = nullptr;
    PRK_CHECK(s.alloc((void**)&err, sizeof(uint32_t)));
    PRK_CHECK(cudaMemsetAsync(err, 0, sizeof(uint32_t), st));
    k_validate<RP><<<grid_for(std::max(n + 1, nnz), g->sm_count), kBlock, 0, st>>>(rp, n, nnz, ci, err);
    uint32_t herr = 0;
    PRK_CHECK(cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, st));
    PRK_CHECK(cudaStreamSynchronize(st));
    if (herr) {
        std::string why;
        if (herr & 1u) why += " rowptr[0] != 0;";
        if (herr & 2u) why += " rowptr[n] != nnz;";
        if (herr & 4u) why += " rowptr decreases;";
        if (herr & 8u) why += " colidx out of [0, n);";
        return fail(PR_ERR_INVALID_GRAPH, "pr_create_graph: invalid CSR:" + why);
    }
    if (g->out_layout) {
        RP* rp_in = nullptr;
        int32_t* ci_in = nullptr;
        PRK_CHECK(transpose_to_in_csr<RP>(g, rp, ci, s, st, &rp_in, &ci_in));
        rp = rp_in;
        ci = ci_in;
    }
    if (g->idx64) return build_layout<RP, int64_t>(g, rp, ci, st, s);
    return build_layout<RP, int32_t>(g, rp, ci, st, s);
}

}  // namespace

std::vector<Tile> tiles_with_threshold(const pr_graph* g, int heavy_degree, int64_t* heavy_rows,
                                       int64_t max_edges, int64_t max_rows) {
    int lh = 0;
    while ((1LL << lh) < (int64_t)heavy_degree) ++lh;
    *heavy_rows = g->bin_start[(size_t)(kTopClass + 1 - lh)];
    return make_tiles(g->bin_start, lh, max_edges, max_rows);
}

cudaError_t scan_counts_i32(const int64_t* counts, int64_t count, int32_t* offsets, cudaStream_t st) {
    Scratch s(st);
    cudaError_t e = exclusive_scan<int32_t>(s, counts, count, offsets, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // before the temporaries are freed
    return e;
}

}  // namespace prk

extern "C" pr_status pr_create_graph(int64_t n, int64_t nnz, const void* rowptr, int rowptr_is_64,
                                     const int32_t* colidx, const float* weights, int layout,
                                     void* stream, pr_graph** out) {
    using namespace prk;
    if (!out) return fail(PR_ERR_INVALID_ARG, "pr_create_graph: out is NULL");
    *out = nullptr;
    if (n < 1 || n > 0x7fffffffLL) return fail(PR_ERR_INVALID_ARG, "pr_create_graph: n must be in [1, 2^31-1]");
    if (nnz < 0) return fail(PR_ERR_INVALID_ARG, "pr_create_graph: nnz < 0");
    if (!rowptr) return fail(PR_ERR_INVALID_ARG, "pr_create_graph: rowptr is NULL");
    if (nnz > 0 && !colidx) return fail(PR_ERR_INVALID_ARG, "pr_create_graph: colidx is NULL");
    if (!rowptr_is_64 && nnz > 0x7fffffffLL)
        return fail(PR_ERR_INVALID_ARG, "pr_create_graph: nnz >= 2^31 needs int64 rowptr");
    if (layout != PR_IN_CSR && layout != PR_OUT_CSR)
        return fail(PR_ERR_INVALID_ARG, "pr_create_graph: layout must be PR_IN_CSR or PR_OUT_CSR");
    if (layout == PR_OUT_CSR && nnz > 0x7fffffffLL)
        return fail(PR_ERR_UNSUPPORTED, "pr_create_graph: PR_OUT_CSR needs nnz < 2^31");
    if (weights)
        return fail(PR_ERR_UNSUPPORTED,
                    "pr_create_graph: edge weights belong to the weighted graph object; use pr_create_wgraph");

    pr_graph* g = new (std::nothrow) pr_graph();
    if (!g) return fail(PR_ERR_OOM, "pr_create_graph: host allocation failed");
    cudaStream_t st = (cudaStream_t)stream;
    pr_status rc = PR_OK;
    do {
        cudaError_t e = cudaGetDevice(&g->device);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaGetDevice"); break; }
        e = cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaDeviceGetAttribute"); break; }
        g->n = n;
        g->nnz = nnz;
        g->out_layout = layout == PR_OUT_CSR;
        g->idx64 = nnz > 0x7fffffffLL || thread_force_index64();
        g->heavy_degree = thread_heavy_degree();
        e = cudaEventCreate(&g->ev_start);
        if (e == cudaSuccess) e = cudaEventCreate(&g->ev_stop);
        if (e == cudaSuccess) e = cudaEventCreate(&g->ev_loop0);
        if (e == cudaSuccess) e = cudaEventCreate(&g->ev_loop1);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaEventCreate"); break; }
        e = cudaEventRecord(g->ev_start, st);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaEventRecord"); break; }
        rc = rowptr_is_64 ? create_typed<int64_t>(g, rowptr, colidx, st)
                          : create_typed<int32_t>(g, rowptr, colidx, st);
        if (rc != PR_OK) break;
        rc = alloc_solver(g);
        if (rc != PR_OK) break;
        e = cudaEventRecord(g->ev_stop, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(g->ev_stop);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&g->setup_ms, g->ev_start, g->ev_stop);
        if (e != cudaSuccess) { rc = cuda_fail(e, "set-up timing"); break; }
    } while (0);
    if (rc != PR_OK) {
        pr_destroy_graph(g);
        return rc;
    }
    *out = g;
    return PR_OK;
}
