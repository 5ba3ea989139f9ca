// pr_ceiling.cu -- pr_measure_gather_rate: how fast this GPU serves random
// 4-byte loads from a vector that stays in L2.
//
// Every kernel of the pull gather (Eq. 1 summed over in-edges) spends its time
// on one irregular load per edge, y(colidx[e]).  On a graph whose quotient
// vector y fits in L2, DRAM is not the limit: each load that misses L1 is one
// request from the SM to L2, and the rate at which an SM can issue those
// requests bounds the iteration.  This entry point measures that rate
// directly, with no graph: warps stream random indices in 16-byte vectors
// (as the row kernels stream colidx) and keep 16 independent gathers in
// flight per lane, summing what they load so that no load can be dropped.
// Dividing a workload's L1-missing gathers by the measured rate gives the
// shortest time any pull-gather kernel can take on it.
//
// The indices are drawn on the device by SplitMix64 (Steele, Lea and Flood,
// "Fast splittable pseudorandom number generators", OOPSLA 2014), reduced
// modulo the vector length.
#include <algorithm>

#include "pr_common.cuh"

namespace prk {
namespace {

constexpr int kGrThreads = 256;
constexpr int kGrChunk = 512;            // indices per warp per chunk: four 16-byte vectors per lane
constexpr int32_t kGrMaxChunks = 65536;  // chunks per warp in one launch
constexpr int kGrMaxBlocksPerSm = 8;

__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_gr_fill(int32_t* __restrict__ idx, int64_t n_idx, int64_t n_values, uint64_t seed) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_idx; i += stride)
        idx[i] = (int32_t)(splitmix64(seed + (uint64_t)i) % (uint64_t)n_values);
}

template <bool kCached>
__device__ __forceinline__ float gr_load(const float* p) {
    return kCached ? __ldg(p) : __ldcg(p);
}

// Warp w takes chunks w, w + W, w + 2W, ... (W warps in the grid), wrapping
// around the index array; chunk c covers idx[512c, 512c + 512).
template <bool kCached>
__global__ void __launch_bounds__(kGrThreads) k_gr_gather(const float* __restrict__ y,
                                                          const int32_t* __restrict__ idx,
                                                          int64_t n_chunks, int32_t chunks,
                                                          float* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t gtid = (int64_t)blockIdx.x * kGrThreads + threadIdx.x;
    const int64_t warp = gtid >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * kGrThreads) >> 5;
    float acc = 0.f;
    for (int32_t c = 0; c < chunks; ++c) {
        const int64_t chunk = (warp + (int64_t)c * n_warps) % n_chunks;
        const int32_t* p = idx + chunk * kGrChunk + 4 * lane;
        int4 v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = __ldcs(reinterpret_cast<const int4*>(p + 128 * j));
#pragma unroll
        for (int j = 0; j < 4; ++j)
            acc += (gr_load<kCached>(y + v[j].x) + gr_load<kCached>(y + v[j].y)) +
                   (gr_load<kCached>(y + v[j].z) + gr_load<kCached>(y + v[j].w));
    }
    out[gtid] = acc;
}

struct DeviceBuffers {
    void* p[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t ev[2] = {nullptr, nullptr};
    ~DeviceBuffers() {
        for (void* q : p)
            if (q) cudaFree(q);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
};

}  // namespace
}  // namespace prk

using namespace prk;

extern "C" pr_status pr_measure_gather_rate(int64_t n_values, int64_t n_indices, int cached,
                                            int blocks_per_sm, int32_t chunks, uint64_t seed,
                                            double* out, void* stream) {
    if (!out) return fail(PR_ERR_INVALID_ARG, "pr_measure_gather_rate: out is NULL");
    if (n_values < 1 || n_values > INT32_MAX)
        return fail(PR_ERR_INVALID_ARG, "pr_measure_gather_rate: n_values must be in [1, 2^31 - 1]");
    if (n_indices < 2 * kGrChunk || n_indices > INT32_MAX || n_indices % kGrChunk != 0)
        return fail(PR_ERR_INVALID_ARG,
                    "pr_measure_gather_rate: n_indices must be a multiple of 512 in [1024, 2^31 - 1]");
    if (cached != 0 && cached != 1)
        return fail(PR_ERR_INVALID_ARG, "pr_measure_gather_rate: cached must be 0 or 1");
    if (blocks_per_sm < 1 || blocks_per_sm > kGrMaxBlocksPerSm)
        return fail(PR_ERR_INVALID_ARG, "pr_measure_gather_rate: blocks_per_sm must be in [1, 8]");
    if (chunks < 1 || chunks > kGrMaxChunks)
        return fail(PR_ERR_INVALID_ARG, "pr_measure_gather_rate: chunks must be in [1, 65536]");

    int dev = 0, sms = 0, occ = 0;
    PRK_CHECK(cudaGetDevice(&dev));
    PRK_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PRK_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ, cached ? (const void*)k_gr_gather<true> : (const void*)k_gr_gather<false>, kGrThreads, 0));
    if (blocks_per_sm > occ)
        return fail(PR_ERR_INVALID_ARG, "pr_measure_gather_rate: blocks_per_sm exceeds the " +
                                            std::to_string(occ) + " blocks that fit on an SM");
    const int grid = sms * blocks_per_sm;
    cudaStream_t s = (cudaStream_t)stream;

    DeviceBuffers b;
    float* y = nullptr;
    int32_t* idx = nullptr;
    float* sink = nullptr;
    PRK_CHECK(cudaMalloc((void**)&y, (size_t)n_values * sizeof(float)));
    b.p[0] = y;
    PRK_CHECK(cudaMalloc((void**)&idx, (size_t)n_indices * sizeof(int32_t)));
    b.p[1] = idx;
    PRK_CHECK(cudaMalloc((void**)&sink, (size_t)grid * kGrThreads * sizeof(float)));
    b.p[2] = sink;
    PRK_CHECK(cudaEventCreate(&b.ev[0]));
    PRK_CHECK(cudaEventCreate(&b.ev[1]));

    PRK_CHECK(cudaMemsetAsync(y, 0, (size_t)n_values * sizeof(float), s));
    k_gr_fill<<<sms * 8, kGrThreads, 0, s>>>(idx, n_indices, n_values, seed);
    PRK_CHECK(cudaGetLastError());
    const int64_t n_chunks = n_indices / kGrChunk;
    auto launch = [&](int32_t c) {
        if (cached)
            k_gr_gather<true><<<grid, kGrThreads, 0, s>>>(y, idx, n_chunks, c, sink);
        else
            k_gr_gather<false><<<grid, kGrThreads, 0, s>>>(y, idx, n_chunks, c, sink);
    };
    launch(std::min<int32_t>(chunks, 4));   // warm-up: the vector and the first chunks into L2
    PRK_CHECK(cudaGetLastError());
    PRK_CHECK(cudaEventRecord(b.ev[0], s));
    launch(chunks);
    PRK_CHECK(cudaGetLastError());
    PRK_CHECK(cudaEventRecord(b.ev[1], s));
    PRK_CHECK(cudaEventSynchronize(b.ev[1]));
    float ms = 0.f;
    PRK_CHECK(cudaEventElapsedTime(&ms, b.ev[0], b.ev[1]));
    const double gathers = (double)grid * kGrThreads * 16.0 * chunks;
    out[0] = ms > 0.f ? gathers / (ms * 1e-3) : 0.0;
    out[1] = ms;
    out[2] = gathers;
    return PR_OK;
}
