// pr_noalloc.cu -- pr_step_noalloc: one synchronous PageRank update that
// allocates no memory at all.
//
// Who needs it: callers that cannot call cudaMalloc (or any allocating
// routine) at the point where they want an update -- for example code running
// inside a memory pool or arena that must not grow, a host process whose
// allocator is owned by another framework, or a real-time loop where an
// allocation's latency or failure is not acceptable.  Those callers bring
// every input and output buffer themselves; the only other memory this entry
// point touches is the fixed scratch array below.
//
// Scratch: g_noalloc_scratch is a file-scope device array of
// kNaScratchBytes (about 128 KiB).  Every GPU that loads this library holds it
// until the process exits.  It carries the per-block partial sums of the two
// reductions (dangling mass, L1 change), the arrival ticket of the
// last-block pattern and the dangling mass of the input.  All calls on a
// device share it: calls that overlap on the GPU (two streams, or two host
// threads) race on it and give wrong sums, so serialise them.  Each call
// clears the ticket before its kernels run.
//
// The device address of the array is looked up with cudaGetSymbolAddress on
// every call, with the caller's device current, and is not remembered: after
// a cudaDeviceReset (or any other teardown of the primary context) the module
// is loaded again, possibly at another address, and a remembered pointer
// would go stale.  The lookup allocates nothing.  The first call on a device
// (or after a reset) is the one that loads the module; make it before any
// stream capture.

#include "pr_tile.cuh"

namespace prk {
namespace {

constexpr int kNaRowsPerBlock = 2048;   // rows handled by one block
constexpr int kNaMaxBlocks = 8192;      // partial-sum slots in the scratch array
constexpr int64_t kNaMaxRows = (int64_t)kNaRowsPerBlock * kNaMaxBlocks;  // 16,777,216

struct NaScratch {
    unsigned int ticket;                 // blocks that have finished (last-block pattern)
    unsigned int pad0;
    double dangling_in;                  // dangling mass of x_in (first kernel -> second)
    double pad1[30];
    double slots[2 * kNaMaxBlocks];      // per-block (a, b) partial sums
};
constexpr size_t kNaScratchBytes = sizeof(NaScratch);
static_assert(kNaScratchBytes <= 160 * 1024, "the fixed scratch stays about 128 KiB");

static __device__ __align__(256) NaScratch g_noalloc_scratch;

// Block sum of (a, b) into slots[2*blockIdx.x]; the last block to arrive gets
// the grid totals, summed over the slots in slot order.
__device__ bool na_pair_to_grid(double a, double b, NaScratch* sc, double* ta, double* tb) {
    return block_pair_to_grid(a, b, sc->slots, &sc->ticket, ta, tb);
}

// sums_out[0] = dangling mass of x_in.
__global__ void __launch_bounds__(kBlock) k_na_dangling(int64_t n, const float* __restrict__ inv,
                                                        const float* __restrict__ x_in,
                                                        NaScratch* sc, double* sums_out) {
    double s = 0.0;
    const int64_t r0 = (int64_t)blockIdx.x * kNaRowsPerBlock;
    const int64_t r1 = min(r0 + kNaRowsPerBlock, n);
    for (int64_t r = r0 + threadIdx.x; r < r1; r += kBlock)
        if (inv[r] == 0.f) s += (double)x_in[r];
    double D, unused;
    if (na_pair_to_grid(s, 0.0, sc, &D, &unused) && threadIdx.x == 0) {
        sc->dangling_in = D;
        sums_out[0] = D;
        sc->ticket = 0;
    }
}

// x_out(v) = (1-d)/n + d (sum_{u->v} x_in(u) inv(u) + D/n); sums_out[1] = dangling
// mass of x_out, sums_out[2] = ||x_out - x_in||_1.  A warp per row.
__global__ void __launch_bounds__(kBlock) k_na_update(int64_t n, const int32_t* __restrict__ rowptr,
                                                      const int32_t* __restrict__ colidx,
                                                      const float* __restrict__ inv, float damping,
                                                      const float* __restrict__ x_in,
                                                      float* __restrict__ x_out, NaScratch* sc,
                                                      double* sums_out) {
    const double d = (double)damping;
    const double inv_n = 1.0 / (double)n;
    const float base = (float)((1.0 - d) * inv_n + d * sc->dangling_in * inv_n);
    const float fd = damping;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * kNaRowsPerBlock;
    const int64_t r1 = min(r0 + kNaRowsPerBlock, n);
    Acc acc;   // L1 change and Kahan-compensated dangling mass of this thread's rows
    for (int64_t r = r0 + warp; r < r1; r += kWarps) {
        const int32_t b = rowptr[r], e = rowptr[r + 1];
        float s = 0.f;
        for (int32_t k = b + lane; k < e; k += 32) {
            const int32_t u = colidx[k];
            s += x_in[u] * inv[u];
        }
        s = warp_sum(s);
        if (lane == 0) {
            const float xn = fmaf(fd, s, base);
            x_out[r] = xn;
            acc.add_r(fabsf(xn - x_in[r]));
            if (inv[r] == 0.f) acc.kahan(xn);
        }
    }
    double D1, L1;
    if (na_pair_to_grid(acc.mass(), acc.resid(), sc, &D1, &L1) && threadIdx.x == 0) {
        sums_out[1] = D1;
        sums_out[2] = L1;
        sc->ticket = 0;
    }
}

}  // namespace
}  // namespace prk

using namespace prk;

extern "C" pr_status pr_step_noalloc(int64_t n, const int32_t* rowptr, const int32_t* colidx,
                                     const float* inv_outdeg, float damping, const float* x_in,
                                     float* x_out, double* sums_out, void* stream) {
    if (n < 1) return fail(PR_ERR_INVALID_ARG, "pr_step_noalloc: n must be >= 1");
    if (n > kNaMaxRows)
        return fail(PR_ERR_INVALID_ARG,
                    "pr_step_noalloc: n exceeds the fixed scratch capacity of 16,777,216 rows "
                    "(8192 blocks of 2048 rows); use pr_create_graph/pr_iterate for larger graphs");
    if (!rowptr || !colidx || !inv_outdeg || !x_in || !x_out || !sums_out)
        return fail(PR_ERR_INVALID_ARG, "pr_step_noalloc: NULL pointer argument");
    {
        // the update reads every x_in(u) while it writes x_out: the two ranges
        // [x_in, x_in + n) and [x_out, x_out + n) must not share an element
        const uintptr_t a0 = (uintptr_t)x_in, b0 = (uintptr_t)x_out;
        const uintptr_t bytes = (uintptr_t)n * sizeof(float);
        if (a0 < b0 + bytes && b0 < a0 + bytes)
            return fail(PR_ERR_INVALID_ARG, "pr_step_noalloc: x_in and x_out overlap; they must be disjoint buffers");
    }
    if (!(damping >= 0.0f && damping < 1.0f))
        return fail(PR_ERR_INVALID_ARG, "pr_step_noalloc: damping must be in [0, 1)");
    const void* ptrs[] = {rowptr, colidx, inv_outdeg, x_in, x_out, sums_out};
    for (const void* p : ptrs)
        if (!is_device_pointer(p))
            return fail(PR_ERR_INVALID_ARG, "pr_step_noalloc: every array must be device memory");

    // The host-side name g_noalloc_scratch is not a device address: ask the
    // runtime where the current device's copy lives.
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "pr_step_noalloc: cudaGetSymbolAddress");
    NaScratch* sc = (NaScratch*)p;
    cudaStream_t s = (cudaStream_t)stream;
    PRK_CHECK(cudaMemsetAsync(&sc->ticket, 0, sizeof(unsigned int), s));
    const int blocks = (int)((n + kNaRowsPerBlock - 1) / kNaRowsPerBlock);
    k_na_dangling<<<blocks, kBlock, 0, s>>>(n, inv_outdeg, x_in, sc, sums_out);
    k_na_update<<<blocks, kBlock, 0, s>>>(n, rowptr, colidx, inv_outdeg, damping, x_in, x_out, sc,
                                          sums_out);
    PRK_CHECK(cudaGetLastError());
    return PR_OK;
}
