// pr_tile.cuh -- device code shared by the synchronous and the barrier-free
// kernels: memory-access policies, the per-row update (epilogue) and the
// gather over a tile of light rows.
//
// Two memory policies:
//   Jacobi (kInPlace = false): the kernel reads x_k, y_k and writes x_{k+1},
//     y_{k+1} in other buffers, so the inputs are read-only for the whole
//     launch and go through the non-coherent path (y gathers may hit L1).
//   In place (kInPlace = true): y is read by every block while its owner
//     rewrites it (the read-write races of No-Sync, Alg. 3).  Those accesses
//     are relaxed gpu-scope atomics -- defined behaviour under the PTX memory
//     model, served by L2.  x, which only its owner touches, uses the same
//     relaxed accesses (one per row per sweep), so no cached copy can be stale.
#pragma once

#include "pr_common.cuh"

namespace prk {

__device__ __forceinline__ float ld_stream(const float* p) {
    float v;
    asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ int32_t ld_stream(const int32_t* p) {
    int32_t v;
    asm("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ int4 ld_stream4(const int32_t* p) {
    int4 v;
    asm("ld.global.nc.L1::no_allocate.v4.s32 {%0, %1, %2, %3}, [%4];"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p));
    return v;
}

// Gathers of the quotient vector through the non-coherent path.  `hot` packs
// an L1 policy (bits 28..31) and a vertex count (bits 0..27): the first
// `count` binned ids -- the rows with the highest in-degree classes, which in
// power-law graphs are also the sources of most edges -- may be given a
// different L1 eviction priority from the rest.  Policy 0 (default) is the
// plain cached load for every id; policy 4 caches only the first `count` ids
// in L1 and reads every other id from L2 (ld.global.cg).
__device__ __forceinline__ float ld_gather(const float* y, int32_t c, int32_t hot) {
    float v;
    const int policy = (int)((uint32_t)hot >> 28);
    const int32_t count = hot & 0x0fffffff;
    if (policy == 0) return __ldg(y + c);
    if (policy == 4) return c < count ? __ldg(y + c) : __ldcg(y + c);
    if (c < count) {
        asm("ld.global.nc.L1::evict_last.f32 %0, [%1];" : "=f"(v) : "l"(y + c));
    } else if (policy == 1) {
        v = __ldg(y + c);
    } else if (policy == 2) {
        asm("ld.global.nc.L1::evict_first.f32 %0, [%1];" : "=f"(v) : "l"(y + c));
    } else {
        asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(y + c));
    }
    return v;
}

__device__ __forceinline__ void st_stream(float* p, float v) {
    asm volatile("st.global.cs.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

__device__ __forceinline__ float ld_relaxed(const float* p) {
    float v;
    asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ void st_relaxed(float* p, float v) {
    asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v));
}

__device__ __forceinline__ double ld_relaxed(const double* p) {
    double v;
    asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ void st_relaxed(double* p, double v) {
    asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v));
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename IdxT>
__device__ __forceinline__ int64_t row_at(const void* rowptr, int64_t r) {
    return (int64_t)__ldg((const IdxT*)rowptr + r);
}

// Constants of the update x' = (1-d) t + d (s + share), share = dangling
// share of this iteration (D/n, or (T - S)/n in the barrier-free form).
struct RowCtx {
    float d;          // damping
    float one_m_d;    // 1 - d
    float d_share;    // d * share
    float base;       // (1-d)/n + d * share (uniform teleport)
    int32_t hot;      // L1 policy of the global gathers (see ld_gather)
    int32_t hot_n;    // binned ids [0, hot_n) are read from hot_sm (shared memory)
    const float* hot_sm;
};

template <bool kInPlace>
struct Mem;

template <>
struct Mem<false> {
    static __device__ __forceinline__ float gather(const float* y, int32_t c, const RowCtx& x) {
        return c < x.hot_n ? x.hot_sm[c] : ld_gather(y, c, x.hot);
    }
    static __device__ __forceinline__ float load_x(const float* p) { return ld_stream(p); }
    static __device__ __forceinline__ void store_x(float* p, float v) { st_stream(p, v); }
    static __device__ __forceinline__ void store_y(float* p, float v) { st_stream(p, v); }
};

template <>
struct Mem<true> {
    static __device__ __forceinline__ float gather(const float* y, int32_t c, const RowCtx& x) {
        return c < x.hot_n ? x.hot_sm[c] : ld_relaxed(y + c);
    }
    static __device__ __forceinline__ float load_x(const float* p) { return ld_relaxed(p); }
    static __device__ __forceinline__ void store_x(float* p, float v) { st_relaxed(p, v); }
    static __device__ __forceinline__ void store_y(float* p, float v) { st_relaxed(p, v); }
};

// Per-thread accumulators.  r: L1 change.  (m, c): Kahan sum of the mass the
// kernel tracks -- the new dangling mass (synchronous form) or the change of
// the non-dangling mass (in-place form).
struct Acc {
    float r = 0.f;
    float m = 0.f;
    float c = 0.f;
    float dd = 0.f;   // in-place form: change of the dangling mass (diagnostic form only)
    __device__ __forceinline__ void kahan(float v) {
        const float yk = v - c;
        const float tk = m + yk;
        c = (tk - m) - yk;
        m = tk;
    }
    __device__ __forceinline__ double mass() const { return (double)m - (double)c; }
};

template <bool kUniform, bool kInPlace>
__device__ __forceinline__ void row_update(int64_t r, float s, float xo, float inv, float tv,
                                           const RowCtx& c, float* x_out, float* y_out, Acc& acc) {
    const float base = kUniform ? c.base : fmaf(c.one_m_d, tv, c.d_share);
    const float xn = fmaf(c.d, s, base);
    Mem<kInPlace>::store_x(x_out + r, xn);
    Mem<kInPlace>::store_y(y_out + r, xn * inv);
    acc.r += fabsf(xn - xo);
    if (kInPlace) {
        if (inv != 0.f) acc.kahan(xn - xo);
        else acc.dd += xn - xo;
    } else {
        if (inv == 0.f) acc.kahan(xn);
    }
}

// Rows without in-edges: thread per row, s = 0.
template <bool kUniform, bool kInPlace>
__device__ __forceinline__ void process_zero_tile(const Tile& tile, const float* inv_out,
                                                  const float* teleport, const float* x_in,
                                                  float* x_out, float* y_out, const RowCtx& c,
                                                  Acc& acc, int tid) {
    for (int64_t r = tile.row_begin + tid; r < tile.row_end; r += kBlock) {
        const float tv = kUniform ? 0.f : ld_stream(teleport + r);
        row_update<kUniform, kInPlace>(r, 0.f, Mem<kInPlace>::load_x(x_in + r), ld_stream(inv_out + r),
                                       tv, c, x_out, y_out, acc);
    }
}

// Tile functions run on a 256-thread (kBlock) group of whole warps; tid is
// the thread's index in that group.
//
// Light rows of one degree class: groups of g = 2^tile.kind lanes gather one
// row each, two rows per group at a time (rows r and r + 256/g), so that a lane
// has up to four colidx loads and four gathers in flight; coalesced colidx
// reads within the group; shuffle reduction; the group's first lane updates
// both rows.
template <typename IdxT, bool kUniform, bool kInPlace>
__device__ __forceinline__ void process_light_tile(const Tile& tile, const void* rowptr,
                                                   const int32_t* colidx, const float* inv_out,
                                                   const float* teleport, const float* x_in,
                                                   const float* y_in, float* x_out, float* y_out,
                                                   const RowCtx& c, Acc& acc, int tid) {
    const int lg = tile.kind;
    const int g = 1 << lg;
    const int rpp = kBlock >> lg;  // rows per pass of the whole group set
    const int grp = tid >> lg;
    const int gl = tid & (g - 1);
    for (int64_t r0 = tile.row_begin; r0 < tile.row_end; r0 += 2 * rpp) {
        int64_t rr[2];
        bool act[2];
        int64_t b[2], e[2];
        float xo[2], inv[2], tv[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            rr[q] = r0 + q * rpp + grp;
            act[q] = rr[q] < tile.row_end;
            b[q] = e[q] = 0;
            xo[q] = inv[q] = tv[q] = 0.f;
            if (act[q]) {
                b[q] = row_at<IdxT>(rowptr, rr[q]);
                e[q] = row_at<IdxT>(rowptr, rr[q] + 1);
                if (gl == 0) {
                    xo[q] = Mem<kInPlace>::load_x(x_in + rr[q]);
                    inv[q] = ld_stream(inv_out + rr[q]);
                    if (!kUniform) tv[q] = ld_stream(teleport + rr[q]);
                }
            }
        }
        float s[2] = {0.f, 0.f};
        const int64_t len = max(e[0] - b[0], e[1] - b[1]);
        for (int64_t k = gl; k < len; k += 2 * g) {
            int32_t cc[2][2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                cc[q][0] = b[q] + k < e[q] ? ld_stream(colidx + b[q] + k) : -1;
                cc[q][1] = b[q] + k + g < e[q] ? ld_stream(colidx + b[q] + k + g) : -1;
            }
            float v[2][2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                v[q][0] = cc[q][0] >= 0 ? Mem<kInPlace>::gather(y_in, cc[q][0], c) : 0.f;
                v[q][1] = cc[q][1] >= 0 ? Mem<kInPlace>::gather(y_in, cc[q][1], c) : 0.f;
            }
            s[0] += v[0][0] + v[0][1];
            s[1] += v[1][0] + v[1][1];
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1)
            if (o < g) {
                s[0] += __shfl_xor_sync(0xffffffffu, s[0], o);
                s[1] += __shfl_xor_sync(0xffffffffu, s[1], o);
            }
        if (gl == 0) {
#pragma unroll
            for (int q = 0; q < 2; ++q)
                if (act[q]) row_update<kUniform, kInPlace>(rr[q], s[q], xo[q], inv[q], tv[q], c, x_out, y_out, acc);
        }
    }
}

// Sum (a, b) over the block and write the block's pair to
// slots[2*blockIdx.x]; returns true in every thread of the block that
// arrives last.  That block then holds the grid totals -- summed over the
// slots in slot order, so the result does not depend on arrival order -- in
// (*ta, *tb) of every thread.
__device__ __forceinline__ bool block_pair_to_grid(double a, double b, double* slots, uint32_t* ticket,
                                                   double* ta, double* tb) {
    __shared__ double sa[32], sb[32];
    const int nw = blockDim.x >> 5;
    __shared__ int last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) {
        sa[warp] = a;
        sb[warp] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0.0, B = 0.0;
        for (int w = 0; w < nw; ++w) {
            A += sa[w];
            B += sb[w];
        }
        slots[2 * blockIdx.x] = A;
        slots[2 * blockIdx.x + 1] = B;
        __threadfence();
        const uint32_t t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double A = 0.0, B = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        A += __ldcg(slots + 2 * i);
        B += __ldcg(slots + 2 * i + 1);
    }
    A = warp_sum(A);
    B = warp_sum(B);
    __syncthreads();
    if (lane == 0) {
        sa[warp] = A;
        sb[warp] = B;
    }
    __syncthreads();
    A = 0.0;
    B = 0.0;
    for (int w = 0; w < nw; ++w) {
        A += sa[w];
        B += sb[w];
    }
    *ta = A;
    *tb = B;
    return true;
}

// Block-wide sum of two doubles; every thread receives the totals.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
    __shared__ double sa[32], sb[32];
    const int nw = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    __syncthreads();
    if (lane == 0) {
        sa[warp] = a;
        sb[warp] = b;
    }
    __syncthreads();
    a = 0.0;
    b = 0.0;
    for (int w = 0; w < nw; ++w) {
        a += sa[w];
        b += sb[w];
    }
}

// Block-wide sum of a float; every thread receives the total.
__device__ __forceinline__ float block_sum(float v) {
    __shared__ float sv[32];
    const int nw = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sv[warp] = v;
    __syncthreads();
    float t = 0.f;
    for (int w = 0; w < nw; ++w) t += sv[w];
    return t;
}

}  // namespace prk
