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

#include <cuda_bf16.h>

#include <type_traits>

#include "pr_common.cuh"

// L2 eviction priority of each access class, as an L2 cache policy made by
// createpolicy: 0 = no hint (plain instruction forms), 1 = evict_first,
// 2 = evict_last, 3 = evict_normal.  The stream class covers what an
// iteration reads once (colidx, x, 1/outdeg, teleport); the gather class the
// quotient vector y that every edge reads; the y-store class the writes of y'
// (gathered by the next iteration; 4 = a plain write-back store).  Keeping y
// resident in L2 while colidx streams past it is what these hints are for:
// on ER-24, where no hub keeps y's lines warm, a quarter of the gathers
// missed L2 with the streamed loads and copies unhinted and y' stored with
// .cs.  Streamed loads and bulk copies evict_first with y' stored plainly
// measured fastest of seven combinations (ER-24 1.41 -> 1.26 ms per
// synchronous iteration, 1.51 -> 1.43 ms per barrier-free sweep; R-MAT-24
// 0.90 -> 0.88 and 0.906 -> 0.892 ms).
#ifndef PRK_L2_STREAM
#define PRK_L2_STREAM 1
#endif
#ifndef PRK_L2_GATHER
#define PRK_L2_GATHER 0
#endif
#ifndef PRK_L2_YSTORE
#define PRK_L2_YSTORE 4
#endif

namespace prk {

template <int P>
__device__ __forceinline__ uint64_t l2_policy() {
    uint64_t p;
    if constexpr (P == 1) asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    else if constexpr (P == 2) asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    else asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ float ld_stream(const float* p) {
    float v;
    if constexpr (PRK_L2_STREAM == 0)
        asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    else
        asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;"
            : "=f"(v) : "l"(p), "l"(l2_policy<PRK_L2_STREAM>()));
    return v;
}

__device__ __forceinline__ int32_t ld_stream(const int32_t* p) {
    int32_t v;
    if constexpr (PRK_L2_STREAM == 0)
        asm("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
    else
        asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;"
            : "=r"(v) : "l"(p), "l"(l2_policy<PRK_L2_STREAM>()));
    return v;
}

__device__ __forceinline__ int4 ld_stream4(const int32_t* p) {
    int4 v;
    if constexpr (PRK_L2_STREAM == 0)
        asm("ld.global.nc.L1::no_allocate.v4.s32 {%0, %1, %2, %3}, [%4];"
            : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
            : "l"(p));
    else
        asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
            : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
            : "l"(p), "l"(l2_policy<PRK_L2_STREAM>()));
    return v;
}

// Column index of a light row gathered by lane groups (gather_row_pair from
// global memory).  The lanes of a warp read one stretch of g indices from each
// of 32/g rows per instruction, and the next instructions of the step read the
// following stretches of the same lines: through L1 (kMode 1: evict_first,
// 2: evict_normal) those lines are requested from L2 once; kMode 0 does not
// allocate in L1.  PRK_NB_COL_L1 is the barrier-free kernel's mode,
// PRK_SYNC_COL_L1 that of the synchronous light-row gathers.
#ifndef PRK_NB_COL_L1
#define PRK_NB_COL_L1 2
#endif
#ifndef PRK_SYNC_COL_L1
#define PRK_SYNC_COL_L1 2
#endif
template <int kMode>
__device__ __forceinline__ int32_t ld_col(const int32_t* p) {
    if constexpr (kMode == 0) {
        return ld_stream(p);
    } else {
        int32_t v;
        if constexpr (kMode == 1)
            asm("ld.global.nc.L1::evict_first.L2::cache_hint.s32 %0, [%1], %2;"
                : "=r"(v) : "l"(p), "l"(l2_policy<PRK_L2_STREAM>()));
        else
            asm("ld.global.nc.L1::evict_normal.L2::cache_hint.s32 %0, [%1], %2;"
                : "=r"(v) : "l"(p), "l"(l2_policy<PRK_L2_STREAM>()));
        return v;
    }
}

// Gathers of y with the gather-class L2 policy: through L1 (ldg) or L2 only (cg).
__device__ __forceinline__ float ld_y_ldg(const float* p) {
    if constexpr (PRK_L2_GATHER == 0) {
        return __ldg(p);
    } else {
        float v;
        asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(l2_policy<PRK_L2_GATHER>()));
        return v;
    }
}

__device__ __forceinline__ float ld_y_cg(const float* p) {
    if constexpr (PRK_L2_GATHER == 0) {
        return __ldcg(p);
    } else {
        float v;
        asm("ld.global.cg.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(l2_policy<PRK_L2_GATHER>()));
        return v;
    }
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
    if (policy == 0) return ld_y_ldg(y + c);
    if (policy == 4) return c < count ? ld_y_ldg(y + c) : ld_y_cg(y + c);
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

// Store of y' (read by the gathers of the next iteration): 0 streaming
// (.cs), 1..3 with the L2 policy of that class, 4 a plain write-back store.
__device__ __forceinline__ void st_y(float* p, float v) {
    if constexpr (PRK_L2_YSTORE == 0)
        asm volatile("st.global.cs.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
    else if constexpr (PRK_L2_YSTORE == 4)
        asm volatile("st.global.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
    else
        asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v),
                     "l"(l2_policy<PRK_L2_YSTORE>()) : "memory");
}

__device__ __forceinline__ float ld_relaxed(const float* p) {
    float v;
    asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ void st_relaxed(float* p, float v) {
    asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v));
}

// Relaxed accesses of the in-place vectors with an L2 policy of class P.
template <int P>
__device__ __forceinline__ float ld_relaxed_p(const float* p) {
    if constexpr (P == 0) {
        return ld_relaxed(p);
    } else {
        float v;
        asm volatile("ld.relaxed.gpu.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p),
                     "l"(l2_policy<P>()));
        return v;
    }
}

template <int P>
__device__ __forceinline__ void st_relaxed_p(float* p, float v) {
    if constexpr (P == 0)
        st_relaxed(p, v);
    else
        asm volatile("st.relaxed.gpu.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v),
                     "l"(l2_policy<P>()));
}

// Weak load that may be served by L1 (possibly an older value of a location
// other SMs write; see the barrier-free kernel for the bound on its age).
__device__ __forceinline__ float ld_weak_l1(const float* p) {
    float v;
    asm volatile("ld.global.ca.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ float4 ld_relaxed4(const float* p) {
    float4 v;
    asm volatile("ld.relaxed.gpu.global.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
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

// Solve-state scalars every thread needs, read once per block by thread 0 and
// broadcast through shared memory: a load of the same word by every thread of
// every block would queue hundreds of thousands of requests on one L2 slice.
struct StateView {
    double d, D, inv_n, t_sum, scale;
    int32_t done, iter, implicit;
};

__device__ __forceinline__ StateView block_state(const SolveState* st) {
    __shared__ StateView sv;
    if (threadIdx.x == 0) {
        sv.done = *(const volatile int32_t*)&st->done;
        sv.iter = *(const volatile int32_t*)&st->iter;
        sv.implicit = st->implicit;
        sv.d = st->d;
        sv.D = st->D;
        sv.inv_n = st->inv_n;
        sv.t_sum = st->t_sum;
        sv.scale = st->scale;
    }
    __syncthreads();
    StateView v = sv;
    __syncthreads();
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
    int32_t lane_mode = kDefaultLaneMode;   // lanes per light row: see light_lanes_log2
};

// Lanes per row of a light tile (log2).  Mode 0: by degree class, 2^min(k, 5)
// lanes for rows of degree in [2^k, 2^(k+1)) (tile.kind).  Mode 1: by the
// tile's row count, the largest power of two g <= 32 with rows <= 2 kBlock / g,
// so the block's groups cover the tile in one pass of two rows per group
// where they can (a tile of more rows takes ceil(rows / 2 kBlock) passes with
// g = 1), and each lane walks about edges / kBlock of the tile's edges.
__device__ __forceinline__ int light_lanes_log2(const Tile& tile, int mode) {
    if (mode == 0) return tile.kind;
    const int rows = tile.row_end - tile.row_begin;
    const int per = rows > 0 ? (2 * kBlock) / rows : 32;
    if (per <= 1) return 0;
    return 31 - __clz((unsigned)(per < 32 ? per : 32));
}

// This lane's share of the sums of two rows: edges b0, b0 + g, ... below e0
// and b1, b1 + g, ... below e1 (b = the row's first edge + the lane's index
// in its group), kU edges of each row per step, so that up to 2 kU gathers
// are in flight; with kU = 4 each step adds ((v0 + v1) + (v2 + v3)) per row.
// col(p) is the source id of edge p.  Every synchronous light-tile path sums
// through this routine with kU = 4, so they agree bit for bit on a row's sum;
// the barrier-free kernel, compiled for fewer registers, takes kU = 2.
template <bool kInPlace, int kU = 4, bool kPrefetch = kInPlace, typename OffT, typename ColAt, typename YT>
__device__ __forceinline__ void gather_row_pair(const ColAt& col, OffT b0, OffT e0, OffT b1, OffT e1, int g,
                                                const YT* y, const RowCtx& c, float& s0, float& s1);

template <bool kInPlace>
struct Mem;

template <>
struct Mem<false> {
    static __device__ __forceinline__ float gather(const float* y, int32_t c, const RowCtx& x) {
        return c < x.hot_n ? x.hot_sm[c] : ld_gather(y, c, x.hot);
    }
    // BF16 quotients (the correction sweeps of the synchronous solver): the hub
    // prefix through L1, the rest from L2, as ld_gather's default policy
    static __device__ __forceinline__ float gather(const __nv_bfloat16* y, int32_t c, const RowCtx& x) {
        const int32_t count = x.hot & 0x0fffffff;
        const unsigned short* p = reinterpret_cast<const unsigned short*>(y) + c;
        const unsigned short h = c < count ? __ldg(p) : __ldcg(p);
        return __uint_as_float((uint32_t)h << 16);
    }
    static __device__ __forceinline__ float load_x(const float* p) { return ld_stream(p); }
    static __device__ __forceinline__ void store_x(float* p, float v) { st_stream(p, v); }
    static __device__ __forceinline__ void store_y(float* p, float v) { st_y(p, v); }
};

template <>
struct Mem<true> {
    static __device__ __forceinline__ float gather(const float* y, int32_t c, const RowCtx& x) {
        if (c < x.hot_n) return x.hot_sm[c];
        if (c < x.hot) return ld_weak_l1(y + c);
        return ld_relaxed_p<PRK_L2_GATHER>(y + c);
    }
    static __device__ __forceinline__ float load_x(const float* p) { return ld_relaxed_p<PRK_L2_STREAM>(p); }
    static __device__ __forceinline__ void store_x(float* p, float v) { st_relaxed_p<PRK_L2_STREAM>(p, v); }
    static __device__ __forceinline__ void store_y(float* p, float v) { st_relaxed_p<PRK_L2_GATHER>(p, v); }
};

template <bool kInPlace, int kU, bool kPrefetch, typename OffT, typename ColAt, typename YT>
__device__ __forceinline__ void gather_row_pair(const ColAt& col, OffT b0, OffT e0, OffT b1, OffT e1, int g,
                                                const YT* y, const RowCtx& c, float& s0, float& s1) {
    static_assert(kU == 2 || kU == 4, "two or four edges per row per step");
    if constexpr (kPrefetch) {
        // column indices read from global memory: the next step's are loaded
        // while this step's gathers are in flight
        int32_t c0[kU], c1[kU];
#pragma unroll
        for (int j = 0; j < kU; ++j) {
            c0[j] = b0 + j * g < e0 ? col(b0 + j * g) : -1;
            c1[j] = b1 + j * g < e1 ? col(b1 + j * g) : -1;
        }
        while (b0 < e0 || b1 < e1) {
            float v0[kU], v1[kU];
#pragma unroll
            for (int j = 0; j < kU; ++j) {
                v0[j] = c0[j] >= 0 ? Mem<kInPlace>::gather(y, c0[j], c) : 0.f;
                v1[j] = c1[j] >= 0 ? Mem<kInPlace>::gather(y, c1[j], c) : 0.f;
            }
            b0 += kU * g;
            b1 += kU * g;
#pragma unroll
            for (int j = 0; j < kU; ++j) {
                c0[j] = b0 + j * g < e0 ? col(b0 + j * g) : -1;
                c1[j] = b1 + j * g < e1 ? col(b1 + j * g) : -1;
            }
            if constexpr (kU == 4) {
                s0 += (v0[0] + v0[1]) + (v0[2] + v0[3]);
                s1 += (v1[0] + v1[1]) + (v1[2] + v1[3]);
            } else {
                s0 += v0[0] + v0[1];
                s1 += v1[0] + v1[1];
            }
        }
        return;
    }
    while (b0 < e0 || b1 < e1) {
        int32_t c0[kU], c1[kU];
#pragma unroll
        for (int j = 0; j < kU; ++j) {
            c0[j] = b0 + j * g < e0 ? col(b0 + j * g) : -1;
            c1[j] = b1 + j * g < e1 ? col(b1 + j * g) : -1;
        }
        float v0[kU], v1[kU];
#pragma unroll
        for (int j = 0; j < kU; ++j) {
            v0[j] = c0[j] >= 0 ? Mem<kInPlace>::gather(y, c0[j], c) : 0.f;
            v1[j] = c1[j] >= 0 ? Mem<kInPlace>::gather(y, c1[j], c) : 0.f;
        }
        if constexpr (kU == 4) {
            s0 += (v0[0] + v0[1]) + (v0[2] + v0[3]);
            s1 += (v1[0] + v1[1]) + (v1[2] + v1[3]);
        } else {
            s0 += v0[0] + v0[1];
            s1 += v1[0] + v1[1];
        }
        b0 += kU * g;
        b1 += kU * g;
    }
}

// Per-thread accumulators, both Kahan-compensated in FP32 (FP64 arithmetic
// is a slow pipe on this GPU) and handed to the FP64 cross-thread reduction:
// (r, rc) the L1 change; (m, c) the mass the kernel tracks -- the new
// dangling mass (synchronous form) or the change of the non-dangling mass
// (in-place form).
struct Acc {
    float r = 0.f;
    float rc = 0.f;
    float m = 0.f;
    float c = 0.f;
    float dd = 0.f;   // in-place form: change of the dangling mass (diagnostic form only)
    __device__ __forceinline__ void kahan(float v) {
        const float yk = v - c;
        const float tk = m + yk;
        c = (tk - m) - yk;
        m = tk;
    }
    __device__ __forceinline__ void add_r(float v) {
        const float yk = v - rc;
        const float tk = r + yk;
        rc = (tk - r) - yk;
        r = tk;
    }
    __device__ __forceinline__ double mass() const { return (double)m - (double)c; }
    __device__ __forceinline__ double resid() const { return (double)r - (double)rc; }
};

// Compensated FP32 sum of one thread's elements (FP32 adds only: FP64
// arithmetic is a slow pipe on this GPU); value() hands it to the FP64
// cross-thread reduction.
struct KahanF {
    float s = 0.f;
    float c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <bool kUniform, bool kInPlace>
__device__ __forceinline__ void row_update(int64_t r, float s, float xo, float inv, float tv,
                                           const RowCtx& c, float* x_out, float* y_out, Acc& acc) {
    const float base = kUniform ? c.base : fmaf(c.one_m_d, tv, c.d_share);
    const float xn = fmaf(c.d, s, base);
    Mem<kInPlace>::store_x(x_out + r, xn);
    Mem<kInPlace>::store_y(y_out + r, xn * inv);
    acc.add_r(fabsf(xn - xo));
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
// Light rows of one degree class: groups of g = 2^light_lanes_log2 lanes
// gather one row each, two rows per group at a time (rows r and r + 256/g),
// each lane up to four edges of each row per step (gather_row_pair);
// coalesced colidx reads within the group; shuffle reduction; the group's
// first lane updates both rows.
template <typename IdxT, bool kUniform, bool kInPlace>
__device__ __forceinline__ void process_light_tile(const Tile& tile, const void* rowptr,
                                                   const int32_t* colidx, const float* inv_out,
                                                   const float* teleport, const float* x_in,
                                                   const float* y_in, float* x_out, float* y_out,
                                                   const RowCtx& c, Acc& acc, int tid) {
    const int lg = light_lanes_log2(tile, c.lane_mode);
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
        gather_row_pair<kInPlace, kInPlace ? PRK_NB_UNROLL : 4, true>(
            [&](int64_t p) { return ld_col<kInPlace ? PRK_NB_COL_L1 : PRK_SYNC_COL_L1>(colidx + p); }, b[0] + gl, e[0],
            b[1] + gl, e[1], g, y_in, c, s[0], s[1]);
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

// ---- loop perforation (Alg. 5), synchronous form --------------------------
// Copies of the row-update paths above for the perforated solve, kept apart so
// the plain paths compile exactly as before.  A frozen row is copied forward
// (its rank still feeds the gathers and, if dangling, the dangling mass); a
// row whose update changed it by a nonzero amount below eps freezes.
struct Perf {
    uint8_t* frozen;   // 1 = row no longer recomputed
    float eps;
};

__device__ __forceinline__ void perf_copy(int64_t r, float xo, float yo, float inv, float* x_out, float* y_out,
                                          Acc& acc) {
    st_stream(x_out + r, xo);
    st_y(y_out + r, yo);
    if (inv == 0.f) acc.kahan(xo);
}

template <bool kUniform>
__device__ __forceinline__ void perf_update(int64_t r, float s, float xo, float inv, float tv, const RowCtx& c,
                                            const Perf& p, float* x_out, float* y_out, Acc& acc) {
    const float base = kUniform ? c.base : fmaf(c.one_m_d, tv, c.d_share);
    const float xn = fmaf(c.d, s, base);
    st_stream(x_out + r, xn);
    st_y(y_out + r, xn * inv);
    acc.add_r(fabsf(xn - xo));
    if (inv == 0.f) acc.kahan(xn);
    const float ch = fabsf(xn - xo);
    if (ch != 0.f && ch < p.eps) p.frozen[r] = 1;
}

template <bool kUniform>
__device__ __forceinline__ void perf_zero_tile(const Tile& tile, const float* inv_out, const float* teleport,
                                               const float* x_in, const float* y_in, float* x_out, float* y_out,
                                               const RowCtx& c, const Perf& p, Acc& acc, int tid) {
    for (int64_t r = tile.row_begin + tid; r < tile.row_end; r += kBlock) {
        const float xo = ld_stream(x_in + r);
        const float inv = ld_stream(inv_out + r);
        if (p.frozen[r]) {
            perf_copy(r, xo, ld_stream(y_in + r), inv, x_out, y_out, acc);
            continue;
        }
        const float tv = kUniform ? 0.f : ld_stream(teleport + r);
        perf_update<kUniform>(r, 0.f, xo, inv, tv, c, p, x_out, y_out, acc);
    }
}

// process_light_tile with frozen rows skipped (Jacobi buffers only).
template <typename IdxT, bool kUniform>
__device__ __forceinline__ void perf_light_tile(const Tile& tile, const void* rowptr, const int32_t* colidx,
                                                const float* inv_out, const float* teleport, const float* x_in,
                                                const float* y_in, float* x_out, float* y_out, const RowCtx& c,
                                                const Perf& p, Acc& acc, int tid) {
    const int lg = light_lanes_log2(tile, c.lane_mode);
    const int g = 1 << lg;
    const int rpp = kBlock >> lg;
    const int grp = tid >> lg;
    const int gl = tid & (g - 1);
    for (int64_t r0 = tile.row_begin; r0 < tile.row_end; r0 += 2 * rpp) {
        int64_t rr[2];
        bool act[2], fz[2];
        int64_t b[2], e[2];
        float xo[2], inv[2], tv[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            rr[q] = r0 + q * rpp + grp;
            act[q] = rr[q] < tile.row_end;
            fz[q] = act[q] && p.frozen[rr[q]] != 0;   // frozen rows gather nothing
            b[q] = e[q] = 0;
            xo[q] = inv[q] = tv[q] = 0.f;
            if (act[q]) {
                if (!fz[q]) {
                    b[q] = row_at<IdxT>(rowptr, rr[q]);
                    e[q] = row_at<IdxT>(rowptr, rr[q] + 1);
                }
                if (gl == 0) {
                    xo[q] = ld_stream(x_in + rr[q]);
                    inv[q] = ld_stream(inv_out + rr[q]);
                    if (!kUniform) tv[q] = ld_stream(teleport + rr[q]);
                }
            }
        }
        float s[2] = {0.f, 0.f};
        gather_row_pair<false, 4, true>([&](int64_t q) { return ld_col<PRK_SYNC_COL_L1>(colidx + q); }, b[0] + gl, e[0], b[1] + gl, e[1],
                               g, y_in, c, s[0], s[1]);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1)
            if (o < g) {
                s[0] += __shfl_xor_sync(0xffffffffu, s[0], o);
                s[1] += __shfl_xor_sync(0xffffffffu, s[1], o);
            }
        if (gl == 0) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (!act[q]) continue;
                if (fz[q]) perf_copy(rr[q], xo[q], ld_stream(y_in + rr[q]), inv[q], x_out, y_out, acc);
                else perf_update<kUniform>(rr[q], s[q], xo[q], inv[q], tv[q], c, p, x_out, y_out, acc);
            }
        }
    }
}

// Staging area of process_staged_tile: the gathered y values of one light
// tile, indexed from the tile's first edge rounded down to a multiple of 4.
constexpr int kStageFloats = kTileEdgesMax + 4;

// Light rows of one degree class, edge-parallel: the 256 threads of the group
// stream the tile's colidx range with 16-byte loads and issue every gather of
// the tile without waiting on any row (up to sixteen in flight per thread),
// park the values in shared memory, and only then reduce row by row (groups
// of g = 2^tile.kind lanes, consecutive lanes on consecutive values).  Every
// gather of a tile is independent of the others, so the tile costs three
// memory latencies (offsets, colidx, y) instead of three per row pair.
// `stage` holds kStageFloats floats, 16-byte aligned; the caller's group must
// be a whole block (the routine uses __syncthreads).  Returns false -- and
// touches nothing -- if the tile does not fit the staging area, which the
// tiling at set-up rules out.
template <typename IdxT, bool kUniform, bool kInPlace>
__device__ __forceinline__ bool process_staged_tile(const Tile& tile, const void* rowptr,
                                                    const int32_t* colidx, const float* inv_out,
                                                    const float* teleport, const float* x_in,
                                                    const float* y_in, float* x_out, float* y_out,
                                                    const RowCtx& c, Acc& acc, int tid, float* stage) {
    const int64_t e0 = row_at<IdxT>(rowptr, tile.row_begin);
    const int64_t e1 = row_at<IdxT>(rowptr, tile.row_end);
    const int64_t a0 = e0 & ~(int64_t)3;   // 16-byte aligned start of the colidx range
    if (e1 - a0 > kStageFloats) return false;
    float4* st4 = reinterpret_cast<float4*>(stage);
    for (int64_t base = a0; base < e1; base += 16 * kBlock) {
        int4 cv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t p = base + 4 * (kBlock * j + tid);
            cv[j] = p < e1 ? ld_stream4(colidx + p) : make_int4(0, 0, 0, 0);
        }
        float4 v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t p = base + 4 * (kBlock * j + tid);
            v[j].x = (p + 0 >= e0 && p + 0 < e1) ? Mem<kInPlace>::gather(y_in, cv[j].x, c) : 0.f;
            v[j].y = (p + 1 >= e0 && p + 1 < e1) ? Mem<kInPlace>::gather(y_in, cv[j].y, c) : 0.f;
            v[j].z = (p + 2 >= e0 && p + 2 < e1) ? Mem<kInPlace>::gather(y_in, cv[j].z, c) : 0.f;
            v[j].w = (p + 3 >= e0 && p + 3 < e1) ? Mem<kInPlace>::gather(y_in, cv[j].w, c) : 0.f;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t p = base + 4 * (kBlock * j + tid);
            if (p < e1) st4[(p - a0) >> 2] = v[j];
        }
    }
    __syncthreads();
    const int lg = tile.kind;
    const int g = 1 << lg;
    const int rpp = kBlock >> lg;
    const int gl = tid & (g - 1);
    // uniform trip count over the block: every lane reaches the shuffles
    for (int64_t r0 = tile.row_begin; r0 < tile.row_end; r0 += rpp) {
        const int64_t r = r0 + (tid >> lg);
        const bool act = r < tile.row_end;
        int32_t b = 0, e = 0;
        if (act) {
            b = (int32_t)(row_at<IdxT>(rowptr, r) - a0);
            e = (int32_t)(row_at<IdxT>(rowptr, r + 1) - a0);
        }
        float xo = 0.f, inv = 0.f, tv = 0.f;
        if (act && gl == 0) {
            xo = Mem<kInPlace>::load_x(x_in + r);
            inv = ld_stream(inv_out + r);
            if (!kUniform) tv = ld_stream(teleport + r);
        }
        float sum = 0.f;
        for (int32_t k = b + gl; k < e; k += g) sum += stage[k];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1)
            if (o < g) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (act && gl == 0) row_update<kUniform, kInPlace>(r, sum, xo, inv, tv, c, x_out, y_out, acc);
    }
    __syncthreads();   // the staging area is reused by the next tile
    return true;
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
