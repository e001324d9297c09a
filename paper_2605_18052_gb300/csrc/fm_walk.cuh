// Device building blocks shared by the streaming kernels: programmatic-dependent-launch
// helpers, evict-first streaming loads, the two keypoint storage formats and the warp-range
// walk over the pair-sorted point pairs.
#pragma once

#include "fm_internal.cuh"

namespace fm {

// ---- programmatic dependent launch --------------------------------------------------------------
// The three kernels of an optimiser iteration are launched with programmatic stream
// serialisation, so a kernel's CTAs can be scheduled while its predecessor drains. Every kernel
// waits (griddepcontrol.wait) before it reads anything its predecessor writes, and lets its own
// dependents launch (griddepcontrol.launch_dependents) only after that wait: when a kernel
// starts, the kernel two places before it has completed, so reads of older data before the
// wait are safe. Both instructions are no-ops for a normal launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
static cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s,
                            bool pdl, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// ---- streaming loads: 16 B vectors, no L1 allocation, evict-first in L2 -----------------------
// The point-pair arrays are read once per pass and are 10-100x larger than L2; marking them
// evict-first keeps the small per-pair and per-camera tables (geometry, partial sums, camera
// lists, poses) resident in L2 across passes, which the latency-bound per-camera step needs.
__device__ __forceinline__ uint64_t evict_first_policy() {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ uint4 ld_stream_v4(const void *p, uint64_t pol) {
    uint4 r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.L2::256B.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(p), "l"(pol));
    return r;
}

__device__ __forceinline__ unsigned ld_stream_u32(const void *p, uint64_t pol) {
    unsigned r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "l"(pol));
    return r;
}

// ---- storage formats -----------------------------------------------------------------------------
template <int STORE>
struct Fmt;

// FP32: one point pair per lane per group, float4 (x1, y1, x2, y2) + float weight
template <>
struct Fmt<FM_STORE_FP32> {
    static constexpr int PPL = 1;
    struct Raw {
        uint4 kp;
        unsigned w;
    };
    __device__ static Raw load(const DevProblem &d, int64_t q, bool need_w, uint64_t pol) {
        Raw r;
        r.kp = ld_stream_v4(static_cast<const float4 *>(d.kp) + q, pol);
        r.w = need_w ? ld_stream_u32(static_cast<const float *>(d.w) + q, pol) : 0u;
        return r;
    }
    __device__ static void get(const Raw &r, int, float &x1, float &y1, float &x2, float &y2,
                               float &w) {
        x1 = __uint_as_float(r.kp.x);
        y1 = __uint_as_float(r.kp.y);
        x2 = __uint_as_float(r.kp.z);
        y2 = __uint_as_float(r.kp.w);
        w = __uint_as_float(r.w);
    }
};

// FP16: two point pairs per lane per group: 16 B = {o1, o2} of pp q and q+1 as half2 pairs,
// weights as one half2 (scaled by s)
template <>
struct Fmt<FM_STORE_FP16> {
    static constexpr int PPL = 2;
    struct Raw {
        uint4 kp;
        unsigned w;
    };
    __device__ static Raw load(const DevProblem &d, int64_t q, bool need_w, uint64_t pol) {
        Raw r;
        r.kp = ld_stream_v4(static_cast<const uint2 *>(d.kp) + q, pol);
        r.w = need_w ? ld_stream_u32(static_cast<const __half *>(d.w) + q, pol) : 0u;
        return r;
    }
    __device__ static void get(const Raw &r, int k, float &x1, float &y1, float &x2, float &y2,
                               float &w) {
        const unsigned a = k == 0 ? r.kp.x : r.kp.z;
        const unsigned b = k == 0 ? r.kp.y : r.kp.w;
        const float2 fa = __half22float2(*reinterpret_cast<const __half2 *>(&a));
        const float2 fb = __half22float2(*reinterpret_cast<const __half2 *>(&b));
        x1 = fa.x;
        y1 = fa.y;
        x2 = fb.x;
        y2 = fb.y;
        const float2 fw = __half22float2(*reinterpret_cast<const __half2 *>(&r.w));
        w = k == 0 ? fw.x : fw.y;
    }
};

__device__ __forceinline__ void load_E(const float *geo, int n, float *E) {
    const float4 *g = reinterpret_cast<const float4 *>(geo + (size_t)n * GEO);
    const float4 a = g[0], b = g[1];
    const float c = geo[(size_t)n * GEO + 8];
    E[0] = a.x; E[1] = a.y; E[2] = a.z; E[3] = a.w;
    E[4] = b.x; E[5] = b.y; E[6] = b.z; E[7] = b.w;
    E[8] = c;
}

// epsilon = o2^T E' o1 with o = (x, y, 1)
__device__ __forceinline__ float epi(const float *E, float x1, float y1, float x2, float y2) {
    const float r0 = fmaf(E[0], x1, fmaf(E[1], y1, E[2]));
    const float r1 = fmaf(E[3], x1, fmaf(E[4], y1, E[5]));
    const float r2 = fmaf(E[6], x1, fmaf(E[7], y1, E[8]));
    return fmaf(x2, r0, fmaf(y2, r1, r2));
}

// ---- the streaming walk ------------------------------------------------------------------------
// Warp `r` streams point pairs [r*WR, min((r+1)*WR, n_pp)). Lane l of group g handles PPL
// consecutive point pairs at g*32*PPL + l*PPL, so every load instruction of the warp reads one
// contiguous 512 B block. The image pair changes only at sorted boundaries: a group that lies
// inside the current pair takes the fast path; a group that crosses a boundary is processed in
// passes, one pass per image pair it meets, and `body.segment_end` closes each finished pair.
template <int STORE, bool NEED_W, class Body>
__device__ __forceinline__ void walk_range(const DevProblem &d, int r, int lane, Body &body) {
    using F = Fmt<STORE>;
    constexpr int PPL = F::PPL;
    constexpr int GROUP = 32 * PPL;
    constexpr int U = 4;
    static_assert(WR % (U * GROUP) == 0, "range must be whole unrolled groups");
    const int64_t p_begin = (int64_t)r * WR;
    const int64_t p_end = min(p_begin + (int64_t)WR, d.n_pp);
    int seg = d.range_pair[r];
    int64_t seg_end = d.pair_off[seg + 1];
    float E[9];
    load_E(d.geo, seg, E);
    body.segment_begin(seg);
    const uint64_t pol = evict_first_policy();
    for (int64_t g0 = p_begin; g0 < p_end; g0 += U * GROUP) {
        typename F::Raw raw[U];
#pragma unroll
        for (int u = 0; u < U; ++u) raw[u] = F::load(d, g0 + u * GROUP + lane * PPL, NEED_W, pol);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t gb = g0 + u * GROUP;
            if (gb >= p_end) break;
            if (gb + GROUP <= seg_end) {
#pragma unroll
                for (int k = 0; k < PPL; ++k) {
                    float x1, y1, x2, y2, w;
                    F::get(raw[u], k, x1, y1, x2, y2, w);
                    body.point(k, epi(E, x1, y1, x2, y2), x1, y1, x2, y2, w);
                }
            } else {
                int64_t lo = gb;
                const int64_t g_end = min(gb + GROUP, p_end);
                while (true) {
                    const int64_t hi = min(seg_end, p_end);
#pragma unroll
                    for (int k = 0; k < PPL; ++k) {
                        const int64_t q = gb + lane * PPL + k;
                        if (q >= lo && q < hi) {
                            float x1, y1, x2, y2, w;
                            F::get(raw[u], k, x1, y1, x2, y2, w);
                            body.point(k, epi(E, x1, y1, x2, y2), x1, y1, x2, y2, w);
                        }
                    }
                    if (seg_end >= g_end) break;
                    body.segment_end(seg, r, lane, false);
                    lo = seg_end;
                    ++seg;
                    seg_end = d.pair_off[seg + 1];
                    load_E(d.geo, seg, E);
                    body.segment_begin(seg);
                }
            }
            body.group_done(gb, p_end, lane);
        }
    }
    body.segment_end(seg, r, lane, true);
}

}  // namespace fm
