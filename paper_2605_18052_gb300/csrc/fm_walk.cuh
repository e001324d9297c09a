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

// Explicitly rounded arithmetic: the compiler never contracts or reassociates these, so a
// formula written with them gives the same bits in every kernel it is inlined into (the fused
// optimiser step and the camera-step kernel must agree bit for bit).
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
// a0 b0 + a1 b1 + a2 b2 as fma(a2, b2, fma(a1, b1, a0 b0))
__device__ __forceinline__ float rdot3(float a0, float b0, float a1, float b1, float a2, float b2) {
    return __fmaf_rn(a2, b2, __fmaf_rn(a1, b1, __fmul_rn(a0, b0)));
}
__device__ __forceinline__ double rdot3(double a0, double b0, double a1, double b1, double a2, double b2) {
    return __fma_rn(a2, b2, __fma_rn(a1, b1, __dmul_rn(a0, b0)));
}

// epsilon = o2^T E' o1 with o = (x, y, 1)
__device__ __forceinline__ float epi(const float *E, float x1, float y1, float x2, float y2) {
    const float r0 = fmaf(E[0], x1, fmaf(E[1], y1, E[2]));
    const float r1 = fmaf(E[3], x1, fmaf(E[4], y1, E[5]));
    const float r2 = fmaf(E[6], x1, fmaf(E[7], y1, E[8]));
    return fmaf(x2, r0, fmaf(y2, r1, r2));
}

// IRLS weight 1/max(|eps|, delta) of a kept point pair. The fast reciprocal (within 2 ulp of
// the rounded quotient; its argument is at least delta, far from the ranges where it differs
// more) is used by every kernel that computes weights, so they agree with each other bit for
// bit; against the exact quotient the difference is far inside the weight tolerance, which is
// set by the residual's FP32 error.
__device__ __forceinline__ float irls_weight(float a, float delta) { return __fdividef(1.0f, fmaxf(a, delta)); }

// *p += v at GPU scope with acquire-release semantics; returns the old value
__device__ __forceinline__ unsigned atomic_add_acq_rel(unsigned *p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// ---- the streaming walk ------------------------------------------------------------------------
// Warp `r` streams point pairs [r*WR, min((r+1)*WR, n_pp)). Lane l of group g handles PPL
// consecutive point pairs at g*32*PPL + l*PPL, so every load instruction of the warp reads one
// contiguous 512 B block. The image pair changes only at sorted boundaries: a group that lies
// inside the current pair takes the fast path; a group that crosses a boundary is processed in
// passes, one pass per image pair it meets, and `body.segment_end` closes each finished pair.
// U groups are loaded before any is processed (loads in flight per warp).
template <int STORE, bool NEED_W, class Body, int U = 4>
__device__ __forceinline__ void walk_range(const DevProblem &d, int r, int lane, Body &body) {
    using F = Fmt<STORE>;
    constexpr int PPL = F::PPL;
    constexpr int GROUP = 32 * PPL;
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

// ---- packed FP32 pairs -----------------------------------------------------------------------------
// Two lanes of FP32 arithmetic in one instruction (fma/mul/add.rn.f32x2): each lane rounds once,
// exactly as the scalar operation, so results keep their bits while the streaming passes, which
// are close to bound by instruction issue, issue one instruction where they issued two.
__device__ __forceinline__ void fma2(float &d0, float &d1, float a0, float a1, float b0, float b1) {
    asm("{\n\t.reg .b64 ra, rb, rc;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rc, {%0, %1};\n\t"
        "fma.rn.f32x2 rc, ra, rb, rc;\n\t"
        "mov.b64 {%0, %1}, rc;\n\t}"
        : "+f"(d0), "+f"(d1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}
__device__ __forceinline__ void mul2(float &d0, float &d1, float a0, float a1, float b0, float b1) {
    asm("{\n\t.reg .b64 ra, rb, rc;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rc, ra, rb;\n\t"
        "mov.b64 {%0, %1}, rc;\n\t}"
        : "=f"(d0), "=f"(d1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}
// d0 += b0, d1 += b1
__device__ __forceinline__ void add2(float &d0, float &d1, float b0, float b1) {
    asm("{\n\t.reg .b64 rb, rc;\n\t"
        "mov.b64 rb, {%2, %3};\n\t"
        "mov.b64 rc, {%0, %1};\n\t"
        "add.rn.f32x2 rc, rc, rb;\n\t"
        "mov.b64 {%0, %1}, rc;\n\t}"
        : "+f"(d0), "+f"(d1)
        : "f"(b0), "f"(b1));
}

// ---- loss + adjoint -----------------------------------------------------------------------------
// acc[0..8] = sum s * o2 o1^T (row-major), acc[9] = sum of loss terms, with s = w*eps (IRLS,
// the factor 2/Z is applied later) or sign(eps) (L1). Each finished (image pair, warp range)
// intersection is reduced by a warp butterfly into its own slot n + r; no atomics, no fences,
// a fixed summation order.
template <int MODE>
struct LossBody {
    const DevProblem &d;
    float acc[10];
    __device__ explicit LossBody(const DevProblem &dd) : d(dd) {
#pragma unroll
        for (int i = 0; i < 10; ++i) acc[i] = 0.f;
    }
    __device__ __forceinline__ void point(int, float e, float x1, float y1, float x2, float y2,
                                          float w) {
        float s;
        if (MODE == MODE_LOSS_IRLS) {
            s = w * e;
            acc[9] = fmaf(s, e, acc[9]);
        } else {
            s = e > 0.f ? 1.f : (e < 0.f ? -1.f : 0.f);
            acc[9] += fabsf(e);
        }
        float a, b;   // s x2, s y2
        mul2(a, b, s, s, x2, y2);
        fma2(acc[0], acc[1], a, a, x1, y1);
        add2(acc[2], acc[5], a, b);
        fma2(acc[3], acc[4], b, b, x1, y1);
        fma2(acc[6], acc[7], s, s, x1, y1);
        acc[8] += s;
    }
    __device__ __forceinline__ void segment_begin(int) {}
    __device__ __forceinline__ void segment_end(int seg, int r, int lane, bool) {
#pragma unroll
        for (int i = 0; i < 10; ++i) {
            float v = acc[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            acc[i] = v;
        }
        if (lane == 0) {
            float4 *s = reinterpret_cast<float4 *>(d.slots + (size_t)(seg + r) * SLOT);
            s[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
            s[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
            s[2] = make_float4(acc[8], acc[9], 0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < 10; ++i) acc[i] = 0.f;
    }
    __device__ __forceinline__ void group_done(int64_t, int64_t, int) {}
};

// ---- per pair: relative pose and folded essential matrix ------------------------------------------
// camera record: R (9), centre as hi (3) + lo (3) floats, s = scale of the normalised keypoints.
// Read at L2 (ld.global.cg): a record may have been written by another block of the same
// launch (the camera step's geometry phase), and L1 is not coherent across SMs.
__device__ __forceinline__ void load_camrec(const float *rec, float *R, float *hi, float *lo, float &s) {
    const float4 *v = reinterpret_cast<const float4 *>(rec);
    const float4 a = __ldcg(v), b = __ldcg(v + 1), c = __ldcg(v + 2), e = __ldcg(v + 3);
    R[0] = a.x; R[1] = a.y; R[2] = a.z; R[3] = a.w;
    R[4] = b.x; R[5] = b.y; R[6] = b.z; R[7] = b.w;
    R[8] = c.x;
    hi[0] = c.y; hi[1] = c.z; hi[2] = c.w;
    lo[0] = e.x; lo[1] = e.y; lo[2] = e.z;
    s = e.w;
}


// Relative pose and centroid-folded matrix of the pair (i, j) from the camera records `cam`
// into the geometry record g (registers): E'_n = T_j^T S_j [t_n/|t_n|]_x R_n S_i T_i,
// R_n = R_j R_i^T, t_n = R_j (c_i - c_j), S = diag(s, s, 1) the cameras' keypoint scales
// (focal refinement; 1 otherwise, which leaves the essential matrix unchanged). Returns false
// (and g with 1/|t_n| = 0) when the baseline is degenerate.
// Record: 0..8 E', 9..17 R_n, 18..20 t_n, 21 1/|t_n|, 22..23 centroid i, 24..32 R_j,
// 33..34 centroid j, 35 s_i, 36 s_j, 37..39 0.
__device__ __forceinline__ bool pair_geometry_regs(const float *cam, const float2 *cen, int i, int j, float *g) {
    float Ri[9], Rj[9], hi_i[3], lo_i[3], hi_j[3], lo_j[3], dc[3], s_i, s_j;
    load_camrec(cam + (size_t)i * CAMREC, Ri, hi_i, lo_i, s_i);
    load_camrec(cam + (size_t)j * CAMREC, Rj, hi_j, lo_j, s_j);
    // c_i - c_j from the two-float representation: the high parts of nearby centres
    // subtract exactly, so the baseline keeps FP32 relative accuracy far from the origin
#pragma unroll
    for (int q = 0; q < 3; ++q) dc[q] = (hi_i[q] - hi_j[q]) + (lo_i[q] - lo_j[q]);
    float Rn[9], tn[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int b = 0; b < 3; ++b)
            Rn[3 * a + b] = rdot3(Rj[3 * a], Ri[3 * b], Rj[3 * a + 1], Ri[3 * b + 1], Rj[3 * a + 2], Ri[3 * b + 2]);
        tn[a] = rdot3(Rj[3 * a], dc[0], Rj[3 * a + 1], dc[1], Rj[3 * a + 2], dc[2]);
    }
    const float nt2 = rdot3(tn[0], tn[0], tn[1], tn[1], tn[2], tn[2]);
    // a baseline below 1e-10 of the centres' magnitude is rounding noise: its direction,
    // and so E_n, is undefined
    float cmax = 1.f;
#pragma unroll
    for (int q = 0; q < 3; ++q) cmax = fmaxf(cmax, fmaxf(fabsf(hi_i[q]), fabsf(hi_j[q])));
    const float floor2 = 1e-20f * cmax * cmax;
    const bool ok = nt2 > floor2 && isfinite(nt2);
    const float inv = ok ? __fdiv_rn(1.0f, __fsqrt_rn(nt2)) : 0.f;
    const float th[3] = {rmul(tn[0], inv), rmul(tn[1], inv), rmul(tn[2], inv)};
    // E = [th]_x R_n, then F = S_j E S_i
    float E[9];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        E[b] = rfma(th[1], Rn[6 + b], rmul(-th[2], Rn[3 + b]));
        E[3 + b] = rfma(-th[0], Rn[6 + b], rmul(th[2], Rn[b]));
        E[6 + b] = rfma(th[0], Rn[3 + b], rmul(-th[1], Rn[b]));
    }
    {
        const float si[3] = {s_i, s_i, 1.f}, sj[3] = {s_j, s_j, 1.f};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) E[3 * a + b] = rmul(rmul(E[3 * a + b], sj[a]), si[b]);
    }
    // E' = T_j^T E T_i with T = [[1,0,cx],[0,1,cy],[0,0,1]] (keypoints stored as offsets o = x - c)
    const float2 cen_i = cen[i], cen_j = cen[j];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        g[3 * a] = E[3 * a];
        g[3 * a + 1] = E[3 * a + 1];
        g[3 * a + 2] = rfma(E[3 * a + 1], cen_i.y, rfma(E[3 * a], cen_i.x, E[3 * a + 2]));
    }
    const float m20 = E[6], m21 = E[7], m22 = rfma(E[7], cen_i.y, rfma(E[6], cen_i.x, E[8]));
    g[6] = rfma(cen_j.y, g[3], rfma(cen_j.x, g[0], m20));
    g[7] = rfma(cen_j.y, g[4], rfma(cen_j.x, g[1], m21));
    g[8] = rfma(cen_j.y, g[5], rfma(cen_j.x, g[2], m22));
#pragma unroll
    for (int k = 0; k < 9; ++k) g[9 + k] = Rn[k];
    g[18] = tn[0];
    g[19] = tn[1];
    g[20] = tn[2];
    g[21] = inv;
    g[22] = cen_i.x;
    g[23] = cen_i.y;
#pragma unroll
    for (int k = 0; k < 9; ++k) g[24 + k] = Rj[k];
    g[33] = cen_j.x;
    g[34] = cen_j.y;
    g[35] = s_i;
    g[36] = s_j;
    g[37] = g[38] = g[39] = 0.f;
    return ok;
}

// the geometry record of pair n = (i, j) at the current camera records, written to d.geo
// (E_out, optional, receives E'_n as well)
__device__ __forceinline__ void pair_geometry(const DevProblem &d, int n, int i, int j, float *E_out = nullptr) {
    float g[GEO];
    if (!pair_geometry_regs(d.cam, d.cen, i, j, g)) atomicOr(d.err, ERR_DEGENERATE);
    if (E_out) {
#pragma unroll
        for (int k = 0; k < 9; ++k) E_out[k] = g[k];
    }
    float4 *out = reinterpret_cast<float4 *>(d.geo + (size_t)n * GEO);
#pragma unroll
    for (int k = 0; k < GEO / 4; ++k) out[k] = make_float4(g[4 * k], g[4 * k + 1], g[4 * k + 2], g[4 * k + 3]);
}

// Loss total of an optimiser step (FP64, fixed order over the n_loss per-camera shares in
// cam_loss) and `count` steps added to the step count. One block of NT threads (NT divides
// FIN_THREADS); the summation order is that of FIN_THREADS threads whatever NT is, so every
// launch that finishes a step produces the same bits.
constexpr int FIN_THREADS = 256;

template <int NT = FIN_THREADS>
__device__ __forceinline__ void finish_step(const DevProblem &d, int n_loss, int count) {
    static_assert(FIN_THREADS % NT == 0, "block must divide FIN_THREADS");
    __shared__ double red[FIN_THREADS];
#pragma unroll
    for (int v = threadIdx.x; v < FIN_THREADS; v += NT) {
        double s = 0.0;
        for (int q = v; q < n_loss; q += FIN_THREADS) s += d.cam_loss[q];
        red[v] = s;
    }
    __syncthreads();
    for (int w = FIN_THREADS / 2; w > 0; w >>= 1) {
        for (int v = threadIdx.x; v < w; v += NT) red[v] += red[v + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *d.loss_out = red[0];
        *d.step += count;
    }
}

}  // namespace fm
