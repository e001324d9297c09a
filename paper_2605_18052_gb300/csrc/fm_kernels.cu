// Per-iteration kernels of the epipolar adjustment (Sec. "Epipolar Adjustment").
//
//   cam_prep    per camera : FP64 pose -> FP32 camera record (R_k, c_k as hi + lo)
//   pair_setup  per pair   : R_n, t_n, 1/|t_n| and the centroid-folded essential matrix E'_n
//   stream_loss per range  : epsilon = o2^T E'_n o1 for every point pair, the loss term and
//                            the adjoint G'_n += s * o2 o1^T, segmented per image pair
//   combine     per pair   : sum the range partials (Kahan), unfold centroids, chain rule to
//                            the two cameras of the pair
//   gather      per camera : FP64 sum of the pair contributions (fixed order) + FP64 loss sum
//   adam        per camera : FP64 Adam step, R_k <- Exp(phi_k) R_k, Gram-Schmidt on rows
//   irls_weights / residuals: the same streaming walk writing one value per point pair
#include <math.h>

#include "fm_internal.cuh"

namespace fm {

// ---- streaming loads: 16 B vectors, no L1 allocation, 256 B L2 prefetch -----------------------
__device__ __forceinline__ uint4 ld_stream_v4(const void *p) {
    uint4 r;
    asm("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0,%1,%2,%3}, [%4];"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(p));
    return r;
}

__device__ __forceinline__ unsigned ld_stream_u32(const void *p) {
    unsigned r;
    asm("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(r) : "l"(p));
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
    __device__ static Raw load(const DevProblem &d, int64_t q, bool need_w) {
        Raw r;
        r.kp = ld_stream_v4(static_cast<const float4 *>(d.kp) + q);
        r.w = need_w ? ld_stream_u32(static_cast<const float *>(d.w) + q) : 0u;
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
    __device__ static Raw load(const DevProblem &d, int64_t q, bool need_w) {
        Raw r;
        r.kp = ld_stream_v4(static_cast<const uint2 *>(d.kp) + q);
        r.w = need_w ? ld_stream_u32(static_cast<const __half *>(d.w) + q) : 0u;
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
    for (int64_t g0 = p_begin; g0 < p_end; g0 += U * GROUP) {
        typename F::Raw raw[U];
#pragma unroll
        for (int u = 0; u < U; ++u) raw[u] = F::load(d, g0 + u * GROUP + lane * PPL, NEED_W);
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
                    body.segment_end(seg, r, lane);
                    lo = seg_end;
                    ++seg;
                    seg_end = d.pair_off[seg + 1];
                    load_E(d.geo, seg, E);
                }
            }
            body.group_done(gb, p_end, lane);
        }
    }
    body.segment_end(seg, r, lane);
}

// ---- loss + adjoint -----------------------------------------------------------------------------
// acc[0..8] = sum s * o2 o1^T (row-major), acc[9] = sum of loss terms, with s = w*eps (IRLS,
// the factor 2/Z is applied in combine) or sign(eps) (L1).
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
        const float a = s * x2, b = s * y2;
        acc[0] = fmaf(a, x1, acc[0]);
        acc[1] = fmaf(a, y1, acc[1]);
        acc[2] += a;
        acc[3] = fmaf(b, x1, acc[3]);
        acc[4] = fmaf(b, y1, acc[4]);
        acc[5] += b;
        acc[6] = fmaf(s, x1, acc[6]);
        acc[7] = fmaf(s, y1, acc[7]);
        acc[8] += s;
    }
    __device__ __forceinline__ void segment_end(int seg, int r, int lane) {
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

template <int STORE, int MODE>
__global__ void __launch_bounds__(CTA_WARPS * 32) k_stream_loss(DevProblem d) {
    const int r = blockIdx.x * CTA_WARPS + (threadIdx.x >> 5);
    if (r >= d.n_ranges) return;
    LossBody<MODE> body(d);
    walk_range<STORE, MODE == MODE_LOSS_IRLS>(d, r, threadIdx.x & 31, body);
}

// ---- per-point-pair maps (IRLS weights, residual export) ------------------------------------------
template <int STORE>
struct WeightBody {
    const DevProblem &d;
    float tau, delta, scale;
    float out[2];
    unsigned kept;
    __device__ WeightBody(const DevProblem &dd, float t) : d(dd), tau(t), delta((float)dd.delta),
                                                            scale(dd.w_scale), kept(0) {
        out[0] = out[1] = 0.f;
    }
    __device__ __forceinline__ void point(int k, float e, float, float, float, float, float) {
        const float a = fabsf(e);
        // filtered (w = 0) when |eps| > tau; NaN residuals are filtered too
        const bool keep = a <= tau;
        out[k] = keep ? 1.0f / fmaxf(a, delta) : 0.f;
        kept += keep ? 1u : 0u;
    }
    __device__ __forceinline__ void segment_end(int, int, int) {}
    __device__ __forceinline__ void group_done(int64_t gb, int64_t p_end, int lane) {
        const int64_t q = gb + lane * Fmt<STORE>::PPL;
        if (STORE == FM_STORE_FP32) {
            static_cast<float *>(d.w)[q] = q < p_end ? out[0] : 0.f;
        } else {
            const float a = q < p_end ? out[0] * scale : 0.f;
            const float b = q + 1 < p_end ? out[1] * scale : 0.f;
            reinterpret_cast<__half2 *>(d.w)[q >> 1] = __floats2half2_rn(a, b);
        }
        out[0] = out[1] = 0.f;
    }
};

template <int STORE>
__global__ void __launch_bounds__(CTA_WARPS * 32) k_irls_weights(DevProblem d, float tau) {
    __shared__ unsigned cta_kept;
    if (threadIdx.x == 0) cta_kept = 0;
    __syncthreads();
    const int r = blockIdx.x * CTA_WARPS + (threadIdx.x >> 5);
    if (r < d.n_ranges) {
        WeightBody<STORE> body(d, tau);
        walk_range<STORE, false>(d, r, threadIdx.x & 31, body);
        unsigned k = body.kept;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&cta_kept, k);
    }
    __syncthreads();
    if (threadIdx.x == 0 && cta_kept) atomicAdd(d.counter, (unsigned long long)cta_kept);
}

template <int STORE>
struct ResidualBody {
    float *out_sorted;
    float out[2];
    __device__ explicit ResidualBody(float *o) : out_sorted(o) { out[0] = out[1] = 0.f; }
    __device__ __forceinline__ void point(int k, float e, float, float, float, float, float) {
        out[k] = e;
    }
    __device__ __forceinline__ void segment_end(int, int, int) {}
    __device__ __forceinline__ void group_done(int64_t gb, int64_t p_end, int lane) {
        const int64_t q = gb + lane * Fmt<STORE>::PPL;
#pragma unroll
        for (int k = 0; k < Fmt<STORE>::PPL; ++k)
            if (q + k < p_end) out_sorted[q + k] = out[k];
    }
};

template <int STORE>
__global__ void __launch_bounds__(CTA_WARPS * 32) k_residuals(DevProblem d, float *out) {
    const int r = blockIdx.x * CTA_WARPS + (threadIdx.x >> 5);
    if (r >= d.n_ranges) return;
    ResidualBody<STORE> body(out);
    walk_range<STORE, false>(d, r, threadIdx.x & 31, body);
}

// ---- per camera: pose record --------------------------------------------------------------------
__device__ __forceinline__ void write_camrec(float *rec, const double *R, const double *c) {
#pragma unroll
    for (int i = 0; i < 9; ++i) rec[i] = (float)R[i];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float hi = (float)c[q];
        rec[9 + q] = hi;
        rec[12 + q] = (float)(c[q] - (double)hi);
    }
    rec[15] = 0.f;
}

__global__ void k_cam_prep(DevProblem d) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.n_cams) return;
    write_camrec(d.cam + (size_t)k * CAMREC, d.R + 9 * (size_t)k, d.c + 3 * (size_t)k);
}

// ---- per pair: relative pose and folded essential matrix ------------------------------------------
__global__ void k_pair_setup(DevProblem d) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= d.n_pairs) return;
    const int i = d.cam_i[n], j = d.cam_j[n];
    const float *ci = d.cam + (size_t)i * CAMREC;
    const float *cj = d.cam + (size_t)j * CAMREC;
    float Ri[9], Rj[9], dc[3];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        Ri[k] = ci[k];
        Rj[k] = cj[k];
    }
    // c_i - c_j from the two-float representation: the high parts of nearby centres
    // subtract exactly, so the baseline keeps FP32 relative accuracy far from the origin
#pragma unroll
    for (int q = 0; q < 3; ++q) dc[q] = (ci[9 + q] - cj[9 + q]) + (ci[12 + q] - cj[12 + q]);
    float Rn[9], tn[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int b = 0; b < 3; ++b)
            Rn[3 * a + b] = Rj[3 * a] * Ri[3 * b] + Rj[3 * a + 1] * Ri[3 * b + 1] + Rj[3 * a + 2] * Ri[3 * b + 2];
        tn[a] = Rj[3 * a] * dc[0] + Rj[3 * a + 1] * dc[1] + Rj[3 * a + 2] * dc[2];
    }
    const float nt2 = tn[0] * tn[0] + tn[1] * tn[1] + tn[2] * tn[2];
    // a baseline below 1e-10 of the centres' magnitude is rounding noise: its direction,
    // and so E_n, is undefined
    float cmax = 1.f;
#pragma unroll
    for (int q = 0; q < 3; ++q) cmax = fmaxf(cmax, fmaxf(fabsf(ci[9 + q]), fabsf(cj[9 + q])));
    const float floor2 = 1e-20f * cmax * cmax;
    float inv = 0.f;
    if (nt2 > floor2 && isfinite(nt2)) {
        inv = 1.0f / sqrtf(nt2);
    } else {
        atomicOr(d.err, ERR_DEGENERATE);
    }
    const float th[3] = {tn[0] * inv, tn[1] * inv, tn[2] * inv};
    // E = [th]_x R_n
    float E[9];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        E[b] = -th[2] * Rn[3 + b] + th[1] * Rn[6 + b];
        E[3 + b] = th[2] * Rn[b] - th[0] * Rn[6 + b];
        E[6 + b] = -th[1] * Rn[b] + th[0] * Rn[3 + b];
    }
    // E' = T_j^T E T_i with T = [[1,0,cx],[0,1,cy],[0,0,1]] (keypoints stored as offsets o = x - c)
    const float2 cen_i = d.cen[i], cen_j = d.cen[j];
    float M[9];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        M[3 * a] = E[3 * a];
        M[3 * a + 1] = E[3 * a + 1];
        M[3 * a + 2] = E[3 * a] * cen_i.x + E[3 * a + 1] * cen_i.y + E[3 * a + 2];
    }
    float *g = d.geo + (size_t)n * GEO;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        g[b] = M[b];
        g[3 + b] = M[3 + b];
        g[6 + b] = cen_j.x * M[b] + cen_j.y * M[3 + b] + M[6 + b];
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) g[9 + k] = Rn[k];
    g[18] = tn[0];
    g[19] = tn[1];
    g[20] = tn[2];
    g[21] = inv;
    g[22] = 0.f;
    g[23] = 0.f;
}

// ---- per pair: combine partials and chain rule ----------------------------------------------------
__device__ __forceinline__ void vee(const float *M, float *v) {
    v[0] = M[7] - M[5];
    v[1] = M[2] - M[6];
    v[2] = M[3] - M[1];
}

__global__ void k_combine(DevProblem d, float gscale, float lscale) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= d.n_pairs) return;
    const int p0 = d.pair_off[n], p1 = d.pair_off[n + 1];
    const int r0 = p0 / WR, r1 = (p1 - 1) / WR;
    float sum[10], cmp[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) sum[k] = cmp[k] = 0.f;
    for (int r = r0; r <= r1; ++r) {
        const float4 *s = reinterpret_cast<const float4 *>(d.slots + (size_t)(n + r) * SLOT);
        const float4 a = s[0], b = s[1], c = s[2];
        const float v[10] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y};
#pragma unroll
        for (int k = 0; k < 10; ++k) {  // Kahan-compensated FP32 sum
            const float y = v[k] - cmp[k];
            const float t = sum[k] + y;
            cmp[k] = (t - sum[k]) - y;
            sum[k] = t;
        }
    }
    float Gp[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Gp[k] = sum[k] * gscale;
    const float loss = sum[9] * lscale;
    const int i = d.cam_i[n], j = d.cam_j[n];
    // G = T_j G' T_i^T (gradient with respect to E from the one with respect to E')
    const float2 cen_i = d.cen[i], cen_j = d.cen[j];
    float M[9], G[9];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        M[3 * a] = Gp[3 * a] + Gp[3 * a + 2] * cen_i.x;
        M[3 * a + 1] = Gp[3 * a + 1] + Gp[3 * a + 2] * cen_i.y;
        M[3 * a + 2] = Gp[3 * a + 2];
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        G[b] = M[b] + cen_j.x * M[6 + b];
        G[3 + b] = M[3 + b] + cen_j.y * M[6 + b];
        G[6 + b] = M[6 + b];
    }
    const float *g = d.geo + (size_t)n * GEO;
    float Rn[9], tn[3];
#pragma unroll
    for (int k = 0; k < 9; ++k) Rn[k] = g[9 + k];
    tn[0] = g[18];
    tn[1] = g[19];
    tn[2] = g[20];
    const float inv = g[21];
    const float th[3] = {tn[0] * inv, tn[1] * inv, tn[2] * inv};
    // A = -[th]_x G
    float A[9];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        A[b] = -(-th[2] * G[3 + b] + th[1] * G[6 + b]);
        A[3 + b] = -(th[2] * G[b] - th[0] * G[6 + b]);
        A[6 + b] = -(-th[1] * G[b] + th[0] * G[3 + b]);
    }
    // g_th = vee(G R_n^T); g_t = (I - th th^T) g_th / |t|
    float GRt[9], ARt[9], RtA[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            GRt[3 * a + b] = G[3 * a] * Rn[3 * b] + G[3 * a + 1] * Rn[3 * b + 1] + G[3 * a + 2] * Rn[3 * b + 2];
            ARt[3 * a + b] = A[3 * a] * Rn[3 * b] + A[3 * a + 1] * Rn[3 * b + 1] + A[3 * a + 2] * Rn[3 * b + 2];
            RtA[3 * a + b] = Rn[a] * A[b] + Rn[3 + a] * A[3 + b] + Rn[6 + a] * A[6 + b];
        }
    float gth[3], gt[3], gpj[3], gpi[3];
    vee(GRt, gth);
    const float dp = th[0] * gth[0] + th[1] * gth[1] + th[2] * gth[2];
#pragma unroll
    for (int q = 0; q < 3; ++q) gt[q] = (gth[q] - dp * th[q]) * inv;
    vee(ARt, gpj);
    gpj[0] += tn[1] * gt[2] - tn[2] * gt[1];
    gpj[1] += tn[2] * gt[0] - tn[0] * gt[2];
    gpj[2] += tn[0] * gt[1] - tn[1] * gt[0];
    vee(RtA, gpi);
    const float *Rj = d.cam + (size_t)j * CAMREC;
    float gc[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) gc[q] = Rj[q] * gt[0] + Rj[3 + q] * gt[1] + Rj[6 + q] * gt[2];
    float4 *out = reinterpret_cast<float4 *>(d.pair_grad + (size_t)n * PG);
    out[0] = make_float4(-gpi[0], -gpi[1], -gpi[2], gc[0]);
    out[1] = make_float4(gc[1], gc[2], gpj[0], gpj[1]);
    out[2] = make_float4(gpj[2], -gc[0], -gc[1], -gc[2]);
    out[3] = make_float4(loss, 0.f, 0.f, 0.f);
    bool ok = isfinite(loss);
#pragma unroll
    for (int q = 0; q < 3; ++q) ok = ok && isfinite(gpi[q]) && isfinite(gpj[q]) && isfinite(gc[q]);
    if (!ok) atomicOr(d.err, ERR_NONFINITE);
}

// ---- per camera: gradient gather (FP64) and the loss sum ------------------------------------------
constexpr int GATHER_THREADS = 256;

__global__ void __launch_bounds__(GATHER_THREADS) k_gather(DevProblem d, int count_step) {
    if (blockIdx.x == gridDim.x - 1) {
        // loss = sum over pairs, FP64, fixed partition and fixed tree order
        __shared__ double red[GATHER_THREADS];
        double s = 0.0;
        for (int n = threadIdx.x; n < d.n_pairs; n += GATHER_THREADS)
            s += (double)d.pair_grad[(size_t)n * PG + 12];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int w = GATHER_THREADS / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            *d.loss_out = red[0];
            if (count_step) *d.step += 1;
        }
        return;
    }
    const int k = blockIdx.x * GATHER_THREADS + threadIdx.x;
    if (k >= d.n_cams) return;
    double g[6] = {0, 0, 0, 0, 0, 0};
    for (int e = d.cam_off[k]; e < d.cam_off[k + 1]; ++e) {
        const int ent = d.cam_ent[e];
        const float *pg = d.pair_grad + (size_t)(ent >> 1) * PG + (ent & 1) * 6;
#pragma unroll
        for (int q = 0; q < 6; ++q) g[q] += (double)pg[q];
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) d.grad[(size_t)k * 6 + q] = g[q];
}

// ---- per camera: Adam + exponential map (FP64) -----------------------------------------------------
__device__ void expmap64(const double *phi, double *R) {
    const double th2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
    const double th = sqrt(th2);
    double a, b;
    if (th < 1e-8) {
        a = 1.0 - th2 / 6.0;
        b = 0.5 - th2 / 24.0;
    } else {
        double s, c;
        sincos(th, &s, &c);
        a = s / th;
        b = (1.0 - c) / th2;
    }
    const double K[9] = {0, -phi[2], phi[1], phi[2], 0, -phi[0], -phi[1], phi[0], 0};
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double k2 = K[3 * r] * K[c] + K[3 * r + 1] * K[3 + c] + K[3 * r + 2] * K[6 + c];
            R[3 * r + c] = (r == c ? 1.0 : 0.0) + a * K[3 * r + c] + b * k2;
        }
}

// Gram-Schmidt on the rows: r0 normalised, r1 orthogonalised and normalised, r2 = r0 x r1
__device__ void orthonormalize_rows(double *R) {
    const double n0 = 1.0 / sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
    for (int q = 0; q < 3; ++q) R[q] *= n0;
    const double dp = R[0] * R[3] + R[1] * R[4] + R[2] * R[5];
    for (int q = 0; q < 3; ++q) R[3 + q] -= dp * R[q];
    const double n1 = 1.0 / sqrt(R[3] * R[3] + R[4] * R[4] + R[5] * R[5]);
    for (int q = 0; q < 3; ++q) R[3 + q] *= n1;
    R[6] = R[1] * R[5] - R[2] * R[4];
    R[7] = R[2] * R[3] - R[0] * R[5];
    R[8] = R[0] * R[4] - R[1] * R[3];
}

__global__ void k_adam(DevProblem d) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.n_cams) return;
    const double lr_r = d.hyper[0], lr_c = d.hyper[1], b1 = d.hyper[2], b2 = d.hyper[3],
                 eps = d.hyper[4];
    const double t = (double)*d.step;
    const double bc1 = 1.0 - pow(b1, t), bc2 = 1.0 - pow(b2, t);
    double delta[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const size_t o = (size_t)k * 6 + q;
        const double g = d.grad[o];
        const double m = b1 * d.m[o] + (1.0 - b1) * g;
        const double v = b2 * d.v[o] + (1.0 - b2) * g * g;
        d.m[o] = m;
        d.v[o] = v;
        delta[q] = -(q < 3 ? lr_r : lr_c) * (m / bc1) / (sqrt(v / bc2) + eps);
    }
    double Ex[9], Rk[9], Rn[9];
    expmap64(delta, Ex);
    double *R = d.R + (size_t)k * 9;
#pragma unroll
    for (int q = 0; q < 9; ++q) Rk[q] = R[q];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            Rn[3 * r + c] = Ex[3 * r] * Rk[c] + Ex[3 * r + 1] * Rk[3 + c] + Ex[3 * r + 2] * Rk[6 + c];
    orthonormalize_rows(Rn);
#pragma unroll
    for (int q = 0; q < 9; ++q) R[q] = Rn[q];
    double *c = d.c + (size_t)k * 3;
#pragma unroll
    for (int q = 0; q < 3; ++q) c[q] += delta[3 + q];
    write_camrec(d.cam + (size_t)k * CAMREC, R, c);
}

// ---- launchers -------------------------------------------------------------------------------------
static inline int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

void launch_cam_prep(const DevProblem &d, cudaStream_t s) {
    k_cam_prep<<<blocks_for(d.n_cams, 128), 128, 0, s>>>(d);
}

void launch_pair_setup(const DevProblem &d, cudaStream_t s) {
    k_pair_setup<<<blocks_for(d.n_pairs, 128), 128, 0, s>>>(d);
}

void launch_stream_loss(const DevProblem &d, cudaStream_t s) {
    const int grid = blocks_for(d.n_ranges, CTA_WARPS);
    if (d.storage == FM_STORE_FP32) {
        if (d.loss == FM_LOSS_IRLS) k_stream_loss<FM_STORE_FP32, MODE_LOSS_IRLS><<<grid, CTA_WARPS * 32, 0, s>>>(d);
        else k_stream_loss<FM_STORE_FP32, MODE_LOSS_L1><<<grid, CTA_WARPS * 32, 0, s>>>(d);
    } else {
        if (d.loss == FM_LOSS_IRLS) k_stream_loss<FM_STORE_FP16, MODE_LOSS_IRLS><<<grid, CTA_WARPS * 32, 0, s>>>(d);
        else k_stream_loss<FM_STORE_FP16, MODE_LOSS_L1><<<grid, CTA_WARPS * 32, 0, s>>>(d);
    }
}

void launch_combine(const DevProblem &d, cudaStream_t s) {
    const double Z = (double)d.n_pp;
    float gscale, lscale;
    if (d.loss == FM_LOSS_IRLS) {  // stored weights are w * s
        gscale = (float)(2.0 / (Z * d.w_scale));
        lscale = (float)(1.0 / (Z * d.w_scale));
    } else {
        gscale = (float)(1.0 / Z);
        lscale = (float)(1.0 / Z);
    }
    k_combine<<<blocks_for(d.n_pairs, 128), 128, 0, s>>>(d, gscale, lscale);
}

void launch_gather(const DevProblem &d, bool count_step, cudaStream_t s) {
    k_gather<<<blocks_for(d.n_cams, GATHER_THREADS) + 1, GATHER_THREADS, 0, s>>>(d, count_step ? 1 : 0);
}

void launch_adam(const DevProblem &d, cudaStream_t s) {
    k_adam<<<blocks_for(d.n_cams, 64), 64, 0, s>>>(d);
}

void launch_irls_weights(const DevProblem &d, float tau, cudaStream_t s) {
    const int grid = blocks_for(d.n_ranges, CTA_WARPS);
    if (d.storage == FM_STORE_FP32) k_irls_weights<FM_STORE_FP32><<<grid, CTA_WARPS * 32, 0, s>>>(d, tau);
    else k_irls_weights<FM_STORE_FP16><<<grid, CTA_WARPS * 32, 0, s>>>(d, tau);
}

void launch_residuals(const DevProblem &d, float *out_sorted, cudaStream_t s) {
    const int grid = blocks_for(d.n_ranges, CTA_WARPS);
    if (d.storage == FM_STORE_FP32) k_residuals<FM_STORE_FP32><<<grid, CTA_WARPS * 32, 0, s>>>(d, out_sorted);
    else k_residuals<FM_STORE_FP16><<<grid, CTA_WARPS * 32, 0, s>>>(d, out_sorted);
}

}  // namespace fm
