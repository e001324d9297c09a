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

#include "fm_step.cuh"

namespace fm {

// prev_loss > 0: this pass follows an optimiser camera step (which also wrote this pass's
// geometry records); block 0 first finishes that step's loss total (over prev_loss per-camera
// shares) and step count.
template <int STORE, int MODE>
__global__ void __launch_bounds__(CTA_WARPS * 32, 4) k_stream_loss(DevProblem d, int prev_loss) {
    pdl_wait();     // pair geometry of this pass
    pdl_trigger();  // the per-camera step may be scheduled once the last wave has started
    if (prev_loss > 0 && blockIdx.x == 0) finish_step(d, prev_loss, 1);
    const int r = blockIdx.x * CTA_WARPS + (threadIdx.x >> 5);
    if (r >= d.n_ranges) return;
    LossBody<MODE> body(d);
    walk_range<STORE, MODE == MODE_LOSS_IRLS>(d, r, threadIdx.x & 31, body);
}

// The first pass of an IRLS round fused with the round's reweighting: the residual at the
// round's starting poses gives the weight (filtered by tau, floored by delta, quantised as the
// storage keeps it), which is written and at once used for the loss and adjoint sums. Same
// arithmetic as the weights kernel followed by the streaming pass, one read of the keypoints
// instead of two. tau comes from d.hyper[6] so one captured graph serves every round.
template <int STORE>
struct ReweightLossBody {
    LossBody<MODE_LOSS_IRLS> loss;
    const DevProblem &d;
    float tau, delta, scale;
    float out[2];
    unsigned kept;
    __device__ ReweightLossBody(const DevProblem &dd, float t)
        : loss(dd), d(dd), tau(t), delta((float)dd.delta), scale(dd.w_scale), kept(0) {
        out[0] = out[1] = 0.f;
    }
    __device__ __forceinline__ void point(int k, float e, float x1, float y1, float x2, float y2, float) {
        const float a = fabsf(e);
        const bool keep = a <= tau;  // NaN residuals are filtered
        const float wf = keep ? irls_weight(a, delta) : 0.f;
        const float w = STORE == FM_STORE_FP32 ? wf : __half2float(__float2half_rn(wf * scale));
        out[k] = w;
        kept += keep ? 1u : 0u;
        loss.point(k, e, x1, y1, x2, y2, w);
    }
    __device__ __forceinline__ void segment_begin(int seg) { loss.segment_begin(seg); }
    __device__ __forceinline__ void segment_end(int seg, int r, int lane, bool last) {
        loss.segment_end(seg, r, lane, last);
    }
    __device__ __forceinline__ void group_done(int64_t gb, int64_t p_end, int lane) {
        const int64_t q = gb + lane * Fmt<STORE>::PPL;
        if (STORE == FM_STORE_FP32) {
            static_cast<float *>(d.w)[q] = q < p_end ? out[0] : 0.f;
        } else {
            // already on the FP16 grid: the conversion is exact
            const float a = q < p_end ? out[0] : 0.f;
            const float b = q + 1 < p_end ? out[1] : 0.f;
            reinterpret_cast<__half2 *>(d.w)[q >> 1] = __floats2half2_rn(a, b);
        }
        out[0] = out[1] = 0.f;
    }
};

template <int STORE>
__global__ void __launch_bounds__(CTA_WARPS * 32, 4) k_stream_reweight(DevProblem d) {
    __shared__ unsigned cta_kept;
    if (threadIdx.x == 0) cta_kept = 0;
    __syncthreads();
    pdl_wait();     // pair geometry of this pass
    pdl_trigger();
    const float tau = (float)d.hyper[6];
    const int r = blockIdx.x * CTA_WARPS + (threadIdx.x >> 5);
    if (r < d.n_ranges) {
        ReweightLossBody<STORE> body(d, tau);
        walk_range<STORE, false>(d, r, threadIdx.x & 31, body);
        unsigned k = body.kept;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&cta_kept, k);
    }
    __syncthreads();
    if (threadIdx.x == 0 && cta_kept) atomicAdd(d.counter, (unsigned long long)cta_kept);
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
        out[k] = keep ? irls_weight(a, delta) : 0.f;
        kept += keep ? 1u : 0u;
    }
    __device__ __forceinline__ void segment_begin(int) {}
    __device__ __forceinline__ void segment_end(int, int, int, bool) {}
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
    __device__ __forceinline__ void segment_begin(int) {}
    __device__ __forceinline__ void segment_end(int, int, int, bool) {}
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

__global__ void k_cam_prep(DevProblem d) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.n_cams) return;
    write_camrec(d.cam + (size_t)k * CAMREC, d.R + 9 * (size_t)k, d.c + 3 * (size_t)k, (float)camera_scale(d, k));
}

// prev_loss > 0: this pass follows an optimiser step with that many per-camera loss shares;
// block 0 (with 256 threads) finishes that step's loss total and step count.
__global__ void __launch_bounds__(256) k_pair_setup(DevProblem d, int prev_loss) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = n < d.n_pairs ? d.cam_i[n] : 0, j = n < d.n_pairs ? d.cam_j[n] : 0;
    pdl_wait();     // camera records of the previous step
    pdl_trigger();
    if (prev_loss > 0 && blockIdx.x == 0) finish_step(d, prev_loss, 1);
    if (n >= d.n_pairs) return;
    pair_geometry(d, n, i, j);
}

// ---- per pair: combine partials and chain rule ----------------------------------------------------
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
// Fused per-camera step, 8 cameras per 256-thread block (all blocks resident at once).
// Before waiting for the streaming pass (griddepcontrol.wait) the block fetches everything that
// is at least two kernels old: its cameras' Adam moments, poses and the step count, and for
// each camera the (pair, role) entries, their range-partial counts and the pairs' geometry
// records (into shared memory). After the wait only the partial sums remain to be read.
// Phase 1: warp w owns camera k = 8*block + w. The chain rule is linear in a pair's sums, so it
// is applied to every (pair, warp-range partial) item separately; the items are spread evenly
// over the lanes (a pair that spans many ranges does not hold up one lane). The warp reduces
// the 6 gradient components and the loss with a compensated (TwoSum) FP32 butterfly, so each
// sum is carried as an unevaluated hi + lo pair.
// Phase 2: warp 0, one camera per lane: the final per-camera gradient hi + lo in FP64, the
// Adam update (FP32 moments), R <- Exp(phi) R and Gram-Schmidt re-orthonormalisation in FP64,
// the centre update in FP64 and the new camera record. Keeping the FP64 work lane-parallel
// matters on GB300, whose FP64 pipe charges a whole warp instruction per operation.
// Geometry comes from the pair records, never from another camera's record, which another
// block may be updating. The loss of a pair is counted by its first camera only; each camera's
// FP64 loss share goes to cam_loss[camera], and the next kernel (the next pass, pair setup or
// the finalize kernel) adds them up in a fixed order and advances the step count.
// Phase 3 (next_geo, with apply): the geometry records of the new poses, so the next pass
// needs no pair-setup launch. Each camera's warp counts its image pairs in d.pair_cnt (one
// acquire-release atomic per (pair, camera); every such step adds 2 to each pair's count); the
// camera that finds an odd count is the pair's second, both records are then written, and it
// computes the pair's record. A record is overwritten only after both of its readers in this
// launch (the pair's two cameras) have passed phase 1, and the pass that read E'_n has
// completed before this kernel's wait.
template <bool FOCAL>
__global__ void __launch_bounds__(STEP_CAMS * 32, 4)
k_camera_step(DevProblem d, float gscale, float lscale, int apply, int next_geo) {
    constexpr int NV = FOCAL ? STEP_VALS : STEP_VALS - 1;   // sums carried per camera
    __shared__ float s_hi[STEP_VALS][STEP_CAMS], s_lo[STEP_VALS][STEP_CAMS];
    __shared__ int4 s_item[STEP_CAMS][32];
    __shared__ __align__(16) float s_geo[STEP_CAMS][32][GEO];
    __shared__ float s_mv[STEP_CAMS][12];     // Adam m (6) and v (6) of the block's cameras
    __shared__ double s_Rc[STEP_CAMS][12];    // R (9) and c (3) of the block's cameras
    __shared__ float s_R32[STEP_CAMS][10];    // their records' rotations (9) and keypoint scale
    __shared__ double s_hyper[6];   // lr_rot, lr_c, beta1, beta2, eps, lr_focal
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = blockIdx.x * STEP_CAMS + warp;
    {
        const int cam0 = blockIdx.x * STEP_CAMS;
        for (int i = threadIdx.x; i < STEP_CAMS * 12; i += STEP_CAMS * 32) {
            const int cc = i / 12, q = i % 12;
            if (cam0 + cc < d.n_cams) {
                s_mv[cc][q] = q < 6 ? d.m[(size_t)(cam0 + cc) * 6 + q] : d.v[(size_t)(cam0 + cc) * 6 + q - 6];
                s_Rc[cc][q] = q < 9 ? d.R[(size_t)(cam0 + cc) * 9 + q] : d.c[(size_t)(cam0 + cc) * 3 + q - 9];
                if (q < 10) s_R32[cc][q] = d.cam[(size_t)(cam0 + cc) * CAMREC + (q < 9 ? q : 15)];
            }
        }
        if (threadIdx.x < 6) s_hyper[threadIdx.x] = d.hyper[threadIdx.x];
    }
    const int e_begin = k < d.n_cams ? d.cam_off[k] : 0;
    const int e_end = k < d.n_cams ? d.cam_off[k + 1] : 0;
    // this camera's entries, 32 at a time: pair, role, first range and number of ranges; the
    // pair's geometry record goes to shared memory
    auto load_chunk = [&](int base) -> int {
        const int e = base + lane;
        int n = 0, role = 0, r0 = 0, cnt = 0;
        if (e < e_end) {
            const int ent = d.cam_ent[e];
            n = ent >> 1;
            role = ent & 1;
            r0 = d.pair_off[n] / WR;
            cnt = (d.pair_off[n + 1] - 1) / WR - r0 + 1;
            const float4 *gv = reinterpret_cast<const float4 *>(d.geo + (size_t)n * GEO);
            float4 *dst = reinterpret_cast<float4 *>(s_geo[warp][lane]);
#pragma unroll
            for (int q = 2; q < GEO / 4; ++q) dst[q] = gv[q];
        }
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += x;
        }
        s_item[warp][lane] = make_int4(incl - cnt, n, role, r0);
        __syncwarp();
        return __shfl_sync(0xffffffffu, incl, 31);
    };
    int total = load_chunk(e_begin);
    pdl_wait();     // partial sums of the streaming pass
    pdl_trigger();
    const long long t_step = *d.step + 1;
    if (k < d.n_cams) {
        float hi[STEP_VALS], lo[STEP_VALS];
#pragma unroll
        for (int q = 0; q < STEP_VALS; ++q) hi[q] = lo[q] = 0.f;
        for (int base = e_begin; base < e_end; base += 32) {
            if (base != e_begin) {
                __syncwarp();
                total = load_chunk(base);
            }
            for (int t = lane; t < total; t += 32) {
                int lo_i = 0, hi_i = 31;
                while (lo_i < hi_i) {
                    const int mid = (lo_i + hi_i + 1) >> 1;
                    if (s_item[warp][mid].x <= t) lo_i = mid;
                    else hi_i = mid - 1;
                }
                const int4 it = s_item[warp][lo_i];
                const float4 *sl = reinterpret_cast<const float4 *>(d.slots + (size_t)(it.y + it.w + (t - it.x)) * SLOT);
                const float4 sa = sl[0], sb = sl[1], sc = sl[2];
                const float sum[10] = {sa.x, sa.y, sa.z, sa.w, sb.x, sb.y, sb.z, sb.w, sc.x, sc.y};
                float contrib[STEP_VALS];
                pair_chain_rule<FOCAL>(s_geo[warp][lo_i], it.z, sum, gscale, lscale, contrib);
#pragma unroll
                for (int q = 0; q < NV; ++q) two_sum_acc(hi[q], lo[q], contrib[q], 0.f);
            }
        }
        warp_two_sum_reduce<NV>(hi, lo);
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < STEP_VALS; ++q) {
                s_hi[q][warp] = q < NV ? hi[q] : 0.f;
                s_lo[q][warp] = lo[q];
            }
        }
    }
    __syncthreads();
    if (warp == 0 && lane < STEP_CAMS) {
        const int kc = blockIdx.x * STEP_CAMS + lane;
        const double bl = kc < d.n_cams
            ? camera_update<FOCAL>(d, kc, &s_hi[0][lane], &s_lo[0][lane], STEP_CAMS, s_mv[lane], s_Rc[lane],
                                   s_R32[lane], s_hyper, t_step, apply, d.cam + (size_t)kc * CAMREC)
            : 0.0;
        if (apply && next_geo) __threadfence();   // the record reaches L2 before any count below
        if (kc < d.n_cams) d.cam_loss[kc] = bl;
    }
    if (!(apply && next_geo)) return;
    __syncthreads();   // the block's new records are written
    if (k < d.n_cams) {
        for (int e = e_begin + lane; e < e_end; e += 32) {
            const int n = d.cam_ent[e] >> 1;
            if (atomic_add_acq_rel(d.pair_cnt + n, 1u) & 1u) pair_geometry(d, n, d.cam_i[n], d.cam_j[n]);
        }
    }
}

// Adam step with a given gradient (d.grad, FP64), one camera per thread: the same update as the
// camera-step kernel (camera_update with the gradient split into FP32 hi + lo parts, whose FP32
// sum is the gradient rounded to FP32, as there); the step count is advanced by k_bump_step.
__global__ void k_apply_gradient(DevProblem d) {
    const int kc = blockIdx.x * blockDim.x + threadIdx.x;
    if (kc >= d.n_cams) return;
    const long long t_step = *d.step + 1;
    float hi[STEP_VALS], lo[STEP_VALS], mv[12], rec[10];
    double Rc[12], hyper[6];
#pragma unroll
    for (int q = 0; q < STEP_VALS; ++q) {
        const double g = q < 6 ? d.grad[(size_t)kc * 6 + q] : 0.0;
        hi[q] = (float)g;
        lo[q] = (float)__dsub_rn(g, (double)hi[q]);
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        mv[q] = d.m[(size_t)kc * 6 + q];
        mv[6 + q] = d.v[(size_t)kc * 6 + q];
        hyper[q] = d.hyper[q];
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        Rc[q] = d.R[(size_t)kc * 9 + q];
        rec[q] = d.cam[(size_t)kc * CAMREC + q];
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) Rc[9 + q] = d.c[(size_t)kc * 3 + q];
    rec[9] = d.cam[(size_t)kc * CAMREC + 15];
    camera_update<false>(d, kc, hi, lo, 1, mv, Rc, rec, hyper, t_step, 1, d.cam + (size_t)kc * CAMREC);
}

__global__ void k_bump_step(DevProblem d) { *d.step += 1; }

// closes a chain of steps: loss of the last step and `count` steps added to the step count
__global__ void __launch_bounds__(FIN_THREADS) k_finalize(DevProblem d, int n_loss, int count) {
    pdl_wait();
    pdl_trigger();
    finish_step(d, n_loss, count);
}

// camera records copied back from the alternate buffer (one float4 per thread)
__global__ void __launch_bounds__(256) k_copy_records(DevProblem d, const float4 *src) {
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < d.n_cams * (CAMREC / 4)) reinterpret_cast<float4 *>(d.cam)[i] = src[i];
}

// ---- launchers -------------------------------------------------------------------------------------
static inline int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

int camera_step_blocks(const DevProblem &d) { return blocks_for(d.n_cams, STEP_CAMS); }

void launch_cam_prep(const DevProblem &d, cudaStream_t s) {
    k_cam_prep<<<blocks_for(d.n_cams, 128), 128, 0, s>>>(d);
}

void launch_pair_setup(const DevProblem &d, cudaStream_t s, bool pdl, bool after_step) {
    launch_k(k_pair_setup, dim3(blocks_for(d.n_pairs, 256)), dim3(256), s, pdl, d, after_step ? d.n_cams : 0);
}

void launch_finalize(const DevProblem &d, bool count_step, cudaStream_t s, bool pdl) {
    launch_finalize_n(d, count_step ? 1 : 0, nullptr, s, pdl);
}

void launch_finalize_n(const DevProblem &d, int count, const float *copy_src, cudaStream_t s, bool pdl) {
    if (copy_src)
        launch_k(k_copy_records, dim3(blocks_for((int64_t)d.n_cams * (CAMREC / 4), 256)), dim3(256), s, pdl, d,
                 reinterpret_cast<const float4 *>(copy_src));
    launch_k(k_finalize, dim3(1), dim3(FIN_THREADS), s, pdl, d, d.n_cams, count);
}

void launch_stream_loss(const DevProblem &d, cudaStream_t s, bool pdl, bool after_step) {
    static_assert(CTA_WARPS * 32 == FIN_THREADS, "block 0 of the pass finishes a step");
    const dim3 grid(blocks_for(d.n_ranges, CTA_WARPS)), block(CTA_WARPS * 32);
    const int prev = after_step ? d.n_cams : 0;
    if (d.storage == FM_STORE_FP32) {
        if (d.loss == FM_LOSS_IRLS) launch_k(k_stream_loss<FM_STORE_FP32, MODE_LOSS_IRLS>, grid, block, s, pdl, d, prev);
        else launch_k(k_stream_loss<FM_STORE_FP32, MODE_LOSS_L1>, grid, block, s, pdl, d, prev);
    } else {
        if (d.loss == FM_LOSS_IRLS) launch_k(k_stream_loss<FM_STORE_FP16, MODE_LOSS_IRLS>, grid, block, s, pdl, d, prev);
        else launch_k(k_stream_loss<FM_STORE_FP16, MODE_LOSS_L1>, grid, block, s, pdl, d, prev);
    }
}

void launch_stream_reweight(const DevProblem &d, cudaStream_t s, bool pdl) {
    const dim3 grid(blocks_for(d.n_ranges, CTA_WARPS)), block(CTA_WARPS * 32);
    if (d.storage == FM_STORE_FP32) launch_k(k_stream_reweight<FM_STORE_FP32>, grid, block, s, pdl, d);
    else launch_k(k_stream_reweight<FM_STORE_FP16>, grid, block, s, pdl, d);
}

void launch_combine(const DevProblem &d, cudaStream_t s) {
    const double Z = d.z > 0.0 ? d.z : (double)d.n_pp;
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

void loss_scales(const DevProblem &d, float &gscale, float &lscale) {
    const double Z = d.z > 0.0 ? d.z : (double)d.n_pp;
    if (d.loss == FM_LOSS_IRLS) {  // stored weights are w * s
        gscale = (float)(2.0 / (Z * d.w_scale));
        lscale = (float)(1.0 / (Z * d.w_scale));
    } else {
        gscale = (float)(1.0 / Z);
        lscale = (float)(1.0 / Z);
    }
}

void launch_apply_gradient(const DevProblem &d, cudaStream_t s) {
    k_apply_gradient<<<blocks_for(d.n_cams, 64), 64, 0, s>>>(d);
    k_bump_step<<<1, 1, 0, s>>>(d);
}

void launch_camera_step(const DevProblem &d, bool apply, cudaStream_t s, bool pdl, bool next_geo) {
    float gscale, lscale;
    loss_scales(d, gscale, lscale);
    const int ng = next_geo && d.pair_cnt ? 1 : 0;
    if (d.refine_focal)
        launch_k(k_camera_step<true>, dim3(blocks_for(d.n_cams, STEP_CAMS)), dim3(STEP_CAMS * 32), s, pdl, d,
                 gscale, lscale, apply ? 1 : 0, ng);
    else
        launch_k(k_camera_step<false>, dim3(blocks_for(d.n_cams, STEP_CAMS)), dim3(STEP_CAMS * 32), s, pdl, d,
                 gscale, lscale, apply ? 1 : 0, ng);
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
