// Pre-aggregated quadratic form of the IRLS objective (Eq. epipolar-objective-l2 and the IRLS
// equation after it): with the weights fixed for a round, the objective of image pair n is a
// quadratic function of e_n = vec(E'_n), so one streaming pass per round collects, per pair,
//   c0 = sum w eps0^2,   g0 = sum w eps0 a,   W = sum w a a^T      (a = vec(o2 o1^T))
// at the anchor e0 (the essential matrices of the poses the pass ran at, eps0 = a^T e0), and
// every iteration of the round evaluates the pair in O(1) from e = e0 + d:
//   sum w eps^2      = c0 + d^T (2 g0 + W d)
//   sum w eps a      = g0 + W d       (the same sums the streaming pass produces)
// Anchoring matters for accuracy: e^T W e on its own cancels by a factor (|a| |e| / eps)^2
// (about 1e5 near the optimum), whereas the anchored form keeps the FP32 error structure of
// the streaming pass (the large W enters only through the step d).
//
// W has Kronecker structure: a a^T = (o2 o2^T) (x) (o1 o1^T), so its 81 entries take only
// 6 x 6 = 36 distinct values M[u][v] = sum w m2_u m1_v over the monomials
//   m2 = (x2^2, x2 y2, x2, y2^2, y2, 1),  m1 = (x1^2, x1 y1, x1, y1^2, y1, 1),
// with W[3p+q][3r+s] = M[sym(p,r)][sym(q,s)], sym the index of the unordered pair in
// (00, 01, 02, 11, 12, 22). Per point pair that is 36 multiply-adds instead of 45, issued as 18
// packed pairs.
#include "fm_step.cuh"

namespace fm {

// REWEIGHT: the IRLS weights are computed from the residual at the same poses (and written,
// quantised as the storage keeps them) before they enter the sums
template <int STORE, bool REWEIGHT>
struct QuadBody {
    const DevProblem &d;
    float tau, delta, scale;
    float acc[QSUMS];
    float out[2];
    unsigned kept;
    __device__ QuadBody(const DevProblem &dd, float t)
        : d(dd), tau(t), delta((float)dd.delta), scale(dd.w_scale), kept(0) {
#pragma unroll
        for (int i = 0; i < QSUMS; ++i) acc[i] = 0.f;
        out[0] = out[1] = 0.f;
    }
    __device__ __forceinline__ void segment_begin(int) {}
    __device__ __forceinline__ void point(int k, float e, float x1, float y1, float x2, float y2, float w) {
        if (REWEIGHT) {
            const float ae = fabsf(e);
            const bool keep = ae <= tau;  // NaN residuals are filtered
            const float wf = keep ? irls_weight(ae, delta) : 0.f;
            w = STORE == FM_STORE_FP32 ? wf : __half2float(__float2half_rn(wf * scale));
            out[k] = w;
            kept += keep ? 1u : 0u;
        }
        // c0 and g0 = sum (w eps o2) (x) o1
        const float we = w * e;
        acc[0] = fmaf(we, e, acc[0]);
        const float t2[3] = {we * x2, we * y2, we};
        const float o1[3] = {x1, y1, 1.f};
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) acc[1 + 3 * p + q] = fmaf(t2[p], o1[q], acc[1 + 3 * p + q]);
        // M[u][v] += (w m2_u) m1_v, two neighbouring entries of a row per packed instruction (the
        // pass is bound by instruction issue, not by the FP32 pipe)
        const float wx2 = w * x2, wy2 = w * y2;
        const float u[6] = {wx2 * x2, wx2 * y2, wx2, wy2 * y2, wy2, w};
        const float v[6] = {x1 * x1, x1 * y1, x1, y1 * y1, y1, 1.f};
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int b = 0; b < 6; b += 2) fma2(acc[10 + 6 * a + b], acc[10 + 6 * a + b + 1], u[a], u[a], v[b], v[b + 1]);
    }
    __device__ __forceinline__ void segment_end(int seg, int r, int lane, bool) {
#pragma unroll
        for (int i = 0; i < QSUMS; ++i) {
            float v = acc[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            acc[i] = v;
        }
        if (lane == 0) {
            float4 *s = reinterpret_cast<float4 *>(d.qslots + (size_t)(seg + r) * QSLOT);
#pragma unroll
            for (int q = 0; q < QSLOT / 4; ++q) {
                float v[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) v[c] = 4 * q + c < QSUMS ? acc[4 * q + c] : 0.f;
                s[q] = make_float4(v[0], v[1], v[2], v[3]);
            }
        }
#pragma unroll
        for (int i = 0; i < QSUMS; ++i) acc[i] = 0.f;
    }
    __device__ __forceinline__ void group_done(int64_t gb, int64_t p_end, int lane) {
        if (!REWEIGHT) return;
        const int64_t q = gb + lane * Fmt<STORE>::PPL;
        if (STORE == FM_STORE_FP32) {
            static_cast<float *>(d.w)[q] = q < p_end ? out[0] : 0.f;
        } else {
            // the values are already multiples of the FP16 grid: the conversion is exact
            const float a = q < p_end ? out[0] : 0.f;
            const float b = q + 1 < p_end ? out[1] : 0.f;
            reinterpret_cast<__half2 *>(d.w)[q >> 1] = __floats2half2_rn(a, b);
        }
        out[0] = out[1] = 0.f;
    }
};

// groups in flight per warp and resident CTAs per SM of the accumulation pass (the 46 running
// sums leave room for few of either)
#ifndef FM_QUAD_UNROLL
#define FM_QUAD_UNROLL 4
#endif
#ifndef FM_QUAD_MIN_CTAS
#define FM_QUAD_MIN_CTAS 2
#endif

template <int STORE, bool REWEIGHT>
__global__ void __launch_bounds__(CTA_WARPS * 32, FM_QUAD_MIN_CTAS) k_quad_accumulate(DevProblem d, float tau) {
    __shared__ unsigned cta_kept;
    if (threadIdx.x == 0) cta_kept = 0;
    __syncthreads();
    const int r = blockIdx.x * CTA_WARPS + (threadIdx.x >> 5);
    if (r < d.n_ranges) {
        QuadBody<STORE, REWEIGHT> body(d, tau);
        walk_range<STORE, !REWEIGHT, QuadBody<STORE, REWEIGHT>, FM_QUAD_UNROLL>(d, r, threadIdx.x & 31, body);
        if (REWEIGHT) {
            unsigned k = body.kept;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
            if ((threadIdx.x & 31) == 0) atomicAdd(&cta_kept, k);
        }
    }
    if (REWEIGHT) {
        __syncthreads();
        if (threadIdx.x == 0 && cta_kept) atomicAdd(d.counter, (unsigned long long)cta_kept);
    }
}

// per pair (one warp, a lane per sum): Kahan-sum the range partials into the pair's record
//   [0..35] M, [36] c0, [37..45] g0, [46..54] e0 = E'_n of the geometry record, [55] 0
// (M first, so that the fused step reads it as 16-byte aligned vectors)
__global__ void k_quad_combine(DevProblem d) {
    const int n = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (n >= d.n_pairs) return;
    const int r0 = d.pair_off[n] / WR, r1 = (d.pair_off[n + 1] - 1) / WR;
    float *rec = d.quad + (size_t)n * QREC;
    for (int q = lane; q < QSUMS; q += 32) {
        float sum = 0.f, c = 0.f;
        for (int r = r0; r <= r1; ++r) {
            const float y = d.qslots[(size_t)(n + r) * QSLOT + q] - c;
            const float t = sum + y;
            c = (t - sum) - y;
            sum = t;
        }
        rec[q < 10 ? 36 + q : q - 10] = sum;
    }
    if (lane < 9) rec[46 + lane] = d.geo[(size_t)n * GEO + lane];
    if (lane == 9) rec[55] = 0.f;
}

// One optimiser iteration on the form, fused into one launch. Warp w owns camera
// k = 8 * block + w; its lanes take the camera's image pairs, each computing the pair's
// geometry from the two camera records (cam_src), the form's sums at the current E'_n,
//   q = g0 + W d,  loss = c0 + d^T (g0 + q),  d = E'_n - e0,
// and the chain rule to camera k. Both cameras of a pair evaluate it (O(1) each), which
// removes a per-pair launch and the wait on it. The warp reduces with compensated butterflies,
// then lanes 0..7 of warp 0 do the FP64 update of the block's cameras and write the new
// records to cam_dst: the records of this step's poses stay intact in cam_src for the other
// blocks. The Adam step count is *d.step + 1 + it; the launch that closes the chain adds
// the chain's length to *d.step.
template <bool FOCAL>
__global__ void __launch_bounds__(STEP_CAMS * 32, 4)
k_quad_step(DevProblem d, int it, const float *cam_src, float *cam_dst, float gscale, float lscale, int apply) {
    constexpr int NV = FOCAL ? STEP_VALS : STEP_VALS - 1;   // sums carried per camera
    __shared__ float s_hi[STEP_VALS][STEP_CAMS], s_lo[STEP_VALS][STEP_CAMS];
    __shared__ float s_mv[STEP_CAMS][12];
    __shared__ double s_Rc[STEP_CAMS][12];
    __shared__ float s_R32[STEP_CAMS][10];    // the cameras' records' rotations (9) and keypoint scale
    __shared__ double s_hyper[6];   // lr_rot, lr_c, beta1, beta2, eps, lr_focal
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = blockIdx.x * STEP_CAMS + warp;
    const int e_begin = k < d.n_cams ? d.cam_off[k] : 0;
    const int e_end = k < d.n_cams ? d.cam_off[k + 1] : 0;
    constexpr int SYM[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    // the camera's first 32 (pair, role) entries and the pairs' cameras are static: fetch them
    // while the previous step finishes
    int e = e_begin + lane;
    int n = 0, role = 0, ci = 0, cj = 0;
    if (e < e_end) {
        const int ent = d.cam_ent[e];
        n = ent >> 1;
        role = ent & 1;
        ci = d.cam_i[n];
        cj = d.cam_j[n];
    }
    pdl_wait();     // camera records, poses and moments of the previous step
    pdl_trigger();
    {
        const int cam0 = blockIdx.x * STEP_CAMS;
        for (int i = threadIdx.x; i < STEP_CAMS * 12; i += STEP_CAMS * 32) {
            const int cc = i / 12, q = i % 12;
            if (cam0 + cc < d.n_cams) {
                s_mv[cc][q] = q < 6 ? d.m[(size_t)(cam0 + cc) * 6 + q] : d.v[(size_t)(cam0 + cc) * 6 + q - 6];
                s_Rc[cc][q] = q < 9 ? d.R[(size_t)(cam0 + cc) * 9 + q] : d.c[(size_t)(cam0 + cc) * 3 + q - 9];
                if (q < 10) s_R32[cc][q] = cam_src[(size_t)(cam0 + cc) * CAMREC + (q < 9 ? q : 15)];
            }
        }
        if (threadIdx.x < 6) s_hyper[threadIdx.x] = d.hyper[threadIdx.x];
    }
    const long long t_step = *d.step + 1 + it;
    if (k < d.n_cams) {
        float hi[STEP_VALS], lo[STEP_VALS];
#pragma unroll
        for (int q = 0; q < STEP_VALS; ++q) hi[q] = lo[q] = 0.f;
        for (; e < e_end; e += 32) {
            if (e >= e_begin + 32) {
                const int ent = d.cam_ent[e];
                n = ent >> 1;
                role = ent & 1;
                ci = d.cam_i[n];
                cj = d.cam_j[n];
            }
            float g[GEO];
            if (!pair_geometry_regs(cam_src, d.cen, ci, cj, g)) atomicOr(d.err, ERR_DEGENERATE);
            const float4 *rec = reinterpret_cast<const float4 *>(d.quad + (size_t)n * QREC);
            float t[20];
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                const float4 x = rec[9 + v];
                t[4 * v] = x.x; t[4 * v + 1] = x.y; t[4 * v + 2] = x.z; t[4 * v + 3] = x.w;
            }
            // t[0] = c0, t[1..9] = g0, t[10..18] = e0
            float dv[9], q[9];
            float loss = t[0];
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                dv[a] = g[a] - t[10 + a];
                q[a] = t[1 + a];
                loss = fmaf(dv[a], t[1 + a], loss);
            }
#pragma unroll
            for (int c = 0; c < 9; ++c) {
                const float4 x = rec[c];
                const float mc[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int u = (4 * c + h) / 6, v = (4 * c + h) % 6;
#pragma unroll
                    for (int pp = 0; pp < 3; ++pp)
#pragma unroll
                        for (int r = 0; r < 3; ++r) {
                            if (SYM[pp][r] != u) continue;
#pragma unroll
                            for (int qq = 0; qq < 3; ++qq)
#pragma unroll
                                for (int ss = 0; ss < 3; ++ss)
                                    if (SYM[qq][ss] == v) q[3 * pp + qq] = fmaf(mc[h], dv[3 * r + ss], q[3 * pp + qq]);
                        }
                }
            }
#pragma unroll
            for (int a = 0; a < 9; ++a) loss = fmaf(dv[a], q[a], loss);
            const float sum[10] = {q[0], q[1], q[2], q[3], q[4], q[5], q[6], q[7], q[8], loss};
            float contrib[STEP_VALS];
            pair_chain_rule<FOCAL>(g, role, sum, gscale, lscale, contrib);
#pragma unroll
            for (int w = 0; w < NV; ++w) two_sum_acc(hi[w], lo[w], contrib[w], 0.f);
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
            ? camera_update<FOCAL>(d, kc, &s_hi[0][lane], &s_lo[0][lane], STEP_CAMS, s_mv[lane], s_Rc[lane], s_R32[lane], s_hyper,
                            t_step, apply, cam_dst + (size_t)kc * CAMREC)
            : 0.0;
        if (kc < d.n_cams) d.cam_loss[kc] = bl;
    }
}

static inline int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

// tau < 0: keep the current weights; otherwise reweight with threshold tau in the same pass
void launch_quad_accumulate(const DevProblem &d, float tau, cudaStream_t s) {
    const int grid = blocks_for(d.n_ranges, CTA_WARPS);
    const dim3 block(CTA_WARPS * 32);
    if (tau < 0.f) {
        if (d.storage == FM_STORE_FP32) k_quad_accumulate<FM_STORE_FP32, false><<<grid, block, 0, s>>>(d, tau);
        else k_quad_accumulate<FM_STORE_FP16, false><<<grid, block, 0, s>>>(d, tau);
    } else {
        if (d.storage == FM_STORE_FP32) k_quad_accumulate<FM_STORE_FP32, true><<<grid, block, 0, s>>>(d, tau);
        else k_quad_accumulate<FM_STORE_FP16, true><<<grid, block, 0, s>>>(d, tau);
    }
}

void launch_quad_combine(const DevProblem &d, cudaStream_t s) {
    k_quad_combine<<<blocks_for(d.n_pairs, 8), 256, 0, s>>>(d);
}

void launch_quad_step(const DevProblem &d, int it, const float *cam_src, float *cam_dst, bool apply,
                      cudaStream_t s, bool pdl) {
    float gscale, lscale;
    loss_scales(d, gscale, lscale);
    if (d.refine_focal)
        launch_k(k_quad_step<true>, dim3(camera_step_blocks(d)), dim3(STEP_CAMS * 32), s, pdl, d, it, cam_src,
                 cam_dst, gscale, lscale, apply ? 1 : 0);
    else
        launch_k(k_quad_step<false>, dim3(camera_step_blocks(d)), dim3(STEP_CAMS * 32), s, pdl, d, it, cam_src,
                 cam_dst, gscale, lscale, apply ? 1 : 0);
}

}  // namespace fm
