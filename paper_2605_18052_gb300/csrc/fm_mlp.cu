// Learned inlier weights: a small MLP (8 -> 32 -> 32 -> 1, ReLU, sigmoid) that predicts the
// probability p that a point pair is an inlier from its residual history, its match score and
// statistics of its image pair; the reweighting step of the IRLS loop (Sec. "Epipolar
// Adjustment") then uses w = p / max(|eps|, delta). The thesis has no learned component; the
// network, its features and its training follow the benchmark's description.
//
// Numerics (shared by inference and training): features, weights and hidden activations are
// rounded to BF16, every product is accumulated in FP32, biases are FP32.
//   * inference runs inside the streaming walk on the tensor cores (mma.sync m16n8k16 BF16,
//     FP32 accumulate): 16 point pairs per tile, 14 MMAs per tile; the FP32 accumulator
//     fragments of one layer are the BF16 A fragments of the next after packing, so no
//     shuffles are needed between layers;
//   * training runs one sample per thread (forward and backward), reduces the gradient per
//     block in a fixed order and applies FP32 Adam to FP32 master parameters.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <string>

#include "fm_tcgen05.cuh"
#include "fm_walk.cuh"

namespace fm {

// ---- per-pair statistics of the current residuals ---------------------------------------------
struct StatsBody {
    const DevProblem &d;
    float tau;
    float acc[2];
    __device__ StatsBody(const DevProblem &dd, float t) : d(dd), tau(t) { acc[0] = acc[1] = 0.f; }
    __device__ __forceinline__ void segment_begin(int) {}
    __device__ __forceinline__ void point(int, float e, float, float, float, float, float) {
        const float a = fabsf(e);
        acc[0] += __logf(a + LOG_FLOOR);
        acc[1] += a <= tau ? 1.f : 0.f;
    }
    __device__ __forceinline__ void segment_end(int seg, int r, int lane, bool) {
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
        if (lane == 0) {
            d.slots[(size_t)(seg + r) * SLOT] = acc[0];
            d.slots[(size_t)(seg + r) * SLOT + 1] = acc[1];
        }
        acc[0] = acc[1] = 0.f;
    }
    __device__ __forceinline__ void group_done(int64_t, int64_t, int) {}
};

template <int STORE>
__global__ void __launch_bounds__(CTA_WARPS * 32) k_pair_stats(DevProblem d, float tau) {
    const int r = blockIdx.x * CTA_WARPS + (threadIdx.x >> 5);
    if (r >= d.n_ranges) return;
    StatsBody body(d, tau);
    walk_range<STORE, false>(d, r, threadIdx.x & 31, body);
}

__global__ void k_pair_stats_combine(DevProblem d) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= d.n_pairs) return;
    const int p0 = d.pair_off[n], p1 = d.pair_off[n + 1];
    float s0 = 0.f, s1 = 0.f;
    for (int r = p0 / WR; r <= (p1 - 1) / WR; ++r) {
        s0 += d.slots[(size_t)(n + r) * SLOT];
        s1 += d.slots[(size_t)(n + r) * SLOT + 1];
    }
    const float cnt = (float)(p1 - p0);
    reinterpret_cast<float4 *>(d.pstat)[n] = make_float4(s0 / cnt, s1 / cnt, logf(cnt) * 0.1f, 0.f);
}

// ---- tensor-core MLP on 16-row tiles ------------------------------------------------------------
__device__ __forceinline__ void mma_bf16(float *c, const unsigned *a, unsigned b0, unsigned b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned *>(&v);
}

// max(lo, 0) and max(hi, 0) rounded to BF16 and packed (lo in the low half): one instruction,
// the same bits as pack_bf16(fmaxf(lo, 0), fmaxf(hi, 0))
__device__ __forceinline__ unsigned pack_relu_bf16(float lo, float hi) {
    unsigned d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// The per-lane B fragments and bias slices of the three layers.
// For lane (g = lane / 4, t = lane % 4): B fragment of an n-tile j holds W[k][8j + g] for
// k = 2t, 2t+1 (b0) and k = 2t+8, 2t+9 (b1); accumulator columns are 8j + 2t, 8j + 2t + 1.
struct MlpFrag {
    unsigned w1[4];        // layer 1: K = 8 (padded to 16: b1 = 0), 4 n-tiles
    unsigned w2[2][4][2];  // layer 2: 2 k-tiles x 4 n-tiles x (b0, b1)
    unsigned w3[2][2];     // layer 3: 2 k-tiles x (b0, b1), only column 0 real
    float b1[4][2], b2[4][2], b3;
};

__device__ __forceinline__ void load_frag(MlpFrag &f, const float *master, const __nv_bfloat16 *wbf, int lane) {
    const int g = lane >> 2, t = lane & 3;
    const __nv_bfloat16 *W1 = wbf, *W2 = wbf + MLP_IN * MLP_H, *W3 = W2 + MLP_H * MLP_H;
    auto pk = [](__nv_bfloat16 lo, __nv_bfloat16 hi) {
        return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
    };
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        f.w1[j] = pk(W1[(2 * t) * MLP_H + 8 * j + g], W1[(2 * t + 1) * MLP_H + 8 * j + g]);
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            const int k0 = 16 * kk + 2 * t;
            f.w2[kk][j][0] = pk(W2[k0 * MLP_H + 8 * j + g], W2[(k0 + 1) * MLP_H + 8 * j + g]);
            f.w2[kk][j][1] = pk(W2[(k0 + 8) * MLP_H + 8 * j + g], W2[(k0 + 9) * MLP_H + 8 * j + g]);
        }
        f.b1[j][0] = master[MLP_OFF_B1 + 8 * j + 2 * t];
        f.b1[j][1] = master[MLP_OFF_B1 + 8 * j + 2 * t + 1];
        f.b2[j][0] = master[MLP_OFF_B2 + 8 * j + 2 * t];
        f.b2[j][1] = master[MLP_OFF_B2 + 8 * j + 2 * t + 1];
    }
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
        const int k0 = 16 * kk + 2 * t;
        f.w3[kk][0] = g == 0 ? pk(W3[k0], W3[k0 + 1]) : 0u;
        f.w3[kk][1] = g == 0 ? pk(W3[k0 + 8], W3[k0 + 9]) : 0u;
    }
    f.b3 = master[MLP_OFF_B3];
}

// p = sigmoid(MLP(x)) for `ntiles` tiles of 16 rows of xs (BF16, 8 features per row)
__device__ __forceinline__ void mlp_tiles(const MlpFrag &f, const __nv_bfloat16 (*xs)[MLP_IN], float *ps,
                                          int ntiles, int lane) {
    const int g = lane >> 2, t = lane & 3;
    for (int tile = 0; tile < ntiles; ++tile) {
        const int r0 = 16 * tile + g, r1 = r0 + 8;
        const unsigned a1[4] = {*reinterpret_cast<const unsigned *>(&xs[r0][2 * t]),
                                *reinterpret_cast<const unsigned *>(&xs[r1][2 * t]), 0u, 0u};
        float h1[4][4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            h1[j][0] = f.b1[j][0];
            h1[j][1] = f.b1[j][1];
            h1[j][2] = f.b1[j][0];
            h1[j][3] = f.b1[j][1];
            mma_bf16(h1[j], a1, f.w1[j], 0u);
        }
        unsigned a2[2][4];
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            a2[kk][0] = pack_relu_bf16(h1[2 * kk][0], h1[2 * kk][1]);
            a2[kk][1] = pack_relu_bf16(h1[2 * kk][2], h1[2 * kk][3]);
            a2[kk][2] = pack_relu_bf16(h1[2 * kk + 1][0], h1[2 * kk + 1][1]);
            a2[kk][3] = pack_relu_bf16(h1[2 * kk + 1][2], h1[2 * kk + 1][3]);
        }
        float h2[4][4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            h2[j][0] = f.b2[j][0];
            h2[j][1] = f.b2[j][1];
            h2[j][2] = f.b2[j][0];
            h2[j][3] = f.b2[j][1];
            mma_bf16(h2[j], a2[0], f.w2[0][j][0], f.w2[0][j][1]);
            mma_bf16(h2[j], a2[1], f.w2[1][j][0], f.w2[1][j][1]);
        }
        unsigned a3[2][4];
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            a3[kk][0] = pack_relu_bf16(h2[2 * kk][0], h2[2 * kk][1]);
            a3[kk][1] = pack_relu_bf16(h2[2 * kk][2], h2[2 * kk][3]);
            a3[kk][2] = pack_relu_bf16(h2[2 * kk + 1][0], h2[2 * kk + 1][1]);
            a3[kk][3] = pack_relu_bf16(h2[2 * kk + 1][2], h2[2 * kk + 1][3]);
        }
        float z[4] = {t == 0 ? f.b3 : 0.f, 0.f, t == 0 ? f.b3 : 0.f, 0.f};
        mma_bf16(z, a3[0], f.w3[0][0], f.w3[0][1]);
        mma_bf16(z, a3[1], f.w3[1][0], f.w3[1][1]);
        if (t == 0) {
            ps[r0] = __frcp_rn(1.f + __expf(-z[0]));
            ps[r1] = __frcp_rn(1.f + __expf(-z[2]));
        }
    }
}

// learned IRLS weight p / max(|eps|, delta) (fast quotient, within 2 ulp; every learned kernel
// uses this one expression, so the fused and separate passes agree bit for bit)
__device__ __forceinline__ float learned_weight(float p, float ae, float delta) {
    return __fdividef(p, fmaxf(ae, delta));
}

// ---- features of a point pair ---------------------------------------------------------------------
//  0 log(|e|+1e-6) - log(tau)      1 log(|e|+1e-6) - pair mean log    2 log(|e_prev|+1e-6) - log(|e|+1e-6)
//  3 match score                   4 pair fraction with |e| <= tau    5 log(pair count) / 10
//  6 round / 10                    7 log(|e_prev|+1e-6) - log(tau)
template <int STORE, bool COLLECT>
struct LearnedBody {
    static constexpr int PPL = Fmt<STORE>::PPL;
    static constexpr int GROUP = 32 * PPL;
    const DevProblem &d;
    float log_tau, tau_cap, delta, wscale, round_f;
    int hist_valid;
    float st_mean, st_frac, st_cnt;
    float ae[PPL], le[PPL], sm[PPL], sf[PPL], sc[PPL];
    unsigned kept;
    MlpFrag frag;     // the network's B fragments, in registers
    __nv_bfloat16 (*xs)[MLP_IN];
    float *ps;
    __nv_bfloat16 *feat_out;
    __device__ LearnedBody(const DevProblem &dd) : d(dd), kept(0) {}
    __device__ __forceinline__ void segment_begin(int seg) {
        const float4 p = reinterpret_cast<const float4 *>(d.pstat)[seg];
        st_mean = p.x;
        st_frac = p.y;
        st_cnt = p.z;
    }
    __device__ __forceinline__ void point(int k, float e, float, float, float, float, float) {
        ae[k] = fabsf(e);
        le[k] = __logf(ae[k] + LOG_FLOOR);
        sm[k] = st_mean;
        sf[k] = st_frac;
        sc[k] = st_cnt;
    }
    __device__ __forceinline__ void segment_end(int, int, int, bool) {}
    __device__ __forceinline__ void group_done(int64_t gb, int64_t p_end, int lane) {
        const int64_t q = gb + lane * PPL;
        float lp[PPL], sco[PPL];
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            lp[k] = hist_valid ? __half2float(d.le_hist[q + k]) : le[k];
            sco[k] = __half2float(d.score[q + k]);
        }
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            float f[MLP_IN];
            f[0] = le[k] - log_tau;
            f[1] = le[k] - sm[k];
            f[2] = lp[k] - le[k];
            f[3] = sco[k];
            f[4] = sf[k];
            f[5] = sc[k];
            f[6] = round_f;
            f[7] = lp[k] - log_tau;
            __align__(16) __nv_bfloat16 fb[MLP_IN];
#pragma unroll
            for (int i = 0; i < MLP_IN; ++i) fb[i] = __float2bfloat16_rn(f[i]);
            if (COLLECT) {
                if (q + k < p_end) {
                    const int64_t dst = d.perm ? d.perm[q + k] : q + k;
                    *reinterpret_cast<uint4 *>(feat_out + dst * MLP_IN) = *reinterpret_cast<const uint4 *>(fb);
                }
            } else {
                *reinterpret_cast<uint4 *>(xs[lane * PPL + k]) = *reinterpret_cast<const uint4 *>(fb);
            }
        }
        if (!COLLECT) {
            __syncwarp();
            mlp_tiles(frag, xs, ps, GROUP / 16, lane);
            __syncwarp();
            float w[PPL];
#pragma unroll
            for (int k = 0; k < PPL; ++k) {
                const bool in = q + k < p_end && ae[k] <= tau_cap;
                w[k] = in ? learned_weight(ps[lane * PPL + k], ae[k], delta) : 0.f;
                kept += in ? 1u : 0u;
            }
            if (STORE == FM_STORE_FP32) {
                static_cast<float *>(d.w)[q] = w[0];
            } else {
                reinterpret_cast<__half2 *>(d.w)[q >> 1] = __floats2half2_rn(w[0] * wscale, w[PPL - 1] * wscale);
            }
            __syncwarp();
        }
#pragma unroll
        for (int k = 0; k < PPL; ++k)
            if (q + k < p_end) d.le_hist[q + k] = __float2half_rn(le[k]);
#pragma unroll
        for (int k = 0; k < PPL; ++k) ae[k] = le[k] = 0.f;
    }
};

template <int STORE, bool COLLECT>
__global__ void __launch_bounds__(CTA_WARPS * 32, 2)
k_learned(DevProblem d, const float *master, const __nv_bfloat16 *wbf, float tau, float tau_cap,
          int round, int hist_valid, __nv_bfloat16 *feat_out) {
    constexpr int GROUP = 32 * Fmt<STORE>::PPL;
    __shared__ __align__(16) __nv_bfloat16 xs[CTA_WARPS][GROUP][MLP_IN];
    __shared__ float ps[CTA_WARPS][GROUP];
    __shared__ unsigned cta_kept;
    if (threadIdx.x == 0) cta_kept = 0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    const int r = blockIdx.x * CTA_WARPS + w;
    if (r < d.n_ranges) {
        LearnedBody<STORE, COLLECT> body(d);
        if (!COLLECT) load_frag(body.frag, master, wbf, lane);
        body.log_tau = __logf(tau);
        body.tau_cap = tau_cap;
        body.delta = (float)d.delta;
        body.wscale = d.w_scale;
        body.round_f = round * 0.1f;
        body.hist_valid = hist_valid;
        body.xs = xs[w];
        body.ps = ps[w];
        body.feat_out = feat_out;
        // one group in flight: the fragments take the registers a deeper unroll would use
        walk_range<STORE, false, LearnedBody<STORE, COLLECT>, 1>(d, r, lane, body);
        unsigned k = body.kept;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
        if (lane == 0) atomicAdd(&cta_kept, k);
    }
    __syncthreads();
    if (!COLLECT && threadIdx.x == 0 && cta_kept) atomicAdd(d.counter, (unsigned long long)cta_kept);
}

// ---- the learned reweighting fused with the round's first loss + adjoint pass -------------------
// Same arithmetic as k_learned followed by k_stream_loss, one read of the keypoints instead of
// two. Every group of 32 * PPL point pairs is handled in two phases:
//   A: residual, features (with the statistics of each point pair's own image pair), the MLP on
//      the group's rows (tensor cores, mma.sync), the weight (written, FP16-quantised for FP16
//      storage), the residual history;
//   B: the loss and adjoint sums of the group with those weights, closing every image pair that
//      ended inside the group (warp butterfly into its slot n + r, as the streaming pass does).
// Phase A walks the group's image pairs forward; phase B revisits the same image pairs from the
// group's first one. The network's B fragments stay in registers for the whole kernel (reading
// them from shared memory for every 16-row tile would move about 330 B of shared memory per
// point pair); to make room, the keypoints stay packed between the phases and the current image
// pair's E'_n and statistics are reloaded (from L1) at the start of every group.
template <int STORE>
__global__ void __launch_bounds__(CTA_WARPS * 32, 2)
k_learned_loss(DevProblem d, const float *master, const __nv_bfloat16 *wbf, float tau, float tau_cap, int round,
               int hist_valid) {
    using F = Fmt<STORE>;
    constexpr int PPL = F::PPL;
    constexpr int GROUP = 32 * PPL;
    __shared__ __align__(16) __nv_bfloat16 xs[CTA_WARPS][GROUP][MLP_IN];
    __shared__ float ps[CTA_WARPS][GROUP];
    __shared__ unsigned cta_kept;
    if (threadIdx.x == 0) cta_kept = 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    MlpFrag frag;
    load_frag(frag, master, wbf, lane);
    pdl_wait();     // pair geometry and statistics of this pass
    pdl_trigger();
    __syncthreads();
    const int r = blockIdx.x * CTA_WARPS + wid;
    unsigned kept = 0;
    if (r < d.n_ranges) {
        const float log_tau = __logf(tau), delta = (float)d.delta, wscale = d.w_scale, round_f = round * 0.1f;
        const int64_t p_begin = (int64_t)r * WR;
        const int64_t p_end = min(p_begin + (int64_t)WR, d.n_pp);
        int seg = d.range_pair[r];
        int64_t seg_end = d.pair_off[seg + 1];
        LossBody<MODE_LOSS_IRLS> loss(d);
        const uint64_t pol = evict_first_policy();
        for (int64_t gb = p_begin; gb < p_end; gb += GROUP) {
            const int64_t q0 = gb + lane * PPL;
            const typename F::Raw raw = F::load(d, q0, false, pol);
            // score and history of the lane's point pairs (PPL consecutive halves)
            float sco[PPL], lp[PPL];
            if (PPL == 2) {
                const float2 sv = __half22float2(reinterpret_cast<const __half2 *>(d.score)[q0 >> 1]);
                const float2 hv = __half22float2(reinterpret_cast<const __half2 *>(d.le_hist)[q0 >> 1]);
                sco[0] = sv.x;
                sco[PPL - 1] = sv.y;
                lp[0] = hv.x;
                lp[PPL - 1] = hv.y;
            } else {
                sco[0] = __half2float(d.score[q0]);
                lp[0] = __half2float(d.le_hist[q0]);
            }
            float e[PPL], le[PPL];
#pragma unroll
            for (int k = 0; k < PPL; ++k) e[k] = le[k] = 0.f;
            // phase A
            const int seg0 = seg;
            const int64_t seg0_end = seg_end;
            const int64_t g_end = min(gb + GROUP, p_end);
            float E[9];
            load_E(d.geo, seg, E);
            float4 st = reinterpret_cast<const float4 *>(d.pstat)[seg];
            int64_t lo = gb;
            while (true) {
                const int64_t hi = min(seg_end, p_end);
#pragma unroll
                for (int k = 0; k < PPL; ++k) {
                    const int64_t q = q0 + k;
                    if (q >= lo && q < hi) {
                        float x1, y1, x2, y2, unused;
                        F::get(raw, k, x1, y1, x2, y2, unused);
                        e[k] = epi(E, x1, y1, x2, y2);
                        le[k] = __logf(fabsf(e[k]) + LOG_FLOOR);
                        const float lpk = hist_valid ? lp[k] : le[k];
                        float f[MLP_IN];
                        f[0] = le[k] - log_tau;
                        f[1] = le[k] - st.x;
                        f[2] = lpk - le[k];
                        f[3] = sco[k];
                        f[4] = st.y;
                        f[5] = st.z;
                        f[6] = round_f;
                        f[7] = lpk - log_tau;
                        __align__(16) __nv_bfloat16 fb[MLP_IN];
#pragma unroll
                        for (int i = 0; i < MLP_IN; ++i) fb[i] = __float2bfloat16_rn(f[i]);
                        *reinterpret_cast<uint4 *>(xs[wid][lane * PPL + k]) = *reinterpret_cast<const uint4 *>(fb);
                    }
                }
                if (seg_end >= g_end) break;
                lo = seg_end;
                ++seg;
                seg_end = d.pair_off[seg + 1];
                load_E(d.geo, seg, E);
                st = reinterpret_cast<const float4 *>(d.pstat)[seg];
            }
#pragma unroll
            for (int k = 0; k < PPL; ++k)   // rows past the end of the range: any finite input
                if (q0 + k >= p_end) *reinterpret_cast<uint4 *>(xs[wid][lane * PPL + k]) = make_uint4(0u, 0u, 0u, 0u);
            __syncwarp();
            mlp_tiles(frag, xs[wid], ps[wid], GROUP / 16, lane);
            __syncwarp();
            float w[PPL];
#pragma unroll
            for (int k = 0; k < PPL; ++k) {
                const float ae = fabsf(e[k]);
                const bool in = q0 + k < p_end && ae <= tau_cap;
                const float wf = in ? learned_weight(ps[wid][lane * PPL + k], ae, delta) : 0.f;
                w[k] = STORE == FM_STORE_FP32 ? wf : __half2float(__float2half_rn(wf * wscale));
                kept += in ? 1u : 0u;
            }
            if (STORE == FM_STORE_FP32) {
                static_cast<float *>(d.w)[q0] = w[0];
                if (q0 < p_end) d.le_hist[q0] = __float2half_rn(le[0]);
            } else {
                reinterpret_cast<__half2 *>(d.w)[q0 >> 1] = __floats2half2_rn(w[0], w[PPL - 1]);
                const __half2 hv = __floats2half2_rn(le[0], le[PPL - 1]);
                if (q0 + 1 < p_end) reinterpret_cast<__half2 *>(d.le_hist)[q0 >> 1] = hv;
                else if (q0 < p_end) d.le_hist[q0] = __low2half(hv);
            }
            __syncwarp();
            // phase B
            int sb = seg0;
            int64_t sb_end = seg0_end;
            lo = gb;
            while (true) {
                const int64_t hi = min(sb_end, p_end);
#pragma unroll
                for (int k = 0; k < PPL; ++k) {
                    const int64_t q = q0 + k;
                    if (q >= lo && q < hi) {
                        float x1, y1, x2, y2, unused;
                        F::get(raw, k, x1, y1, x2, y2, unused);
                        loss.point(k, e[k], x1, y1, x2, y2, w[k]);
                    }
                }
                if (sb == seg) break;
                loss.segment_end(sb, r, lane, false);
                lo = sb_end;
                ++sb;
                sb_end = d.pair_off[sb + 1];
            }
        }
        loss.segment_end(seg, r, lane, true);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
    if (lane == 0 && kept) atomicAdd(&cta_kept, kept);
    __syncthreads();
    if (threadIdx.x == 0 && cta_kept) atomicAdd(d.counter, (unsigned long long)cta_kept);
}

// ---- the learned reweighting on the fifth-generation tensor cores (tcgen05) ---------------------
// A CTA is one warpgroup (4 warps); each warp streams its own warp range as in the other passes,
// and for every group of 32 * PPL point pairs per warp the warpgroup's 128 x PPL rows go through
// the network as MMAs of M = 128 rows with FP32 accumulators in TMEM (k = the lane's k-th point
// pair of the group, one MMA row block per k):
//   L1  D1[k] (128 x 32) = A1[k] (128 x 16: 8 features, three 1s, 5 zeros) . B1^T
//        B1 (32 x 16) = W1^T with b1 in its columns 8..10 as three BF16 parts (hi + mid + lo = b1)
//   L2  D2[k] (128 x 32) = A2[k] (128 x 48: bf16(relu(D1)), three 1s, zeros) . B2^T (W2^T, b2 parts)
//   L3  D3[k] (128 x 16, column 0 used) = A3[k] (A2's layout, from D2) . B3^T (row 0: W3, b3 parts)
// so the biases are added inside the FP32 accumulation and every row's epilogue is one TMEM load,
// one ReLU-and-round instruction per two values and four 16-byte shared-memory stores. One thread
// issues the MMAs and commits them to an mbarrier; the warpgroup waits on it (bounded: a wait that
// runs out records ERR_NONFINITE and the warpgroup leaves the loop together).
// Footprint (the pass is bound by the latency of the MMA round trips, so what matters is how many
// row blocks an SM keeps in flight): D1, D2 and D3 of row block k share TMEM columns 32 k .. 32 k
// + 31 (each layer's result is read before the next layer's MMA is issued), 64 columns per CTA;
// A1 lives inside A2's buffer: the features take A2's first K core matrix and layer 1 reads its
// second K core matrix from A2's fifth (the constant bias inputs), through the descriptor's
// leading byte offset.
// FUSE: also accumulate the loss + adjoint sums with the new weights (the round's first pass).
constexpr int TC_THREADS = 128;
constexpr uint32_t TC_COLS = 64;
constexpr int TC_K1 = 16, TC_K2 = 48;      // padded K of layer 1 and of layers 2 and 3
constexpr long long TC_WAIT_CYCLES = 2000000000LL;   // about one second

struct TcSmem {
    alignas(128) unsigned char a2[2][128 * TC_K2 * 2];
    alignas(128) unsigned char b1[32 * TC_K1 * 2];
    alignas(128) unsigned char b2[32 * TC_K2 * 2];
    alignas(128) unsigned char b3[16 * TC_K2 * 2];
    alignas(8) uint64_t mbar;
    uint32_t tmem;
    int fail;
    unsigned kept;
};

__device__ __forceinline__ void put_bf16(unsigned char *base, uint32_t r, uint32_t k, uint32_t kp, float v) {
    *reinterpret_cast<__nv_bfloat16 *>(base + tc_offset(r, k, kp)) = __float2bfloat16_rn(v);
}

// v = hi + mid + lo with three BF16 values (exact for FP32 v up to the last bit of lo)
__device__ __forceinline__ void bf16_split3(float v, float &hi, float &mid, float &lo) {
    hi = __bfloat162float(__float2bfloat16_rn(v));
    mid = __bfloat162float(__float2bfloat16_rn(v - hi));
    lo = v - hi - mid;
}

// the network's B operands and the constant columns of the A operands, by the whole CTA
__device__ __forceinline__ void tc_setup(TcSmem &sm, const float *master, const __nv_bfloat16 *wbf) {
    const int tid = threadIdx.x;
    const __nv_bfloat16 *W1 = wbf, *W2 = wbf + MLP_IN * MLP_H, *W3 = W2 + MLP_H * MLP_H;
    for (int i = tid; i < 32 * TC_K1; i += TC_THREADS) {
        const int n = i / TC_K1, k = i % TC_K1;
        float v = 0.f;
        if (k < MLP_IN) v = __bfloat162float(W1[k * MLP_H + n]);
        else if (k < MLP_IN + 3) {
            float h, m, l;
            bf16_split3(master[MLP_OFF_B1 + n], h, m, l);
            v = k == MLP_IN ? h : (k == MLP_IN + 1 ? m : l);
        }
        put_bf16(sm.b1, n, k, TC_K1, v);
    }
    for (int i = tid; i < 32 * TC_K2; i += TC_THREADS) {
        const int n = i / TC_K2, k = i % TC_K2;
        float v = 0.f;
        if (k < MLP_H) v = __bfloat162float(W2[k * MLP_H + n]);
        else if (k < MLP_H + 3) {
            float h, m, l;
            bf16_split3(master[MLP_OFF_B2 + n], h, m, l);
            v = k == MLP_H ? h : (k == MLP_H + 1 ? m : l);
        }
        put_bf16(sm.b2, n, k, TC_K2, v);
    }
    for (int i = tid; i < 16 * TC_K2; i += TC_THREADS) {
        const int n = i / TC_K2, k = i % TC_K2;
        float v = 0.f;
        if (n == 0 && k < MLP_H) v = __bfloat162float(W3[k]);
        else if (n == 0 && k < MLP_H + 3) {
            float h, m, l;
            bf16_split3(master[MLP_OFF_B3], h, m, l);
            v = k == MLP_H ? h : (k == MLP_H + 1 ? m : l);
        }
        put_bf16(sm.b3, n, k, TC_K2, v);
    }
    // A2 columns 32..47: three 1s (the bias inputs of every layer) and zeros
    for (int i = tid; i < 2 * 128 * (TC_K2 - MLP_H); i += TC_THREADS) {
        const int kk = i / (128 * (TC_K2 - MLP_H)), rem = i % (128 * (TC_K2 - MLP_H));
        const int r = rem / (TC_K2 - MLP_H), k = MLP_H + rem % (TC_K2 - MLP_H);
        put_bf16(sm.a2[kk], r, k, TC_K2, k < MLP_H + 3 ? 1.f : 0.f);
    }
}

// bf16(relu(x)) of 32 accumulator columns into row `row` of an A operand (K padded to TC_K2)
__device__ __forceinline__ void tc_relu_row(unsigned char *a, int row, const uint32_t (&acc)[32]) {
#pragma unroll
    for (int kb = 0; kb < 4; ++kb) {
        uint4 v;
        v.x = pack_relu_bf16(__uint_as_float(acc[8 * kb + 0]), __uint_as_float(acc[8 * kb + 1]));
        v.y = pack_relu_bf16(__uint_as_float(acc[8 * kb + 2]), __uint_as_float(acc[8 * kb + 3]));
        v.z = pack_relu_bf16(__uint_as_float(acc[8 * kb + 4]), __uint_as_float(acc[8 * kb + 5]));
        v.w = pack_relu_bf16(__uint_as_float(acc[8 * kb + 6]), __uint_as_float(acc[8 * kb + 7]));
        *reinterpret_cast<uint4 *>(a + tc_offset(row, 8 * kb, TC_K2)) = v;
    }
}

// all warpgroup threads: make the A rows visible to the tensor core and hand over to the issuer;
// returns whether an earlier wait ran out (then everybody leaves)
__device__ __forceinline__ bool tc_handover(TcSmem &sm) {
    fence_smem_async();
    tc_fence_before_sync();
    named_sync(1, TC_THREADS);
    return sm.fail != 0;
}

__device__ __forceinline__ void tc_wait(TcSmem &sm, uint32_t &phase) {
    if (!mbar_wait(smem_addr(&sm.mbar), phase, TC_WAIT_CYCLES)) sm.fail = 1;
    phase ^= 1u;
    tc_fence_after_sync();
}

template <int STORE, bool FUSE>
__global__ void __launch_bounds__(TC_THREADS, 5)
k_learned_tc(DevProblem d, const float *master, const __nv_bfloat16 *wbf, float tau, float tau_cap, int round,
             int hist_valid) {
    using F = Fmt<STORE>;
    constexpr int PPL = F::PPL;
    constexpr int GROUP = 32 * PPL;
    constexpr int NG = WR / GROUP;
    __shared__ TcSmem sm;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int row = 32 * wid + lane;
    if (wid == 0) {
        tmem_alloc(smem_addr(&sm.tmem), TC_COLS);
        tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        mbar_init(smem_addr(&sm.mbar), 1);
        sm.fail = 0;
        sm.kept = 0;
    }
    tc_setup(sm, master, wbf);
    pdl_wait();     // pair geometry and statistics of this pass
    pdl_trigger();
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tm = sm.tmem + ((uint32_t)(32 * wid) << 16);   // this warp's TMEM lanes
    const uint32_t id1 = tc_idesc_bf16(128, 32), id3 = tc_idesc_bf16(128, 16);
    // operand descriptors (loop-invariant; K slice sl of layers 2 and 3 adds sl * 2 * TC_LBO to
    // the start address field, i.e. sl * 16 in 16-byte units)
    const uint64_t dA1[2] = {tc_desc(smem_addr(sm.a2[0]), TC_K2 * 16, 4 * TC_LBO),
                             tc_desc(smem_addr(sm.a2[1]), TC_K2 * 16, 4 * TC_LBO)};
    const uint64_t dA2[2] = {tc_desc(smem_addr(sm.a2[0]), TC_K2 * 16), tc_desc(smem_addr(sm.a2[1]), TC_K2 * 16)};
    const uint64_t dB1 = tc_desc(smem_addr(sm.b1), TC_K1 * 16), dB2 = tc_desc(smem_addr(sm.b2), TC_K2 * 16),
                   dB3 = tc_desc(smem_addr(sm.b3), TC_K2 * 16);
    constexpr uint64_t SLICE = (2 * TC_LBO) >> 4;
    uint32_t phase = 0;

    const int r = blockIdx.x * 4 + wid;
    const bool r_ok = r < d.n_ranges;
    const float log_tau = __logf(tau), delta = (float)d.delta, wscale = d.w_scale, round_f = round * 0.1f;
    const int64_t p_begin = (int64_t)r * WR;
    const int64_t p_end = r_ok ? min(p_begin + (int64_t)WR, d.n_pp) : p_begin;
    int seg = r_ok ? d.range_pair[r] : 0;
    int64_t seg_end = r_ok ? d.pair_off[seg + 1] : 0;
    LossBody<MODE_LOSS_IRLS> loss(d);
    unsigned kept = 0;
    const uint64_t pol = evict_first_policy();
    // the keypoints, scores and history of the next group are loaded one group ahead, so their
    // latency overlaps the current group's MMAs
    typename F::Raw nraw;
    unsigned nsc = 0u, nhi = 0u;
    auto fetch = [&](int64_t gq) {
        nraw = F::load(d, gq, false, pol);
        if (PPL == 2) {
            nsc = *reinterpret_cast<const unsigned *>(d.score + gq);
            nhi = *reinterpret_cast<const unsigned *>(d.le_hist + gq);
        } else {
            nsc = __half_as_ushort(d.score[gq]);
            nhi = __half_as_ushort(d.le_hist[gq]);
        }
    };
    if (p_begin < p_end) fetch(p_begin + lane * PPL);
    for (int g = 0; g < NG; ++g) {
        const int64_t gb = p_begin + (int64_t)g * GROUP;
        const bool active = gb < p_end;   // warp-uniform
        const int64_t q0 = gb + lane * PPL;
        typename F::Raw raw = nraw;
        const unsigned csc = nsc, chi = nhi;
        if (gb + GROUP < p_end) fetch(q0 + GROUP);
        float sco[PPL], lp[PPL], e[PPL], le[PPL];
#pragma unroll
        for (int k = 0; k < PPL; ++k) sco[k] = lp[k] = e[k] = le[k] = 0.f;
        int seg0 = seg;
        int64_t seg0_end = seg_end;
        // ---- phase A: features of the lane's point pairs into A1[k], row `row`
        uint4 feat[PPL];
#pragma unroll
        for (int k = 0; k < PPL; ++k) feat[k] = make_uint4(0u, 0u, 0u, 0u);
        if (active) {
            if (PPL == 2) {
                const float2 sv = __half22float2(*reinterpret_cast<const __half2 *>(&csc));
                const float2 hv = __half22float2(*reinterpret_cast<const __half2 *>(&chi));
                sco[0] = sv.x;
                sco[PPL - 1] = sv.y;
                lp[0] = hv.x;
                lp[PPL - 1] = hv.y;
            } else {
                sco[0] = __half2float(__ushort_as_half((unsigned short)csc));
                lp[0] = __half2float(__ushort_as_half((unsigned short)chi));
            }
            const int64_t g_end = min(gb + GROUP, p_end);
            float E[9];
            load_E(d.geo, seg, E);
            float4 st = reinterpret_cast<const float4 *>(d.pstat)[seg];
            int64_t lo = gb;
            while (true) {
                const int64_t hi = min(seg_end, p_end);
#pragma unroll
                for (int k = 0; k < PPL; ++k) {
                    const int64_t q = q0 + k;
                    if (q >= lo && q < hi) {
                        float x1, y1, x2, y2, unused;
                        F::get(raw, k, x1, y1, x2, y2, unused);
                        e[k] = epi(E, x1, y1, x2, y2);
                        le[k] = __logf(fabsf(e[k]) + LOG_FLOOR);
                        const float lpk = hist_valid ? lp[k] : le[k];
                        feat[k] = make_uint4(pack_bf16(le[k] - log_tau, le[k] - st.x),
                                             pack_bf16(lpk - le[k], sco[k]), pack_bf16(st.y, st.z),
                                             pack_bf16(round_f, lpk - log_tau));
                    }
                }
                if (seg_end >= g_end) break;
                lo = seg_end;
                ++seg;
                seg_end = d.pair_off[seg + 1];
                load_E(d.geo, seg, E);
                st = reinterpret_cast<const float4 *>(d.pstat)[seg];
            }
        }
#pragma unroll
        for (int k = 0; k < PPL; ++k) *reinterpret_cast<uint4 *>(sm.a2[k] + tc_offset(row, 0, TC_K2)) = feat[k];
        // ---- layer 1
        if (tc_handover(sm)) break;
        if (threadIdx.x == 0) {
            tc_fence_after_sync();
#pragma unroll
            for (int k = 0; k < PPL; ++k)
                tc_mma_bf16(sm.tmem + 32 * k, dA1[k], dB1, id1, 0u);
            tc_commit(smem_addr(&sm.mbar));
        }
        tc_wait(sm, phase);
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            uint32_t acc[32];
            tmem_ld32(tm + 32 * k, acc);
            tc_relu_row(sm.a2[k], row, acc);
        }
        // ---- layer 2
        if (tc_handover(sm)) break;
        if (threadIdx.x == 0) {
            tc_fence_after_sync();
#pragma unroll
            for (int k = 0; k < PPL; ++k)
#pragma unroll
                for (int sl = 0; sl < TC_K2 / 16; ++sl)
                    tc_mma_bf16(sm.tmem + 32 * k, dA2[k] + sl * SLICE, dB2 + sl * SLICE, id1, sl > 0 ? 1u : 0u);
            tc_commit(smem_addr(&sm.mbar));
        }
        tc_wait(sm, phase);
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            uint32_t acc[32];
            tmem_ld32(tm + 32 * k, acc);
            tc_relu_row(sm.a2[k], row, acc);
        }
        // ---- layer 3
        if (tc_handover(sm)) break;
        if (threadIdx.x == 0) {
            tc_fence_after_sync();
#pragma unroll
            for (int k = 0; k < PPL; ++k)
#pragma unroll
                for (int sl = 0; sl < TC_K2 / 16; ++sl)
                    tc_mma_bf16(sm.tmem + 32 * k, dA2[k] + sl * SLICE, dB3 + sl * SLICE, id3, sl > 0 ? 1u : 0u);
            tc_commit(smem_addr(&sm.mbar));
        }
        tc_wait(sm, phase);
        float z[PPL];
#pragma unroll
        for (int k = 0; k < PPL; ++k) z[k] = __uint_as_float(tmem_ld1(tm + 32 * k));
        tc_fence_before_sync();
        if (!active) continue;
        // ---- weights, history, kept count
        float w[PPL];
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            const float pk = __frcp_rn(1.f + __expf(-z[k]));
            const float ae = fabsf(e[k]);
            const bool in = q0 + k < p_end && ae <= tau_cap;
            const float wf = in ? learned_weight(pk, ae, delta) : 0.f;
            w[k] = STORE == FM_STORE_FP32 ? wf : __half2float(__float2half_rn(wf * wscale));
            kept += in ? 1u : 0u;
        }
        if (STORE == FM_STORE_FP32) {
            static_cast<float *>(d.w)[q0] = w[0];
            if (q0 < p_end) d.le_hist[q0] = __float2half_rn(le[0]);
        } else {
            reinterpret_cast<__half2 *>(d.w)[q0 >> 1] = __floats2half2_rn(w[0], w[PPL - 1]);
            const __half2 hv = __floats2half2_rn(le[0], le[PPL - 1]);
            if (q0 + 1 < p_end) reinterpret_cast<__half2 *>(d.le_hist)[q0 >> 1] = hv;
            else if (q0 < p_end) d.le_hist[q0] = __low2half(hv);
        }
        if (!FUSE) continue;
        // ---- phase B: loss and adjoint sums with the new weights
        int sb = seg0;
        int64_t sb_end = seg0_end, lo = gb;
        while (true) {
            const int64_t hi = min(sb_end, p_end);
#pragma unroll
            for (int k = 0; k < PPL; ++k) {
                const int64_t q = q0 + k;
                if (q >= lo && q < hi) {
                    float x1, y1, x2, y2, unused;
                    F::get(raw, k, x1, y1, x2, y2, unused);
                    loss.point(k, e[k], x1, y1, x2, y2, w[k]);
                }
            }
            if (sb == seg) break;
            loss.segment_end(sb, r, lane, false);
            lo = sb_end;
            ++sb;
            sb_end = d.pair_off[sb + 1];
        }
    }
    if (FUSE && r_ok) loss.segment_end(seg, r, lane, true);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
    if (lane == 0 && kept) atomicAdd(&sm.kept, kept);
    tc_fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0) {
        if (sm.kept) atomicAdd(d.counter, (unsigned long long)sm.kept);
        if (sm.fail) atomicOr(d.err, ERR_NONFINITE);
    }
    if (wid == 0) {
        tc_fence_after_sync();
        tmem_dealloc(sm.tmem, TC_COLS);
    }
}

static inline int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

void launch_learned_loss(const DevProblem &d, const float *master, const __nv_bfloat16 *wbf, float tau,
                         float tau_cap, int round, int hist_valid, cudaStream_t s, bool pdl) {
    const dim3 grid(blocks_for(d.n_ranges, TC_THREADS / 32)), block(TC_THREADS);
    if (d.storage == FM_STORE_FP32)
        launch_k(k_learned_tc<FM_STORE_FP32, true>, grid, block, s, pdl, d, master, wbf, tau, tau_cap, round, hist_valid);
    else
        launch_k(k_learned_tc<FM_STORE_FP16, true>, grid, block, s, pdl, d, master, wbf, tau, tau_cap, round, hist_valid);
}

void launch_pair_stats(const DevProblem &d, float tau, cudaStream_t s) {
    const int grid = blocks_for(d.n_ranges, CTA_WARPS);
    if (d.storage == FM_STORE_FP32) k_pair_stats<FM_STORE_FP32><<<grid, CTA_WARPS * 32, 0, s>>>(d, tau);
    else k_pair_stats<FM_STORE_FP16><<<grid, CTA_WARPS * 32, 0, s>>>(d, tau);
    k_pair_stats_combine<<<blocks_for(d.n_pairs, 128), 128, 0, s>>>(d);
}

void launch_learned_weights(const DevProblem &d, const float *master, const __nv_bfloat16 *wbf, float tau,
                            float tau_cap, int round, int hist_valid, cudaStream_t s) {
    const dim3 grid(blocks_for(d.n_ranges, TC_THREADS / 32)), block(TC_THREADS);
    if (d.storage == FM_STORE_FP32)
        launch_k(k_learned_tc<FM_STORE_FP32, false>, grid, block, s, false, d, master, wbf, tau, tau_cap, round, hist_valid);
    else
        launch_k(k_learned_tc<FM_STORE_FP16, false>, grid, block, s, false, d, master, wbf, tau, tau_cap, round, hist_valid);
}

void launch_collect_features(const DevProblem &d, float tau, int round, int hist_valid,
                             __nv_bfloat16 *feat, cudaStream_t s) {
    const int grid = blocks_for(d.n_ranges, CTA_WARPS);
    if (d.storage == FM_STORE_FP32)
        k_learned<FM_STORE_FP32, true><<<grid, CTA_WARPS * 32, 0, s>>>(d, nullptr, nullptr, tau, INFINITY, round, hist_valid, feat);
    else
        k_learned<FM_STORE_FP16, true><<<grid, CTA_WARPS * 32, 0, s>>>(d, nullptr, nullptr, tau, INFINITY, round, hist_valid, feat);
}

// ---- training: one sample per thread, block-level gradient sums, FP32 Adam ----------------------
constexpr int TRAIN_THREADS = 128;
constexpr int TRAIN_SMEM_FLOATS = MLP_NPARAM + TRAIN_THREADS * (MLP_IN + 4 * MLP_H + 2);

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// forward with BF16 weights (wf, from the BF16 copies) and FP32 biases; returns z3 and fills
// h1b, h2b (BF16-rounded activations) and the ReLU masks
__device__ __forceinline__ float mlp_forward_thread(const float *wf, const float *x, float *h1b, float *h2b,
                                                    unsigned &m1, unsigned &m2) {
    const float *W1 = wf + MLP_OFF_W1, *b1 = wf + MLP_OFF_B1, *W2 = wf + MLP_OFF_W2, *b2 = wf + MLP_OFF_B2,
                *W3 = wf + MLP_OFF_W3;
    m1 = m2 = 0u;
    for (int j = 0; j < MLP_H; ++j) {
        float z = b1[j];
#pragma unroll
        for (int k = 0; k < MLP_IN; ++k) z = fmaf(x[k], W1[k * MLP_H + j], z);
        if (z > 0.f) m1 |= 1u << j;
        h1b[j] = bf16r(fmaxf(z, 0.f));
    }
    for (int j = 0; j < MLP_H; ++j) {
        float z = b2[j];
        for (int k = 0; k < MLP_H; ++k) z = fmaf(h1b[k], W2[k * MLP_H + j], z);
        if (z > 0.f) m2 |= 1u << j;
        h2b[j] = bf16r(fmaxf(z, 0.f));
    }
    float z3 = wf[MLP_OFF_B3];
    for (int k = 0; k < MLP_H; ++k) z3 = fmaf(h2b[k], W3[k], z3);
    return z3;
}

__device__ __forceinline__ void load_weights_smem(float *wf, const float *master, const __nv_bfloat16 *wbf) {
    for (int q = threadIdx.x; q < MLP_NPARAM; q += blockDim.x) {
        float v;
        if (q < MLP_OFF_B1) v = __bfloat162float(wbf[q]);
        else if (q < MLP_OFF_W2) v = master[q];
        else if (q < MLP_OFF_B2) v = __bfloat162float(wbf[q - MLP_H]);
        else if (q < MLP_OFF_W3) v = master[q];
        else if (q < MLP_OFF_B3) v = __bfloat162float(wbf[q - 2 * MLP_H]);
        else v = master[q];
        wf[q] = v;
    }
}

__global__ void __launch_bounds__(TRAIN_THREADS)
k_mlp_grad(const float *master, const __nv_bfloat16 *wbf, const __nv_bfloat16 *feat, const float *labels, int n,
           float inv_n, float *gpart, float *lpart) {
    extern __shared__ float sm[];
    float *wf = sm;
    float *xs = wf + MLP_NPARAM;                  // [T][8]
    float *h1s = xs + TRAIN_THREADS * MLP_IN;     // [T][32]
    float *h2s = h1s + TRAIN_THREADS * MLP_H;
    float *dz1s = h2s + TRAIN_THREADS * MLP_H;
    float *dz2s = dz1s + TRAIN_THREADS * MLP_H;
    float *dz3s = dz2s + TRAIN_THREADS * MLP_H;   // [T]
    float *ls = dz3s + TRAIN_THREADS;             // [T]
    load_weights_smem(wf, master, wbf);
    __syncthreads();
    const int tid = threadIdx.x;
    const int s = blockIdx.x * TRAIN_THREADS + tid;
    const bool valid = s < n;
    float x[MLP_IN];
#pragma unroll
    for (int k = 0; k < MLP_IN; ++k) x[k] = valid ? __bfloat162float(feat[(size_t)s * MLP_IN + k]) : 0.f;
    float *h1b = h1s + tid * MLP_H, *h2b = h2s + tid * MLP_H;
    unsigned m1, m2;
    const float z3 = mlp_forward_thread(wf, x, h1b, h2b, m1, m2);
    const float y = valid ? labels[s] : 0.f;
    const float p = 1.f / (1.f + expf(-z3));
    ls[tid] = valid ? fmaxf(z3, 0.f) - z3 * y + log1pf(expf(-fabsf(z3))) : 0.f;
    const float dz3 = valid ? (p - y) * inv_n : 0.f;
    dz3s[tid] = dz3;
#pragma unroll
    for (int k = 0; k < MLP_IN; ++k) xs[tid * MLP_IN + k] = x[k];
    const float *W2 = wf + MLP_OFF_W2, *W3 = wf + MLP_OFF_W3;
    float *dz2 = dz2s + tid * MLP_H, *dz1 = dz1s + tid * MLP_H;
    for (int j = 0; j < MLP_H; ++j) dz2[j] = ((m2 >> j) & 1u) ? W3[j] * dz3 : 0.f;
    for (int k = 0; k < MLP_H; ++k) {
        float a = 0.f;
        for (int j = 0; j < MLP_H; ++j) a = fmaf(W2[k * MLP_H + j], dz2[j], a);
        dz1[k] = ((m1 >> k) & 1u) ? a : 0.f;
    }
    __syncthreads();
    // gradient sums over the block's samples, in sample order
    float *gout = gpart + (size_t)blockIdx.x * MLP_NPARAM;
    for (int q = tid; q < MLP_NPARAM; q += TRAIN_THREADS) {
        float acc = 0.f;
        if (q < MLP_OFF_B1) {
            const int k = q / MLP_H, j = q % MLP_H;
            for (int t = 0; t < TRAIN_THREADS; ++t) acc = fmaf(xs[t * MLP_IN + k], dz1s[t * MLP_H + j], acc);
        } else if (q < MLP_OFF_W2) {
            const int j = q - MLP_OFF_B1;
            for (int t = 0; t < TRAIN_THREADS; ++t) acc += dz1s[t * MLP_H + j];
        } else if (q < MLP_OFF_B2) {
            const int k = (q - MLP_OFF_W2) / MLP_H, j = (q - MLP_OFF_W2) % MLP_H;
            for (int t = 0; t < TRAIN_THREADS; ++t) acc = fmaf(h1s[t * MLP_H + k], dz2s[t * MLP_H + j], acc);
        } else if (q < MLP_OFF_W3) {
            const int j = q - MLP_OFF_B2;
            for (int t = 0; t < TRAIN_THREADS; ++t) acc += dz2s[t * MLP_H + j];
        } else if (q < MLP_OFF_B3) {
            const int k = q - MLP_OFF_W3;
            for (int t = 0; t < TRAIN_THREADS; ++t) acc = fmaf(h2s[t * MLP_H + k], dz3s[t], acc);
        } else {
            for (int t = 0; t < TRAIN_THREADS; ++t) acc += dz3s[t];
        }
        gout[q] = acc;
    }
    if (tid == 0) {
        float l = 0.f;
        for (int t = 0; t < TRAIN_THREADS; ++t) l += ls[t];
        lpart[blockIdx.x] = l;
    }
}

__global__ void k_mlp_refresh(const float *master, __nv_bfloat16 *wbf) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < MLP_NPARAM; q += gridDim.x * blockDim.x) {
        if (q < MLP_OFF_B1) wbf[q] = __float2bfloat16_rn(master[q]);
        else if (q >= MLP_OFF_W2 && q < MLP_OFF_B2) wbf[q - MLP_H] = __float2bfloat16_rn(master[q]);
        else if (q >= MLP_OFF_W3 && q < MLP_OFF_B3) wbf[q - 2 * MLP_H] = __float2bfloat16_rn(master[q]);
    }
}

__global__ void k_mlp_adam(float *master, float *m, float *v, const float *gpart, const float *lpart, int nblocks,
                           float lr, float bc1, float bc2, float inv_n, float *loss_out) {
    for (int q = threadIdx.x; q < MLP_NPARAM; q += blockDim.x) {
        float g = 0.f;
        for (int b = 0; b < nblocks; ++b) g += gpart[(size_t)b * MLP_NPARAM + q];
        const float mq = 0.9f * m[q] + 0.1f * g;
        const float vq = 0.999f * v[q] + 0.001f * g * g;
        m[q] = mq;
        v[q] = vq;
        master[q] -= lr * (mq / bc1) / (sqrtf(vq / bc2) + 1e-8f);
    }
    if (threadIdx.x == 0) {
        float l = 0.f;
        for (int b = 0; b < nblocks; ++b) l += lpart[b];
        *loss_out = l * inv_n;
    }
}

__global__ void __launch_bounds__(TRAIN_THREADS)
k_mlp_forward(const float *master, const __nv_bfloat16 *wbf, const __nv_bfloat16 *feat, int n, float *p_out) {
    extern __shared__ float sm[];
    float *wf = sm;
    float *h = wf + MLP_NPARAM;
    load_weights_smem(wf, master, wbf);
    __syncthreads();
    const int s = blockIdx.x * TRAIN_THREADS + threadIdx.x;
    if (s >= n) return;
    float x[MLP_IN];
#pragma unroll
    for (int k = 0; k < MLP_IN; ++k) x[k] = __bfloat162float(feat[(size_t)s * MLP_IN + k]);
    unsigned m1, m2;
    const float z3 = mlp_forward_thread(wf, x, h + threadIdx.x * 2 * MLP_H, h + threadIdx.x * 2 * MLP_H + MLP_H, m1, m2);
    p_out[s] = 1.f / (1.f + expf(-z3));
}

}  // namespace fm

// ====================================== C ABI ======================================================
using namespace fm;

void fm_internal_set_error(const char *msg);

struct fm_mlp {
    float *master = nullptr, *m = nullptr, *v = nullptr, *gpart = nullptr, *lpart = nullptr, *loss = nullptr;
    __nv_bfloat16 *wbf = nullptr;
    int max_blocks = 0;
    long long step = 0;
};

namespace {
fm_status mlp_fail(fm_status s, const std::string &m) {
    fm_internal_set_error(m.c_str());
    return s;
}
#define MLP_CUDA(call)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return mlp_fail(FM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

constexpr int MLP_MAX_BATCH = 1 << 16;
}  // namespace

// device pointers of a network, for fm_learned_weights (fm_api.cu)
void fm_internal_mlp_params(const fm_mlp *net, const float **master, const __nv_bfloat16 **wbf) {
    *master = net->master;
    *wbf = net->wbf;
}

extern "C" {

FM_API fm_status fm_mlp_create(const float *params, fm_mlp **out) {
    if (!out || !params) return mlp_fail(FM_EINVAL, "fm_mlp_create: params and out must not be NULL");
    *out = nullptr;
    for (int q = 0; q < MLP_NPARAM; ++q)
        if (!std::isfinite(params[q])) return mlp_fail(FM_EINVAL, "fm_mlp_create: parameters must be finite");
    fm_mlp *n = new fm_mlp();
    n->max_blocks = MLP_MAX_BATCH / TRAIN_THREADS;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&n->master, sizeof(float) * MLP_NPARAM);
    if (e == cudaSuccess) e = cudaMalloc(&n->m, sizeof(float) * MLP_NPARAM);
    if (e == cudaSuccess) e = cudaMalloc(&n->v, sizeof(float) * MLP_NPARAM);
    if (e == cudaSuccess) e = cudaMalloc(&n->gpart, sizeof(float) * MLP_NPARAM * n->max_blocks);
    if (e == cudaSuccess) e = cudaMalloc(&n->lpart, sizeof(float) * n->max_blocks);
    if (e == cudaSuccess) e = cudaMalloc(&n->loss, sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&n->wbf, sizeof(__nv_bfloat16) * MLP_NPARAM);
    if (e == cudaSuccess) e = cudaMemcpy(n->master, params, sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(n->m, 0, sizeof(float) * MLP_NPARAM);
    if (e == cudaSuccess) e = cudaMemset(n->v, 0, sizeof(float) * MLP_NPARAM);
    if (e == cudaSuccess) {
        k_mlp_refresh<<<2, 1024>>>(n->master, n->wbf);
        e = cudaDeviceSynchronize();
    }
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)(sizeof(float) * TRAIN_SMEM_FLOATS));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)(sizeof(float) * (MLP_NPARAM + TRAIN_THREADS * 2 * MLP_H)));
    if (e != cudaSuccess) {
        fm_mlp_destroy(n);
        return mlp_fail(e == cudaErrorMemoryAllocation ? FM_ENOMEM : FM_ECUDA,
                        std::string("fm_mlp_create: ") + cudaGetErrorString(e));
    }
    *out = n;
    return FM_OK;
}

FM_API void fm_mlp_destroy(fm_mlp *n) {
    if (!n) return;
    cudaDeviceSynchronize();
    cudaFree(n->master);
    cudaFree(n->m);
    cudaFree(n->v);
    cudaFree(n->gpart);
    cudaFree(n->lpart);
    cudaFree(n->loss);
    cudaFree(n->wbf);
    delete n;
}

FM_API fm_status fm_mlp_get_params(fm_mlp *n, float *params) {
    if (!n || !params) return mlp_fail(FM_EINVAL, "fm_mlp_get_params: NULL argument");
    MLP_CUDA(cudaMemcpy(params, n->master, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost));
    return FM_OK;
}

FM_API fm_status fm_mlp_set_params(fm_mlp *n, const float *params) {
    if (!n || !params) return mlp_fail(FM_EINVAL, "fm_mlp_set_params: NULL argument");
    for (int q = 0; q < MLP_NPARAM; ++q)
        if (!std::isfinite(params[q])) return mlp_fail(FM_EINVAL, "fm_mlp_set_params: parameters must be finite");
    MLP_CUDA(cudaMemcpy(n->master, params, sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice));
    k_mlp_refresh<<<2, 1024>>>(n->master, n->wbf);
    MLP_CUDA(cudaDeviceSynchronize());
    return FM_OK;
}

FM_API fm_status fm_mlp_train_step(fm_mlp *n, const void *d_features, const float *d_labels, int32_t count,
                                   float lr, float *loss, void *stream) {
    if (!n || !d_features || !d_labels) return mlp_fail(FM_EINVAL, "fm_mlp_train_step: NULL argument");
    if (count < 1 || count > MLP_MAX_BATCH) return mlp_fail(FM_EINVAL, "fm_mlp_train_step: count must be in [1, 65536]");
    if (!(lr >= 0.f) || !std::isfinite(lr)) return mlp_fail(FM_EINVAL, "fm_mlp_train_step: lr must be finite and >= 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nb = (count + TRAIN_THREADS - 1) / TRAIN_THREADS;
    const float inv_n = 1.f / (float)count;
    k_mlp_grad<<<nb, TRAIN_THREADS, sizeof(float) * TRAIN_SMEM_FLOATS, s>>>(
        n->master, n->wbf, static_cast<const __nv_bfloat16 *>(d_features), d_labels, count, inv_n, n->gpart, n->lpart);
    n->step += 1;
    const float bc1 = 1.f - powf(0.9f, (float)n->step), bc2 = 1.f - powf(0.999f, (float)n->step);
    k_mlp_adam<<<1, 512, 0, s>>>(n->master, n->m, n->v, n->gpart, n->lpart, nb, lr, bc1, bc2, 1.f / (float)count, n->loss);
    k_mlp_refresh<<<2, 1024, 0, s>>>(n->master, n->wbf);
    MLP_CUDA(cudaGetLastError());
    if (loss) {
        MLP_CUDA(cudaMemcpyAsync(loss, n->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
        MLP_CUDA(cudaStreamSynchronize(s));
    }
    return FM_OK;
}

FM_API fm_status fm_mlp_gradient(fm_mlp *n, const void *d_features, const float *d_labels, int32_t count,
                                 float *grad, float *loss) {
    if (!n || !d_features || !d_labels || !grad) return mlp_fail(FM_EINVAL, "fm_mlp_gradient: NULL argument");
    if (count < 1 || count > MLP_MAX_BATCH) return mlp_fail(FM_EINVAL, "fm_mlp_gradient: count must be in [1, 65536]");
    const int nb = (count + TRAIN_THREADS - 1) / TRAIN_THREADS;
    k_mlp_grad<<<nb, TRAIN_THREADS, sizeof(float) * TRAIN_SMEM_FLOATS>>>(
        n->master, n->wbf, static_cast<const __nv_bfloat16 *>(d_features), d_labels, count, 1.f / (float)count,
        n->gpart, n->lpart);
    MLP_CUDA(cudaGetLastError());
    float *gp = new float[(size_t)nb * MLP_NPARAM];
    float *lp = new float[nb];
    cudaError_t e = cudaMemcpy(gp, n->gpart, sizeof(float) * nb * MLP_NPARAM, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(lp, n->lpart, sizeof(float) * nb, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
        for (int q = 0; q < MLP_NPARAM; ++q) {
            float g = 0.f;
            for (int b = 0; b < nb; ++b) g += gp[(size_t)b * MLP_NPARAM + q];
            grad[q] = g;
        }
        if (loss) {
            float l = 0.f;
            for (int b = 0; b < nb; ++b) l += lp[b];
            *loss = l / (float)count;
        }
    }
    delete[] gp;
    delete[] lp;
    if (e != cudaSuccess) return mlp_fail(FM_ECUDA, cudaGetErrorString(e));
    return FM_OK;
}

FM_API fm_status fm_mlp_forward(fm_mlp *n, const void *d_features, int32_t count, float *d_p, void *stream) {
    if (!n || !d_features || !d_p) return mlp_fail(FM_EINVAL, "fm_mlp_forward: NULL argument");
    if (count < 1) return mlp_fail(FM_EINVAL, "fm_mlp_forward: count must be >= 1");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_mlp_forward<<<(count + TRAIN_THREADS - 1) / TRAIN_THREADS, TRAIN_THREADS,
                    sizeof(float) * (MLP_NPARAM + TRAIN_THREADS * 2 * MLP_H), s>>>(
        n->master, n->wbf, static_cast<const __nv_bfloat16 *>(d_features), count, d_p);
    MLP_CUDA(cudaGetLastError());
    return FM_OK;
}

FM_API int32_t fm_mlp_num_params(void) { return MLP_NPARAM; }

}  // extern "C"
