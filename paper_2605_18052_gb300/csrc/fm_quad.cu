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
// (00, 01, 02, 11, 12, 22). Per point pair that is 36 multiply-adds instead of 45.
#include "fm_walk.cuh"

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
            const float wf = keep ? 1.0f / fmaxf(ae, delta) : 0.f;
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
        // M[u][v] += (w m2_u) m1_v
        const float wx2 = w * x2, wy2 = w * y2;
        const float u[6] = {wx2 * x2, wx2 * y2, wx2, wy2 * y2, wy2, w};
        const float v[6] = {x1 * x1, x1 * y1, x1, y1 * y1, y1, 1.f};
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int b = 0; b < 6; ++b) acc[10 + 6 * a + b] = fmaf(u[a], v[b], acc[10 + 6 * a + b]);
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

template <int STORE, bool REWEIGHT>
__global__ void __launch_bounds__(CTA_WARPS * 32, 2) k_quad_accumulate(DevProblem d, float tau) {
    __shared__ unsigned cta_kept;
    if (threadIdx.x == 0) cta_kept = 0;
    __syncthreads();
    const int r = blockIdx.x * CTA_WARPS + (threadIdx.x >> 5);
    if (r < d.n_ranges) {
        QuadBody<STORE, REWEIGHT> body(d, tau);
        walk_range<STORE, !REWEIGHT>(d, r, threadIdx.x & 31, body);
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

// per pair (one warp, a lane per sum): Kahan-sum the range partials; keep the anchor
// e0 = E'_n of the geometry record. The records are stored component-major (entry q of pair n
// at q * n_pairs + n), so that the per-iteration kernel reads them coalesced.
__global__ void k_quad_combine(DevProblem d) {
    const int n = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (n >= d.n_pairs) return;
    const int r0 = d.pair_off[n] / WR, r1 = (d.pair_off[n + 1] - 1) / WR;
    const size_t np = (size_t)d.n_pairs;
    for (int q = lane; q < QSUMS; q += 32) {
        float sum = 0.f, c = 0.f;
        for (int r = r0; r <= r1; ++r) {
            const float y = d.qslots[(size_t)(n + r) * QSLOT + q] - c;
            const float t = sum + y;
            c = (t - sum) - y;
            sum = t;
        }
        d.quad[q * np + n] = sum;
    }
    if (lane < 9) d.quad[(QSUMS + lane) * np + n] = d.geo[(size_t)n * GEO + lane];
}

// one iteration's per-pair evaluation: geometry at the current poses, then the quadratic form;
// writes the pair's sums (G'(9), loss) in the layout of the streaming partials
constexpr int QPAIR_THREADS = 128;

__global__ void __launch_bounds__(QPAIR_THREADS) k_quad_pair(DevProblem d, int prev_blocks) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = n < d.n_pairs ? d.cam_i[n] : 0, j = n < d.n_pairs ? d.cam_j[n] : 0;
    pdl_wait();     // camera records of the previous step
    pdl_trigger();
    if (prev_blocks > 0 && blockIdx.x == 0) finish_step<QPAIR_THREADS>(d, prev_blocks, 1);
    if (n >= d.n_pairs) return;
    float e[9];
    pair_geometry(d, n, i, j, e);
    const size_t np = (size_t)d.n_pairs;
    const float *Qn = d.quad + n;
    auto Q = [&](int k) { return Qn[k * np]; };
    float dv[9], q[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        dv[a] = e[a] - Q(QSUMS + a);
        q[a] = Q(1 + a);
    }
    // q = g0 + W d, W[3p+q][3r+s] = M[sym(p,r)][sym(q,s)]
    constexpr int SYM[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
#pragma unroll
    for (int u = 0; u < 6; ++u)
#pragma unroll
        for (int v = 0; v < 6; ++v) {
            const float m = Q(10 + 6 * u + v);
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    if (SYM[p][r] != u) continue;
#pragma unroll
                    for (int qq = 0; qq < 3; ++qq)
#pragma unroll
                        for (int ss = 0; ss < 3; ++ss)
                            if (SYM[qq][ss] == v) q[3 * p + qq] = fmaf(m, dv[3 * r + ss], q[3 * p + qq]);
                }
        }
    // loss = c0 + d^T (g0 + q)
    float loss = Q(0);
#pragma unroll
    for (int a = 0; a < 9; ++a) loss = fmaf(dv[a], Q(1 + a) + q[a], loss);
    float4 *out = reinterpret_cast<float4 *>(d.pair_rec + (size_t)n * SLOT);
    out[0] = make_float4(q[0], q[1], q[2], q[3]);
    out[1] = make_float4(q[4], q[5], q[6], q[7]);
    out[2] = make_float4(q[8], loss, 0.f, 0.f);
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
    k_quad_combine<<<blocks_for(d.n_pairs, 8), 256, 0, s>>>(d);
}

void launch_quad_pair(const DevProblem &d, cudaStream_t s, bool pdl, bool after_step) {
    launch_k(k_quad_pair, dim3(blocks_for(d.n_pairs, QPAIR_THREADS)), dim3(QPAIR_THREADS), s, pdl, d,
             after_step ? camera_step_blocks(d) : 0);
}

}  // namespace fm
