// Per-camera pieces shared by the optimiser-step kernels (the streaming path's camera step
// and the quadratic form's fused step): compensated sums, the chain rule from an image pair's
// sums to one of its cameras, and the FP64 Adam / exponential-map update of one camera.
#pragma once

#include <math.h>

#include "fm_walk.cuh"

namespace fm {

constexpr int STEP_CAMS = 8;   // cameras (warps) per block of the step kernels
constexpr int STEP_VALS = 8;   // per camera: 6 pose gradient components, loss, scale gradient

// (hi, lo) += (bhi, blo) with the rounding error of the high parts kept (Knuth's TwoSum)
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float bhi, float blo) {
    const float s = hi + bhi;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (bhi - bb);
    const float l = lo + blo + err;
    hi = s + l;
    lo = l - (hi - s);
}

// ---- per camera: pose record --------------------------------------------------------------------
// R (9 floats), centre as hi + lo floats (3 + 3), keypoint scale s (focal refinement)
__device__ __forceinline__ void write_camrec(float *rec, const double *R, const double *c, float s) {
#pragma unroll
    for (int i = 0; i < 9; ++i) rec[i] = (float)R[i];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float hi = (float)c[q];
        rec[9 + q] = hi;
        rec[12 + q] = (float)__dsub_rn(c[q], (double)hi);
    }
    rec[15] = s;
}

// keypoint scale of camera k: exp(rho_k), 1 without focal state
__device__ __forceinline__ double camera_scale(const DevProblem &d, int k) {
    return d.rho ? exp(d.rho[k]) : 1.0;
}

__device__ __forceinline__ void vee(const float *M, float *v) {
    v[0] = M[7] - M[5];
    v[1] = M[2] - M[6];
    v[2] = M[3] - M[1];
}

// 1/sqrt(x) in FP64: an FP32 seed refined by two Newton steps (the relative error squares
// each step: ~2e-7 -> ~1e-13 -> below FP64 rounding)
__device__ __forceinline__ double rsqrt64(double x) {
    double y = (double)rsqrtf((float)x);
    const double hx = __dmul_rn(-0.5, x);
    y = __dmul_rn(y, __fma_rn(hx, __dmul_rn(y, y), 1.5));
    y = __dmul_rn(y, __fma_rn(hx, __dmul_rn(y, y), 1.5));
    return y;
}

// Exp(phi) - I = a K + b K^2 (K = [phi]_x) in FP32. A rotation increment is small, so its
// FP32 relative error (a few ulp) is an absolute error of a few 1e-7 |phi|, the same order as
// that of phi itself, which Adam computes in FP32. For |phi| < 0.1 the Taylor series of a and b
// through the t^6 terms (truncation below 1e-13); otherwise sin and b = 2 sin^2(t/2) / t^2.
__device__ __forceinline__ void so3_exp_minus_identity(const float *phi, float *A) {
    const float th2 = rdot3(phi[0], phi[0], phi[1], phi[1], phi[2], phi[2]);
    float a, b;
    if (th2 < 0.01f) {
        a = rfma(-rmul(th2, 1.f / 6.f), rfma(-rmul(th2, 1.f / 20.f), radd(1.f, -rmul(th2, 1.f / 42.f)), 1.f), 1.f);
        b = rmul(0.5f, rfma(-rmul(th2, 1.f / 12.f), rfma(-rmul(th2, 1.f / 30.f), radd(1.f, -rmul(th2, 1.f / 56.f)), 1.f), 1.f));
    } else {
        const float th = __fsqrt_rn(th2);
        const float sh = sinf(rmul(0.5f, th));
        a = __fdiv_rn(sinf(th), th);
        b = __fdiv_rn(rmul(rmul(2.f, sh), sh), th2);
    }
    const float K[9] = {0.f, -phi[2], phi[1], phi[2], 0.f, -phi[0], -phi[1], phi[0], 0.f};
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float k2 = rdot3(K[3 * r], K[c], K[3 * r + 1], K[3 + c], K[3 * r + 2], K[6 + c]);
            A[3 * r + c] = rfma(b, k2, rmul(a, K[3 * r + c]));
        }
}

// Gram-Schmidt on the rows: r0 normalised, r1 orthogonalised and normalised, r2 = r0 x r1
__device__ __forceinline__ void orthonormalize_rows(double *R) {
    const double n0 = rsqrt64(rdot3(R[0], R[0], R[1], R[1], R[2], R[2]));
    for (int q = 0; q < 3; ++q) R[q] = __dmul_rn(R[q], n0);
    const double dp = rdot3(R[0], R[3], R[1], R[4], R[2], R[5]);
    for (int q = 0; q < 3; ++q) R[3 + q] = __fma_rn(-dp, R[q], R[3 + q]);
    const double n1 = rsqrt64(rdot3(R[3], R[3], R[4], R[4], R[5], R[5]));
    for (int q = 0; q < 3; ++q) R[3 + q] = __dmul_rn(R[3 + q], n1);
    R[6] = __fma_rn(R[1], R[5], -__dmul_rn(R[2], R[4]));
    R[7] = __fma_rn(R[2], R[3], -__dmul_rn(R[0], R[5]));
    R[8] = __fma_rn(R[0], R[4], -__dmul_rn(R[1], R[3]));
}

// Chain rule of one image pair (or one range partial of it) to one of its cameras.
// gr = the pair's geometry record, sum[0..8] = sum s * o2 o1^T over the point pairs,
// sum[9] = their loss terms. Writes the camera's 6 pose gradient components, (for the first
// camera only) the loss in contrib[6], and in contrib[7] the gradient with respect to the
// camera's keypoint scale s: with F = S_j E S_i, dL/dE = S_j G S_i (G = dL/dF) and
// dL/ds_i = sum_{a, b<2} G_ab E_ab (S_j)_a, dL/ds_j = sum_{a<2, b} G_ab E_ab (S_i)_b.
// FOCAL = false: the scale gradient is not formed (contrib[7] = 0); the pair matrix still
// carries the scales, so dL/dE = S_j G S_i either way.
template <bool FOCAL>
__device__ __forceinline__ void pair_chain_rule(const float *gr, int role, const float *sum,
                                                float gscale, float lscale, float *contrib) {
    float Gp[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) Gp[q] = rmul(sum[q], gscale);
    const float2 cen_i = make_float2(gr[22], gr[23]), cen_j = make_float2(gr[33], gr[34]);
    float M[9], G[9];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        M[3 * a] = rfma(Gp[3 * a + 2], cen_i.x, Gp[3 * a]);
        M[3 * a + 1] = rfma(Gp[3 * a + 2], cen_i.y, Gp[3 * a + 1]);
        M[3 * a + 2] = Gp[3 * a + 2];
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        G[b] = rfma(cen_j.x, M[6 + b], M[b]);
        G[3 + b] = rfma(cen_j.y, M[6 + b], M[3 + b]);
        G[6 + b] = M[6 + b];
    }
    const float *Rn = gr + 9;
    const float tn[3] = {gr[18], gr[19], gr[20]};
    const float inv = gr[21];
    const float *Rj = gr + 24;
    const float th[3] = {rmul(tn[0], inv), rmul(tn[1], inv), rmul(tn[2], inv)};
    // focal: E = [th]_x R_n, the scale gradient from G = dL/dF, then G <- dL/dE
    const float s_i = gr[35], s_j = gr[36];
    {
        const float si[3] = {s_i, s_i, 1.f}, sj[3] = {s_j, s_j, 1.f};
        float gs = 0.f;
        if (FOCAL) {
            float E[9];
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                E[b] = rfma(th[1], Rn[6 + b], rmul(-th[2], Rn[3 + b]));
                E[3 + b] = rfma(-th[0], Rn[6 + b], rmul(th[2], Rn[b]));
                E[6 + b] = rfma(th[0], Rn[3 + b], rmul(-th[1], Rn[b]));
            }
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const float ge = rmul(G[3 * a + b], E[3 * a + b]);
                    if (role == 0 ? b < 2 : a < 2) gs = rfma(ge, role == 0 ? sj[a] : si[b], gs);
                }
        }
        contrib[7] = gs;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) G[3 * a + b] = rmul(rmul(G[3 * a + b], sj[a]), si[b]);
    }
    float A[9];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        A[b] = -rfma(th[1], G[6 + b], rmul(-th[2], G[3 + b]));
        A[3 + b] = -rfma(-th[0], G[6 + b], rmul(th[2], G[b]));
        A[6 + b] = -rfma(th[0], G[3 + b], rmul(-th[1], G[b]));
    }
    float GRt[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            GRt[3 * a + b] = rdot3(G[3 * a], Rn[3 * b], G[3 * a + 1], Rn[3 * b + 1], G[3 * a + 2], Rn[3 * b + 2]);
    float gth[3], gt[3], gc[3], gp[3];
    vee(GRt, gth);
    const float dp = rdot3(th[0], gth[0], th[1], gth[1], th[2], gth[2]);
#pragma unroll
    for (int q = 0; q < 3; ++q) gt[q] = rmul(rfma(-dp, th[q], gth[q]), inv);
#pragma unroll
    for (int q = 0; q < 3; ++q) gc[q] = rdot3(Rj[q], gt[0], Rj[3 + q], gt[1], Rj[6 + q], gt[2]);
    if (role == 0) {
        float RtA[9];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) RtA[3 * a + b] = rdot3(Rn[a], A[b], Rn[3 + a], A[3 + b], Rn[6 + a], A[6 + b]);
        vee(RtA, gp);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            contrib[q] = -gp[q];
            contrib[3 + q] = gc[q];
        }
        contrib[6] = rmul(sum[9], lscale);
    } else {
        float ARt[9];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                ARt[3 * a + b] = rdot3(A[3 * a], Rn[3 * b], A[3 * a + 1], Rn[3 * b + 1], A[3 * a + 2], Rn[3 * b + 2]);
        vee(ARt, gp);
        contrib[0] = radd(gp[0], rfma(tn[1], gt[2], rmul(-tn[2], gt[1])));
        contrib[1] = radd(gp[1], rfma(tn[2], gt[0], rmul(-tn[0], gt[2])));
        contrib[2] = radd(gp[2], rfma(tn[0], gt[1], rmul(-tn[1], gt[0])));
#pragma unroll
        for (int q = 0; q < 3; ++q) contrib[3 + q] = -gc[q];
        contrib[6] = 0.f;
    }
}


// warp-wide TwoSum butterfly of N (hi, lo) pairs: every lane ends with the total
template <int N>
__device__ __forceinline__ void warp_two_sum_reduce(float *hi, float *lo) {
#pragma unroll
    for (int q = 0; q < N; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float bh = __shfl_xor_sync(0xffffffffu, hi[q], o);
            const float bl = __shfl_xor_sync(0xffffffffu, lo[q], o);
            two_sum_acc(hi[q], lo[q], bh, bl);
        }
}

// Phase 2 of a step for camera kc, one lane. apply = 0: the gradient (FP64 sum of its hi + lo
// parts) and the focal gradient are written, nothing else. apply = 1: one Adam step (FP32
// moments) and the new pose: R <- R + (Exp(phi) - I) R and c <- c + delta_c in FP64, where the
// small increment (Exp(phi) - I) R is formed in FP32 from the camera's FP32 record rotation R32
// (its error, a few 1e-7 |phi|, is of the order of phi's own FP32 error), then Gram-Schmidt on
// the rows in FP64 on every eighth step (steps 1, 9, 17, ...) and the new camera record at
// rec_out. hi/lo hold STEP_VALS values (6 pose gradient components, the loss, the
// keypoint-scale gradient) `stride` apart; mv = the camera's Adam m (6) and v (6); Rc = its R
// (9) and c (3) in FP64; rec = its current record's rotation (9 floats) and keypoint scale
// (rec[9]); hyper = lr_rot, lr_c, beta1, beta2, eps, lr_focal. With focal refinement
// rho = log s takes its own Adam step (gradient s dL/ds); without, the record keeps its scale.
// Returns the camera's loss share.
// GB300 executes FP64 on a narrow pipe at whole-warp cost per instruction, and every block of a
// step reaches this phase at the same moment, so the update keeps its FP64 work to the state
// itself: the two sums and the record (about 45 operations), and the re-orthonormalisation
// (about 40) only every eighth step. Between two of them R leaves SO(3) by the FP32 rounding of
// the increments, a few 1e-7 |phi| per step, far below the FP32 camera record's resolution.
template <bool FOCAL>
__device__ __forceinline__ double camera_update(const DevProblem &d, int kc, const float *hi, const float *lo,
                                                int stride, const float *mv, const double *Rc, const float *rec,
                                                const double *hyper, long long t_step, int apply,
                                                float *rec_out) {
    const float *R32 = rec;
    const double bl = (double)hi[6 * stride] + (double)lo[6 * stride];
    const double s_cur = FOCAL ? camera_scale(d, kc) : 1.0;
    const double g_rho = FOCAL ? s_cur * ((double)hi[7 * stride] + (double)lo[7 * stride]) : 0.0;
    if (!apply) {
        bool ok = isfinite(hi[6 * stride]);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const double g = (double)hi[q * stride] + (double)lo[q * stride];
            ok = ok && isfinite(g);
            d.grad[(size_t)kc * 6 + q] = g;
        }
        if (!ok) atomicOr(d.err, ERR_NONFINITE);
        if (d.grad_rho) d.grad_rho[kc] = g_rho;
        return bl;
    }
    // the FP32 gradient: hi is the rounded value of hi + lo (TwoSum keeps |lo| within half an
    // ulp of hi), so hi + lo in FP32 is the same number the FP64 sum would round to
    float gq[6];
    bool ok = isfinite(hi[6 * stride]);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        gq[q] = radd(hi[q * stride], lo[q * stride]);
        ok = ok && isfinite(gq[q]);
    }
    if (!ok) atomicOr(d.err, ERR_NONFINITE);
    float s_new = rec[9];
    const float b1 = (float)hyper[2], b2 = (float)hyper[3], eps = (float)hyper[4];
    const float lr_r = (float)hyper[0], lr_c = (float)hyper[1];
    const float bc1 = radd(1.f, -powf(b1, (float)t_step)), bc2 = radd(1.f, -powf(b2, (float)t_step));
    if (FOCAL) {
        const float g1 = (float)g_rho;
        const float mo = rfma(b1, d.rho_m[kc], rmul(radd(1.f, -b1), g1));
        const float vo = rfma(b2, d.rho_v[kc], rmul(rmul(radd(1.f, -b2), g1), g1));
        d.rho_m[kc] = mo;
        d.rho_v[kc] = vo;
        const double r = d.rho[kc] - (double)__fdiv_rn(rmul((float)hyper[5], __fdiv_rn(mo, bc1)),
                                                       radd(__fsqrt_rn(__fdiv_rn(vo, bc2)), eps));
        d.rho[kc] = r;
        d.grad_rho[kc] = g_rho;
        s_new = (float)exp(r);
    }
    float dl[6], mo[6], vo[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        mo[q] = rfma(b1, mv[q], rmul(radd(1.f, -b1), gq[q]));
        vo[q] = rfma(b2, mv[6 + q], rmul(rmul(radd(1.f, -b2), gq[q]), gq[q]));
        dl[q] = __fdiv_rn(rmul(-(q < 3 ? lr_r : lr_c), __fdiv_rn(mo[q], bc1)),
                          radd(__fsqrt_rn(__fdiv_rn(vo[q], bc2)), eps));
    }
    float A[9];
    so3_exp_minus_identity(dl, A);
    double Rn[9], cn[3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            Rn[3 * r + c] = __dadd_rn(Rc[3 * r + c], (double)rdot3(A[3 * r], R32[c], A[3 * r + 1], R32[3 + c],
                                                                     A[3 * r + 2], R32[6 + c]));
    if ((t_step & 7) == 1) orthonormalize_rows(Rn);
#pragma unroll
    for (int q = 0; q < 3; ++q) cn[q] = __dadd_rn(Rc[9 + q], (double)dl[3 + q]);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const size_t o = (size_t)kc * 6 + q;
        d.m[o] = mo[q];
        d.v[o] = vo[q];
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) d.R[(size_t)kc * 9 + q] = Rn[q];
#pragma unroll
    for (int q = 0; q < 3; ++q) d.c[(size_t)kc * 3 + q] = cn[q];
    write_camrec(rec_out, Rn, cn, s_new);
    return bl;
}

}  // namespace fm
