// Global rotation stage (Sec. "Global Rotation", Eq. fastmap-rotation-objective):
// world-to-camera rotations from relative rotations R_{i->j} of the image pairs.
//
// Initialisation (paragraph "Initialization details", column-wise least squares): column 1 of
// every rotation minimises sum_p ||x_j - R_p x_i||^2, column 2 the same (scaled by 1/|P|) plus
// (1/N) sum_k (x_k^T y_k)^2; camera 0's column is held at e1 / e2 (the gauge, R_0 = I), which
// leaves a symmetric positive definite system in the other cameras' columns:
//   A v = w_pair (deg_k v_k - sum_{p: k=j} R_p v_i - sum_{p: k=i} R_p^T v_j) + D_k v_k = b,
// solved by preconditioned conjugate gradients with the operator applied per camera from the
// CSR of the pair table (no matrix stored) and the 3x3 diagonal blocks as preconditioner.
// Columns are then normalised, column 2 orthogonalised to column 1, column 3 = 1 x 2.
//
// Refinement: L_R = (1/|P|) sum_p d(R_j, R_p R_i), d = geodesic distance, with each R_k given
// by the 6D representation (a1, a2): b1 = a1/|a1|, b2 = (a2 - (b1.a2) b1)/|.|, b3 = b1 x b2.
// Per iteration k_rot_pair computes every pair's distance and its gradient with respect to R_i
// and R_j, and k_rot_cam gathers a camera's gradient, maps it through the 6D representation and
// takes the Adam step. All in FP64 (per pair a few hundred flops; O(pairs) per iteration).
#include <cmath>
#include <string>
#include <vector>

#include "fm_walk.cuh"

void fm_internal_set_error(const char *msg);

using namespace fm;

namespace {

constexpr int RT_THREADS = 256;
constexpr int RT_CAMS = 8;    // cameras (warps) per block of the per-camera kernels
constexpr double C_MAX = 1.0 - 1e-12;

struct DevRot {
    int n_cams, n_pairs;
    const int *cam_i, *cam_j, *cam_off, *cam_ent;
    const double *Rrel;      // n_pairs x 9 (row-major)
    double *a;               // n_cams x 6: the 6D parameters
    double *R;               // n_cams x 9: rotations of the current parameters
    float *m, *v;            // Adam moments, n_cams x 6
    double *pgrad;           // n_pairs x 18: d d_p / d R_i (9), d d_p / d R_j (9)
    double *pdist;           // n_pairs: d_p
    double *blk;             // per-block partial sums (loss, CG dot products)
    double *loss;
    double *hyper;           // lr, beta1, beta2, eps
    long long *step;
    // conjugate gradients: vectors n_cams x 3 and scalars
    double *x, *r, *z, *p, *q, *col1, *scal;   // scal: rz, rz_new, pq, w_pair, w_pen
    unsigned *err;
};

__host__ __device__ inline int cam_blocks(int n) { return (n + RT_CAMS - 1) / RT_CAMS; }

// ---- small FP64 3x3 helpers ---------------------------------------------------------------------
__device__ __forceinline__ void mat_vec(const double *M, const double *v, double *o) {
#pragma unroll
    for (int a = 0; a < 3; ++a) o[a] = M[3 * a] * v[0] + M[3 * a + 1] * v[1] + M[3 * a + 2] * v[2];
}
__device__ __forceinline__ void mat_t_vec(const double *M, const double *v, double *o) {
#pragma unroll
    for (int a = 0; a < 3; ++a) o[a] = M[a] * v[0] + M[3 + a] * v[1] + M[6 + a] * v[2];
}

// warp-wide sum of n doubles (fixed butterfly order)
template <int N>
__device__ __forceinline__ void warp_sum(double *v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < N; ++q) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
}

// ---- conjugate gradients on the anchored column system ----------------------------------------
// (A v)_k for camera k != 0 (camera 0's entries are fixed and excluded: its row is not part of
// the system and its column contributes to the right-hand side only)
__device__ void apply_A(const DevRot &t, const double *v, int k, int lane, bool skip_anchor, double *out) {
    const int e_begin = t.cam_off[k], e_end = t.cam_off[k + 1];
    double s[3] = {0.0, 0.0, 0.0};
    for (int e = e_begin + lane; e < e_end; e += 32) {
        const int ent = t.cam_ent[e];
        const int n = ent >> 1, role = ent & 1;
        const int other = role ? t.cam_i[n] : t.cam_j[n];
        if (skip_anchor && other == 0) continue;
        double o[3];
        const double *vo = v + (size_t)other * 3;
        if (role) mat_vec(t.Rrel + (size_t)n * 9, vo, o);      // k = j: R_p v_i
        else mat_t_vec(t.Rrel + (size_t)n * 9, vo, o);         // k = i: R_p^T v_j
#pragma unroll
        for (int a = 0; a < 3; ++a) s[a] += o[a];
    }
    warp_sum<3>(s);
    const double wp = t.scal[3], wq = t.scal[4];
    const double deg = (double)(e_end - e_begin);
    const double *vk = v + (size_t)k * 3, *ck = t.col1 + (size_t)k * 3;
    const double dot = ck[0] * vk[0] + ck[1] * vk[1] + ck[2] * vk[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) out[a] = wp * (deg * vk[a] - s[a]) + wq * ck[a] * dot;
}

// z = M^-1 r with M the 3x3 diagonal block w_pair deg I + w_pen c c^T:
// (alpha I + beta c c^T)^-1 = (I - beta/(alpha + beta |c|^2) c c^T) / alpha
__device__ __forceinline__ void precondition(const DevRot &t, int k, const double *rk, double *zk) {
    const double deg = (double)(t.cam_off[k + 1] - t.cam_off[k]);
    const double al = t.scal[3] * deg, be = t.scal[4];
    const double *c = t.col1 + (size_t)k * 3;
    const double cc = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    const double cr = c[0] * rk[0] + c[1] * rk[1] + c[2] * rk[2];
    const double f = be / (al + be * cc);
#pragma unroll
    for (int a = 0; a < 3; ++a) zk[a] = (rk[a] - f * c[a] * cr) / al;
}

// setup: x = 0 except the anchor, r = b - A x = -(A x_anchor) on cameras != 0, z = M^-1 r, p = z;
// block partial sums of r.z
__global__ void __launch_bounds__(RT_CAMS * 32) k_cg_init(DevRot t) {
    __shared__ double s_blk[RT_CAMS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = blockIdx.x * RT_CAMS + warp;
    double rz = 0.0;
    if (k < t.n_cams) {
        if (k == 0) {
            if (lane == 0)
#pragma unroll
                for (int a = 0; a < 3; ++a) t.r[a] = t.z[a] = t.p[a] = 0.0;
        } else {
            // b_k = (contribution of the fixed anchor column): sum over pairs with camera 0
            double s[3] = {0.0, 0.0, 0.0};
            for (int e = t.cam_off[k] + lane; e < t.cam_off[k + 1]; e += 32) {
                const int ent = t.cam_ent[e];
                const int n = ent >> 1, role = ent & 1;
                const int other = role ? t.cam_i[n] : t.cam_j[n];
                if (other != 0) continue;
                double o[3];
                if (role) mat_vec(t.Rrel + (size_t)n * 9, t.x, o);
                else mat_t_vec(t.Rrel + (size_t)n * 9, t.x, o);
#pragma unroll
                for (int a = 0; a < 3; ++a) s[a] += o[a];
            }
            warp_sum<3>(s);
            if (lane == 0) {
                double rk[3], zk[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) rk[a] = t.scal[3] * s[a];   // b - A x with x_k = 0
                precondition(t, k, rk, zk);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    t.x[(size_t)k * 3 + a] = 0.0;
                    t.r[(size_t)k * 3 + a] = rk[a];
                    t.z[(size_t)k * 3 + a] = zk[a];
                    t.p[(size_t)k * 3 + a] = zk[a];
                }
                rz = rk[0] * zk[0] + rk[1] * zk[1] + rk[2] * zk[2];
            }
        }
    }
    if (lane == 0) s_blk[warp] = rz;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < RT_CAMS; ++w) b += s_blk[w];
        t.blk[blockIdx.x] = b;
    }
}

// sum of the per-block partials into scal[slot] (one block, fixed order). advance: first make
// the last iteration's new r.z (scal[1]) the current one (scal[0]); only this single-block
// launch writes scal[0], after every reader of the previous value has finished
__global__ void __launch_bounds__(RT_THREADS) k_block_sum(DevRot t, int n_blocks, int slot, int advance) {
    __shared__ double red[RT_THREADS];
    pdl_wait();
    pdl_trigger();
    if (advance && threadIdx.x == 0) t.scal[0] = t.scal[1];
    double s = 0.0;
    for (int b = threadIdx.x; b < n_blocks; b += RT_THREADS) s += t.blk[b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = RT_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) t.scal[slot] = red[0];
}

// q = A p on cameras != 0; block partials of p.q
__global__ void __launch_bounds__(RT_CAMS * 32) k_cg_matvec(DevRot t) {
    __shared__ double s_blk[RT_CAMS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = blockIdx.x * RT_CAMS + warp;
    pdl_wait();
    pdl_trigger();
    double pq = 0.0;
    if (k > 0 && k < t.n_cams) {
        double o[3];
        apply_A(t, t.p, k, lane, true, o);
        if (lane == 0) {
#pragma unroll
            for (int a = 0; a < 3; ++a) t.q[(size_t)k * 3 + a] = o[a];
            pq = o[0] * t.p[(size_t)k * 3] + o[1] * t.p[(size_t)k * 3 + 1] + o[2] * t.p[(size_t)k * 3 + 2];
        }
    }
    if (lane == 0) s_blk[warp] = pq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < RT_CAMS; ++w) b += s_blk[w];
        t.blk[blockIdx.x] = b;
    }
}

// x += alpha p, r -= alpha q, z = M^-1 r (alpha = rz / pq); block partials of the new r.z
__global__ void __launch_bounds__(RT_THREADS) k_cg_update(DevRot t) {
    __shared__ double red[RT_THREADS];
    pdl_wait();
    pdl_trigger();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const double pq = t.scal[2];
    const double alpha = pq > 0.0 ? t.scal[0] / pq : 0.0;
    double rz = 0.0;
    if (k > 0 && k < t.n_cams) {
        double rk[3], zk[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const size_t o = (size_t)k * 3 + a;
            t.x[o] += alpha * t.p[o];
            rk[a] = t.r[o] - alpha * t.q[o];
            t.r[o] = rk[a];
        }
        precondition(t, k, rk, zk);
#pragma unroll
        for (int a = 0; a < 3; ++a) t.z[(size_t)k * 3 + a] = zk[a];
        rz = rk[0] * zk[0] + rk[1] * zk[1] + rk[2] * zk[2];
    }
    red[threadIdx.x] = rz;
    __syncthreads();
    for (int w = RT_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) t.blk[blockIdx.x] = red[0];
}

// p = z + beta p (beta = rz_new / rz), then rz = rz_new
__global__ void __launch_bounds__(RT_THREADS) k_cg_direction(DevRot t) {
    pdl_wait();
    pdl_trigger();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const double rz = t.scal[0], rzn = t.scal[1];
    const double beta = rz > 0.0 ? rzn / rz : 0.0;
    if (k > 0 && k < t.n_cams)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const size_t o = (size_t)k * 3 + a;
            t.p[o] = t.z[o] + beta * t.p[o];
        }
}

// normalise the solved column into col (n_cams x 3); `orth`: first remove its component along
// t.col1 (column 2)
__global__ void k_finish_column(DevRot t, double *col, int orth) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= t.n_cams) return;
    double v[3] = {t.x[(size_t)k * 3], t.x[(size_t)k * 3 + 1], t.x[(size_t)k * 3 + 2]};
    double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (!(n > 0.0) || !isfinite(n)) {
        atomicOr(t.err, ERR_DEGENERATE);
        n = 1.0;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) v[a] /= n;
    if (orth) {
        const double *c = t.col1 + (size_t)k * 3;
        const double d = c[0] * v[0] + c[1] * v[1] + c[2] * v[2];
#pragma unroll
        for (int a = 0; a < 3; ++a) v[a] -= d * c[a];
        n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (!(n > 0.0) || !isfinite(n)) {
            atomicOr(t.err, ERR_DEGENERATE);
            n = 1.0;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) v[a] /= n;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) col[(size_t)k * 3 + a] = v[a];
}

// ---- 6D representation and the geodesic objective ----------------------------------------------
__device__ __forceinline__ void cross3(const double *u, const double *v, double *o) {
    o[0] = u[1] * v[2] - u[2] * v[1];
    o[1] = u[2] * v[0] - u[0] * v[2];
    o[2] = u[0] * v[1] - u[1] * v[0];
}

// R (row-major) with columns b1, b2, b3 from a = (a1, a2)
__device__ void rot_from_6d(const double *a, double *R) {
    double b1[3], u[3], b2[3], b3[3];
    const double n1 = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
#pragma unroll
    for (int q = 0; q < 3; ++q) b1[q] = a[q] / n1;
    const double d = b1[0] * a[3] + b1[1] * a[4] + b1[2] * a[5];
#pragma unroll
    for (int q = 0; q < 3; ++q) u[q] = a[3 + q] - d * b1[q];
    const double nu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
#pragma unroll
    for (int q = 0; q < 3; ++q) b2[q] = u[q] / nu;
    cross3(b1, b2, b3);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        R[3 * r] = b1[r];
        R[3 * r + 1] = b2[r];
        R[3 * r + 2] = b3[r];
    }
}

// gradient with respect to a of a scalar whose gradient with respect to R is gR (row-major)
__device__ void rot_6d_backward(const double *a, const double *gR, double *ga) {
    double b1[3], u[3], b2[3], g1[3], g2[3], g3[3], gb1[3], gb2[3], gu[3], t1[3], t2[3];
    const double n1 = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
#pragma unroll
    for (int q = 0; q < 3; ++q) b1[q] = a[q] / n1;
    const double d = b1[0] * a[3] + b1[1] * a[4] + b1[2] * a[5];
#pragma unroll
    for (int q = 0; q < 3; ++q) u[q] = a[3 + q] - d * b1[q];
    const double nu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        b2[q] = u[q] / nu;
        g1[q] = gR[3 * q];
        g2[q] = gR[3 * q + 1];
        g3[q] = gR[3 * q + 2];
    }
    cross3(b2, g3, t1);      // b3 = b1 x b2: gradient b2 x g3 on b1, g3 x b1 on b2
    cross3(g3, b1, t2);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        gb1[q] = g1[q] + t1[q];
        gb2[q] = g2[q] + t2[q];
    }
    const double b2g = b2[0] * gb2[0] + b2[1] * gb2[1] + b2[2] * gb2[2];
#pragma unroll
    for (int q = 0; q < 3; ++q) gu[q] = (gb2[q] - b2[q] * b2g) / nu;
    const double b1gu = b1[0] * gu[0] + b1[1] * gu[1] + b1[2] * gu[2];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        ga[3 + q] = gu[q] - b1[q] * b1gu;
        gb1[q] = gb1[q] - gu[q] * d - a[3 + q] * b1gu;
    }
    const double b1g = b1[0] * gb1[0] + b1[1] * gb1[1] + b1[2] * gb1[2];
#pragma unroll
    for (int q = 0; q < 3; ++q) ga[q] = (gb1[q] - b1[q] * b1g) / n1;
}

__global__ void k_rot_from_params(DevRot t) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= t.n_cams) return;
    double R[9];
    rot_from_6d(t.a + (size_t)k * 6, R);
#pragma unroll
    for (int q = 0; q < 9; ++q) t.R[(size_t)k * 9 + q] = R[q];
}

// per pair: X = R_p R_i, c = (tr(R_j^T X) - 1)/2, d = arccos(c);
// d d/d R_j = s X, d d/d R_i = s R_p^T R_j with s = -1/(2 sqrt(1 - c^2)) (c clamped below 1)
__global__ void __launch_bounds__(RT_THREADS) k_rot_pair(DevRot t) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = n < t.n_pairs ? t.cam_i[n] : 0, j = n < t.n_pairs ? t.cam_j[n] : 0;
    pdl_wait();     // rotations of the previous step
    pdl_trigger();
    if (n >= t.n_pairs) return;
    const double *Rp = t.Rrel + (size_t)n * 9, *Ri = t.R + (size_t)i * 9, *Rj = t.R + (size_t)j * 9;
    double X[9], Y[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            X[3 * a + b] = Rp[3 * a] * Ri[b] + Rp[3 * a + 1] * Ri[3 + b] + Rp[3 * a + 2] * Ri[6 + b];
            Y[3 * a + b] = Rp[a] * Rj[b] + Rp[3 + a] * Rj[3 + b] + Rp[6 + a] * Rj[6 + b];   // R_p^T R_j
        }
    double tr = 0.0;
#pragma unroll
    for (int q = 0; q < 9; ++q) tr += Rj[q] * X[q];
    const double c = 0.5 * (tr - 1.0);
    const double cc = fmin(fmax(c, -1.0), C_MAX);
    const double s = -0.5 / sqrt(1.0 - cc * cc);
    t.pdist[n] = acos(fmin(fmax(c, -1.0), 1.0));
    double *g = t.pgrad + (size_t)n * 18;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        g[q] = s * Y[q];
        g[9 + q] = s * X[q];
    }
}

// warp per camera: gather d L/d R_k from its pairs (scaled 1/|P|); then lanes 0..RT_CAMS-1 of
// warp 0 map the block's cameras through the 6D representation and take the Adam step (apply)
// or write the gradient (apply = 0: grad_out holds n_cams x 6 gradients), one camera per lane:
// GB300's FP64 pipe charges a whole warp instruction per operation, so the FP64 tail runs once
// per block instead of once per camera. Block partials of the loss.
__global__ void __launch_bounds__(RT_CAMS * 32) k_rot_cam(DevRot t, int it, int apply, double *grad_out) {
    __shared__ double s_g[RT_CAMS][10];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = blockIdx.x * RT_CAMS + warp;
    pdl_wait();     // pair gradients of this step
    pdl_trigger();
    {
        double g[10];
#pragma unroll
        for (int q = 0; q < 10; ++q) g[q] = 0.0;
        if (k < t.n_cams) {
            for (int e = t.cam_off[k] + lane; e < t.cam_off[k + 1]; e += 32) {
                const int ent = t.cam_ent[e];
                const int n = ent >> 1, role = ent & 1;
                const double *pg = t.pgrad + (size_t)n * 18 + (role ? 9 : 0);
#pragma unroll
                for (int q = 0; q < 9; ++q) g[q] += pg[q];
                if (role == 0) g[9] += t.pdist[n];     // each pair's distance counted once
            }
            warp_sum<10>(g);
        }
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < 10; ++q) s_g[warp][q] = g[q];
        }
    }
    __syncthreads();
    if (warp != 0 || lane >= RT_CAMS) return;
    const int kc = blockIdx.x * RT_CAMS + lane;
    if (kc < t.n_cams) {
        const double inv_b = 1.0 / (double)t.n_pairs;
        double g[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) g[q] = s_g[lane][q] * inv_b;
        double ga[6];
        rot_6d_backward(t.a + (size_t)kc * 6, g, ga);
        if (!apply) {
#pragma unroll
            for (int q = 0; q < 6; ++q) grad_out[(size_t)kc * 6 + q] = ga[q];
        } else {
            const long long ts = *t.step + 1 + it;
            const float lr = (float)t.hyper[0], b1 = (float)t.hyper[1], b2 = (float)t.hyper[2],
                        eps = (float)t.hyper[3];
            const float bc1 = 1.f - powf(b1, (float)ts), bc2 = 1.f - powf(b2, (float)ts);
            double *ak = t.a + (size_t)kc * 6;
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const size_t o = (size_t)kc * 6 + q;
                const float gq = (float)ga[q];
                const float mo = b1 * t.m[o] + (1.f - b1) * gq;
                const float vo = b2 * t.v[o] + (1.f - b2) * gq * gq;
                t.m[o] = mo;
                t.v[o] = vo;
                ak[q] -= (double)(lr * (mo / bc1) / (sqrtf(vo / bc2) + eps));
            }
        }
    }
    if (lane == 0) {   // loss partial of the block, cameras in order
        double b = 0.0;
        for (int w = 0; w < RT_CAMS; ++w) b += s_g[w][9];
        t.blk[blockIdx.x] = b;
    }
}


// rotations of the updated parameters (after a step) + loss of the step's evaluation
__global__ void __launch_bounds__(RT_THREADS) k_rot_finish(DevRot t, int count) {
    __shared__ double red[RT_THREADS];
    pdl_wait();
    pdl_trigger();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < t.n_cams) {
        double R[9];
        rot_from_6d(t.a + (size_t)k * 6, R);
#pragma unroll
        for (int q = 0; q < 9; ++q) t.R[(size_t)k * 9 + q] = R[q];
    }
    if (blockIdx.x == 0) {
        const int nb = cam_blocks(t.n_cams);
        double s = 0.0;
        for (int b = threadIdx.x; b < nb; b += RT_THREADS) s += t.blk[b];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int w = RT_THREADS / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            *t.loss = red[0] / (double)t.n_pairs;
            *t.step += count;
        }
    }
}

// between iterations inside a chain: rotations of the updated parameters
__global__ void __launch_bounds__(RT_THREADS) k_rot_refresh(DevRot t) {
    pdl_wait();
    pdl_trigger();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= t.n_cams) return;
    double R[9];
    rot_from_6d(t.a + (size_t)k * 6, R);
#pragma unroll
    for (int q = 0; q < 9; ++q) t.R[(size_t)k * 9 + q] = R[q];
}

// 6D parameters from rotations (columns 1 and 2)
__global__ void k_params_from_rot(DevRot t) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= t.n_cams) return;
    const double *R = t.R + (size_t)k * 9;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        t.a[(size_t)k * 6 + q] = R[3 * q];
        t.a[(size_t)k * 6 + 3 + q] = R[3 * q + 1];
    }
}

// R_k from the two solved columns: [c1 c2 c1 x c2]
__global__ void k_rot_from_columns(DevRot t, const double *c1, const double *c2) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= t.n_cams) return;
    const double *x = c1 + (size_t)k * 3, *y = c2 + (size_t)k * 3;
    double z[3];
    cross3(x, y, z);
    double *R = t.R + (size_t)k * 9;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        R[3 * r] = x[r];
        R[3 * r + 1] = y[r];
        R[3 * r + 2] = z[r];
    }
}

}  // namespace

struct fm_rotation {
    DevRot d{};
    fm_rotation_options opt{};
    cudaStream_t user = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t graph = nullptr, graph8 = nullptr;
    double *col2 = nullptr;
    double *grad6 = nullptr;
    std::vector<void *> allocs;
    int cg_iters_last = 0;
    double cg_resid_last = 0.0;
};

namespace {

fm_status rfail(fm_status s, const std::string &msg) {
    fm_internal_set_error(msg.c_str());
    return s;
}

#define RT_CUDA(call)                                                                         \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return rfail(e_ == cudaErrorMemoryAllocation ? FM_ENOMEM : FM_ECUDA,              \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                 \
    } while (0)

template <class T>
cudaError_t ralloc(fm_rotation *p, T **ptr, size_t count) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(ptr), sizeof(T) * (count ? count : 1));
    if (e == cudaSuccess) p->allocs.push_back(*ptr);
    return e;
}

cudaError_t rjoin_in(fm_rotation *p) {
    cudaError_t e = cudaEventRecord(p->ev_in, p->user);
    if (e != cudaSuccess) return e;
    return cudaStreamWaitEvent(p->s, p->ev_in, 0);
}

cudaError_t rjoin_out(fm_rotation *p) {
    cudaError_t e = cudaEventRecord(p->ev_out, p->s);
    if (e != cudaSuccess) return e;
    return cudaStreamWaitEvent(p->user, p->ev_out, 0);
}

fm_status rcheck_errors(fm_rotation *p) {
    unsigned err = 0;
    RT_CUDA(cudaMemcpyAsync(&err, p->d.err, sizeof err, cudaMemcpyDeviceToHost, p->s));
    RT_CUDA(cudaStreamSynchronize(p->s));
    if (err & ERR_DEGENERATE) {
        const unsigned zero = 0;
        RT_CUDA(cudaMemcpyAsync(p->d.err, &zero, sizeof zero, cudaMemcpyHostToDevice, p->s));
        RT_CUDA(cudaStreamSynchronize(p->s));
        return rfail(FM_EDEGENERATE, "a solved rotation column vanished or is not finite (last solve: " +
                                         std::to_string(p->cg_iters_last) + " conjugate-gradient iterations, " +
                                         "relative residual " + std::to_string(p->cg_resid_last) + ")");
    }
    return FM_OK;
}

int cblocks(const fm_rotation *p) { return cam_blocks(p->d.n_cams); }
int tblocks(const fm_rotation *p) { return (p->d.n_cams + RT_THREADS - 1) / RT_THREADS; }

// one iteration: pair terms, camera gathers + Adam, rotations of the new parameters
void enqueue_steps(fm_rotation *p, int iters) {
    const dim3 gp((p->d.n_pairs + RT_THREADS - 1) / RT_THREADS);
    for (int it = 0; it < iters; ++it) {
        launch_k(k_rot_pair, gp, dim3(RT_THREADS), p->s, true, p->d);
        launch_k(k_rot_cam, dim3(cblocks(p)), dim3(RT_CAMS * 32), p->s, true, p->d, it, 1, (double *)nullptr);
        if (it + 1 < iters) launch_k(k_rot_refresh, dim3(tblocks(p)), dim3(RT_THREADS), p->s, true, p->d);
    }
    launch_k(k_rot_finish, dim3(tblocks(p)), dim3(RT_THREADS), p->s, true, p->d, iters);
}

fm_status build_rgraph(fm_rotation *p, int iters, cudaGraphExec_t *out) {
    cudaGraph_t g = nullptr;
    RT_CUDA(cudaStreamBeginCapture(p->s, cudaStreamCaptureModeThreadLocal));
    enqueue_steps(p, iters);
    cudaError_t e = cudaStreamEndCapture(p->s, &g);
    if (e != cudaSuccess) return rfail(FM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *out = nullptr;
        return rfail(FM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    return FM_OK;
}

void free_rot(fm_rotation *p) {
    if (!p) return;
    if (p->s) cudaStreamSynchronize(p->s);
    for (void *a : p->allocs) cudaFree(a);
    if (p->graph) cudaGraphExecDestroy(p->graph);
    if (p->graph8) cudaGraphExecDestroy(p->graph8);
    if (p->ev_in) cudaEventDestroy(p->ev_in);
    if (p->ev_out) cudaEventDestroy(p->ev_out);
    if (p->s) cudaStreamDestroy(p->s);
    delete p;
}

bool rfinite(const double *a, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

fm_status upload_hyper(fm_rotation *p) {
    const double h[4] = {p->opt.lr, p->opt.beta1, p->opt.beta2, p->opt.adam_eps};
    RT_CUDA(cudaMemcpyAsync(p->d.hyper, h, sizeof h, cudaMemcpyHostToDevice, p->s));
    RT_CUDA(cudaStreamSynchronize(p->s));
    return FM_OK;
}

// one anchored column system by preconditioned CG; the anchor column x_0 = e_axis;
// w_pair / w_pen weight the data term and the orthogonality penalty (along t.col1)
fm_status solve_column(fm_rotation *p, int axis, double w_pair, double w_pen, int max_iters, double tol) {
    DevRot &d = p->d;
    double e[3] = {0.0, 0.0, 0.0};
    e[axis] = 1.0;
    const double sc[2] = {w_pair, w_pen};
    RT_CUDA(cudaMemcpyAsync(d.x, e, sizeof e, cudaMemcpyHostToDevice, p->s));
    RT_CUDA(cudaMemcpyAsync(d.scal + 3, sc, sizeof sc, cudaMemcpyHostToDevice, p->s));
    k_cg_init<<<cblocks(p), RT_CAMS * 32, 0, p->s>>>(d);
    k_block_sum<<<1, RT_THREADS, 0, p->s>>>(d, cblocks(p), 1, 0);
    RT_CUDA(cudaGetLastError());
    double rz0 = 0.0;
    RT_CUDA(cudaMemcpyAsync(&rz0, d.scal + 1, sizeof rz0, cudaMemcpyDeviceToHost, p->s));
    RT_CUDA(cudaStreamSynchronize(p->s));
    // iterate in chunks; the host checks the residual between chunks
    constexpr int CHUNK = 32;
    int it = 0;
    double rz = rz0;
    while (it < max_iters && rz > tol * tol * rz0 && rz > 0.0) {
        for (int c = 0; c < CHUNK; ++c) {
            launch_k(k_cg_matvec, dim3(cblocks(p)), dim3(RT_CAMS * 32), p->s, true, d);
            launch_k(k_block_sum, dim3(1), dim3(RT_THREADS), p->s, true, d, cblocks(p), 2, 1);
            launch_k(k_cg_update, dim3(tblocks(p)), dim3(RT_THREADS), p->s, true, d);
            launch_k(k_block_sum, dim3(1), dim3(RT_THREADS), p->s, true, d, tblocks(p), 1, 0);
            launch_k(k_cg_direction, dim3(tblocks(p)), dim3(RT_THREADS), p->s, true, d);
        }
        RT_CUDA(cudaGetLastError());
        it += CHUNK;
        RT_CUDA(cudaMemcpyAsync(&rz, d.scal + 1, sizeof rz, cudaMemcpyDeviceToHost, p->s));
        RT_CUDA(cudaStreamSynchronize(p->s));
    }
    p->cg_iters_last = it;
    p->cg_resid_last = rz0 > 0.0 ? std::sqrt(rz / rz0) : 0.0;
    return FM_OK;
}

fm_status create_rot(fm_rotation *p, int32_t n_cams, int32_t n_pairs, const int32_t *cam_i, const int32_t *cam_j,
                     const double *R_rel) {
    DevRot &d = p->d;
    d.n_cams = n_cams;
    d.n_pairs = n_pairs;
    RT_CUDA(cudaStreamCreateWithFlags(&p->s, cudaStreamNonBlocking));
    RT_CUDA(cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming));
    RT_CUDA(cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming));
    RT_CUDA(rjoin_in(p));
    std::vector<int> cam_off(n_cams + 1, 0), cam_ent(2 * (size_t)n_pairs);
    for (int n = 0; n < n_pairs; ++n) {
        cam_off[cam_i[n] + 1]++;
        cam_off[cam_j[n] + 1]++;
    }
    for (int k = 0; k < n_cams; ++k) cam_off[k + 1] += cam_off[k];
    {
        std::vector<int> fill(cam_off.begin(), cam_off.end() - 1);
        for (int n = 0; n < n_pairs; ++n) {
            cam_ent[fill[cam_i[n]]++] = 2 * n;
            cam_ent[fill[cam_j[n]]++] = 2 * n + 1;
        }
    }
    int *ci = nullptr, *cj = nullptr, *co = nullptr, *ce = nullptr;
    double *rr = nullptr;
    RT_CUDA(ralloc(p, &ci, (size_t)n_pairs));
    RT_CUDA(ralloc(p, &cj, (size_t)n_pairs));
    RT_CUDA(ralloc(p, &co, (size_t)n_cams + 1));
    RT_CUDA(ralloc(p, &ce, 2 * (size_t)n_pairs));
    RT_CUDA(ralloc(p, &rr, 9 * (size_t)n_pairs));
    d.cam_i = ci;
    d.cam_j = cj;
    d.cam_off = co;
    d.cam_ent = ce;
    d.Rrel = rr;
    const size_t nc = (size_t)n_cams;
    RT_CUDA(ralloc(p, &d.a, 6 * nc));
    RT_CUDA(ralloc(p, &d.R, 9 * nc));
    RT_CUDA(ralloc(p, &d.m, 6 * nc));
    RT_CUDA(ralloc(p, &d.v, 6 * nc));
    RT_CUDA(ralloc(p, &d.pgrad, 18 * (size_t)n_pairs));
    RT_CUDA(ralloc(p, &d.pdist, (size_t)n_pairs));
    RT_CUDA(ralloc(p, &d.blk, (size_t)std::max(cam_blocks(n_cams), (n_cams + RT_THREADS - 1) / RT_THREADS)));
    RT_CUDA(ralloc(p, &d.loss, 1));
    RT_CUDA(ralloc(p, &d.hyper, 4));
    RT_CUDA(ralloc(p, &d.step, 1));
    RT_CUDA(ralloc(p, &d.x, 3 * nc));
    RT_CUDA(ralloc(p, &d.r, 3 * nc));
    RT_CUDA(ralloc(p, &d.z, 3 * nc));
    RT_CUDA(ralloc(p, &d.p, 3 * nc));
    RT_CUDA(ralloc(p, &d.q, 3 * nc));
    RT_CUDA(ralloc(p, &d.col1, 3 * nc));
    RT_CUDA(ralloc(p, &p->col2, 3 * nc));
    RT_CUDA(ralloc(p, &p->grad6, 6 * nc));
    RT_CUDA(ralloc(p, &d.scal, 8));
    RT_CUDA(ralloc(p, &d.err, 1));
    RT_CUDA(cudaMemcpyAsync(ci, cam_i, sizeof(int) * n_pairs, cudaMemcpyHostToDevice, p->s));
    RT_CUDA(cudaMemcpyAsync(cj, cam_j, sizeof(int) * n_pairs, cudaMemcpyHostToDevice, p->s));
    RT_CUDA(cudaMemcpyAsync(co, cam_off.data(), sizeof(int) * (n_cams + 1), cudaMemcpyHostToDevice, p->s));
    RT_CUDA(cudaMemcpyAsync(ce, cam_ent.data(), sizeof(int) * 2 * n_pairs, cudaMemcpyHostToDevice, p->s));
    RT_CUDA(cudaMemcpyAsync(rr, R_rel, sizeof(double) * 9 * n_pairs, cudaMemcpyHostToDevice, p->s));
    RT_CUDA(cudaMemsetAsync(d.m, 0, sizeof(float) * 6 * nc, p->s));
    RT_CUDA(cudaMemsetAsync(d.v, 0, sizeof(float) * 6 * nc, p->s));
    RT_CUDA(cudaMemsetAsync(d.step, 0, sizeof(long long), p->s));
    RT_CUDA(cudaMemsetAsync(d.err, 0, sizeof(unsigned), p->s));
    RT_CUDA(cudaMemsetAsync(d.col1, 0, sizeof(double) * 3 * nc, p->s));
    RT_CUDA(cudaMemsetAsync(d.scal, 0, sizeof(double) * 8, p->s));
    if (fm_status st = upload_hyper(p)) return st;
    RT_CUDA(rjoin_out(p));
    return FM_OK;
}

fm_status rcheck(const fm_rotation *p) {
    if (!p) return rfail(FM_EINVAL, "rotation problem is NULL");
    return FM_OK;
}

}  // namespace

extern "C" {

FM_API void fm_rotation_default_options(fm_rotation_options *opt) {
    if (!opt) return;
    opt->lr = 1e-3;
    opt->beta1 = 0.9;
    opt->beta2 = 0.999;
    opt->adam_eps = 1e-12;
    opt->cg_tol = 1e-9;
    opt->cg_max_iters = 20000;
    opt->use_graph = 1;
}

FM_API fm_status fm_rotation_create(int32_t n_cams, int32_t n_pairs, const int32_t *cam_i, const int32_t *cam_j,
                                    const double *R_rel, const fm_rotation_options *opt, void *stream,
                                    fm_rotation **out) {
    if (!out) return rfail(FM_EINVAL, "out must not be NULL");
    *out = nullptr;
    if (n_cams < 2) return rfail(FM_EINVAL, "n_cams must be >= 2");
    if (n_pairs < 1) return rfail(FM_EINVAL, "n_pairs must be >= 1");
    if (!cam_i || !cam_j || !R_rel) return rfail(FM_EINVAL, "array arguments must not be NULL");
    for (int n = 0; n < n_pairs; ++n)
        if (cam_i[n] < 0 || cam_i[n] >= n_cams || cam_j[n] < 0 || cam_j[n] >= n_cams || cam_i[n] == cam_j[n])
            return rfail(FM_EINVAL, "camera indices must be in [0, n_cams) with cam_i != cam_j");
    if (!rfinite(R_rel, 9 * (size_t)n_pairs)) return rfail(FM_EINVAL, "relative rotations must be finite");
    for (int n = 0; n < n_pairs; ++n) {
        const double *M = R_rel + 9 * (size_t)n;
        double worst = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                const double dot = M[a] * M[b] + M[3 + a] * M[3 + b] + M[6 + a] * M[6 + b];
                worst = std::max(worst, std::fabs(dot - (a == b ? 1.0 : 0.0)));
            }
        const double det = M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
                           M[2] * (M[3] * M[7] - M[4] * M[6]);
        if (worst > 1e-6 || std::fabs(det - 1.0) > 1e-6)
            return rfail(FM_EINVAL, "relative rotations must be rotation matrices (orthonormal, det +1)");
    }
    {
        // the image graph must be connected (the anchored systems are singular otherwise)
        std::vector<int> parent(n_cams);
        for (int k = 0; k < n_cams; ++k) parent[k] = k;
        auto find = [&](int k) {
            while (parent[k] != k) k = parent[k] = parent[parent[k]];
            return k;
        };
        int comps = n_cams;
        for (int n = 0; n < n_pairs; ++n) {
            const int a = find(cam_i[n]), b = find(cam_j[n]);
            if (a != b) {
                parent[a] = b;
                --comps;
            }
        }
        if (comps != 1) return rfail(FM_EINVAL, "the image graph must be connected");
    }
    fm_rotation_options o;
    fm_rotation_default_options(&o);
    if (opt) o = *opt;
    if (!(o.lr > 0.0) || !(o.beta1 >= 0.0 && o.beta1 < 1.0) || !(o.beta2 >= 0.0 && o.beta2 < 1.0) ||
        !(o.adam_eps > 0.0) || !(o.cg_tol > 0.0) || o.cg_max_iters < 1 || (o.use_graph != 0 && o.use_graph != 1))
        return rfail(FM_EINVAL, "invalid options");
    fm_rotation *p = new (std::nothrow) fm_rotation();
    if (!p) return rfail(FM_ENOMEM, "host allocation failed");
    p->opt = o;
    p->user = static_cast<cudaStream_t>(stream);
    fm_status st = create_rot(p, n_cams, n_pairs, cam_i, cam_j, R_rel);
    if (st != FM_OK) {
        free_rot(p);
        return st;
    }
    *out = p;
    return FM_OK;
}

FM_API void fm_rotation_destroy(fm_rotation *p) { free_rot(p); }

FM_API fm_status fm_rotation_initialize(fm_rotation *p, int32_t *cg_iters, double *cg_residual) {
    if (fm_status st = rcheck(p)) return st;
    RT_CUDA(rjoin_in(p));
    const int blocks = tblocks(p);
    const double n_pairs = (double)p->d.n_pairs, n_cams = (double)p->d.n_cams;
    int iters_total = 0;
    double resid = 0.0;
    // column 1: sum ||x_j - R_p x_i||^2, anchored x_0 = e1
    if (fm_status st = solve_column(p, 0, 1.0, 0.0, p->opt.cg_max_iters, p->opt.cg_tol)) return st;
    iters_total += p->cg_iters_last;
    resid = std::max(resid, p->cg_resid_last);
    k_finish_column<<<blocks, RT_THREADS, 0, p->s>>>(p->d, p->d.col1, 0);
    if (fm_status st = rcheck_errors(p)) return st;
    // column 2: (1/|P|) sum ||y_j - R_p y_i||^2 + (1/N) sum (x_k^T y_k)^2, anchored y_0 = e2
    if (fm_status st = solve_column(p, 1, 1.0 / n_pairs, 1.0 / n_cams, p->opt.cg_max_iters, p->opt.cg_tol))
        return st;
    iters_total += p->cg_iters_last;
    resid = std::max(resid, p->cg_resid_last);
    k_finish_column<<<blocks, RT_THREADS, 0, p->s>>>(p->d, p->col2, 1);
    k_rot_from_columns<<<blocks, RT_THREADS, 0, p->s>>>(p->d, p->d.col1, p->col2);
    k_params_from_rot<<<blocks, RT_THREADS, 0, p->s>>>(p->d);
    RT_CUDA(cudaGetLastError());
    RT_CUDA(cudaMemsetAsync(p->d.m, 0, sizeof(float) * 6 * p->d.n_cams, p->s));
    RT_CUDA(cudaMemsetAsync(p->d.v, 0, sizeof(float) * 6 * p->d.n_cams, p->s));
    RT_CUDA(cudaMemsetAsync(p->d.step, 0, sizeof(long long), p->s));
    if (fm_status st = rcheck_errors(p)) return st;
    if (cg_iters) *cg_iters = iters_total;
    if (cg_residual) *cg_residual = resid;
    return FM_OK;
}

FM_API fm_status fm_rotation_set_rotations(fm_rotation *p, const double *R) {
    if (fm_status st = rcheck(p)) return st;
    if (!R) return rfail(FM_EINVAL, "R must not be NULL");
    if (!rfinite(R, 9 * (size_t)p->d.n_cams)) return rfail(FM_EINVAL, "rotations must be finite");
    RT_CUDA(rjoin_in(p));
    RT_CUDA(cudaMemcpyAsync(p->d.R, R, sizeof(double) * 9 * p->d.n_cams, cudaMemcpyHostToDevice, p->s));
    k_params_from_rot<<<tblocks(p), RT_THREADS, 0, p->s>>>(p->d);
    k_rot_from_params<<<tblocks(p), RT_THREADS, 0, p->s>>>(p->d);
    RT_CUDA(cudaGetLastError());
    RT_CUDA(cudaMemsetAsync(p->d.m, 0, sizeof(float) * 6 * p->d.n_cams, p->s));
    RT_CUDA(cudaMemsetAsync(p->d.v, 0, sizeof(float) * 6 * p->d.n_cams, p->s));
    RT_CUDA(cudaMemsetAsync(p->d.step, 0, sizeof(long long), p->s));
    RT_CUDA(cudaStreamSynchronize(p->s));
    return FM_OK;
}

FM_API fm_status fm_rotation_set_params(fm_rotation *p, const double *a6) {
    if (fm_status st = rcheck(p)) return st;
    if (!a6) return rfail(FM_EINVAL, "a6 must not be NULL");
    if (!rfinite(a6, 6 * (size_t)p->d.n_cams)) return rfail(FM_EINVAL, "parameters must be finite");
    RT_CUDA(rjoin_in(p));
    RT_CUDA(cudaMemcpyAsync(p->d.a, a6, sizeof(double) * 6 * p->d.n_cams, cudaMemcpyHostToDevice, p->s));
    k_rot_from_params<<<tblocks(p), RT_THREADS, 0, p->s>>>(p->d);
    RT_CUDA(cudaGetLastError());
    RT_CUDA(cudaMemsetAsync(p->d.m, 0, sizeof(float) * 6 * p->d.n_cams, p->s));
    RT_CUDA(cudaMemsetAsync(p->d.v, 0, sizeof(float) * 6 * p->d.n_cams, p->s));
    RT_CUDA(cudaMemsetAsync(p->d.step, 0, sizeof(long long), p->s));
    RT_CUDA(cudaStreamSynchronize(p->s));
    return FM_OK;
}

FM_API fm_status fm_rotation_loss_grad(fm_rotation *p, double *loss, double *grad6) {
    if (fm_status st = rcheck(p)) return st;
    if (!loss) return rfail(FM_EINVAL, "loss must not be NULL");
    RT_CUDA(rjoin_in(p));
    const dim3 gp((p->d.n_pairs + RT_THREADS - 1) / RT_THREADS);
    launch_k(k_rot_pair, gp, dim3(RT_THREADS), p->s, false, p->d);
    launch_k(k_rot_cam, dim3(cblocks(p)), dim3(RT_CAMS * 32), p->s, true, p->d, 0, 0, p->grad6);
    launch_k(k_rot_finish, dim3(tblocks(p)), dim3(RT_THREADS), p->s, true, p->d, 0);
    RT_CUDA(cudaGetLastError());
    RT_CUDA(cudaMemcpyAsync(loss, p->d.loss, sizeof(double), cudaMemcpyDeviceToHost, p->s));
    if (grad6)
        RT_CUDA(cudaMemcpyAsync(grad6, p->grad6, sizeof(double) * 6 * p->d.n_cams, cudaMemcpyDeviceToHost, p->s));
    return rcheck_errors(p);
}

FM_API fm_status fm_rotation_step(fm_rotation *p, int32_t n_iters) {
    if (fm_status st = rcheck(p)) return st;
    if (n_iters < 0) return rfail(FM_EINVAL, "n_iters must be >= 0");
    if (n_iters == 0) return FM_OK;
    RT_CUDA(rjoin_in(p));
    if (!p->opt.use_graph) {
        enqueue_steps(p, n_iters);
        RT_CUDA(cudaGetLastError());
    } else {
        if (!p->graph)
            if (fm_status st = build_rgraph(p, 1, &p->graph)) return st;
        if (n_iters >= 8 && !p->graph8)
            if (fm_status st = build_rgraph(p, 8, &p->graph8)) return st;
        int left = n_iters;
        for (; left >= 8; left -= 8) RT_CUDA(cudaGraphLaunch(p->graph8, p->s));
        for (; left > 0; --left) RT_CUDA(cudaGraphLaunch(p->graph, p->s));
    }
    RT_CUDA(rjoin_out(p));
    return FM_OK;
}

FM_API fm_status fm_rotation_set_learning_rate(fm_rotation *p, double lr) {
    if (fm_status st = rcheck(p)) return st;
    if (!(lr > 0.0) || std::isinf(lr)) return rfail(FM_EINVAL, "lr must be finite and > 0");
    RT_CUDA(rjoin_in(p));
    p->opt.lr = lr;
    return upload_hyper(p);
}

FM_API fm_status fm_rotation_get_rotations(fm_rotation *p, double *R) {
    if (fm_status st = rcheck(p)) return st;
    if (!R) return rfail(FM_EINVAL, "R must not be NULL");
    RT_CUDA(rjoin_in(p));
    RT_CUDA(cudaMemcpyAsync(R, p->d.R, sizeof(double) * 9 * p->d.n_cams, cudaMemcpyDeviceToHost, p->s));
    return rcheck_errors(p);
}

FM_API fm_status fm_rotation_get_params(fm_rotation *p, double *a6) {
    if (fm_status st = rcheck(p)) return st;
    if (!a6) return rfail(FM_EINVAL, "a6 must not be NULL");
    RT_CUDA(rjoin_in(p));
    RT_CUDA(cudaMemcpyAsync(a6, p->d.a, sizeof(double) * 6 * p->d.n_cams, cudaMemcpyDeviceToHost, p->s));
    return rcheck_errors(p);
}

}  // extern "C"
