/*
 * Oracle for the epipolar adjustment of FastMap: a plain, slow FP64 CPU restatement of the
 * objective, its gradient, the IRLS reweighting with outlier filtering and the first-order
 * optimisation loop.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path links, loads or calls this file;
 * only the tests, the smoke check and the benchmark's CPU-baseline leg do. It shares no
 * code, header or constant with the CUDA library.
 *
 * Notation (Sec. "Epipolar Adjustment"):
 *   camera k is world-to-camera, x_cam = R_k X + t_k; its centre is c_k = -R_k^T t_k.
 *   image pair n = (i, j) = (i_n, j_n); point pair m of pair n is (x1, x2) with x1 in image
 *   i and x2 in image j, both normalized homogeneous coordinates (x, y, 1).
 *   R_n = R_j R_i^T, t_n = t_j - R_n t_i = R_j (c_i - c_j), t^_n = t_n / |t_n|,
 *   E_n = [t^_n]_x R_n  (the essential matrix "computed from the global rotations and
 *   translations", Eq. epipolar-objective; its translation is taken with unit length).
 *   epsilon_nm = x2^T E_n x1.
 *
 * Losses (Z = total number of point pairs, a constant):
 *   L1   : L_e = (1/Z) sum |epsilon|                         (Eq. epipolar-objective)
 *   IRLS : L^_e = (1/Z) sum w * epsilon^2, w held fixed       (Eq. after the IRLS paragraph)
 *
 * Parameters: per camera a left rotation increment phi_k (R_k <- Exp(phi_k) R_k) and the
 * camera centre c_k. Gradients are d/d(phi_k, c_k) at phi = 0, ordered
 * [phi_x, phi_y, phi_z, c_x, c_y, c_z].
 *
 * Every loop runs in input order; nothing is blocked, fused or reordered.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

/* ---- 3x3 helpers (row-major) ---------------------------------------------------------- */
static void mat_mul(const double *A, const double *B, double *C) {
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * r + k] * B[3 * k + c];
            C[3 * r + c] = s;
        }
}

static void mat_mul_bt(const double *A, const double *B, double *C) { /* C = A B^T */
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * r + k] * B[3 * c + k];
            C[3 * r + c] = s;
        }
}

static void mat_mul_at(const double *A, const double *B, double *C) { /* C = A^T B */
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * k + r] * B[3 * k + c];
            C[3 * r + c] = s;
        }
}

static void mat_vec(const double *A, const double *v, double *out) {
    for (int r = 0; r < 3; ++r) out[r] = A[3 * r] * v[0] + A[3 * r + 1] * v[1] + A[3 * r + 2] * v[2];
}

static void mat_tvec(const double *A, const double *v, double *out) { /* A^T v */
    for (int r = 0; r < 3; ++r) out[r] = A[r] * v[0] + A[3 + r] * v[1] + A[6 + r] * v[2];
}

static void hat(const double *v, double *K) { /* [v]_x */
    K[0] = 0.0;   K[1] = -v[2]; K[2] = v[1];
    K[3] = v[2];  K[4] = 0.0;   K[5] = -v[0];
    K[6] = -v[1]; K[7] = v[0];  K[8] = 0.0;
}

static void vee(const double *M, double *v) { /* the v with <[v]_x, M> = v . vee(M) */
    v[0] = M[7] - M[5];
    v[1] = M[2] - M[6];
    v[2] = M[3] - M[1];
}

static void cross(const double *a, const double *b, double *out) {
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

/* ---- relative pose and essential matrix of one image pair ----------------------------- */
/* R_n = R_j R_i^T and t_n = R_j (c_i - c_j). Returns |t_n|. */
static double relative_pose(const double *Ri, const double *ci, const double *Rj,
                            const double *cj, double *Rn, double *tn) {
    double d[3] = {ci[0] - cj[0], ci[1] - cj[1], ci[2] - cj[2]};
    mat_mul_bt(Rj, Ri, Rn);
    mat_vec(Rj, d, tn);
    return sqrt(tn[0] * tn[0] + tn[1] * tn[1] + tn[2] * tn[2]);
}

/* E_n = [t^_n]_x R_n for every pair; also returns 0 if every |t_n| > 0, else -1. */
int or_essential(int n_pairs, const int32_t *cam_i, const int32_t *cam_j, const double *R,
                 const double *c, double *E) {
    int status = 0;
    for (int n = 0; n < n_pairs; ++n) {
        const int i = cam_i[n], j = cam_j[n];
        double Rn[9], tn[3], K[9];
        const double nt = relative_pose(R + 9 * i, c + 3 * i, R + 9 * j, c + 3 * j, Rn, tn);
        if (!(nt > 0.0)) status = -1;
        const double th[3] = {tn[0] / nt, tn[1] / nt, tn[2] / nt};
        hat(th, K);
        mat_mul(K, Rn, E + 9 * n);
    }
    return status;
}

/* epsilon = x2^T E x1 with x = (x, y, 1). */
static double epipolar(const double *E, const double *x1, const double *x2) {
    const double a[3] = {x1[0], x1[1], 1.0};
    const double b[3] = {x2[0], x2[1], 1.0};
    double s = 0.0;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) s += b[r] * E[3 * r + c] * a[c];
    return s;
}

/* Residuals epsilon_nm of every point pair (input order). */
int or_residuals(int n_cams, const double *R, const double *c, int n_pairs,
                 const int32_t *cam_i, const int32_t *cam_j, int64_t n_pp,
                 const int32_t *pair_id, const double *x1, const double *x2, double *E_work,
                 double *eps) {
    (void)n_cams;
    const int st = or_essential(n_pairs, cam_i, cam_j, R, c, E_work);
    for (int64_t p = 0; p < n_pp; ++p)
        eps[p] = epipolar(E_work + 9 * pair_id[p], x1 + 2 * p, x2 + 2 * p);
    return st;
}

/*
 * Loss and gradient.
 *   mode 0 (IRLS): loss = (1/Z) sum w eps^2, dloss/deps = (2/Z) w eps  (w must be given)
 *   mode 1 (L1)  : loss = (1/Z) sum |eps|,   dloss/deps = (1/Z) sign(eps)
 * G_n = dloss/dE_n = sum_m dloss/deps * x2 x1^T, then the chain rule through
 * E_n = [t^]_x R_n, t^ = t_n/|t_n|, t_n = R_j (c_i - c_j), R_n = R_j R_i^T with left
 * perturbations R_k <- Exp(phi_k) R_k:
 *   A = dloss/dR_n (through E's R_n factor) = [t^]_x^T G = -[t^]_x G
 *   g_t^ = vee(G R_n^T),  g_t = (I - t^ t^^T) g_t^ / |t_n|
 *   g_ci = R_j^T g_t,  g_cj = -R_j^T g_t
 *   g_phi_j = vee(A R_n^T) + t_n x g_t,  g_phi_i = -vee(R_n^T A)
 * G_work must hold 9 * n_pairs doubles. Returns 0, or -1 if some |t_n| is zero.
 */
int or_loss_grad(int n_cams, const double *R, const double *c, int n_pairs,
                 const int32_t *cam_i, const int32_t *cam_j, int64_t n_pp,
                 const int32_t *pair_id, const double *x1, const double *x2, const double *w,
                 int mode, double *E_work, double *G_work, double *loss, double *grad) {
    const int st = or_essential(n_pairs, cam_i, cam_j, R, c, E_work);
    const double Z = (double)n_pp;
    memset(G_work, 0, sizeof(double) * 9 * (size_t)n_pairs);
    memset(grad, 0, sizeof(double) * 6 * (size_t)n_cams);
    double L = 0.0;
    for (int64_t p = 0; p < n_pp; ++p) {
        const int n = pair_id[p];
        const double *a = x1 + 2 * p, *b = x2 + 2 * p;
        const double e = epipolar(E_work + 9 * n, a, b);
        double d;
        if (mode == 0) {
            L += w[p] * e * e / Z;
            d = 2.0 * w[p] * e / Z;
        } else {
            L += fabs(e) / Z;
            d = (e > 0.0 ? 1.0 : (e < 0.0 ? -1.0 : 0.0)) / Z;
        }
        const double av[3] = {a[0], a[1], 1.0};
        const double bv[3] = {b[0], b[1], 1.0};
        for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 3; ++q) G_work[9 * n + 3 * r + q] += d * bv[r] * av[q];
    }
    *loss = L;
    for (int n = 0; n < n_pairs; ++n) {
        const int i = cam_i[n], j = cam_j[n];
        const double *Ri = R + 9 * i, *Rj = R + 9 * j;
        double Rn[9], tn[3];
        const double nt = relative_pose(Ri, c + 3 * i, Rj, c + 3 * j, Rn, tn);
        const double th[3] = {tn[0] / nt, tn[1] / nt, tn[2] / nt};
        const double *G = G_work + 9 * n;
        double K[9], A[9], M[9], gth[3], gt[3], tmp[3];
        hat(th, K);
        mat_mul(K, G, A);
        for (int k = 0; k < 9; ++k) A[k] = -A[k];
        mat_mul_bt(G, Rn, M);
        vee(M, gth);
        const double dp = th[0] * gth[0] + th[1] * gth[1] + th[2] * gth[2];
        for (int k = 0; k < 3; ++k) gt[k] = (gth[k] - dp * th[k]) / nt;
        /* centres */
        mat_tvec(Rj, gt, tmp);
        for (int k = 0; k < 3; ++k) {
            grad[6 * i + 3 + k] += tmp[k];
            grad[6 * j + 3 + k] -= tmp[k];
        }
        /* rotation of camera j: through R_n and through t_n */
        double ARt[9], gpj[3], txg[3];
        mat_mul_bt(A, Rn, ARt);
        vee(ARt, gpj);
        cross(tn, gt, txg);
        for (int k = 0; k < 3; ++k) grad[6 * j + k] += gpj[k] + txg[k];
        /* rotation of camera i: through R_n */
        double RtA[9], gpi[3];
        mat_mul_at(Rn, A, RtA);
        vee(RtA, gpi);
        for (int k = 0; k < 3; ++k) grad[6 * i + k] -= gpi[k];
    }
    return st;
}

/*
 * IRLS weights with outlier filtering (Sec. "Epipolar Adjustment", IRLS and filtering
 * paragraphs): a point pair whose |epsilon^| exceeds the round's threshold tau is filtered
 * (w = 0); otherwise w = 1 / max(|epsilon^|, delta). Returns the number of kept pairs.
 */
int64_t or_irls_weights(int64_t n_pp, const double *eps_hat, double tau, double delta,
                        double *w) {
    int64_t kept = 0;
    for (int64_t p = 0; p < n_pp; ++p) {
        const double a = fabs(eps_hat[p]);
        if (a <= tau) {
            w[p] = 1.0 / (a > delta ? a : delta);
            ++kept;
        } else {
            w[p] = 0.0;
        }
    }
    return kept;
}

/* Exp(phi) by Rodrigues' formula: I + sin(th)/th K + (1 - cos(th))/th^2 K^2, K = [phi]_x. */
void or_expmap(const double *phi, double *Rout) {
    const double th2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
    const double th = sqrt(th2);
    double a, b;
    if (th < 1e-8) {
        a = 1.0 - th2 / 6.0;
        b = 0.5 - th2 / 24.0;
    } else {
        a = sin(th) / th;
        b = (1.0 - cos(th)) / th2;
    }
    double K[9], K2[9];
    hat(phi, K);
    mat_mul(K, K, K2);
    for (int k = 0; k < 9; ++k) Rout[k] = (k % 4 == 0 ? 1.0 : 0.0) + a * K[k] + b * K2[k];
}

/*
 * One Adam step (Kingma & Ba; the adaptive first-order optimiser the method relies on) on
 * every camera's (phi_k, c_k), then R_k <- Exp(phi_k) R_k and phi_k <- 0. `step` is the
 * 1-based step number used in the bias corrections. lr[0] applies to phi, lr[1] to c.
 * The rotation is not re-orthonormalised here; or_project_rotations does that.
 */
void or_adam_step(int n_cams, double *R, double *c, const double *grad, double *m, double *v,
                  int64_t step, const double *lr, double beta1, double beta2, double eps) {
    const double bc1 = 1.0 - pow(beta1, (double)step);
    const double bc2 = 1.0 - pow(beta2, (double)step);
    for (int k = 0; k < n_cams; ++k) {
        double delta[6];
        for (int q = 0; q < 6; ++q) {
            const double g = grad[6 * k + q];
            m[6 * k + q] = beta1 * m[6 * k + q] + (1.0 - beta1) * g;
            v[6 * k + q] = beta2 * v[6 * k + q] + (1.0 - beta2) * g * g;
            const double mh = m[6 * k + q] / bc1, vh = v[6 * k + q] / bc2;
            delta[q] = -lr[q < 3 ? 0 : 1] * mh / (sqrt(vh) + eps);
        }
        double Ex[9], Rn[9];
        or_expmap(delta, Ex);
        mat_mul(Ex, R + 9 * k, Rn);
        memcpy(R + 9 * k, Rn, sizeof Rn);
        for (int q = 0; q < 3; ++q) c[3 * k + q] += delta[3 + q];
    }
}
