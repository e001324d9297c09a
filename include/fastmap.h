/*
 * fastmap.h - C ABI of the GB300 epipolar-adjustment library (libfastmap.so).
 *
 * The library refines global camera poses by FastMap's re-weighting epipolar adjustment
 * (Sec. "Epipolar Adjustment"): it minimises, over world-to-camera rotations and
 * translations, the mean absolute epipolar error
 *     L_e = (1/Z) sum_n sum_m | x2_nm^T E_n x1_nm |                (Eq. epipolar-objective)
 * through iteratively re-weighted least squares
 *     L^_e = (1/Z) sum_n sum_m w_nm (x2_nm^T E_n x1_nm)^2,  w_nm = 1/|eps^_nm|
 * (the IRLS objective of the same section) with periodic filtering of point pairs whose
 * error exceeds a shrinking threshold, using a first-order optimiser (Adam; Sec.
 * "First-order Optimization"). Every per-point-pair pass runs in the library's CUDA kernels.
 *
 * Conventions shared by all entry points
 *   - Camera k is world-to-camera: x_cam = R_k X + t_k; R is row-major 3x3, FP64. The
 *     library optimises R_k (by left increments, R_k <- Exp(phi_k) R_k) and the camera
 *     centre c_k = -R_k^T t_k. Poses cross the ABI as (R, t).
 *   - Image pair n = (cam_i[n], cam_j[n]), cam_i != cam_j. Point pair p belongs to pair
 *     pair_id[p]; x1[2p..2p+1] is its keypoint in image cam_i, x2[2p..2p+1] in image cam_j,
 *     both in normalized image coordinates ((u - cx)/f, (v - cy)/f) (Sec. "Camera
 *     Assumptions": principal point at the centre, intrinsics known).
 *   - E_n = [t_n/|t_n|]_x R_n with R_n = R_j R_i^T, t_n = t_j - R_n t_i (the essential
 *     matrix computed from the global poses; its translation is taken with unit length so
 *     the objective is invariant to the global scale).
 *   - Z = n_pp, the total number of point pairs (filtered pairs keep counting).
 *   - Gradients are with respect to (phi_k, c_k) at phi = 0, FP64, n_cams x 6, ordered
 *     [phi_x, phi_y, phi_z, c_x, c_y, c_z].
 *   - "Input order" means the order of the point pairs passed to fm_create_problem.
 *
 * Ownership and streams
 *   - fm_create_problem copies every input; the caller keeps its buffers. The problem owns
 *     all device memory it allocates and frees it in fm_destroy_problem.
 *   - Each problem runs its kernels on a private non-blocking stream, ordered after the
 *     work already queued on the caller's stream at call time (the `stream` argument of
 *     fm_create_problem, a cudaStream_t; NULL means the legacy default stream). Calls that
 *     return host data block until that data is ready; fm_step only enqueues.
 *   - A problem is not thread-safe; one host thread at a time may use it.
 *
 * Errors
 *   - No C++ exception crosses the ABI. Every entry point returns fm_status; FM_OK is 0.
 *   - Invalid arguments (NULL pointers, sizes out of range, pair indices out of range,
 *     cam_i == cam_j, an image pair without point pairs, non-finite or |coordinate| > 8
 *     keypoints) return FM_EINVAL and leave outputs untouched.
 *   - Device-detected problems (a relative translation of zero length, non-finite
 *     residuals) are recorded on the device and returned as FM_EDEGENERATE by the next call
 *     that synchronises (fm_synchronize, fm_get_poses, fm_loss_grad, ...).
 *   - fm_last_error() returns a thread-local message describing the last failure.
 */
#ifndef FASTMAP_H_
#define FASTMAP_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define FM_API __attribute__((visibility("default")))
#else
#define FM_API
#endif

typedef struct fm_problem fm_problem;

typedef enum {
    FM_OK = 0,
    FM_EINVAL = -1,      /* invalid argument or input data */
    FM_ENOMEM = -2,      /* device or host allocation failed */
    FM_ECUDA = -3,       /* a CUDA runtime call failed */
    FM_EDEGENERATE = -4, /* zero-length relative translation or non-finite value on device */
    FM_ESTATE = -5       /* call not valid in the problem's current state */
} fm_status;

/* Keypoint storage in device memory. */
enum {
    FM_STORE_FP32 = 0,   /* (x1, y1, x2, y2) as 4 x FP32 = 16 B per point pair + FP32 weight */
    FM_STORE_FP16 = 1    /* FP16 offsets from per-image centroids, 8 B + FP16 weight (2 B) */
};

/* Objective minimised by fm_step and returned by fm_loss_grad. */
enum {
    FM_LOSS_IRLS = 0,    /* (1/Z) sum w eps^2 with the current weights (all 1 until reweighted) */
    FM_LOSS_L1 = 1       /* (1/Z) sum |eps| */
};

typedef struct {
    int32_t storage;     /* FM_STORE_FP32 or FM_STORE_FP16 */
    int32_t loss;        /* FM_LOSS_IRLS or FM_LOSS_L1 */
    double delta;        /* IRLS weight floor: w = 1/max(|eps^|, delta); > 0 */
    double lr_rot;       /* Adam step size for phi (radians) */
    double lr_c;         /* Adam step size for camera centres (scene units) */
    double beta1, beta2; /* Adam moment decay rates, in [0, 1) */
    double adam_eps;     /* Adam denominator epsilon, >= 0 */
    int32_t use_graph;   /* 1: replay captured CUDA graphs of chained iterations in fm_step */
    int32_t refine_focal; /* 1: optimise each camera's focal length with the poses (0 or 1) */
    int64_t z_total;     /* Z of the objective; 0 means n_pp. A shard of a problem split across
                            processes sets the total point-pair count of all shards. */
} fm_options;

typedef struct {
    int32_t n_cams, n_pairs;
    int64_t n_pp;
    int32_t storage, loss;
    int64_t n_warp_ranges;      /* work units of the streaming kernels */
    int64_t stream_bytes;       /* algorithmic bytes read by one loss+gradient pass */
    int64_t device_bytes;       /* device memory held by the problem */
    int32_t input_was_sorted;   /* 1 if point pairs arrived grouped by pair_id */
    int32_t reserved;
} fm_info;

/* Defaults: FP32 storage, IRLS loss, delta 1e-6, lr_rot 1e-2, lr_c 1e-2, betas 0.9/0.999,
 * adam_eps 1e-12, use_graph 1. */
FM_API void fm_default_options(fm_options *opt);

/*
 * Build a problem (Sec. "Epipolar Adjustment": image pairs P = {(i_n, j_n)} and point-pair
 * sets Q_n). R (n_cams x 9) and t (n_cams x 3) are the initial poses, host FP64.
 * cam_i, cam_j (n_pairs) are host int32. pair_id (n_pp, int32), x1, x2 (n_pp x 2, FP32)
 * are host pointers, or device pointers when pp_on_device is 1. Point pairs may come in
 * any order; they are sorted by pair on the device (stable). Requires n_cams >= 2,
 * n_pairs >= 1, 1 <= n_pp < 2^31 - 2^16. Blocks until the device layout is built.
 */
FM_API fm_status fm_create_problem(int32_t n_cams, const double *R, const double *t,
                                   int32_t n_pairs, const int32_t *cam_i, const int32_t *cam_j,
                                   int64_t n_pp, const int32_t *pair_id, const float *x1,
                                   const float *x2, int32_t pp_on_device, const fm_options *opt,
                                   void *stream, fm_problem **out);

/* Free all device and host memory of the problem (after finishing its queued work). */
FM_API void fm_destroy_problem(fm_problem *p);

FM_API fm_status fm_problem_info(const fm_problem *p, fm_info *info);

/* Current poses (host FP64, R n_cams x 9, t n_cams x 3). Synchronises. */
FM_API fm_status fm_get_poses(fm_problem *p, double *R, double *t);
/* Replace the poses (host FP64); keeps the optimiser state. */
FM_API fm_status fm_set_poses(fm_problem *p, const double *R, const double *t);

/*
 * The optimiser's own parameters: rotations R (n_cams x 9) and camera centres c (n_cams x 3),
 * host FP64, copied without conversion. Together with fm_get_state/fm_set_state and the
 * weights they make an exact checkpoint (fm_get_poses/fm_set_poses convert t = -R c and
 * round in the last bit). fm_get_params synchronises.
 */
FM_API fm_status fm_get_params(fm_problem *p, double *R, double *c);
FM_API fm_status fm_set_params(fm_problem *p, const double *R, const double *c);
/* fm_set_params from device memory (d_R n_cams x 9, d_c n_cams x 3, FP64), asynchronous and
 * ordered on the caller's stream; R must be a rotation (not checked here). */
FM_API fm_status fm_set_params_device(fm_problem *p, const double *d_R, const double *d_c);

/*
 * Replace the per-point-pair weights w of the IRLS objective (n_pp FP32, input order; host,
 * or device when on_device is 1). FP16 storage keeps fp16_rn(w * s)/s with the power of
 * two s = 2^floor(log2(32768 * delta)); weights must be finite and in [0, 1/delta].
 */
FM_API fm_status fm_set_weights(fm_problem *p, const float *w, int32_t on_device);
/* Current weights as stored (n_pp FP32, input order, host). Synchronises. */
FM_API fm_status fm_get_weights(fm_problem *p, float *w);

/*
 * IRLS reweighting with outlier filtering at the current poses (Sec. "Epipolar Adjustment",
 * IRLS and filtering paragraphs): eps^ = x2^T E_n x1 for every point pair, then
 * w = 1/max(|eps^|, delta) if |eps^| <= tau, else w = 0. tau may be +inf (no filtering).
 * Writes the number of kept point pairs to *n_active (may be NULL). Synchronises.
 */
FM_API fm_status fm_irls_weights(fm_problem *p, double tau, int64_t *n_active);

/*
 * Objective and gradient at the current poses with the current weights (the objective
 * selected by opt.loss). loss: host FP64 scalar; grad: host FP64 n_cams x 6 (may be NULL).
 * Synchronises.
 */
FM_API fm_status fm_loss_grad(fm_problem *p, double *loss, double *grad);
/* Same, asynchronous, into device memory the caller owns (either pointer may be NULL). */
FM_API fm_status fm_loss_grad_device(fm_problem *p, double *d_loss, double *d_grad);

/* Residuals eps = x2^T E_n x1 at the current poses, FP32, input order, host. Synchronises. */
FM_API fm_status fm_residuals(fm_problem *p, float *eps);

/*
 * n_iters optimiser iterations, each: objective gradient at the current poses, one Adam
 * step on (phi_k, c_k) (FP32 moments), R_k <- Exp(phi_k) R_k with FP64 exponential map and
 * re-orthonormalisation, c_k updated in FP64 (with opt.refine_focal also rho_k, see the focal
 * section below). Only enqueues work; errors found on the device surface at the next
 * synchronising call.
 */
FM_API fm_status fm_step(fm_problem *p, int32_t n_iters);

/*
 * One IRLS round: fm_irls_weights(tau) followed by fm_step(n_iters), with the reweighting fused
 * into the first iteration's pass over the point pairs (the weights come from the residuals at
 * the round's starting poses, which that pass computes anyway): the same arithmetic, bit for
 * bit, and one read of the keypoints less. n_iters >= 1; IRLS objective only. Writes the
 * number of kept point pairs to *n_active if it is not NULL (then synchronises; otherwise
 * only enqueues work).
 */
FM_API fm_status fm_step_irls(fm_problem *p, double tau, int32_t n_iters, int64_t *n_active);

/* Objective value of the most recent iteration of fm_step (or fm_loss_grad). Synchronises. */
FM_API fm_status fm_last_loss(fm_problem *p, double *loss);

/*
 * One optimiser step with a gradient computed elsewhere (for example the sum of the gradients
 * of a problem's shards on several processes): grad is n_cams x 6 FP64, host, or device when
 * on_device is 1. Same update as one fm_step iteration. With a host gradient it synchronises;
 * with a device gradient it only enqueues, ordered after the work queued on the caller's stream
 * (so a collective that wrote the gradient on that stream needs no host wait), and a non-finite
 * device gradient surfaces as FM_EDEGENERATE at the next synchronising call.
 */
FM_API fm_status fm_apply_gradient(fm_problem *p, const double *grad, int32_t on_device);

/* Change the Adam step sizes used by later iterations (a learning-rate schedule). */
FM_API fm_status fm_set_learning_rate(fm_problem *p, double lr_rot, double lr_c);

/* Zero the Adam moments (poses and focal scales) and the step counter. */
FM_API fm_status fm_reset_optimizer(fm_problem *p);

/*
 * Optimiser state for checkpoint/resume: m and v (n_cams x 6, host FP64 arrays; the device
 * keeps them in FP32, so values round-trip exactly when they came from fm_get_state) and the
 * number of Adam steps taken. Resuming from a saved (poses, weights, state) gives bit-identical
 * trajectories because every reduction runs in a fixed order. (With focal refinement the scales
 * are saved and restored with fm_get_focal_scales / fm_set_focal_scales, which resets their
 * moments, so such a resume is not bit-identical.)
 */
FM_API fm_status fm_get_state(fm_problem *p, double *m, double *v, int64_t *step);
FM_API fm_status fm_set_state(fm_problem *p, const double *m, const double *v, int64_t step);

/* ---- focal refinement (last paragraph of Sec. "Epipolar Adjustment") ------------------------------
 * The focal lengths can be optimised with the poses by building them into the pair matrices,
 * which then are fundamental matrices. Keypoints are normalised with initial focal lengths f0_k;
 * a refined f_k rescales camera k's normalised coordinates by s_k = f0_k / f_k, so
 *   eps = x2^T F_n x1,  F_n = S_j E_n S_i,  S = diag(s, s, 1),
 * and with opt.refine_focal = 1 every optimiser step (fm_step, fm_step_quadratic) also takes an
 * Adam step on rho_k = log s_k (FP32 moments, FP64 rho; step size set below, default 1e-3).
 * With refine_focal = 0 the scales stay as set (1 by default) and results are identical to the
 * pose-only adjustment. fm_apply_gradient and fm_loss_grad_noalloc do not touch the scales.
 */
FM_API fm_status fm_set_focal_learning_rate(fm_problem *p, double lr);
/* Per-camera scales s_k (host FP64 n_cams). Synchronises. */
FM_API fm_status fm_get_focal_scales(fm_problem *p, double *s);
/* Set the scales (host FP64 n_cams, > 0) and reset their Adam moments. Synchronises. */
FM_API fm_status fm_set_focal_scales(fm_problem *p, const double *s);
/* d loss / d rho_k (host FP64 n_cams) of the last fm_loss_grad or optimiser step. Synchronises. */
FM_API fm_status fm_get_focal_gradient(fm_problem *p, double *g);

/* ---- focal-length vote (Sec. "Intrinsics Estimation", Eq. fastmap-focal-vote) -------------------
 * A 3x3 matrix is an essential matrix exactly when its two largest singular values are equal
 * (and the third is zero). For fundamental matrices F_i of image pairs and a candidate focal
 * length f, E_i = K_2^T F_i K_1 with K = diag(f, f, 1) (principal point at the image centre) and
 *   v(f) = sum_i exp((1 - lambda_1^(i) / lambda_2^(i)) / tau)
 * scores the candidate; the estimate is the candidate with the largest vote (chosen by the
 * caller from the votes). A pair side whose focal length is already known uses that value
 * instead of the candidate (the paper's procedure for several cameras).
 *   F: n_pairs x 9 FP64 host, row-major, x2^T F x1 = 0 with x in pixels from the image centre
 *      (each F is normalised to unit norm internally; the ratio is scale-free); finite, non-zero.
 *   f1_known, f2_known: n_pairs FP64 host known focal length of side 1 / side 2 of each pair,
 *      0 = use the candidate; either may be NULL (the candidate on that side for every pair).
 *   cand: n_cand FP64 host candidates (> 0); tau > 0 the temperature.
 *   votes: n_cand FP64 host output. elapsed_ms: if not NULL, the device time of the vote
 *      kernels (CUDA events on `stream`).
 * Numerics: FP32 per (candidate, pair) term (E, E^T E, four cyclic Jacobi sweeps for its
 * eigenvalues), per-block FP32 sums in a fixed order, FP64 total per candidate: bit-reproducible.
 * A pair with lambda_2 = 0 contributes 0. Allocates and frees its device buffers on `stream`
 * (a cudaStream_t, NULL = legacy default) and synchronises it. FM_EINVAL on bad arguments.
 */
FM_API fm_status fm_focal_vote(int32_t n_pairs, const double *F, const double *f1_known,
                               const double *f2_known, int32_t n_cand, const double *cand, double tau,
                               double *votes, float *elapsed_ms, void *stream);

/* ---- pre-aggregated quadratic form (Eq. epipolar-objective-l2 with the IRLS weights) ---------
 * With the weights held fixed, the objective of image pair n is quadratic in the 9 entries
 * e_n = vec(E_n) of its essential matrix, with eps = a^T e_n and a = vec(x2 x1^T). One pass over
 * the point pairs collects, per image pair, the weighted second moments anchored at the
 * essential matrix e0 of the poses of that pass:
 *   c0 = sum w eps0^2,  g0 = sum w eps0 a,  W = sum w a a^T   (FP32, 64 floats per pair)
 * and every later evaluation costs O(1) per image pair, independent of its point-pair count:
 *   objective = c0 + 2 d^T g0 + d^T W d,   d/de = 2 (g0 + W d),   d = e_n - e0.
 * Within FP32 rounding this is the IRLS objective of fm_loss_grad with the weights of the
 * pass; it goes stale when the weights change (fm_set_weights, fm_irls_weights,
 * fm_learned_weights), and the calls below then return FM_EINVAL. Needs opt.loss ==
 * FM_LOSS_IRLS. The device memory (about 224 B per 2048 point pairs and 320 B per image pair)
 * is allocated by the first call.
 */
/* Collect the form at the current poses with the current weights. Asynchronous. */
FM_API fm_status fm_preaggregate(fm_problem *p);
/* fm_irls_weights(tau) and fm_preaggregate in one pass over the point pairs (the weights are
 * written and, for FP16 storage, quantised before they enter the sums). Synchronises. */
FM_API fm_status fm_irls_preaggregate(fm_problem *p, double tau, int64_t *n_active);
/* Objective and gradient from the form, as fm_loss_grad (host outputs; grad may be NULL). */
FM_API fm_status fm_loss_grad_quadratic(fm_problem *p, double *loss, double *grad);
/* n_iters optimiser iterations of fm_step with the gradient taken from the form. Asynchronous. */
FM_API fm_status fm_step_quadratic(fm_problem *p, int32_t n_iters);

/* ---- learned inlier weights ------------------------------------------------------------------
 * The thesis has no learned component. These entry points implement the learned variant of the
 * reweighting step the benchmark describes: an MLP 8 -> 32 -> 32 -> 1 (ReLU, sigmoid) predicts
 * the probability p that a point pair is an inlier, and the IRLS weight becomes
 * w = p / max(|eps^|, delta) (0 where |eps^| > tau_cap). Features of a point pair, from the
 * residuals eps^ at the current poses (Sec. "Epipolar Adjustment" notation):
 *   0 log(|e|+1e-6) - log(tau)        1 log(|e|+1e-6) - mean over its image pair of log(|e|+1e-6)
 *   2 log(|e_prev|+1e-6) - log(|e|+1e-6)   (e_prev: residual at the previous reweighting call)
 *   3 match score                     4 fraction of its image pair's point pairs with |e| <= tau
 *   5 log(image-pair size)/10         6 round/10        7 log(|e_prev|+1e-6) - log(tau)
 * Numerics: features, weights and hidden activations in BF16, FP32 accumulation, FP32 biases.
 * Parameters: 1377 FP32 values, W1 (8 x 32, row k = input), b1 (32), W2 (32 x 32), b2 (32),
 * W3 (32), b3 (1).
 */
typedef struct fm_mlp fm_mlp;

FM_API int32_t fm_mlp_num_params(void);
/* Network from host FP32 parameters (copied); the device keeps FP32 masters and BF16 copies. */
FM_API fm_status fm_mlp_create(const float *params, fm_mlp **out);
FM_API void fm_mlp_destroy(fm_mlp *net);
FM_API fm_status fm_mlp_get_params(fm_mlp *net, float *params);
FM_API fm_status fm_mlp_set_params(fm_mlp *net, const float *params);
/* One Adam step (beta 0.9/0.999, eps 1e-8) on the mean binary cross-entropy of count samples:
 * d_features (count x 8 BF16, device), d_labels (count FP32 in {0,1}, device), count <= 65536.
 * Writes the batch loss before the step to *loss (host; may be NULL, then nothing syncs). */
FM_API fm_status fm_mlp_train_step(fm_mlp *net, const void *d_features, const float *d_labels,
                                   int32_t count, float lr, float *loss, void *stream);
/* Gradient of the mean cross-entropy (host, fm_mlp_num_params() floats) without a step. */
FM_API fm_status fm_mlp_gradient(fm_mlp *net, const void *d_features, const float *d_labels,
                                 int32_t count, float *grad, float *loss);
/* p for count feature rows (device BF16 in, device FP32 out), asynchronous on `stream`. */
FM_API fm_status fm_mlp_forward(fm_mlp *net, const void *d_features, int32_t count, float *d_p,
                                void *stream);
/* Match scores in [0, 1] (n_pp FP32, input order; host, or device when on_device is 1). */
FM_API fm_status fm_set_scores(fm_problem *p, const float *score, int32_t on_device);
/* Features of every point pair at the current poses (d_features: n_pp x 8 BF16, device, input
 * order), then remember the residuals as the history of the next call. Synchronises. */
FM_API fm_status fm_collect_features(fm_problem *p, double tau, int32_t round, void *d_features);
/* Learned reweighting (replaces fm_irls_weights): features -> MLP (tensor cores) -> weights;
 * n_active counts point pairs with |eps^| <= tau_cap. Synchronises. */
FM_API fm_status fm_learned_weights(fm_problem *p, const fm_mlp *net, double tau, double tau_cap,
                                    int32_t round, int64_t *n_active);
/* One learned IRLS round: fm_learned_weights(net, tau, tau_cap, round) followed by
 * fm_step(n_iters), with the learned reweighting (features, MLP, weights, history) fused into the
 * first iteration's pass over the point pairs: the same arithmetic, bit for bit, and one read of
 * the keypoints less. n_iters >= 1; IRLS objective only. Writes the number of point pairs with
 * |eps^| <= tau_cap to *n_active if it is not NULL (then synchronises; otherwise only enqueues). */
FM_API fm_status fm_step_learned(fm_problem *p, const fm_mlp *net, double tau, double tau_cap,
                                 int32_t round, int32_t n_iters, int64_t *n_active);
/* Forget the residual history (the next call uses the current residuals as history). */
FM_API fm_status fm_reset_history(fm_problem *p);

/* Wait for all queued work of the problem; returns FM_EDEGENERATE if the device flagged one. */
FM_API fm_status fm_synchronize(fm_problem *p);

/*
 * Kernel timing: when enabled, the library records CUDA events around every launch of each
 * pass over the point pairs listed below (fm_step and fm_step_irls then replay no graph, and a
 * timed pass is launched without overlap with its neighbours). fm_pass_time returns, for one
 * pass, the summed event time in milliseconds and the number of timed launches since enabling
 * (or since the last fm_pass_time of that pass), and resets both; fm_kernel_time is
 * fm_pass_time(FM_PASS_STREAM_LOSS). Synchronises.
 */
enum {
    FM_PASS_STREAM_LOSS = 0,      /* loss + adjoint pass of an iteration (fm_step, fm_step_irls) */
    FM_PASS_STREAM_REWEIGHT = 1,  /* the first pass of fm_step_irls (reweighting fused) */
    FM_PASS_QUAD_ACCUMULATE = 2,  /* the form pass of fm_preaggregate / fm_irls_preaggregate */
    FM_PASS_LEARNED_LOSS = 3,     /* the first pass of fm_step_learned (learned reweighting fused) */
    FM_PASS_PAIR_STATS = 4,       /* the image-pair statistics pass of fm_step_learned */
    FM_NUM_PASSES = 5
};
FM_API fm_status fm_enable_kernel_timing(fm_problem *p, int32_t enable);
FM_API fm_status fm_pass_time(fm_problem *p, int32_t pass, double *ms, int64_t *launches);
FM_API fm_status fm_kernel_time(fm_problem *p, double *ms, int64_t *launches);

/* ---- global translation (Sec. "Global Translation") ----------------------------------------------
 * With the world-to-camera rotations R_k fixed and a unit relative translation t_{i->j} per
 * image pair (in camera j's frame), the world direction from camera i's centre to camera j's
 * is o_{i->j} = -R_j^T t_{i->j}, and the centres o_k minimise
 *   L_t = (1/|P|) sum_n || (o_j - o_i)/||o_j - o_i|| - o_{i->j} ||_1
 * (Eq. fastmap-global-translation-objective). Several runs from random initial centres are
 * advanced together and merged (paragraph "Multiple initializations"): every run is centred
 * at the origin and scaled to unit mean norm, and each camera takes its centre from the run in
 * which the mean of its pairs' L1 terms is lowest (the lower run index on ties); the merged
 * centres continue as one run with fresh Adam state.
 * Numerics: centres and their update FP64; per-pair terms FP32 from the FP64 difference of the
 * two centres; subgradient of |x| at 0 is 0; per-camera sums FP32 in a fixed order; loss FP64.
 */
typedef struct fm_translation fm_translation;

typedef struct {
    double lr;          /* Adam step size (units of the centres; 1e-2) */
    double beta1;       /* 0.9 */
    double beta2;       /* 0.999 */
    double adam_eps;    /* 1e-12 */
    int32_t use_graph;  /* 1: replay CUDA graphs of chained iterations */
    int32_t reserved;
} fm_translation_options;

FM_API void fm_translation_default_options(fm_translation_options *opt);
/*
 * n_cams >= 2 cameras with rotations R (host FP64 n_cams x 9, row-major, world-to-camera);
 * n_pairs >= 1 image pairs (cam_i, cam_j host int32, distinct, in range) with unit relative
 * translations t_rel (host FP64 n_pairs x 3, |t| = 1 within 1e-6); n_runs (1..65535) initial
 * centre sets o_init (host FP64 n_runs x n_cams x 3, drawn by the caller). Everything is
 * copied; work runs on a private stream ordered after and before `stream` (a cudaStream_t).
 * FM_EINVAL on bad arguments.
 */
FM_API fm_status fm_translation_create(int32_t n_cams, const double *R, int32_t n_pairs,
                                       const int32_t *cam_i, const int32_t *cam_j,
                                       const double *t_rel, int32_t n_runs, const double *o_init,
                                       const fm_translation_options *opt, void *stream,
                                       fm_translation **out);
FM_API void fm_translation_destroy(fm_translation *tp);
/* Number of runs currently advanced (n_runs, or 1 after fm_translation_merge). */
FM_API int32_t fm_translation_num_runs(const fm_translation *tp);
/* Per run (host outputs): loss[runs]; grad[runs x n_cams x 3] and cam_loss[runs x n_cams]
 * (mean L1 term of each camera's pairs, 0 for a camera in no pair) may be NULL. Synchronises;
 * FM_EDEGENERATE if two cameras of a pair share a centre. */
FM_API fm_status fm_translation_loss_grad(fm_translation *tp, double *loss, double *grad,
                                          double *cam_loss);
/* n_iters Adam iterations of every run. Asynchronous. */
FM_API fm_status fm_translation_step(fm_translation *tp, int32_t n_iters);
/* Merge the runs into one (see above); the merged centres are normalised. Synchronises. */
FM_API fm_status fm_translation_merge(fm_translation *tp);
FM_API fm_status fm_translation_set_learning_rate(fm_translation *tp, double lr);
/* Centres of the current runs (host FP64 runs x n_cams x 3). Synchronises. */
FM_API fm_status fm_translation_get_centres(fm_translation *tp, double *o);
/* Replace the centres of the current runs (host, same layout) and reset the Adam state. */
FM_API fm_status fm_translation_set_centres(fm_translation *tp, const double *o);

/* ---- global rotation (Sec. "Global Rotation") -----------------------------------------------------
 * World-to-camera rotations R_k from relative rotations R_{i->j} of the image pairs, minimising
 *   L_R = (1/|P|) sum_n d(R_j, R_{i->j} R_i),   d(R, R') = arccos((tr(R^T R') - 1)/2)
 * (Eq. fastmap-rotation-objective) with every R_k in the 6D representation (a1, a2): columns
 * b1 = a1/|a1|, b2 = the normalised part of a2 orthogonal to b1, b3 = b1 x b2.
 * Initialisation (paragraph "Initialization details", column-wise least squares): column 1
 * from min sum ||x_j - R_{i->j} x_i||^2, column 2 from min (1/|P|) sum ||y_j - R_{i->j} y_i||^2
 * + (1/N) sum (x_k^T y_k)^2, each with camera 0's column held at e1 / e2 (gauge: R_0 = I), solved
 * by preconditioned conjugate gradients on the GPU; columns normalised, column 2 orthogonalised
 * to column 1, column 3 their cross product. All FP64; for the gradient the arccos argument is
 * clamped to 1 - 1e-12 (finite at d = 0).
 */
typedef struct fm_rotation fm_rotation;

typedef struct {
    double lr;            /* Adam step size on the 6D parameters (1e-3) */
    double beta1;         /* 0.9 */
    double beta2;         /* 0.999 */
    double adam_eps;      /* 1e-12 */
    double cg_tol;        /* stop when the preconditioned residual norm falls by this factor (1e-9) */
    int32_t cg_max_iters; /* per column system (20000) */
    int32_t use_graph;    /* 1: replay CUDA graphs of chained iterations */
} fm_rotation_options;

FM_API void fm_rotation_default_options(fm_rotation_options *opt);
/*
 * n_cams >= 2, n_pairs >= 1 image pairs (cam_i, cam_j host int32, distinct, in range) forming a
 * connected graph, relative rotations R_rel (host FP64 n_pairs x 9, row-major, orthonormal with
 * det +1 within 1e-6, mapping camera i's frame to camera j's). Copied. FM_EINVAL otherwise.
 */
FM_API fm_status fm_rotation_create(int32_t n_cams, int32_t n_pairs, const int32_t *cam_i,
                                    const int32_t *cam_j, const double *R_rel,
                                    const fm_rotation_options *opt, void *stream,
                                    fm_rotation **out);
FM_API void fm_rotation_destroy(fm_rotation *rp);
/* The column-wise initialisation; resets the Adam state. Writes the total number of conjugate-
 * gradient iterations and the worse relative residual of the two systems (either may be NULL).
 * Synchronises; FM_EDEGENERATE if a solved column vanishes. */
FM_API fm_status fm_rotation_initialize(fm_rotation *rp, int32_t *cg_iters, double *cg_residual);
/* L_R (host scalar) and its gradient with respect to the 6D parameters (host n_cams x 6,
 * may be NULL). Synchronises. */
FM_API fm_status fm_rotation_loss_grad(fm_rotation *rp, double *loss, double *grad6);
/* n_iters Adam iterations on the 6D parameters. Asynchronous. */
FM_API fm_status fm_rotation_step(fm_rotation *rp, int32_t n_iters);
FM_API fm_status fm_rotation_set_learning_rate(fm_rotation *rp, double lr);
/* Rotations (host FP64 n_cams x 9) / 6D parameters (n_cams x 6) of the current state. */
FM_API fm_status fm_rotation_get_rotations(fm_rotation *rp, double *R);
FM_API fm_status fm_rotation_get_params(fm_rotation *rp, double *a6);
/* Replace the state by rotations (their first two columns become the parameters) or by 6D
 * parameters; resets the Adam state. */
FM_API fm_status fm_rotation_set_rotations(fm_rotation *rp, const double *R);
FM_API fm_status fm_rotation_set_params(fm_rotation *rp, const double *a6);

/*
 * Loss and gradient without any device allocation, for callers that cannot call cudaMalloc:
 * code whose device memory is owned by another memory manager (a framework's caching
 * allocator, a fixed arena), or a loop that cannot afford cudaMalloc's implicit device
 * synchronisation. The paper has no counterpart; this is an interface convenience that
 * computes the same quantities as fm_loss_grad.
 *
 * All pointers are device pointers the caller owns:
 *   d_R (n_cams x 9 FP64) rotations and d_c (n_cams x 3 FP64) camera centres c = -R^T t;
 *   d_cam_i, d_cam_j (n_pairs int32) image pairs; d_pair_off (n_pairs + 1 int32) offsets of
 *   each pair's point pairs, rising strictly from 0 to n_pp (point pairs sorted by pair);
 *   d_kp (n_pp x 4 FP32, 16-byte aligned) rows (x1, y1, x2, y2) in normalized coordinates;
 *   d_w (n_pp FP32) IRLS weights, or NULL for all ones (ignored when loss is FM_LOSS_L1);
 *   outputs d_loss (1 FP64) and d_grad (n_cams x 6 FP64, ordered as for fm_loss_grad).
 * Limits: 2 <= n_cams <= 4096, 1 <= n_pairs <= 32768, n_pairs <= n_pp <= 2^26; larger
 * problems return FM_EINVAL (use fm_create_problem for them).
 *
 * Intermediates live in one fixed 10.9 MiB __device__ array of the library, held on every
 * device that loads it until the process exits. The first call on a device looks up the
 * array's device address with that device current; make that first call before any stream
 * capture. Every call shares the array, so calls that overlap on the GPU (other streams,
 * other host threads on the same device) race and must be serialised by the caller.
 * Runs on `stream` (a cudaStream_t, NULL = legacy default) and synchronises it before
 * returning. Invalid device data returns FM_EINVAL with nothing written to d_loss/d_grad
 * that the caller may rely on: offsets not rising, a camera index out of range, cam_i ==
 * cam_j, a keypoint coordinate that is not finite or exceeds 8 in magnitude, a weight that is
 * negative or not finite (the same input rules as fm_create_problem and fm_set_weights; no
 * upper bound is imposed on the weights here, since no IRLS floor delta is given). A
 * zero-length relative translation or a non-finite result returns FM_EDEGENERATE.
 * Cost: besides the pass over the point pairs, O(n_pairs + n_cams) work to build each
 * camera's list of image pairs plus O(d_k^2) for camera k of degree d_k to put its list into
 * pair order.
 */
FM_API fm_status fm_loss_grad_noalloc(int32_t n_cams, const double *d_R, const double *d_c,
                                      int32_t n_pairs, const int32_t *d_cam_i,
                                      const int32_t *d_cam_j, const int32_t *d_pair_off,
                                      int64_t n_pp, const float *d_kp, const float *d_w,
                                      int32_t loss, double *d_loss, double *d_grad, void *stream);

FM_API const char *fm_status_string(fm_status s);
FM_API const char *fm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FASTMAP_H_ */
