// Internal layout and kernel declarations of libfastmap (not part of the C ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "fastmap.h"

namespace fm {

// ---- work decomposition --------------------------------------------------------------------
// The sorted point-pair array is cut into warp ranges of WR point pairs; each warp streams one
// range. A range that meets k image pairs produces k partial sums ("slots"). Slot (n, r) of
// pair n and range r lives at index n + r: along the sorted array every range or pair boundary
// advances n or r, so n + r is unique per non-empty intersection and there are at most
// n_pairs + n_ranges slots.
constexpr int WR = 2048;           // point pairs per warp range
constexpr int CTA_WARPS = 8;       // warps per CTA of the streaming kernels
constexpr int SLOT = 12;           // floats per slot: G'(9), loss, 2 pad (48 B)
constexpr int GEO = 40;            // floats per pair geometry record (160 B)
constexpr int CAMREC = 16;         // floats per camera record
constexpr int PG = 16;             // floats per pair gradient record
constexpr float COORD_LIMIT = 8.0f;  // |normalized coordinate| bound (fixed-point centroids)
constexpr int FIXED_SHIFT = 32;    // centroid sums use trunc(x * 2^32) in int64

// geometry record of pair n (written by pair_setup, read by the streaming and combine kernels)
//   [0..8]  E'_n = T_j^T E_n T_i (centroid-folded essential matrix, row-major)
//   [9..17] R_n = R_j R_i^T
//   [18..20] t_n = R_j (c_i - c_j)
//   [21] 1/|t_n|, [22..23] centroid of image i, [33..34] centroid of image j
//   [24..32] R_j (the second camera's rotation, so the per-camera step never reads another
//            camera's record while that record is being updated)
// camera record k (written by the per-camera step kernel)
//   [0..8] R_k (FP32), [9..11] c_k high part, [12..14] c_k low part (c = hi + lo), [15] 0
// pair gradient record n: [0..2] g_phi_i, [3..5] g_c_i, [6..8] g_phi_j, [9..11] g_c_j, [12] loss

enum StreamMode { MODE_LOSS_IRLS = 0, MODE_LOSS_L1 = 1 };

enum ErrBits : unsigned {
    ERR_DEGENERATE = 1u,   // |t_n| == 0 or non-finite pose data
    ERR_NONFINITE = 2u,    // non-finite loss or gradient
    ERR_PAIR_RANGE = 4u,   // pair_id out of range
    ERR_COORD = 8u,        // non-finite or too large keypoint coordinate
    ERR_EMPTY_PAIR = 16u,  // image pair without point pairs
    ERR_UNSORTED = 32u,    // input not grouped by pair (not an error: triggers the sort)
    ERR_WEIGHT = 64u,      // weight outside [0, 1/delta] or non-finite
};

struct DevProblem {
    int n_cams, n_pairs;
    int64_t n_pp;
    int64_t n_pad;          // allocated point pairs (multiple of WR)
    int n_ranges;
    int storage, loss;
    double delta;
    double z;               // Z of the objective (n_pp, or the total over all shards)
    float w_scale;          // FP16 weight scale s (1 for FP32 storage)
    // poses (FP64) and Adam moments (FP32)
    double *R, *c, *hyper;   // hyper: lr_rot, lr_c, beta1, beta2, eps, lr_focal, tau (fused reweighting)
    // focal refinement: per camera rho = log(f0 / f), the scale of its normalised keypoints
    // is exp(rho) (1 when rho is null); Adam moments of rho and its last gradient
    double *rho, *grad_rho;
    float *rho_m, *rho_v;
    int refine_focal;
    float *m, *v;
    long long *step;
    double *cam_loss;        // per-camera loss shares of the last optimiser step (FP64)
    float *cam;             // camera records
    float2 *cen;            // per-camera centroids (zeros for FP32 storage)
    int *cam_i, *cam_j, *pair_off, *range_pair;
    int *cam_off, *cam_ent;
    void *kp;               // float4[n_pad] or uint2[n_pad]
    void *w;                // float[n_pad] or __half[n_pad]
    int *perm;              // sorted position -> input index, or nullptr (identity)
    float *geo, *slots, *pair_grad;
    double *grad, *loss_out;
    unsigned *err;
    unsigned long long *counter;
    float *fbuf;            // n_pad floats of scratch (residual export)
    // learned inlier weights
    __half *score;          // per point pair: matcher confidence (0.5 until set)
    __half *le_hist;        // per point pair: log(|eps| + 1e-6) at the previous reweighting
    float *pstat;           // per pair: mean log residual, inlier fraction, log(count)/10, 0
    // pre-aggregated quadratic form (Eq. epipolar-objective-l2), anchored at the reweighting
    // point: per (pair, range) partials and per pair records
    float *qslots;          // (n_pairs + n_ranges) x QSLOT
    float *quad;            // n_pairs x QREC: c0, g0(9), M(36), e0(9), pad
    float *cam_alt;         // n_cams x CAMREC: second camera-record buffer of the fused step
    unsigned *pair_cnt;     // per pair: cameras updated by camera steps with the geometry phase
};

// c0 = sum w eps0^2, g0 = sum w eps0 a (9), M = the 36 distinct entries of W = sum w a a^T
// (a = vec(o2 o1^T); W = (o2 o2^T) (x) (o1 o1^T) summed), e0 = vec(E'_n) at the anchor
constexpr int QSUMS = 46;
constexpr int QSLOT = 48;
constexpr int QREC = 56;

// ---- learned inlier-weight MLP (fm_mlp.cu) ------------------------------------------------------
constexpr int MLP_IN = 8;
constexpr int MLP_H = 32;
constexpr int MLP_OFF_W1 = 0;                                // W1[k][n], 8 x 32
constexpr int MLP_OFF_B1 = MLP_OFF_W1 + MLP_IN * MLP_H;      // 32
constexpr int MLP_OFF_W2 = MLP_OFF_B1 + MLP_H;               // W2[k][n], 32 x 32
constexpr int MLP_OFF_B2 = MLP_OFF_W2 + MLP_H * MLP_H;       // 32
constexpr int MLP_OFF_W3 = MLP_OFF_B2 + MLP_H;               // W3[k], 32
constexpr int MLP_OFF_B3 = MLP_OFF_W3 + MLP_H;               // 1
constexpr int MLP_NPARAM = MLP_OFF_B3 + 1;                   // 1377
constexpr float LOG_FLOOR = 1e-6f;

// quadratic form: accumulate at the current poses and weights (range partials), combine them
// into per-pair records; per-iteration evaluation
void launch_quad_accumulate(const DevProblem &d, float tau, cudaStream_t s);
void launch_quad_combine(const DevProblem &d, cudaStream_t s);
// one fused step on the form: iteration `it` of a chain (Adam step count *d.step + 1 + it),
// camera records read from cam_src and written to cam_dst (apply = false: gradient and loss only)
void launch_quad_step(const DevProblem &d, int it, const float *cam_src, float *cam_dst, bool apply,
                      cudaStream_t s, bool pdl);

// pair statistics of the current residuals (pstat), then features -> MLP -> weights, or the
// features themselves (input order) for training
void launch_pair_stats(const DevProblem &d, float tau, cudaStream_t s);
void launch_learned_weights(const DevProblem &d, const float *mlp_master, const __nv_bfloat16 *mlp_bf16,
                            float tau, float tau_cap, int round, int hist_valid, cudaStream_t s);
void launch_collect_features(const DevProblem &d, float tau, int round, int hist_valid,
                             __nv_bfloat16 *feat_input_order, cudaStream_t s);
// the learned reweighting fused with the loss + adjoint pass (slots, weights, history, kept count)
void launch_learned_loss(const DevProblem &d, const float *mlp_master, const __nv_bfloat16 *mlp_bf16, float tau,
                         float tau_cap, int round, int hist_valid, cudaStream_t s, bool pdl);

// ---- kernels launched by the API layer (fm_kernels.cu) ----------------------------------------
void launch_cam_prep(const DevProblem &d, cudaStream_t s);
// pdl: launch with programmatic stream serialisation (overlaps the predecessor's tail)
// after_step: the previous kernel was an optimiser camera step whose loss total and step
// count this launch finishes
void launch_pair_setup(const DevProblem &d, cudaStream_t s, bool pdl = false, bool after_step = false);
// loss total of the last camera step (and the step count after an optimiser step)
void launch_finalize(const DevProblem &d, bool count_step, cudaStream_t s, bool pdl = false);
// the same with `count` steps added, and camera records copied back from copy_src if not null
void launch_finalize_n(const DevProblem &d, int count, const float *copy_src, cudaStream_t s, bool pdl);
int camera_step_blocks(const DevProblem &d);
// factors applied to the raw sums of the loss (Sum w eps^2 or Sum |eps|, weights stored as
// w * s): gradient 2/(Z s) and loss 1/(Z s) for IRLS, 1/Z for L1
void loss_scales(const DevProblem &d, float &gscale, float &lscale);
// streaming loss + adjoint: per (image pair, CTA range) partial sums in d.slots; after_step:
// the previous kernel was an optimiser camera step whose loss total and step count this
// launch finishes
void launch_stream_loss(const DevProblem &d, cudaStream_t s, bool pdl = false, bool after_step = false);
// the same pass fused with the IRLS reweighting at threshold d.hyper[6]; kept count in d.counter
void launch_stream_reweight(const DevProblem &d, cudaStream_t s, bool pdl = false);
void launch_combine(const DevProblem &d, cudaStream_t s);
void launch_gather(const DevProblem &d, bool count_step, cudaStream_t s);
// fused per-camera step: combine this camera's pair partials, chain rule, FP64 sum, Adam,
// exponential map, camera record; the last block sums the loss and advances the step count
// Adam step of every camera with the gradient in d.grad (FP64, n_cams x 6); advances the step
void launch_apply_gradient(const DevProblem &d, cudaStream_t s);
// apply = false computes the gradient and loss only (no Adam step, no step count); next_geo
// (with apply, when d.pair_cnt is allocated): also the geometry records of the new poses
void launch_camera_step(const DevProblem &d, bool apply, cudaStream_t s, bool pdl = false, bool next_geo = false);
void launch_irls_weights(const DevProblem &d, float tau, cudaStream_t s);
void launch_residuals(const DevProblem &d, float *out_sorted, cudaStream_t s);

// ---- layout kernels (fm_layout.cu) -------------------------------------------------------------
// Validate pair ids / coordinates and detect whether the input is grouped by pair.
void launch_validate(const int *pair_id, const float2 *x1, const float2 *x2, int64_t n_pp,
                     int n_pairs, unsigned *err, cudaStream_t s);
// Stable sort of point pairs by pair id: writes perm (sorted -> input) and sorted keys.
cudaError_t sort_by_pair(const int *pair_id, int64_t n_pp, int n_pairs, int *keys_out,
                         int *perm_out, cudaStream_t s);
void launch_pair_offsets(const int *sorted_keys, int64_t n_pp, int n_pairs, int *pair_off,
                         unsigned *err, cudaStream_t s);
void launch_range_pairs(const int *pair_off, int n_pairs, int n_ranges, int *range_pair,
                        cudaStream_t s);
// FP16 storage: per-image centroids into d.cen (needs d.cam_off/cam_ent/pair_off/range_pair/perm);
// `sums` is scratch for 2 * n_cams int64.
void launch_centroids(const DevProblem &d, const int *sorted_keys, const float2 *x1,
                      const float2 *x2, unsigned long long *sums, cudaStream_t s);
void launch_pack(const DevProblem &d, const int *sorted_keys, const float2 *x1, const float2 *x2,
                 cudaStream_t s);
void launch_fill_weights(const DevProblem &d, float value, cudaStream_t s);
void launch_set_weights(const DevProblem &d, const float *w_input_order, cudaStream_t s);
void launch_get_weights(const DevProblem &d, float *w_input_order, cudaStream_t s);
void launch_unpermute(const DevProblem &d, const float *sorted, float *input_order,
                      cudaStream_t s);
void launch_fill_half(__half *p, int64_t n, float value, cudaStream_t s);
// match scores in input order -> d.score (sorted order, FP16); values outside [0, 1] -> ERR_WEIGHT
void launch_set_scores(const DevProblem &d, const float *score_input_order, cudaStream_t s);

}  // namespace fm
