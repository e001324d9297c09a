"""Oracle of focal refinement inside the epipolar adjustment (TEST INFRASTRUCTURE ONLY).

The last paragraph of Sec. "Epipolar Adjustment" notes that the focal lengths can be optimised
together with the poses by building them into the essential matrices (which then are
fundamental matrices). With keypoints normalised by a focal length f0_k (principal point at
the centre, Sec. "Camera Assumptions"), a refined focal length f_k rescales camera k's
normalised coordinates by s_k = f0_k / f_k:

    eps = (S_j x2)^T E_n (S_i x1) = x2^T (S_j E_n S_i) x1,   S = diag(s, s, 1),

so F_n = S_j E_n S_i. The optimised per-camera variable is rho_k = log s_k (positive scale,
step sizes relative). Readings: the loss is the IRLS objective (1/Z) sum w eps^2 with the
weights held fixed, as for the poses; rho starts at 0 (the initial focal lengths).

Independent of the per-point-pair C loops in epipolar.c: the objective at scales s is the
plain objective on rescaled keypoints, and the scale gradient is summed here per point pair
in NumPy (FP64).
"""
from __future__ import annotations

import numpy as np

from . import Problem, essential
from . import loss_grad as _pose_loss_grad


def scaled_problem(prob: Problem, s) -> Problem:
    """The same point pairs with camera i's keypoints scaled by s_i (x1) and camera j's by s_j (x2)."""
    s = np.asarray(s, np.float64)
    si = s[prob.cam_i][prob.pair_id][:, None]
    sj = s[prob.cam_j][prob.pair_id][:, None]
    return Problem(prob.n_cams, prob.cam_i, prob.cam_j, prob.pair_id, prob.x1 * si, prob.x2 * sj)


def fundamental(prob: Problem, R, c, s) -> np.ndarray:
    """F_n = S_j E_n S_i, (B, 3, 3)."""
    s = np.asarray(s, np.float64)
    E = essential(prob, R, c)
    sig = np.stack([s, s, np.ones_like(s)], axis=1)
    return sig[prob.cam_j][:, :, None] * E * sig[prob.cam_i][:, None, :]


def loss_grad(prob: Problem, R, c, rho, w=None):
    """IRLS objective at scales s = exp(rho): (loss, pose gradient (N, 6), d loss / d rho (N,))."""
    s = np.exp(np.asarray(rho, np.float64))
    sp = scaled_problem(prob, s)
    loss, g_pose = _pose_loss_grad(sp, R, c, w)
    # d eps / d s_i = (S_j x2)^T E (x1, y1, 0);  d eps / d s_j = (x2, y2, 0)^T E (S_i x1)
    E = essential(prob, R, c)[prob.pair_id]
    o1 = np.concatenate([sp.x1, np.ones((prob.n_pp, 1))], 1)
    o2 = np.concatenate([sp.x2, np.ones((prob.n_pp, 1))], 1)
    eps = np.einsum("pa,pab,pb->p", o2, E, o1)
    wv = np.ones(prob.n_pp) if w is None else np.asarray(w, np.float64)
    u1 = np.concatenate([prob.x1, np.zeros((prob.n_pp, 1))], 1)
    u2 = np.concatenate([prob.x2, np.zeros((prob.n_pp, 1))], 1)
    de_dsi = np.einsum("pa,pab,pb->p", o2, E, u1)
    de_dsj = np.einsum("pa,pab,pb->p", u2, E, o1)
    k = 2.0 * wv * eps / prob.n_pp
    g_s = np.bincount(prob.cam_i[prob.pair_id], weights=k * de_dsi, minlength=prob.n_cams) \
        + np.bincount(prob.cam_j[prob.pair_id], weights=k * de_dsj, minlength=prob.n_cams)
    return loss, g_pose, g_s * s


def residuals(prob: Problem, R, c, rho) -> np.ndarray:
    """eps = x2^T F_n x1 at scales exp(rho), input order."""
    F = fundamental(prob, R, c, np.exp(np.asarray(rho, np.float64)))[prob.pair_id]
    o1 = np.concatenate([prob.x1, np.ones((prob.n_pp, 1))], 1)
    o2 = np.concatenate([prob.x2, np.ones((prob.n_pp, 1))], 1)
    return np.einsum("pa,pab,pb->p", o2, F, o1)
