"""Oracle of the focal-length vote (TEST INFRASTRUCTURE ONLY).

Sec. "Intrinsics Estimation", paragraph "Focal Length Estimation": a 3x3 matrix is an
essential matrix exactly when its two largest singular values are equal and the third is zero.
For a fundamental matrix F of an image pair and the intrinsics K of a candidate focal length,
E = K^T F K should therefore have lambda_1 / lambda_2 = 1 (lambda_1 >= lambda_2 >= lambda_3 its
singular values), and a candidate f is scored over the image pairs i by

    v(f) = sum_i exp((1 - lambda_1^(i) / lambda_2^(i)) / tau)          (Eq. fastmap-focal-vote)

with a temperature tau; the candidate with the largest vote is the estimate.

Readings (the passage fixes no more):
  * K = diag(f, f, 1): the principal point is the image centre (Sec. "Camera Assumptions"), so
    F acts on keypoints in pixels measured from the image centre.
  * Several cameras: for the camera being estimated, an image pair uses the candidate f on the
    side(s) that belong to that camera and the already known focal length on the other side:
    E = K_2^T F K_1 with F mapping image-1 keypoints to epipolar lines in image 2
    (x2^T F x1 = 0). Known focal lengths are passed per pair and side; 0 marks "the candidate".
  * A pair whose lambda_2 is zero (F of rank below 2) contributes exp(-inf) = 0.

Plain FP64 NumPy; the singular values come from the library SVD (numpy.linalg.svd).
"""
from __future__ import annotations

import numpy as np


def essential_from_fundamental(F, f1, f2):
    """E = diag(f2, f2, 1) F diag(f1, f1, 1) for every pair; F (B, 3, 3), f1 and f2 (B,)."""
    F = np.asarray(F, np.float64)
    s1 = np.stack([f1, f1, np.ones_like(f1)], axis=1)
    s2 = np.stack([f2, f2, np.ones_like(f2)], axis=1)
    return s2[:, :, None] * F * s1[:, None, :]


def singular_ratio(E):
    """lambda_1 / lambda_2 of every 3x3 matrix (inf where lambda_2 is zero)."""
    sv = np.linalg.svd(np.asarray(E, np.float64), compute_uv=False)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = sv[:, 0] / sv[:, 1]
    return np.where(sv[:, 1] > 0, r, np.inf)


def votes(F, candidates, tau, f1_known=None, f2_known=None):
    """v(f) for every candidate f (Eq. fastmap-focal-vote), FP64 array (n_candidates,).

    F: (B, 3, 3) fundamental matrices (x2^T F x1 = 0, pixels from the image centre).
    f1_known, f2_known: (B,) known focal lengths of side 1 / side 2 of each pair, 0 where that
    side uses the candidate (default: every side uses it, the single-camera case).
    """
    F = np.asarray(F, np.float64)
    B = F.shape[0]
    k1 = np.zeros(B) if f1_known is None else np.asarray(f1_known, np.float64)
    k2 = np.zeros(B) if f2_known is None else np.asarray(f2_known, np.float64)
    out = np.empty(len(candidates))
    for c, f in enumerate(np.asarray(candidates, np.float64)):
        f1 = np.where(k1 > 0, k1, f)
        f2 = np.where(k2 > 0, k2, f)
        r = singular_ratio(essential_from_fundamental(F, f1, f2))
        out[c] = np.exp((1.0 - r) / tau).sum()
    return out


def estimate(F, candidates, tau, f1_known=None, f2_known=None):
    """The candidate with the largest vote (the first one on ties) and all votes."""
    v = votes(F, candidates, tau, f1_known, f2_known)
    return float(np.asarray(candidates, np.float64)[int(np.argmax(v))]), v


def fundamental_from_poses(R, C, cam_i, cam_j, f):
    """Fundamental matrices of image pairs (i, j) from world-to-camera rotations R (N, 3, 3),
    centres C (N, 3) and per-camera focal lengths f (N,): F = K_j^-T [t]_x R_n K_i^-1 with
    R_n = R_j R_i^T, t = R_j (c_i - c_j) (a test-input helper: true two-view geometry)."""
    R = np.asarray(R, np.float64)
    C = np.asarray(C, np.float64)
    f = np.asarray(f, np.float64)
    Rn = np.einsum("nab,ncb->nac", R[cam_j], R[cam_i])
    t = np.einsum("nab,nb->na", R[cam_j], C[cam_i] - C[cam_j])
    tx = np.zeros((len(cam_i), 3, 3))
    tx[:, 0, 1], tx[:, 0, 2] = -t[:, 2], t[:, 1]
    tx[:, 1, 0], tx[:, 1, 2] = t[:, 2], -t[:, 0]
    tx[:, 2, 0], tx[:, 2, 1] = -t[:, 1], t[:, 0]
    E = tx @ Rn
    inv_i = np.stack([1.0 / f[cam_i], 1.0 / f[cam_i], np.ones(len(cam_i))], axis=1)
    inv_j = np.stack([1.0 / f[cam_j], 1.0 / f[cam_j], np.ones(len(cam_j))], axis=1)
    return inv_j[:, :, None] * E * inv_i[:, None, :]
