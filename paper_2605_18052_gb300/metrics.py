"""Pose-accuracy metrics (evaluation only, FP64 on the host).

Rotation error: geodesic distance d(R, R') = arccos((tr(R^T R') - 1)/2) (Sec. "Global
Rotation"), per camera, after the global rotation that best aligns the estimate with the
reference (the objective is invariant to a world rotation). Translation error: angle between
estimated and reference unit relative translations of each image pair.
"""
from __future__ import annotations

import numpy as np


def _nearest_rotation(M: np.ndarray) -> np.ndarray:
    U, _, Vt = np.linalg.svd(M)
    D = np.diag([1.0, 1.0, np.sign(np.linalg.det(U @ Vt))])
    return U @ D @ Vt


def rotation_error_deg(R_est, R_ref) -> np.ndarray:
    Re = np.asarray(R_est, dtype=np.float64).reshape(-1, 3, 3)
    Rr = np.asarray(R_ref, dtype=np.float64).reshape(-1, 3, 3)
    Q = _nearest_rotation(np.einsum("nba,nbc->ac", Re, Rr))
    tr = np.einsum("nab,nab->n", Rr, Re @ Q)
    return np.degrees(np.arccos(np.clip((tr - 1.0) / 2.0, -1.0, 1.0)))


def translation_error_deg(R_est, t_est, R_ref, t_ref, cam_i, cam_j) -> np.ndarray:
    def unit_rel(R, t):
        R = np.asarray(R, dtype=np.float64).reshape(-1, 3, 3)
        t = np.asarray(t, dtype=np.float64).reshape(-1, 3)
        Rn = np.einsum("nab,ncb->nac", R[cam_j], R[cam_i])
        tn = t[cam_j] - np.einsum("nab,nb->na", Rn, t[cam_i])
        return tn / np.linalg.norm(tn, axis=1, keepdims=True)
    a, b = unit_rel(R_est, t_est), unit_rel(R_ref, t_ref)
    return np.degrees(np.arccos(np.clip((a * b).sum(1), -1.0, 1.0)))
