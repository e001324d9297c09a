"""Oracle of the global translation stage (TEST INFRASTRUCTURE ONLY).

Sec. "Global Translation" of the FastMap chapter: with the world-to-camera rotations R_k fixed
and a unit relative translation t_{i->j} per image pair, the world-frame direction from the
centre of camera i to that of camera j is o_{i->j} = -R_j^T t_{i->j} (the equation before
Eq. fastmap-global-translation-objective). The camera centres o_k minimise

    L_t = (1/|P|) sum_{(i,j) in P} || (o_j - o_i) / ||o_j - o_i||_2  -  o_{i->j} ||_1

(Eq. fastmap-global-translation-objective) by first-order steps from random initial centres.
Several independent runs are merged (paragraph "Multiple initializations"): every solution is
centred at the origin and scaled to unit mean norm, and each camera takes its centre from the
run in which its mean per-pair loss is lowest; the merged centres start a final run.

Plain FP64 NumPy, for checking the CUDA kernels. Readings where the thesis is silent: the
optimiser is Adam (the same first-order method as the epipolar adjustment) with a constant step
size; the subgradient of |x| at 0 is 0; a camera's loss for the merge is the mean of the L1 terms
of the image pairs it belongs to (0 for a camera in no pair); ties in the merge go to the lower
run index. Random initial centres are inputs (drawn by the caller).
"""
from __future__ import annotations

import numpy as np


def relative_directions(R, t_rel, cam_j) -> np.ndarray:
    """o_{i->j} = -R_j^T t_{i->j} for every pair, (B, 3)."""
    R = np.asarray(R, np.float64).reshape(-1, 3, 3)
    t = np.asarray(t_rel, np.float64).reshape(-1, 3)
    return -np.einsum("nba,nb->na", R[np.asarray(cam_j)], t)


def pair_terms(o, cam_i, cam_j, o_ij):
    """Per pair: the L1 term ||u/|u| - o_ij||_1 and its gradient with respect to u = o_j - o_i
    (the L1 subgradient sign(r), projected orthogonally to u and divided by |u|)."""
    o = np.asarray(o, np.float64).reshape(-1, 3)
    u = o[np.asarray(cam_j)] - o[np.asarray(cam_i)]
    nrm = np.linalg.norm(u, axis=1)
    if np.any(nrm == 0.0):
        raise FloatingPointError("two cameras at the same centre")
    uh = u / nrm[:, None]
    r = uh - np.asarray(o_ij, np.float64).reshape(-1, 3)
    term = np.abs(r).sum(1)
    s = np.sign(r)
    g_u = (s - uh * (uh * s).sum(1, keepdims=True)) / nrm[:, None]
    return term, g_u


def loss_grad(o, cam_i, cam_j, o_ij):
    """L_t and its gradient with respect to the centres, (N, 3)."""
    o = np.asarray(o, np.float64).reshape(-1, 3)
    term, g_u = pair_terms(o, cam_i, cam_j, o_ij)
    B = term.shape[0]
    g = np.zeros_like(o)
    np.add.at(g, np.asarray(cam_j), g_u / B)
    np.add.at(g, np.asarray(cam_i), -g_u / B)
    return float(term.sum() / B), g


def camera_losses(o, cam_i, cam_j, o_ij) -> np.ndarray:
    """Mean L1 term over the pairs of each camera (0 for a camera in no pair), (N,)."""
    o = np.asarray(o, np.float64).reshape(-1, 3)
    term, _ = pair_terms(o, cam_i, cam_j, o_ij)
    n = o.shape[0]
    s = np.bincount(cam_i, weights=term, minlength=n) + np.bincount(cam_j, weights=term, minlength=n)
    c = np.bincount(cam_i, minlength=n) + np.bincount(cam_j, minlength=n)
    return np.where(c > 0, s / np.maximum(c, 1), 0.0)


def adam(o0, cam_i, cam_j, o_ij, iters: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-12):
    """`iters` Adam steps on the centres from o0; returns (centres, last loss)."""
    o = np.asarray(o0, np.float64).reshape(-1, 3).copy()
    m = np.zeros_like(o)
    v = np.zeros_like(o)
    loss = float("nan")
    for k in range(1, iters + 1):
        loss, g = loss_grad(o, cam_i, cam_j, o_ij)
        m = beta1 * m + (1 - beta1) * g
        v = beta2 * v + (1 - beta2) * g * g
        o -= lr * (m / (1 - beta1 ** k)) / (np.sqrt(v / (1 - beta2 ** k)) + eps)
    return o, loss


def normalize(o) -> np.ndarray:
    """Centred at the origin and scaled to unit mean norm."""
    o = np.asarray(o, np.float64).reshape(-1, 3)
    c = o - o.mean(0)
    return c / np.linalg.norm(c, axis=1).mean()


def merge(solutions, cam_losses) -> np.ndarray:
    """Per camera, the normalised centre of the run with the lowest camera loss."""
    sols = np.stack([normalize(s) for s in solutions])
    best = np.argmin(np.asarray(cam_losses, np.float64), axis=0)   # first minimum on ties
    return sols[best, np.arange(sols.shape[1])]


def solve(o_inits, cam_i, cam_j, o_ij, iters: int, final_iters: int, lr: float, **adam_kw):
    """Independent runs from each initialisation, merge, final run from the merged centres."""
    sols, losses = [], []
    for o0 in o_inits:
        o, _ = adam(o0, cam_i, cam_j, o_ij, iters, lr, **adam_kw)
        sols.append(o)
        losses.append(camera_losses(o, cam_i, cam_j, o_ij))
    merged = merge(sols, losses)
    return adam(merged, cam_i, cam_j, o_ij, final_iters, lr, **adam_kw)
