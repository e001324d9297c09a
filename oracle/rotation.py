"""Oracle of the global rotation stage (TEST INFRASTRUCTURE ONLY).

Sec. "Global Rotation" of the FastMap chapter: given relative rotations R_{i->j} of the image
pairs, find world-to-camera rotations R_k minimising

    L_R = (1/|P|) sum_{(i,j)} d(R_j, R_{i->j} R_i),   d(R, R') = arccos((tr(R^T R') - 1) / 2)

(Eq. fastmap-rotation-objective, geodesic distance), with each R_k parameterised by the 6D
representation (two 3-vectors, Gram-Schmidt, third column their cross product), from the
column-wise initialisation (paragraph "Initialization details", a variant of Martinec and
Pajdla): column 1 of every rotation from the least-squares problem sum ||x_j - R_{i->j} x_i||^2,
then normalised; column 2 from the same problem plus the orthogonality penalty
(1/|I|) sum (x_i^T y_i)^2 with the data term scaled by 1/|P|, then normalised and
Gram-Schmidt-orthogonalised to column 1; column 3 = column 1 x column 2.

Readings where the thesis is silent: the least-squares problems fix the gauge (a global
rotation) and exclude the zero solution by holding camera 0's column at its value for
R_0 = I (e1, then e2); they are solved exactly here (sparse direct solve). (With inconsistent
relative rotations this anchored solution shrinks with the distance from camera 0; on long
chains with wrong pairs it can vanish, which the thesis' upstream pair filtering avoids.) For the gradient the
arccos argument is clamped to 1 - 1e-12, so it stays finite at d = 0. The optimiser is
Adam on the 6D parameters with a constant step size. Plain FP64 NumPy/SciPy.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

C_MAX = 1.0 - 1e-12


# ---- column-wise initialisation ---------------------------------------------------------------
def connection_matrix(n_cams, cam_i, cam_j, R_rel, w_pair=1.0, diag_blocks=None):
    """Matrix of the quadratic form w_pair * sum_p ||v_j - R_p v_i||^2 (+ block-diagonal extra
    terms) over the stacked 3-vectors v (3N x 3N, sparse): blocks deg_k I on the diagonal and
    -R_p at (j, i), -R_p^T at (i, j)."""
    R_rel = np.asarray(R_rel, np.float64).reshape(-1, 3, 3)
    rows, cols, vals = [], [], []
    deg = np.bincount(cam_i, minlength=n_cams) + np.bincount(cam_j, minlength=n_cams)
    for k in range(n_cams):
        blk = w_pair * deg[k] * np.eye(3)
        if diag_blocks is not None:
            blk = blk + diag_blocks[k]
        for a in range(3):
            for b in range(3):
                rows.append(3 * k + a)
                cols.append(3 * k + b)
                vals.append(blk[a, b])
    for p, (i, j) in enumerate(zip(cam_i, cam_j)):
        for a in range(3):
            for b in range(3):
                rows += [3 * j + a, 3 * i + b]
                cols += [3 * i + b, 3 * j + a]
                vals += [-w_pair * R_rel[p, a, b], -w_pair * R_rel[p, a, b]]
    return sp.csr_matrix((vals, (rows, cols)), shape=(3 * n_cams, 3 * n_cams))


def _solve_anchored(A, v0):
    """Minimise v^T A v with the 3-vector of camera 0 held at v0."""
    n3 = A.shape[0]
    free = np.arange(3, n3)
    rhs = -A[free][:, :3] @ v0
    vf = spla.spsolve(A[free][:, free].tocsc(), rhs)
    return np.concatenate([v0, vf]).reshape(-1, 3)


def initial_rotations(n_cams, cam_i, cam_j, R_rel):
    """Column-wise initialisation; returns (N, 3, 3) world-to-camera rotations with R_0 = I."""
    cam_i = np.asarray(cam_i)
    cam_j = np.asarray(cam_j)
    A1 = connection_matrix(n_cams, cam_i, cam_j, R_rel)
    x = _solve_anchored(A1, np.array([1.0, 0.0, 0.0]))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    B = len(cam_i)
    pen = np.einsum("ka,kb->kab", x, x) / n_cams
    A2 = connection_matrix(n_cams, cam_i, cam_j, R_rel, w_pair=1.0 / B, diag_blocks=pen)
    y = _solve_anchored(A2, np.array([0.0, 1.0, 0.0]))
    y /= np.linalg.norm(y, axis=1, keepdims=True)
    y -= x * (x * y).sum(1, keepdims=True)
    y /= np.linalg.norm(y, axis=1, keepdims=True)
    z = np.cross(x, y)
    return np.stack([x, y, z], axis=2)      # columns


# ---- 6D representation ---------------------------------------------------------------------------
def rot_from_6d(a):
    """a: (N, 6) = (a1, a2); R = [b1 b2 b3] with b1 = a1/|a1|, b2 = normalised a2 minus its b1
    component, b3 = b1 x b2 (columns)."""
    a = np.asarray(a, np.float64).reshape(-1, 6)
    a1, a2 = a[:, :3], a[:, 3:]
    b1 = a1 / np.linalg.norm(a1, axis=1, keepdims=True)
    u = a2 - b1 * (b1 * a2).sum(1, keepdims=True)
    b2 = u / np.linalg.norm(u, axis=1, keepdims=True)
    b3 = np.cross(b1, b2)
    return np.stack([b1, b2, b3], axis=2)


def six_d_from_rot(R):
    """The 6D parameters of rotations (their first two columns), the inverse of rot_from_6d
    on SO(3) (6D representation of Sec. "Global Rotation")."""
    R = np.asarray(R, np.float64).reshape(-1, 3, 3)
    return np.concatenate([R[:, :, 0], R[:, :, 1]], axis=1)


def rot_6d_backward(a, gR):
    """Gradient with respect to the 6D parameters a (N, 6) of a scalar with gradient gR
    (N, 3, 3) with respect to R = rot_from_6d(a)."""
    a = np.asarray(a, np.float64).reshape(-1, 6)
    a1, a2 = a[:, :3], a[:, 3:]
    n1 = np.linalg.norm(a1, axis=1, keepdims=True)
    b1 = a1 / n1
    u = a2 - b1 * (b1 * a2).sum(1, keepdims=True)
    nu = np.linalg.norm(u, axis=1, keepdims=True)
    b2 = u / nu
    g1, g2, g3 = gR[:, :, 0], gR[:, :, 1], gR[:, :, 2]
    # b3 = b1 x b2:  d<g3, b1 x b2> = <b2 x g3, db1> + <g3 x b1, db2>
    gb1 = g1 + np.cross(b2, g3)
    gb2 = g2 + np.cross(g3, b1)
    # b2 = u/|u|
    gu = (gb2 - b2 * (b2 * gb2).sum(1, keepdims=True)) / nu
    # u = a2 - b1 (b1 . a2)
    d = (b1 * a2).sum(1, keepdims=True)
    ga2 = gu - b1 * (b1 * gu).sum(1, keepdims=True)
    gb1 = gb1 - gu * d - a2 * (b1 * gu).sum(1, keepdims=True)
    # b1 = a1/|a1|
    ga1 = (gb1 - b1 * (b1 * gb1).sum(1, keepdims=True)) / n1
    return np.concatenate([ga1, ga2], axis=1)


# ---- objective -------------------------------------------------------------------------------
def geodesic(Ra, Rb):
    """d(Ra, Rb) = arccos((tr(Ra^T Rb) - 1) / 2) per pair, radians (the geodesic distance of
    Eq. fastmap-rotation-objective)."""
    c = (np.einsum("nab,nab->n", Ra, Rb) - 1.0) / 2.0
    return np.arccos(np.clip(c, -1.0, 1.0))


def loss_grad_R(R, cam_i, cam_j, R_rel):
    """L_R and its gradient with respect to the rotation matrices (N, 3, 3)."""
    R = np.asarray(R, np.float64).reshape(-1, 3, 3)
    Rr = np.asarray(R_rel, np.float64).reshape(-1, 3, 3)
    ci, cj = np.asarray(cam_i), np.asarray(cam_j)
    X = Rr @ R[ci]                                        # R_{i->j} R_i
    c = (np.einsum("nab,nab->n", R[cj], X) - 1.0) / 2.0   # (tr(R_j^T X) - 1)/2
    d = np.arccos(np.clip(c, -1.0, 1.0))
    cc = np.clip(c, -1.0, C_MAX)
    dd = -0.5 / np.sqrt(1.0 - cc * cc)                    # d d / d tr, finite at d = 0
    B = len(ci)
    g = np.zeros_like(R)
    np.add.at(g, cj, (dd / B)[:, None, None] * X)                          # d tr / d R_j = X
    np.add.at(g, ci, (dd / B)[:, None, None] * np.einsum("nba,nbc->nac", Rr, R[cj]))  # R_rel^T R_j
    return float(d.sum() / B), g


def loss_grad_6d(a, cam_i, cam_j, R_rel):
    """L_R (Eq. fastmap-rotation-objective) and its gradient with respect to the 6D
    parameters a (N, 6), by the chain rule through rot_from_6d."""
    R = rot_from_6d(a)
    loss, gR = loss_grad_R(R, cam_i, cam_j, R_rel)
    return loss, rot_6d_backward(a, gR)


def adam(a0, cam_i, cam_j, R_rel, iters: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-12):
    """`iters` Adam steps on the 6D parameters from a0 (the first-order optimisation of the
    rotation objective, Sec. "Global Rotation"); returns (parameters, last loss)."""
    a = np.asarray(a0, np.float64).reshape(-1, 6).copy()
    m = np.zeros_like(a)
    v = np.zeros_like(a)
    loss = float("nan")
    for k in range(1, iters + 1):
        loss, g = loss_grad_6d(a, cam_i, cam_j, R_rel)
        m = beta1 * m + (1 - beta1) * g
        v = beta2 * v + (1 - beta2) * g * g
        a -= lr * (m / (1 - beta1 ** k)) / (np.sqrt(v / (1 - beta2 ** k)) + eps)
    return a, loss
