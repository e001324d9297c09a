"""Oracle: plain FP64 CPU reference of FastMap's epipolar adjustment.

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's CPU-baseline
leg may import this package. The CUDA library never loads it, and the two share no code.

The per-point-pair loops live in plain C (``epipolar.c``, FP64, input order, no blocking);
this module loads it with ctypes and adds the small dense pieces in NumPy:

* residuals, L1 / IRLS losses and the analytic gradient (Eq. epipolar-objective and the
  IRLS objective of Sec. "Epipolar Adjustment"),
* IRLS weights with outlier filtering (IRLS and filtering paragraphs of the same section),
* the Adam + exponential-map optimisation loop (first-order optimisation, Sec.
  "First-order Optimization"),
* the pre-aggregated quadratic form e_n^T W_n e_n (Eq. epipolar-objective-l2),
* the FP16 centroid-offset storage rule the CUDA path promises to implement, so the oracle
  can evaluate the exact dequantized inputs without reading anything from the GPU,
* pose-error metrics (geodesic rotation distance after global alignment, Eq. of the
  geodesic distance in Sec. "Global Rotation"; relative-translation direction angle).

Where the paper is silent the readings are: E_n uses the unit translation t_n/|t_n|; the
quadratic-form factor is 1/Z (the printed 2/Z does not match (w^T e)^2 = e^T w w^T e);
w = 1/max(|eps^|, delta); filtered pairs keep counting in Z; the filter threshold shrinks
by a constant factor each round down to a floor; Adam state persists across rounds; the per-camera parameters
are a left rotation increment and the camera centre.

Pinned by the not-gpu tests against: zero residual at the true poses of noise-free scenes,
the rectified-stereo closed form, brute-force quadratic form, similarity and pair-swap
invariance, the three gauge identities of the gradient, central finite differences,
the IRLS = L1 identity at the reweighting point, Rodrigues vs a library rotation, the
closed-form first Adam step and convergence on noise-free scenes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "epipolar.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lib = None

__all__ = [
    "build", "centres_from_poses", "poses_from_centres", "essential", "residuals",
    "loss_grad", "irls_weights", "threshold_schedule", "expmap", "project_rotation",
    "adam_step", "refine", "quadratic_form_loss", "pair_W", "fp16_centroid_storage",
    "fp16_weight_scale", "quantize_weights_fp16", "rotation_error_deg",
    "translation_error_deg",
]


def build(force: bool = False) -> str:
    """Compile epipolar.c into a shared library next to it (gcc, strict IEEE)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        lib.or_essential.argtypes = [ctypes.c_int, P, P, P, P, P]
        lib.or_essential.restype = ctypes.c_int
        lib.or_residuals.argtypes = [ctypes.c_int, P, P, ctypes.c_int, P, P, ctypes.c_int64, P, P, P, P, P]
        lib.or_residuals.restype = ctypes.c_int
        lib.or_loss_grad.argtypes = [ctypes.c_int, P, P, ctypes.c_int, P, P, ctypes.c_int64, P, P, P, P,
                                     ctypes.c_int, P, P, P, P]
        lib.or_loss_grad.restype = ctypes.c_int
        lib.or_irls_weights.argtypes = [ctypes.c_int64, P, ctypes.c_double, ctypes.c_double, P]
        lib.or_irls_weights.restype = ctypes.c_int64
        lib.or_expmap.argtypes = [P, P]
        lib.or_expmap.restype = None
        lib.or_adam_step.argtypes = [ctypes.c_int, P, P, P, P, P, ctypes.c_int64, P,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double]
        lib.or_adam_step.restype = None
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


class Problem:
    """Point pairs of one scene as contiguous FP64/int32 arrays (input order kept)."""

    def __init__(self, n_cams, cam_i, cam_j, pair_id, x1, x2):
        self.n_cams = int(n_cams)
        self.cam_i = _i32(cam_i)
        self.cam_j = _i32(cam_j)
        self.pair_id = _i32(pair_id)
        self.x1 = _f64(x1).reshape(-1, 2)
        self.x2 = _f64(x2).reshape(-1, 2)
        self.n_pairs = int(self.cam_i.shape[0])
        self.n_pp = int(self.pair_id.shape[0])
        self._E = np.empty((self.n_pairs, 9))
        self._G = np.empty((self.n_pairs, 9))

    @classmethod
    def from_scene(cls, sc):
        return cls(sc.n_cams, sc.cam_i.cpu().numpy(), sc.cam_j.cpu().numpy(),
                   sc.pair_id.cpu().numpy(), sc.x1.cpu().numpy(), sc.x2.cpu().numpy())


# ---- pose conventions -----------------------------------------------------------------
def centres_from_poses(R, t):
    """c_k = -R_k^T t_k: the camera centre of a world-to-camera pose (the translations of
    Eq. epipolar-objective are optimised through it; a reading, see the module notes)."""
    R = _f64(R).reshape(-1, 3, 3)
    return -np.einsum("nba,nb->na", R, _f64(t).reshape(-1, 3))


def poses_from_centres(R, c):
    """t_k = -R_k c_k, the inverse of centres_from_poses."""
    R = _f64(R).reshape(-1, 3, 3)
    return -np.einsum("nab,nb->na", R, _f64(c).reshape(-1, 3))


# ---- objective --------------------------------------------------------------------------
def essential(prob: Problem, R, c) -> np.ndarray:
    """E_n = [t_n/|t_n|]_x R_j R_i^T for every pair, (B, 3, 3): the essential matrix of image
    pair n computed from the global poses (Eq. epipolar-objective; the unit translation is a
    reading, see the module notes)."""
    R = _f64(R).reshape(-1, 9)
    c = _f64(c).reshape(-1, 3)
    E = np.empty((prob.n_pairs, 9))
    if _load().or_essential(prob.n_pairs, _p(prob.cam_i), _p(prob.cam_j), _p(R), _p(c), _p(E)):
        raise FloatingPointError("zero-length relative translation")
    return E.reshape(-1, 3, 3)


def residuals(prob: Problem, R, c) -> np.ndarray:
    """epsilon_nm = x2^T E_n x1 for every point pair, input order (the epipolar error inside
    Eq. epipolar-objective)."""
    R = _f64(R).reshape(-1, 9)
    c = _f64(c).reshape(-1, 3)
    eps = np.empty(prob.n_pp)
    st = _load().or_residuals(prob.n_cams, _p(R), _p(c), prob.n_pairs, _p(prob.cam_i), _p(prob.cam_j),
                              prob.n_pp, _p(prob.pair_id), _p(prob.x1), _p(prob.x2), _p(prob._E), _p(eps))
    if st:
        raise FloatingPointError("zero-length relative translation")
    return eps


def loss_grad(prob: Problem, R, c, w=None, mode: str = "irls"):
    """Loss and gradient d/d(phi_k, c_k), (n_cams, 6).

    mode "irls": (1/Z) sum w eps^2 with the given weights (w=None means all ones, the plain
    L2 objective of Eq. epipolar-objective-l2); mode "l1": (1/Z) sum |eps|.
    """
    R = _f64(R).reshape(-1, 9)
    c = _f64(c).reshape(-1, 3)
    if mode == "irls":
        wv = np.ones(prob.n_pp) if w is None else _f64(w)
        m = 0
    elif mode == "l1":
        wv = np.zeros(1)
        m = 1
    else:
        raise ValueError(mode)
    loss = ctypes.c_double()
    grad = np.empty((prob.n_cams, 6))
    st = _load().or_loss_grad(prob.n_cams, _p(R), _p(c), prob.n_pairs, _p(prob.cam_i), _p(prob.cam_j),
                              prob.n_pp, _p(prob.pair_id), _p(prob.x1), _p(prob.x2), _p(wv), m,
                              _p(prob._E), _p(prob._G), ctypes.byref(loss), _p(grad))
    if st:
        raise FloatingPointError("zero-length relative translation")
    return loss.value, grad


def irls_weights(eps_hat, tau: float, delta: float):
    """w = [|eps^| <= tau] / max(|eps^|, delta); returns (w, number kept). The IRLS weight
    1/|eps^| of Sec. "Epipolar Adjustment" (IRLS paragraph; the floor delta is a reading) with
    the filtering paragraph's threshold: pairs above tau get weight 0."""
    e = _f64(eps_hat)
    w = np.empty_like(e)
    kept = _load().or_irls_weights(e.shape[0], _p(e), float(tau), float(delta), _p(w))
    return w, int(kept)


def threshold_schedule(r: int, tau0: float, tau_min: float, factor: float = 0.8) -> float:
    """Filtering threshold of round r: starts large and shrinks by `factor` each round down to
    a fixed floor (filtering paragraph of Sec. "Epipolar Adjustment", which gives no values)."""
    return max(tau_min, tau0 * factor ** r)


# ---- optimiser ----------------------------------------------------------------------------
def expmap(phi) -> np.ndarray:
    """Exp(phi) of one rotation vector by Rodrigues' formula (the rotation increment of the
    first-order loop, Sec. "First-order Optimization"); a series near 0 (epipolar.c)."""
    phi = _f64(phi).reshape(3)
    R = np.empty(9)
    _load().or_expmap(_p(phi), _p(R))
    return R.reshape(3, 3)


def project_rotation(R) -> np.ndarray:
    """Nearest rotation matrix (SVD polar factor with det +1), applied per camera: keeps the
    rotations of the first-order loop (Sec. "First-order Optimization") on SO(3)."""
    R = _f64(R).reshape(-1, 3, 3)
    U, _, Vt = np.linalg.svd(R)
    d = np.sign(np.linalg.det(U @ Vt))
    D = np.ones((R.shape[0], 3))
    D[:, 2] = d
    return np.einsum("nab,nb,nbc->nac", U, D, Vt)


def adam_step(R, c, grad, m, v, step: int, lr_rot: float, lr_c: float,
              beta1=0.9, beta2=0.999, eps=1e-12):
    """One Adam step in place on (R, c, m, v); R is re-orthonormalised afterwards. Adam is the
    adaptive first-order method Sec. "First-order Optimization" cites; rotations move by
    R <- Exp(step) R, centres additively."""
    lr = np.array([lr_rot, lr_c], dtype=np.float64)
    _load().or_adam_step(R.shape[0], _p(R), _p(c), _p(_f64(grad)), _p(m), _p(v), int(step), _p(lr),
                         float(beta1), float(beta2), float(eps))
    R[:] = project_rotation(R).reshape(R.shape)


def refine(prob: Problem, R0, c0, n_rounds: int, iters_per_round: int, tau0: float,
           tau_min: float, delta: float, lr_rot: float, lr_c: float, decay: float = 1.0,
           beta1=0.9, beta2=0.999, adam_eps=1e-12, weight_fn=None, callback=None,
           tau_factor: float = 0.8):
    """IRLS epipolar adjustment: per round, reweight at the current poses (with filtering),
    then `iters_per_round` Adam steps on the weighted objective. Learning rates are
    multiplied by `decay` after every round. `weight_fn(w)` may post-process the weights
    (e.g. the FP16 storage rounding). Returns (R, c, last loss)."""
    R = _f64(R0).reshape(-1, 3, 3).copy()
    c = _f64(c0).reshape(-1, 3).copy()
    m = np.zeros((R.shape[0], 6))
    v = np.zeros((R.shape[0], 6))
    step = 0
    loss = float("nan")
    for r in range(n_rounds):
        tau = threshold_schedule(r, tau0, tau_min, tau_factor)
        w, _ = irls_weights(residuals(prob, R, c), tau, delta)
        if weight_fn is not None:
            w = weight_fn(w)
        scale = decay ** r
        for _ in range(iters_per_round):
            loss, g = loss_grad(prob, R, c, w)
            step += 1
            adam_step(R, c, g, m, v, step, lr_rot * scale, lr_c * scale, beta1, beta2, adam_eps)
        if callback is not None:
            callback(r, R, c, loss)
    return R, c, loss


# ---- pre-aggregated quadratic form (Eq. epipolar-objective-l2) -----------------------------
def pair_W(prob: Problem, w=None) -> np.ndarray:
    """W_n = sum_m w_m vec(x2 x1^T) vec(x2 x1^T)^T (row-major flatten), (B, 9, 9)."""
    a = np.concatenate([prob.x1, np.ones((prob.n_pp, 1))], 1)
    b = np.concatenate([prob.x2, np.ones((prob.n_pp, 1))], 1)
    v = np.einsum("pr,pc->prc", b, a).reshape(-1, 9)
    wt = np.ones(prob.n_pp) if w is None else _f64(w)
    W = np.zeros((prob.n_pairs, 9, 9))
    np.add.at(W, prob.pair_id, wt[:, None, None] * v[:, :, None] * v[:, None, :])
    return W


def quadratic_form_loss(prob: Problem, R, c, w=None) -> float:
    """(1/Z) sum_n e_n^T W_n e_n with e_n = vec(E_n)."""
    e = essential(prob, R, c).reshape(-1, 9)
    W = pair_W(prob, w)
    return float(np.einsum("na,nab,nb->", e, W, e) / prob.n_pp)


# ---- FP16 centroid-offset storage rule ------------------------------------------------------
FIXED_POINT_SHIFT = 32


def fp16_centroid_storage(prob: Problem, x1_f32, x2_f32):
    """The storage the FP16 path promises: per-image centroid c_k and FP16 offsets.

    c_k is the mean of all keypoints of image k over all its pairs, computed exactly as
    sum(trunc(x * 2^32)) in integers, converted to FP64 (round to nearest), divided by the
    count, scaled by 2^-32 and rounded to FP32. Offsets are fp16_rn(fp32(x) - c_k) with the
    subtraction in FP32. Returns (centroids (N,2) f32, dequantized x1, x2 as FP64)."""
    x1 = np.asarray(x1_f32, dtype=np.float32).reshape(-1, 2)
    x2 = np.asarray(x2_f32, dtype=np.float32).reshape(-1, 2)
    ci = prob.cam_i[prob.pair_id]
    cj = prob.cam_j[prob.pair_id]
    S = np.zeros((prob.n_cams, 2), dtype=np.int64)
    cnt = np.zeros(prob.n_cams, dtype=np.int64)
    # exact integer sums: per image pair first (segments of the pair-sorted list), then per image
    order = None if np.all(prob.pair_id[1:] >= prob.pair_id[:-1]) else np.argsort(prob.pair_id, kind="stable")
    pid = prob.pair_id if order is None else prob.pair_id[order]
    starts = np.flatnonzero(np.r_[True, pid[1:] != pid[:-1]])
    seg_pair = pid[starts]
    seg_cnt = np.diff(np.r_[starts, len(pid)])
    for cams, x in ((prob.cam_i, x1), (prob.cam_j, x2)):
        xs = x if order is None else x[order]
        fx = np.trunc(xs.astype(np.float64) * 2.0 ** FIXED_POINT_SHIFT).astype(np.int64)
        seg_sum = np.add.reduceat(fx, starts, axis=0)
        np.add.at(S, cams[seg_pair], seg_sum)
        np.add.at(cnt, cams[seg_pair], seg_cnt)
    cen = np.zeros((prob.n_cams, 2), dtype=np.float32)
    has = cnt > 0
    cen[has] = ((S[has].astype(np.float64) / cnt[has, None].astype(np.float64))
                * 2.0 ** -FIXED_POINT_SHIFT).astype(np.float32)
    o1 = (x1 - cen[ci]).astype(np.float16)
    o2 = (x2 - cen[cj]).astype(np.float16)
    d1 = cen[ci].astype(np.float64) + o1.astype(np.float64)
    d2 = cen[cj].astype(np.float64) + o2.astype(np.float64)
    return cen, d1, d2


def fp16_weight_scale(delta: float) -> float:
    """Power-of-two scale s with (1/delta) * s <= 32768, so FP16 holds w * s without overflow
    (the FP16 storage the CUDA path promises; not from the paper, which stores FP32)."""
    return 2.0 ** np.floor(np.log2(32768.0 * delta))


def quantize_weights_fp16(w, delta: float) -> np.ndarray:
    """w as stored by the FP16 path: fp16_rn(fp32(w) * s) / s (a storage rule of the CUDA
    path, restated here so the oracle computes on the same weights)."""
    s = np.float32(fp16_weight_scale(delta))
    q = (np.asarray(w, dtype=np.float32) * s).astype(np.float16)
    return q.astype(np.float64) / float(s)


# ---- metrics --------------------------------------------------------------------------------
def _geodesic_deg(Ra, Rb):
    """d(Ra, Rb) = arccos((tr(Ra^T Rb) - 1)/2), degrees (Sec. "Global Rotation")."""
    tr = np.einsum("nab,nab->n", Ra, Rb)
    return np.degrees(np.arccos(np.clip((tr - 1.0) / 2.0, -1.0, 1.0)))


def rotation_error_deg(R_est, R_gt):
    """Per-camera rotation error after the best global rotation Q (gauge):
    Q = proj_SO3(sum_k R_est_k^T R_gt_k), error_k = d(R_gt_k, R_est_k Q)."""
    Re = _f64(R_est).reshape(-1, 3, 3)
    Rg = _f64(R_gt).reshape(-1, 3, 3)
    Q = project_rotation(np.einsum("nba,nbc->ac", Re, Rg)[None])[0]
    return _geodesic_deg(Rg, Re @ Q)


def translation_error_deg(R_est, c_est, R_gt, c_gt, cam_i, cam_j):
    """Angle between estimated and true unit relative translations t_n/|t_n| per pair (the
    relative-translation error the thesis' accuracy metrics cite)."""
    def tdir(R, c):
        R = _f64(R).reshape(-1, 3, 3)
        c = _f64(c).reshape(-1, 3)
        t = np.einsum("nab,nb->na", R[cam_j], c[cam_i] - c[cam_j])
        return t / np.linalg.norm(t, axis=1, keepdims=True)
    a, b = tdir(R_est, c_est), tdir(R_gt, c_gt)
    return np.degrees(np.arccos(np.clip((a * b).sum(1), -1.0, 1.0)))
