"""Parity bounds shared by the GPU tests (imported by the test modules; not a test itself).

Gradient bound, derived from the arithmetic: every per-camera gradient is a sum over the
camera's image pairs of chain-rule terms, each built from FP32 sums over the pair's point
pairs. The FP32 rounding of those sums leaves an error of about 1e-7 of the sum's gross
magnitude, so two checks are made on the n_cams x 6 gradient, separately for the rotation
block (phi) and the centre block (c) of every camera, whose units differ:

  * whole vector:  max |g - g_ref| <= tol * max |g_ref|                    (tol = 1e-4);
  * per camera:    |g_k - g_ref,k| <= tol * |g_ref,k| + floor * max_k |g_ref,k|   (floor = 1e-7)

The per-camera check catches a mistake confined to a few cameras (a wrong term in the chain
rule of one pair orientation, a lost scatter) that the whole-vector bound would hide behind the
camera with the largest gradient; the floor term (1e-3 of the whole-vector bound) only admits
the FP32 rounding of cameras whose own gradient nearly cancels. For the L1 objective the
subgradient takes sign(eps), a decision the CUDA path makes in FP32 and the oracle in FP64;
point pairs whose residual lies within the residual's FP32 error of zero may go either way, and
`l1_flip_allowance` adds, per camera, the largest change those decisions can make.
"""
import numpy as np


def l1_flip_allowance(prob, R, c, eps, atol):
    """Per-camera, per-block bound (n_cams x 2) on how far the L1 gradient can move when the
    signs of the residuals within `atol` of zero are decided the other way (the CUDA path takes
    sign(eps) in FP32, the oracle in FP64). A point pair's residual eps = o2^T [t^]_x R_n o1 moves
    by at most 2 |o1| |o2| per radian of either camera's rotation and by |o1| |o2| / |c_i - c_j|
    per unit move of either centre (unit |t^|, orthonormal R); one flipped sign changes the
    gradient by twice that over Z. eps are the oracle's FP64 residuals (input order)."""
    eps = np.asarray(eps, np.float64)
    und = np.abs(eps) <= atol
    out = np.zeros((prob.n_cams, 2))
    if not und.any():
        return out
    pid = prob.pair_id[und]
    o1 = np.sqrt(1.0 + (prob.x1[und] ** 2).sum(1))
    o2 = np.sqrt(1.0 + (prob.x2[und] ** 2).sum(1))
    ci, cj = prob.cam_i[pid], prob.cam_j[pid]
    base = np.linalg.norm(c[ci] - c[cj], axis=1)
    rot = 2.0 * 2.0 * o1 * o2 / prob.n_pp
    cen = 2.0 * o1 * o2 / base / prob.n_pp
    for cams in (ci, cj):
        out[:, 0] += np.bincount(cams, weights=rot, minlength=prob.n_cams)
        out[:, 1] += np.bincount(cams, weights=cen, minlength=prob.n_cams)
    return out


def assert_grad_close(g, ref, tol=1e-4, floor=1e-7, what="gradient", allowance=None):
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    assert g.shape == ref.shape, (g.shape, ref.shape)
    err = np.abs(g - ref).max()
    assert err <= tol * np.abs(ref).max(), (what, err, np.abs(ref).max())
    if ref.ndim == 2 and ref.shape[1] == 6:
        d = np.linalg.norm((g - ref).reshape(-1, 2, 3), axis=2)
        r = np.linalg.norm(ref.reshape(-1, 2, 3), axis=2)
        bound = tol * r + floor * r.max(axis=0, keepdims=True)
        if allowance is not None:
            bound = bound + allowance
        bad = d > bound
        if bad.any():
            k, b = np.argwhere(bad)[0]
            raise AssertionError(f"{what}: camera {k} {'phi' if b == 0 else 'centre'} block off by "
                                 f"{d[k, b]:.3e} (own norm {r[k, b]:.3e}, bound {bound[k, b]:.3e}); "
                                 f"{int(bad.sum())} blocks out of bound")


def grad_bound_ratio(g, ref, tol=1e-4, floor=1e-7):
    """Largest per-camera error as a fraction of its bound (diagnostics; < 1 passes)."""
    d = np.linalg.norm((np.asarray(g) - np.asarray(ref)).reshape(-1, 2, 3), axis=2)
    r = np.linalg.norm(np.asarray(ref).reshape(-1, 2, 3), axis=2)
    return float((d / (tol * r + floor * r.max(axis=0, keepdims=True))).max())


def bf16_spacing(v):
    """Distance between neighbouring BF16 values at |v| (8 significant bits)."""
    a = np.maximum(np.abs(np.asarray(v, np.float64)), 1e-30)
    return 2.0 ** (np.floor(np.log2(a)) - 7)


def mlp_output_bound(L, params, X, dX):
    """First-order bound, per row, on |p_gpu - p_oracle| for the network of the library's
    numerics (BF16 inputs, weights and hidden activations, FP32 accumulation; L = oracle.learned).
    The two sides may differ by (1) the input features before rounding (dX, per feature, from
    the residual's FP32 error), which can move a BF16-rounded input by dX plus one BF16 spacing,
    (2) the FP32 summation order of each dot product, which can move a BF16-rounded hidden
    activation across one rounding boundary (one BF16 spacing), (3) the fast exponential and
    reciprocal of the sigmoid (1e-6). Each is weighted by the oracle's own |dp/d.| at the row
    (back-propagation through the BF16 network with its ReLU masks), and the sum is taken with a
    factor 1.5 for the linearisation. Returns (p_oracle, bound)."""
    p, (xb, z1, h1, z2, h2, z3, qp) = L.forward_bf16(params, X, keep=True)
    s = p * (1.0 - p)
    dh2 = s[:, None] * qp["W3"][:, 0][None, :]
    dz2 = dh2 * (z2 > 0)
    dh1 = dz2 @ qp["W2"].T
    dz1 = dh1 * (z1 > 0)
    dx = dz1 @ qp["W1"].T
    b = (np.abs(dx) * (dX + bf16_spacing(xb))).sum(1)
    b += (np.abs(dh1) * bf16_spacing(h1) * (h1 > 0)).sum(1) + (np.abs(dh2) * bf16_spacing(h2) * (h2 > 0)).sum(1)
    return p, 1.5 * b + 1e-6
