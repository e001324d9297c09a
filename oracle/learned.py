"""Oracle of the learned inlier-weight variant (TEST INFRASTRUCTURE ONLY).

The thesis has no learned component; this restates the variant the benchmark asks for: a
small MLP (8 -> 32 -> 32 -> 1) predicts, from a point pair's residual history, its match
score and statistics of its image pair, the probability p that the pair is an inlier. The
reweighting step of the IRLS loop (Sec. "Epipolar Adjustment") then uses
w = p / max(|eps^|, delta) in place of the hard threshold mask. Labels come from the method
itself: the IRLS mask |eps| <= tau_min at the poses a long plain-IRLS run converged to.

Everything here is plain FP64 NumPy, written for checking the CUDA kernels. The trained
network itself: parity unpinned (it depends on data and initialisation; its only judge is the
pose error it reaches). The forward and backward passes are pinned by finite differences in
the tests.
"""
from __future__ import annotations

import numpy as np

N_FEAT = 8
HIDDEN = 32
LOG_FLOOR = 1e-6


def pair_statistics(abs_eps, pair_id, n_pairs, tau):
    """Per image pair: mean of log(|eps| + 1e-6), fraction of point pairs with |eps| <= tau,
    and the point-pair count."""
    le = np.log(abs_eps + LOG_FLOOR)
    cnt = np.bincount(pair_id, minlength=n_pairs).astype(np.float64)
    mean_log = np.bincount(pair_id, weights=le, minlength=n_pairs) / np.maximum(cnt, 1)
    frac = np.bincount(pair_id, weights=(abs_eps <= tau).astype(np.float64), minlength=n_pairs) / np.maximum(cnt, 1)
    return mean_log, frac, cnt


def features(abs_eps, abs_eps_prev, score, pair_id, n_pairs, tau, round_index):
    """The 8 features of every point pair (float64, (P, 8)):
    0 log(|e|+1e-6) - log(tau)            residual against the round's threshold
    1 log(|e|+1e-6) - mean_pair(log)      residual against its image pair's log-scale
    2 log(|e_prev|+1e-6) - log(|e|+1e-6)  change since the previous reweighting
    3 score                               matcher confidence
    4 frac_pair(|e| <= tau)               image-pair inlier fraction at this threshold
    5 log(count_pair) / 10                image-pair size
    6 round / 10                          reweighting round
    7 log(|e_prev|+1e-6) - log(tau)       previous residual against the threshold
    """
    mean_log, frac, cnt = pair_statistics(abs_eps, pair_id, n_pairs, tau)
    le = np.log(abs_eps + LOG_FLOOR)
    lp = np.log(abs_eps_prev + LOG_FLOOR)
    lt = np.log(tau)
    f = np.empty((abs_eps.shape[0], N_FEAT))
    f[:, 0] = le - lt
    f[:, 1] = le - mean_log[pair_id]
    f[:, 2] = lp - le
    f[:, 3] = score
    f[:, 4] = frac[pair_id]
    f[:, 5] = np.log(cnt[pair_id]) / 10.0
    f[:, 6] = round_index / 10.0
    f[:, 7] = lp - lt
    return f


# ---- flat parameter vector (the library's layout) and BF16 emulation -----------------------------
SHAPES = (("W1", (N_FEAT, HIDDEN)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
          ("W3", (HIDDEN, 1)), ("b3", (1,)))


def flatten(params) -> np.ndarray:
    """Parameters as one vector in the library's order (W1, b1, W2, b2, W3, b3; row-major)."""
    return np.concatenate([np.asarray(params[k], np.float64).reshape(-1) for k, _ in SHAPES])


def unflatten(vec) -> dict:
    """The inverse of flatten."""
    vec = np.asarray(vec, np.float64)
    out, o = {}, 0
    for k, shp in SHAPES:
        n = int(np.prod(shp))
        out[k] = vec[o:o + n].reshape(shp).copy()
        o += n
    return out


def bf16_round(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64: the FP32 bit pattern
    with the low 16 bits rounded away."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def quantized(params) -> dict:
    """Weights rounded to BF16 (biases stay as they are), as the library uses them."""
    q = {k: np.asarray(v, np.float64).copy() for k, v in params.items()}
    for k in ("W1", "W2", "W3"):
        q[k] = bf16_round(q[k])
    return q


def forward_bf16(params, X, keep=False):
    """The library's numerics: BF16 inputs, weights and hidden activations, exact products."""
    qp = quantized(params)
    xb = bf16_round(X)
    z1 = xb @ qp["W1"] + qp["b1"]
    h1 = bf16_round(np.maximum(z1, 0.0))
    z2 = h1 @ qp["W2"] + qp["b2"]
    h2 = bf16_round(np.maximum(z2, 0.0))
    z3 = (h2 @ qp["W3"])[:, 0] + qp["b3"][0]
    p = 1.0 / (1.0 + np.exp(-z3))
    if keep:
        return p, (xb, z1, h1, z2, h2, z3, qp)
    return p


def bce_loss_grad_bf16(params, X, y):
    """Cross-entropy gradient of forward_bf16 with the roundings passed straight through."""
    p, (xb, z1, h1, z2, h2, z3, qp) = forward_bf16(params, X, keep=True)
    n = X.shape[0]
    loss = np.mean(np.maximum(z3, 0) - z3 * y + np.log1p(np.exp(-np.abs(z3))))
    dz3 = (p - y) / n
    g = {"W3": h2.T @ dz3[:, None], "b3": np.array([dz3.sum()])}
    dz2 = dz3[:, None] * qp["W3"][:, 0][None, :] * (z2 > 0)
    g["W2"] = h1.T @ dz2
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ qp["W2"].T) * (z1 > 0)
    g["W1"] = xb.T @ dz1
    g["b1"] = dz1.sum(0)
    return loss, g


def init_params(seed=0):
    """He-normal weights (variance 2/fan-in for the ReLU layers, 1/fan-in for the output) and
    zero biases, seeded."""
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.normal(0, np.sqrt(2.0 / N_FEAT), (N_FEAT, HIDDEN)),
        "b1": np.zeros(HIDDEN),
        "W2": rng.normal(0, np.sqrt(2.0 / HIDDEN), (HIDDEN, HIDDEN)),
        "b2": np.zeros(HIDDEN),
        "W3": rng.normal(0, np.sqrt(1.0 / HIDDEN), (HIDDEN, 1)),
        "b3": np.zeros(1),
    }


def forward(params, X, keep=False):
    """p = sigmoid(W3^T relu(W2^T relu(W1^T x + b1) + b2) + b3)."""
    z1 = X @ params["W1"] + params["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ params["W2"] + params["b2"]
    h2 = np.maximum(z2, 0.0)
    z3 = (h2 @ params["W3"])[:, 0] + params["b3"][0]
    p = 1.0 / (1.0 + np.exp(-z3))
    if keep:
        return p, (X, z1, h1, z2, h2, z3)
    return p


def bce_loss_grad(params, X, y):
    """Mean binary cross-entropy of p against labels y and its gradient (backpropagation)."""
    p, (X, z1, h1, z2, h2, z3) = forward(params, X, keep=True)
    n = X.shape[0]
    # log(1 + e^-z) written stably
    loss = np.mean(np.maximum(z3, 0) - z3 * y + np.log1p(np.exp(-np.abs(z3))))
    dz3 = (p - y) / n
    g = {"W3": h2.T @ dz3[:, None], "b3": np.array([dz3.sum()])}
    dh2 = dz3[:, None] * params["W3"][:, 0][None, :]
    dz2 = dh2 * (z2 > 0)
    g["W2"] = h1.T @ dz2
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ params["W2"].T
    dz1 = dh1 * (z1 > 0)
    g["W1"] = X.T @ dz1
    g["b1"] = dz1.sum(0)
    return loss, g


def adam_init(params):
    """Zero first and second moments for adam_update."""
    return {k: np.zeros_like(v) for k, v in params.items()}, {k: np.zeros_like(v) for k, v in params.items()}


def adam_update(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba, bias-corrected; `step` is 1-based) on every parameter,
    in place: the training optimiser of the network."""
    bc1 = 1 - beta1 ** step
    bc2 = 1 - beta2 ** step
    for k in params:
        m[k] = beta1 * m[k] + (1 - beta1) * grads[k]
        v[k] = beta2 * v[k] + (1 - beta2) * grads[k] ** 2
        params[k] = params[k] - lr * (m[k] / bc1) / (np.sqrt(v[k] / bc2) + eps)


def learned_weights(params, abs_eps, feats, delta, tau_cap=np.inf):
    """w = p / max(|eps|, delta), and 0 beyond tau_cap."""
    p = forward(params, feats)
    w = p / np.maximum(abs_eps, delta)
    w[abs_eps > tau_cap] = 0.0
    return w, p
