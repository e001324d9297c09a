"""The learned inlier-weight kernels against the oracle: SIMT forward and training gradient,
the tensor-core inference inside the streaming pass, the per-point-pair features, and that
training with the library's kernels reduces the loss.

Tolerances: both sides use BF16 inputs, weights and hidden activations; they differ in the
FP32 summation order of each dot product and, rarely, in a hidden activation that lands on
the other side of a BF16 rounding boundary, which moves p by a few 1e-3 at most. Features
are computed in FP32 on the GPU (FP64 in the oracle) from residuals that differ by the FP32
forward error (2e-6, as in test_gpu_parity); every feature and every weight is held to a bound
derived per point pair from those errors (see test_features_and_learned_weights_match_oracle);
the history is stored in FP16.
"""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import learned as L
import scenegen
import paper_2605_18052_gb300 as fm
from paper_2605_18052_gb300 import build, learned

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    build.build()
    fm.load_library()


def _params(seed):
    v = learned.init_params(seed)
    rng = np.random.default_rng(seed + 100)
    return (v + 0.05 * rng.normal(size=v.shape)).astype(np.float32)


def test_forward_and_gradient_match_oracle():
    rng = np.random.default_rng(0)
    n = 5000
    X = L.bf16_round(rng.normal(0, 2, (n, 8)))
    y = (rng.random(n) < 0.6).astype(np.float32)
    pv = _params(1)
    net = fm.Mlp(pv)
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda").to(torch.bfloat16)
    Yd = torch.tensor(y, device="cuda")
    p_gpu = torch.empty(n, dtype=torch.float32, device="cuda")
    net.forward(Xd, p_gpu)
    torch.cuda.synchronize()
    params = L.unflatten(pv.astype(np.float64))
    p_or = L.forward_bf16(params, X)
    assert np.abs(p_gpu.cpu().numpy() - p_or).max() < 5e-3
    loss, g = net.gradient(Xd, Yd)
    l_or, g_or = L.bce_loss_grad_bf16(params, X, y.astype(np.float64))
    g_or = L.flatten(g_or)
    assert loss == pytest.approx(l_or, rel=1e-3)
    assert np.abs(g - g_or).max() <= 2e-3 * np.abs(g_or).max()


def test_training_reduces_loss():
    rng = np.random.default_rng(2)
    n = 40000
    X = rng.normal(0, 1, (n, 8))
    y = ((X[:, 0] + 0.5 * X[:, 3] - 0.3 * X[:, 5] ** 2) > 0).astype(np.float32)
    net = fm.Mlp(learned.init_params(3))
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda").to(torch.bfloat16)
    Yd = torch.tensor(y, device="cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    losses = learned.train(net, Xd, Yd, 400, 4096, 3e-3, g, log_every=100)
    assert losses[-1][1] < 0.35 * losses[0][1]
    p = torch.empty(n, dtype=torch.float32, device="cuda")
    net.forward(Xd, p)
    acc = ((p.cpu().numpy() > 0.5) == (y > 0.5)).mean()
    assert acc > 0.95


def _feature_errors(L, e_now, e_prev16, pair_id, n_pairs, tau):
    """Per point pair and feature, a bound on the FP32 error of the GPU's feature before BF16
    rounding (the oracle computes it in FP64 from FP64 residuals): the residual's FP32 error
    (2e-6 absolute) moves log(|e| + 1e-6) by at most 2e-6 / (|e| + 1e-6), the fast logarithm adds
    3 ulp; an image pair's mean log and inlier fraction inherit the worst of their point pairs
    (the fraction moves by one count for every residual within 2e-6 of tau); the FP16 history
    moves by one FP16 spacing of the stored log."""
    le = np.log(e_now + 1e-6)
    dle = 2e-6 / (e_now + 1e-6) + 3 * 2.0 ** -23 * np.abs(le) + 1e-6
    cnt = np.bincount(pair_id, minlength=n_pairs).astype(np.float64)
    dmean = np.zeros(n_pairs)
    np.maximum.at(dmean, pair_id, dle)
    und = np.bincount(pair_id, weights=(np.abs(e_now - tau) <= 2e-6).astype(np.float64), minlength=n_pairs)
    lp = np.log(e_prev16 + 1e-6)
    dlp = 2.0 ** (np.floor(np.log2(np.maximum(np.abs(lp), 2.0 ** -14))) - 10) + 3e-6 / (e_prev16 + 1e-6) + 1e-6
    dX = np.zeros((e_now.shape[0], 8))
    dX[:, 0] = dle + 1e-6
    dX[:, 1] = dle + dmean[pair_id] + 1e-5
    dX[:, 2] = dlp + dle
    dX[:, 4] = (und / cnt)[pair_id] + 1e-6
    dX[:, 5] = 1e-6
    dX[:, 6] = 1e-7
    dX[:, 7] = dlp + 1e-6
    return dX


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
@pytest.mark.parametrize("fused", [False, True])
def test_features_and_learned_weights_match_oracle(storage, fused):
    """Every feature and every learned weight against the oracle, element by element: features
    within their FP32 error bound plus one BF16 spacing; weights within the first-order bound of
    tests/bounds.py (mlp_output_bound) carried through w = p / max(|e|, delta), plus the FP16
    weight quantisation; the mask |e| <= tau_cap exact outside the residual's FP32 band."""
    from bounds import bf16_spacing, mlp_output_bound
    sc = scenegen.make_scene("sphere128", seed=5)
    R0, t0 = sc.R_init.numpy(), sc.t_init.numpy()
    c0 = O.centres_from_poses(R0, t0)
    prob = O.Problem.from_scene(sc)
    if storage == "fp16":
        _, d1, d2 = O.fp16_centroid_storage(prob, sc.x1.numpy(), sc.x2.numpy())
        prob = O.Problem(sc.n_cams, prob.cam_i, prob.cam_j, prob.pair_id, d1, d2)
    score = sc.score.numpy()
    tau0, tau1, delta = 0.3, 0.2, 1e-6
    pv = _params(7)
    net = fm.Mlp(pv)
    feats = torch.empty(sc.n_pp, 8, dtype=torch.bfloat16, device="cuda")
    with fm.Problem(R0, t0, sc.cam_i, sc.cam_j, sc.pair_id, sc.x1, sc.x2,
                    options=fm.default_options(storage=storage, delta=delta)) as gp:
        gp.set_scores(score)
        gp.collect_features(tau0, 0, feats)          # round 0: history = current residuals
        f0 = feats.to(torch.float32).cpu().numpy()
        gp.step(5)                                    # move the poses
        R5, c5 = gp.get_params()
        if fused:                                     # round 1, history from round 0
            kept = gp.step_learned(net, tau1, tau1, 1, 1, count=True)
        else:
            kept = gp.learned_weights(net, tau1, tau1, 1)
        w_gpu = gp.get_weights().astype(np.float64)
    e0 = np.abs(O.residuals(prob, R0, c0))
    e5 = np.abs(O.residuals(prob, R5, c5))
    sc16 = score.astype(np.float16).astype(np.float64)
    # round-0 features: every one within its FP32 error plus one BF16 spacing
    F0 = L.features(e0, e0, sc16, prob.pair_id, prob.n_pairs, tau0, 0)
    dX0 = _feature_errors(L, e0, e0, prob.pair_id, prob.n_pairs, tau0)
    dX0[:, 2] = 2 * (2e-6 / (e0 + 1e-6) + 3 * 2.0 ** -23 * np.abs(np.log(e0 + 1e-6)) + 1e-6)
    dX0[:, 7] = dX0[:, 0]
    assert (np.abs(f0 - L.bf16_round(F0)) <= dX0 + bf16_spacing(F0) + 1e-12).all()
    # round-1 weights with the round-0 residuals as history (stored in FP16)
    hist = np.log(e0 + 1e-6).astype(np.float16).astype(np.float64)
    e_prev = np.exp(hist) - 1e-6
    F1 = L.features(e5, e_prev, sc16, prob.pair_id, prob.n_pairs, tau1, 1)
    dX1 = _feature_errors(L, e5, e0, prob.pair_id, prob.n_pairs, tau1)
    params = L.unflatten(pv.astype(np.float64))
    p_or, dp = mlp_output_bound(L, params, F1, dX1)
    m = np.maximum(e5, delta)
    w_or = np.where(e5 <= tau1, p_or / m, 0.0)
    dw = dp / m + p_or * 2e-6 / (m * m) + 4 * 2.0 ** -24 * w_or
    if storage == "fp16":
        dw += 2.0 ** -11 * w_or + 2.0 ** -24
    decided = np.abs(e5 - tau1) > 2e-6
    assert ((w_gpu > 0) == (e5 <= tau1))[decided].all()
    err = np.abs(w_gpu - w_or)[decided]
    assert (err <= dw[decided]).all(), (err / dw[decided]).max()
    assert abs(kept - (e5 <= tau1).sum()) <= int((~decided).sum())


def test_trained_network_gains_over_plain_reweighting():
    # held-out scene of the training shape (128-camera sphere, here with 30% outliers; the
    # network was trained on seeds 1000-1199): after the same 10 rounds the learned weights
    # leave a clearly smaller rotation error than the hard IRLS mask
    import os
    from paper_2605_18052_gb300 import metrics
    path = os.path.join(os.path.dirname(fm.__file__), "data", "mlp_inlier.npy")
    sc = scenegen.make_scene("sphere128_o30", seed=8, device="cuda")
    sch = learned.default_schedule(sc, 10)
    Rg = sc.R_gt.cpu().numpy()
    err = {}
    for arm in ("irls", "learned"):
        with fm.Problem(sc.R_init.cpu(), sc.t_init.cpu(), sc.cam_i.cpu(), sc.cam_j.cpu(), sc.pair_id, sc.x1,
                        sc.x2, options=sch.options(storage="fp16")) as gp:
            gp.set_scores(sc.score)
            if arm == "irls":
                fm.refine(gp, sch)
            else:
                net = fm.Mlp(np.load(path))
                learned.refine_learned(gp, net, sch)
                net.close()
            err[arm] = float(metrics.rotation_error_deg(gp.get_poses()[0], Rg).mean())
    assert err["learned"] < 0.5 * err["irls"], err


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_fused_learned_round_is_bit_identical(storage):
    # fm_step_learned = fm_learned_weights + fm_step with the learned reweighting inside the first
    # pass; two rounds, so the second one reads the residual history the first one wrote
    sc = scenegen.make_scene("sphere128", seed=9)
    R0, t0 = sc.R_init.numpy(), sc.t_init.numpy()
    net = fm.Mlp(_params(11))
    res = []
    for fused in (False, True):
        with fm.Problem(R0, t0, sc.cam_i, sc.cam_j, sc.pair_id, sc.x1, sc.x2,
                        options=fm.default_options(storage=storage)) as gp:
            gp.set_scores(sc.score.numpy())
            kept = []
            for rnd, tau in enumerate((0.3, 0.2)):
                if fused:
                    kept.append(gp.step_learned(net, tau, tau, rnd, 7, count=True))
                else:
                    kept.append(gp.learned_weights(net, tau, tau, rnd))
                    gp.step(7)
            res.append((kept, gp.get_weights(), gp.get_params(), gp.last_loss(), gp.get_state()[2]))
    (k0, w0, p0, l0, s0), (k1, w1, p1, l1, s1) = res
    assert k0 == k1 and s0 == s1 == 14 and l0 == l1
    np.testing.assert_array_equal(w0, w1)
    np.testing.assert_array_equal(p0[0], p1[0])
    np.testing.assert_array_equal(p0[1], p1[1])
