"""Pins for the FP64 oracle, each against something other than the oracle itself:
closed forms, invariances the geometry fixes, brute force, finite differences and
library routines. None of these needs a GPU."""
import math

import numpy as np
import pytest

import oracle as O
import scenegen


def _tiny_problem(seed=0, n_cams=4, per_pair=40, noise=0.0, outlier=0.0):
    """A handful of cameras around the unit ball, all pairs, FP64 keypoints projected here
    (independently of the oracle) from known points."""
    rng = np.random.default_rng(seed)
    ang = np.arange(n_cams) * 2 * np.pi / n_cams + rng.uniform(-0.2, 0.2, n_cams)
    C = np.stack([3 * np.cos(ang), 3 * np.sin(ang), rng.uniform(-0.5, 0.5, n_cams)], 1)
    R = []
    for k in range(n_cams):
        z = -C[k] / np.linalg.norm(C[k])
        y = -(np.array([0, 0, 1.0]) - z[2] * z)
        y /= np.linalg.norm(y)
        x = np.cross(y, z)
        Rk = np.stack([x, y, z])
        Rk = O.expmap(rng.normal(0, 0.05, 3)) @ Rk
        R.append(Rk)
    R = np.array(R)
    pairs = [(i, j) for i in range(n_cams) for j in range(i + 1, n_cams)]
    cam_i = np.array([p[0] for p in pairs], np.int32)
    cam_j = np.array([p[1] for p in pairs], np.int32)
    pid, x1, x2 = [], [], []
    for n, (i, j) in enumerate(pairs):
        X = rng.normal(0, 0.4, (per_pair, 3))
        for k, xs in ((i, x1), (j, x2)):
            Xc = (R[k] @ (X - C[k]).T).T
            xs.append(Xc[:, :2] / Xc[:, 2:3] + noise * rng.normal(size=(per_pair, 2)))
        pid.append(np.full(per_pair, n, np.int32))
    x1, x2, pid = np.concatenate(x1), np.concatenate(x2), np.concatenate(pid)
    if outlier:
        bad = rng.random(len(pid)) < outlier
        x2[bad] = rng.uniform(-0.6, 0.6, (bad.sum(), 2))
    return O.Problem(n_cams, cam_i, cam_j, pid, x1, x2), R, C


def _perturb(R, C, rng, rot=0.05, tr=0.1):
    R2 = np.array([O.expmap(rng.normal(0, rot, 3)) @ r for r in R])
    return R2, C + rng.normal(0, tr, C.shape)


# ---- residual ---------------------------------------------------------------------------------
def test_zero_residual_at_true_poses_noise_free():
    prob, R, C = _tiny_problem()
    eps = O.residuals(prob, R, C)
    assert np.abs(eps).max() < 1e-13


def test_zero_residual_scene_generator():
    # the generator's FP32 keypoints are exact projections up to FP32 rounding
    sc = scenegen.make_scene("ring16", seed=2, sigma_px=0.0, outlier=0.0)
    prob = O.Problem.from_scene(sc)
    R = sc.R_gt.numpy()
    c = O.centres_from_poses(R, sc.t_gt.numpy())
    assert np.abs(O.residuals(prob, R, c)).max() < 2e-7


def test_rectified_stereo_closed_form():
    # R_i = R_j = I, camera j one unit along -x from camera i: t_n = (1,0,0),
    # E = [e1]_x, and x2^T E x1 = y1 - y2 (textbook rectified pair).
    rng = np.random.default_rng(1)
    x1 = rng.uniform(-1, 1, (50, 2))
    x2 = rng.uniform(-1, 1, (50, 2))
    prob = O.Problem(2, [0], [1], np.zeros(50, np.int32), x1, x2)
    R = np.stack([np.eye(3), np.eye(3)])
    c = np.array([[0.0, 0, 0], [-1.0, 0, 0]])
    np.testing.assert_allclose(O.residuals(prob, R, c), x1[:, 1] - x2[:, 1], rtol=0, atol=1e-15)
    E = O.essential(prob, R, c)[0]
    np.testing.assert_allclose(E, [[0, 0, 0], [0, 0, -1], [0, 1, 0]], atol=1e-15)


def test_translation_scale_does_not_change_residual():
    prob, R, C = _tiny_problem(noise=0.01)
    rng = np.random.default_rng(3)
    R1, C1 = _perturb(R, C, rng)
    np.testing.assert_allclose(O.residuals(prob, R1, C1), O.residuals(prob, R1, 7.5 * C1),
                               rtol=1e-12, atol=1e-15)


# ---- losses -------------------------------------------------------------------------------------
def test_quadratic_form_identity_brute_force():
    # (1/Z) sum_m (x2^T E x1)^2 == (1/Z) sum_n e_n^T W_n e_n (Eq. epipolar-objective-l2, factor 1/Z)
    prob, R, C = _tiny_problem(noise=0.01, outlier=0.2)
    rng = np.random.default_rng(4)
    R1, C1 = _perturb(R, C, rng)
    w = rng.uniform(0.1, 3.0, prob.n_pp)
    direct, _ = O.loss_grad(prob, R1, C1, w)
    brute = sum(w[p] * O.residuals(prob, R1, C1)[p] ** 2 for p in range(prob.n_pp)) / prob.n_pp
    qf = O.quadratic_form_loss(prob, R1, C1, w)
    assert direct == pytest.approx(brute, rel=1e-12)
    assert direct == pytest.approx(qf, rel=1e-12)


def test_l1_loss_is_mean_absolute_residual():
    prob, R, C = _tiny_problem(noise=0.02)
    rng = np.random.default_rng(5)
    R1, C1 = _perturb(R, C, rng)
    l1, _ = O.loss_grad(prob, R1, C1, mode="l1")
    assert l1 == pytest.approx(np.abs(O.residuals(prob, R1, C1)).mean(), rel=1e-13)


def test_similarity_invariance():
    prob, R, C = _tiny_problem(noise=0.01, outlier=0.1)
    rng = np.random.default_rng(6)
    R1, C1 = _perturb(R, C, rng)
    w = rng.uniform(0.5, 2.0, prob.n_pp)
    base_l2, _ = O.loss_grad(prob, R1, C1, w)
    base_l1, _ = O.loss_grad(prob, R1, C1, mode="l1")
    for trial in range(3):
        s = 10 ** rng.uniform(-1, 1)
        Q = O.expmap(rng.normal(0, 1, 3))
        d = rng.normal(0, 5, 3)
        # world X' = s Q X + d: rotations R Q^T, centres s Q c + d
        R2 = np.einsum("nab,cb->nac", R1, Q)
        C2 = s * (C1 @ Q.T) + d
        assert O.loss_grad(prob, R2, C2, w)[0] == pytest.approx(base_l2, rel=1e-11)
        assert O.loss_grad(prob, R2, C2, mode="l1")[0] == pytest.approx(base_l1, rel=1e-11)


def test_pair_orientation_swap_invariance():
    prob, R, C = _tiny_problem(noise=0.01)
    rng = np.random.default_rng(7)
    R1, C1 = _perturb(R, C, rng)
    swapped = O.Problem(prob.n_cams, prob.cam_j, prob.cam_i, prob.pair_id, prob.x2, prob.x1)
    np.testing.assert_allclose(O.residuals(swapped, R1, C1), O.residuals(prob, R1, C1),
                               rtol=1e-11, atol=1e-14)
    g1 = O.loss_grad(prob, R1, C1)[1]
    g2 = O.loss_grad(swapped, R1, C1)[1]
    np.testing.assert_allclose(g1, g2, rtol=1e-9, atol=1e-13 * np.abs(g1).max())


def test_camera_permutation_invariance():
    prob, R, C = _tiny_problem(noise=0.01, n_cams=5)
    rng = np.random.default_rng(8)
    R1, C1 = _perturb(R, C, rng)
    perm = rng.permutation(5)
    inv = np.argsort(perm)  # new index of old camera k is inv[k]
    p2 = O.Problem(5, inv[prob.cam_i], inv[prob.cam_j], prob.pair_id, prob.x1, prob.x2)
    l1, g1 = O.loss_grad(prob, R1, C1)
    l2, g2 = O.loss_grad(p2, R1[perm], C1[perm])
    assert l2 == pytest.approx(l1, rel=1e-13)
    np.testing.assert_allclose(g2, g1[perm], rtol=1e-10, atol=1e-14)


# ---- gradient -------------------------------------------------------------------------------------
def _fd_grad(prob, R, C, w, mode, h_rot=1e-6, h_c=1e-6):
    g = np.zeros((prob.n_cams, 6))
    for k in range(prob.n_cams):
        for q in range(6):
            Rp, Rm, Cp, Cm = R.copy(), R.copy(), C.copy(), C.copy()
            if q < 3:
                e = np.zeros(3)
                e[q] = h_rot
                Rp[k] = O.expmap(e) @ R[k]
                Rm[k] = O.expmap(-e) @ R[k]
                h = h_rot
            else:
                Cp[k, q - 3] += h_c
                Cm[k, q - 3] -= h_c
                h = h_c
            g[k, q] = (O.loss_grad(prob, Rp, Cp, w, mode)[0] - O.loss_grad(prob, Rm, Cm, w, mode)[0]) / (2 * h)
    return g


@pytest.mark.parametrize("mode", ["irls", "l1"])
def test_gradient_central_differences(mode):
    prob, R, C = _tiny_problem(noise=0.02, outlier=0.1)
    rng = np.random.default_rng(9)
    R1, C1 = _perturb(R, C, rng)
    w = rng.uniform(0.2, 2.0, prob.n_pp) if mode == "irls" else None
    _, g = O.loss_grad(prob, R1, C1, w, mode)
    fd = _fd_grad(prob, R1, C1, w, mode)
    assert np.abs(fd - g).max() <= 1e-6 * np.abs(g).max()


def test_gradient_gauge_identities():
    # the loss is invariant to world similarities, so the gradient is orthogonal to the
    # 7 gauge directions: sum_k g_c = 0 (translation), sum_k c.g_c = 0 (scale),
    # sum_k (-R_k^T g_phi + c_k x g_c) = 0 (rotation).
    prob, R, C = _tiny_problem(noise=0.02, outlier=0.1, n_cams=5)
    rng = np.random.default_rng(10)
    R1, C1 = _perturb(R, C, rng)
    _, g = O.loss_grad(prob, R1, C1, rng.uniform(0.5, 2, prob.n_pp))
    scale = np.abs(g).max() * max(1.0, np.abs(C1).max())
    assert np.abs(g[:, 3:].sum(0)).max() < 1e-12 * scale
    assert abs((C1 * g[:, 3:]).sum()) < 1e-12 * scale
    rot = -np.einsum("nba,nb->a", R1, g[:, :3]) + np.cross(C1, g[:, 3:]).sum(0)
    assert np.abs(rot).max() < 1e-12 * scale


def test_gradient_zero_at_true_poses_noise_free():
    prob, R, C = _tiny_problem()
    _, g = O.loss_grad(prob, R, C)
    assert np.abs(g).max() < 1e-14


# ---- IRLS ---------------------------------------------------------------------------------------
def test_irls_equals_l1_at_reweighting_point():
    # with w = 1/|eps^| taken at the current poses (no filtering, floor inactive) the
    # weighted L2 loss equals the L1 loss and its gradient is twice the L1 gradient.
    prob, R, C = _tiny_problem(noise=0.02, outlier=0.1)
    rng = np.random.default_rng(11)
    R1, C1 = _perturb(R, C, rng)
    eps = O.residuals(prob, R1, C1)
    assert np.abs(eps).min() > 1e-9
    w, kept = O.irls_weights(eps, math.inf, 1e-12)
    assert kept == prob.n_pp
    lw, gw = O.loss_grad(prob, R1, C1, w)
    l1, g1 = O.loss_grad(prob, R1, C1, mode="l1")
    assert lw == pytest.approx(l1, rel=1e-12)
    np.testing.assert_allclose(gw, 2 * g1, rtol=1e-10, atol=1e-12 * np.abs(g1).max())


def test_irls_filter_and_floor_closed_form():
    eps = np.array([0.0, 1e-9, -2e-6, 0.01, -0.02, 0.05, 0.5, -0.5000001])
    w, kept = O.irls_weights(eps, 0.5, 1e-6)
    expect = [1e6, 1e6, 5e5, 100.0, 50.0, 20.0, 2.0, 0.0]
    np.testing.assert_allclose(w, expect, rtol=1e-15)
    assert kept == 7


def test_threshold_schedule():
    assert [O.threshold_schedule(r, 0.05, 0.004, 0.5) for r in range(6)] == \
        [0.05, 0.025, 0.0125, 0.00625, 0.004, 0.004]
    assert O.threshold_schedule(3, 0.5, 0.008) == pytest.approx(0.5 * 0.8 ** 3)
    assert O.threshold_schedule(40, 0.5, 0.008) == 0.008


# ---- optimiser ----------------------------------------------------------------------------------
def test_expmap_against_library_and_series():
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(12)
    for _ in range(20):
        phi = rng.normal(0, 1.0, 3)
        np.testing.assert_allclose(O.expmap(phi), Rot.from_rotvec(phi).as_matrix(), atol=1e-14)
    phi = np.array([1e-9, -2e-9, 3e-9])
    K = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
    np.testing.assert_allclose(O.expmap(phi), np.eye(3) + K + K @ K / 2, atol=1e-17)
    Rm = O.expmap(rng.normal(0, 2, 3))
    assert np.abs(Rm.T @ Rm - np.eye(3)).max() < 1e-14
    assert np.linalg.det(Rm) == pytest.approx(1.0, abs=1e-14)


def test_adam_first_step_closed_form():
    # first Adam step: m^ = g, v^ = g^2, so each parameter moves by -lr * sign(g)
    R = np.stack([np.eye(3), O.expmap([0.1, 0.2, 0.3])])
    c = np.array([[0.0, 1, 2], [3, 4, 5]])
    g = np.array([[0.5, -2.0, 1e-3, 3.0, -1.0, 2.0], [-1, 1, -1, 1, -1, 1.0]])
    m = np.zeros((2, 6))
    v = np.zeros((2, 6))
    R0, c0 = R.copy(), c.copy()
    O.adam_step(R, c, g, m, v, 1, 0.01, 0.1, eps=0.0)
    np.testing.assert_allclose(c, c0 - 0.1 * np.sign(g[:, 3:]), atol=1e-15)
    for k in range(2):
        np.testing.assert_allclose(R[k], O.expmap(-0.01 * np.sign(g[k, :3])) @ R0[k], atol=1e-14)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_adam_bias_correction_under_a_constant_gradient():
    # with the same gradient every step, the bias-corrected moments are exactly g and g^2 at
    # every step number, so each step moves every parameter by lr * sign(g); a wrong bias
    # correction (or step count) changes the step length from the second step on
    rng = np.random.default_rng(21)
    g = rng.normal(size=(3, 6))
    R = np.stack([O.expmap(rng.normal(size=3)) for _ in range(3)])
    c = rng.normal(size=(3, 3))
    m = np.zeros((3, 6))
    v = np.zeros((3, 6))
    R0, c0 = R.copy(), c.copy()
    lr_r, lr_c = 1e-3, 2e-2
    for k in range(1, 8):
        O.adam_step(R, c, g, m, v, k, lr_r, lr_c, beta1=0.8, beta2=0.95, eps=0.0)
        np.testing.assert_allclose(c, c0 - k * lr_c * np.sign(g[:, 3:]), atol=1e-13)
        for q in range(3):
            # the same increment k times about a fixed axis is one turn of k times its angle
            np.testing.assert_allclose(R[q], O.expmap(-k * lr_r * np.sign(g[q, :3])) @ R0[q], atol=1e-12)


def test_project_rotation_nearest():
    rng = np.random.default_rng(13)
    Q = O.expmap(rng.normal(size=3))
    noisy = Q + 1e-4 * rng.normal(size=(3, 3))
    P = O.project_rotation(noisy)[0]
    assert np.abs(P.T @ P - np.eye(3)).max() < 1e-14
    assert np.abs(P - Q).max() < 3e-4


def test_refine_moves_towards_truth_noise_free():
    sc = scenegen.make_scene("ring16", seed=3, sigma_px=0.0, outlier=0.0)
    prob = O.Problem.from_scene(sc)
    Rg = sc.R_gt.numpy()
    cg = O.centres_from_poses(Rg, sc.t_gt.numpy())
    R0 = sc.R_init.numpy()
    c0 = O.centres_from_poses(R0, sc.t_init.numpy())
    l0 = O.loss_grad(prob, R0, c0)[0]
    e0 = O.rotation_error_deg(R0, Rg).mean()
    base = np.median(np.linalg.norm(cg[prob.cam_i] - cg[prob.cam_j], axis=1))
    R, c, _ = O.refine(prob, R0, c0, 12, 25, 1.0, 1.0, 1e-9, 1e-2, 1e-2 * base, 0.95,
                       weight_fn=lambda w: np.ones_like(w))
    assert O.loss_grad(prob, R, c)[0] < 1e-2 * l0
    assert O.rotation_error_deg(R, Rg).mean() < e0 / 3


# ---- metrics -------------------------------------------------------------------------------------
def test_rotation_error_gauge_and_known_error():
    rng = np.random.default_rng(14)
    Rg = np.array([O.expmap(rng.normal(size=3)) for _ in range(200)])
    Q = O.expmap(rng.normal(size=3))
    assert O.rotation_error_deg(Rg @ Q, Rg).max() < 1e-5  # arccos near 1: ~sqrt(ulp)
    Rb = Rg @ Q
    Rb[5] = O.expmap(np.radians(2.0) * np.array([0, 0, 1.0])) @ Rb[5]
    e = O.rotation_error_deg(Rb, Rg)
    assert e[5] == pytest.approx(2.0, abs=0.03)
    assert np.median(e) < 0.03


def test_translation_error_similarity_invariant():
    prob, R, C = _tiny_problem()
    rng = np.random.default_rng(15)
    Q = O.expmap(rng.normal(size=3))
    R2 = np.einsum("nab,cb->nac", R, Q)
    C2 = 3.0 * (C @ Q.T) + rng.normal(size=3)
    assert O.translation_error_deg(R2, C2, R, C, prob.cam_i, prob.cam_j).max() < 1e-5


# ---- FP16 storage rule ---------------------------------------------------------------------------
def test_fp16_centroid_rule_brute_force():
    from fractions import Fraction
    sc = scenegen.make_scene("ring16", seed=4)
    sub = sc.pair_id.numpy() < 6
    prob = O.Problem(sc.n_cams, sc.cam_i.numpy(), sc.cam_j.numpy(), sc.pair_id.numpy()[sub],
                     sc.x1.numpy()[sub], sc.x2.numpy()[sub])
    x1 = sc.x1.numpy()[sub]
    x2 = sc.x2.numpy()[sub]
    cen, d1, d2 = O.fp16_centroid_storage(prob, x1, x2)
    for k in range(prob.n_cams):
        vals = [x1[p] for p in range(prob.n_pp) if prob.cam_i[prob.pair_id[p]] == k]
        vals += [x2[p] for p in range(prob.n_pp) if prob.cam_j[prob.pair_id[p]] == k]
        if not vals:
            assert (cen[k] == 0).all()
            continue
        for a in range(2):
            exact = sum(Fraction(float(v[a])) for v in vals) / len(vals)
            assert abs(float(exact) - float(cen[k, a])) <= 2.0 ** -31 + abs(float(exact)) * 2.0 ** -23
    # dequantized offsets are within half an FP16 ulp of the FP32 difference
    for x, d, cam in ((x1, d1, prob.cam_i), (x2, d2, prob.cam_j)):
        off = x.astype(np.float32) - cen[cam[prob.pair_id]]
        ulp = np.spacing(np.abs(off).astype(np.float16)).astype(np.float64)
        stored = d - cen[cam[prob.pair_id]].astype(np.float64)
        assert (np.abs(stored - off) <= 0.5 * ulp + 1e-12).all()
        # and the stored offsets are FP16 numbers (the storage is FP16, not merely close to it)
        assert np.array_equal(stored.astype(np.float16).astype(np.float64), stored)


def test_fp16_weight_quantization():
    delta = 1e-6
    s = O.fp16_weight_scale(delta)
    assert s == 2.0 ** -5 and (1 / delta) * s <= 32768
    w = np.array([0.0, 1.0, 20.0, 1e3, 5e5, 1e6])
    q = O.quantize_weights_fp16(w, delta)
    np.testing.assert_allclose(q, w, rtol=2.0 ** -11)
    assert q[0] == 0.0
