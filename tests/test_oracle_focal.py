"""Pins of the focal-refinement oracle (fundamental matrices F = S_j E S_i with per-camera
scales of the normalised keypoints) against facts that do not restate its formulas."""
import numpy as np
import pytest

import oracle as O
from oracle import focal as Fo
import scenegen


def _scene(seed=0):
    sc = scenegen.make_scene("ring16", seed=seed)
    prob = O.Problem.from_scene(sc)
    return sc, prob


def test_unit_scales_reduce_to_the_pose_objective():
    sc, prob = _scene()
    R, t = sc.R_init.numpy(), sc.t_init.numpy()
    c = O.centres_from_poses(R, t)
    w = np.random.default_rng(0).uniform(0, 5, prob.n_pp)
    l0, g0 = O.loss_grad(prob, R, c, w)
    l1, g1, gr = Fo.loss_grad(prob, R, c, np.zeros(sc.n_cams), w)
    assert l1 == l0
    np.testing.assert_array_equal(g1, g0)
    np.testing.assert_allclose(Fo.residuals(prob, R, c, np.zeros(sc.n_cams)), O.residuals(prob, R, c), atol=1e-15)


def test_wrongly_normalised_keypoints_are_undone_by_the_true_scales():
    # keypoints normalised with f0 = f (1 + d_k): the residuals at the true poses vanish (noise
    # free) exactly when s_k = f0_k / f = 1 + d_k
    sc = scenegen.make_scene("ring16", seed=1, sigma_px=0.0, outlier=0.0)
    prob = O.Problem.from_scene(sc)
    d = np.random.default_rng(1).uniform(-0.1, 0.1, sc.n_cams)
    s_true = 1.0 + d
    ci, cj = prob.cam_i[prob.pair_id], prob.cam_j[prob.pair_id]
    bad = O.Problem(sc.n_cams, prob.cam_i, prob.cam_j, prob.pair_id, prob.x1 / s_true[ci][:, None],
                    prob.x2 / s_true[cj][:, None])
    R = sc.R_gt.numpy()
    c = O.centres_from_poses(R, sc.t_gt.numpy())
    assert np.abs(Fo.residuals(bad, R, c, np.log(s_true))).max() < 1e-6   # FP32 keypoints
    assert np.abs(Fo.residuals(bad, R, c, np.zeros(sc.n_cams))).max() > 1e-3


def test_scale_gradient_central_differences():
    sc, prob = _scene(2)
    R, t = sc.R_init.numpy(), sc.t_init.numpy()
    c = O.centres_from_poses(R, t)
    rng = np.random.default_rng(3)
    rho = 0.05 * rng.normal(size=sc.n_cams)
    w = rng.uniform(0, 5, prob.n_pp)
    _, _, g = Fo.loss_grad(prob, R, c, rho, w)
    h = 1e-6
    for k in (0, 5, 11):
        rp, rm = rho.copy(), rho.copy()
        rp[k] += h
        rm[k] -= h
        fd = (Fo.loss_grad(prob, R, c, rp, w)[0] - Fo.loss_grad(prob, R, c, rm, w)[0]) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-6, abs=1e-12)


def test_fundamental_matrix_has_the_essential_rank():
    sc, prob = _scene(3)
    R, t = sc.R_init.numpy(), sc.t_init.numpy()
    F = Fo.fundamental(prob, R, O.centres_from_poses(R, t), np.exp(0.1 * np.random.default_rng(4).normal(size=sc.n_cams)))
    sv = np.linalg.svd(F, compute_uv=False)
    assert np.abs(sv[:, 2]).max() < 1e-12 * np.abs(sv[:, 0]).max()
