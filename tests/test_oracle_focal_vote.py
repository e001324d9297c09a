"""Pins of the focal-vote oracle (Sec. "Intrinsics Estimation", Eq. fastmap-focal-vote) against
facts that do not restate its formula: on noise-free fundamental matrices the true focal length
makes every pair an essential matrix (ratio 1, vote = number of pairs, the maximum); for a
rank-2 matrix the singular-value ratio has a closed form from the characteristic polynomial of
E^T E; the vote does not change when a fundamental matrix is rescaled or its pair is read in
the other order; with two cameras of different focal lengths, the known side fixed at its true
value makes the other camera's true focal length win. CPU only."""
import numpy as np
import pytest

import oracle as O
from oracle import focal_vote as V
import scenegen


def _scene_F(f_per_cam=None, seed=0):
    sc = scenegen.make_scene("sphere128", seed=seed)
    R = sc.R_gt.numpy()
    C = O.centres_from_poses(R, sc.t_gt.numpy())
    ci, cj = sc.cam_i.numpy(), sc.cam_j.numpy()
    f = np.full(sc.n_cams, 500.0) if f_per_cam is None else f_per_cam
    return V.fundamental_from_poses(R, C, ci, cj, f), ci, cj, sc.n_cams


def test_true_focal_length_makes_every_pair_essential():
    F, _, _, _ = _scene_F()
    B = F.shape[0]
    r = V.singular_ratio(V.essential_from_fundamental(F, np.full(B, 500.0), np.full(B, 500.0)))
    np.testing.assert_allclose(r, 1.0, atol=1e-9)
    cands = np.linspace(300.0, 800.0, 101)            # contains 500 exactly
    f_hat, v = V.estimate(F, cands, tau=0.05)
    assert f_hat == 500.0
    assert v.max() == pytest.approx(B, rel=1e-9)
    assert (v <= B * (1 + 1e-12)).all()
    # away from the truth the essential-matrix property is lost on most pairs
    assert v[np.abs(cands - 500.0) >= 50.0].max() < 0.9 * B


def test_ratio_matches_rank_two_closed_form():
    # det(K2^T F K1) = 0 for any K, so the squared singular values are the non-zero roots of
    # mu^2 - tr(M) mu + m2 = 0, M = E^T E and m2 its sum of principal 2x2 minors
    F, _, _, _ = _scene_F(seed=1)
    for f in (350.0, 500.0, 720.0):
        E = V.essential_from_fundamental(F, np.full(len(F), f), np.full(len(F), f))
        M = np.einsum("nba,nbc->nac", E, E)
        tr = np.trace(M, axis1=1, axis2=2)
        m2 = (M[:, 0, 0] * M[:, 1, 1] - M[:, 0, 1] * M[:, 1, 0] + M[:, 0, 0] * M[:, 2, 2] - M[:, 0, 2] * M[:, 2, 0]
              + M[:, 1, 1] * M[:, 2, 2] - M[:, 1, 2] * M[:, 2, 1])
        disc = np.sqrt(np.maximum(tr * tr - 4 * m2, 0.0))
        ratio = np.sqrt((tr + disc) / np.maximum(tr - disc, 1e-300))
        np.testing.assert_allclose(V.singular_ratio(E), ratio, rtol=1e-7)


def test_vote_invariant_to_scale_and_pair_order():
    F, _, _, _ = _scene_F(seed=2)
    rng = np.random.default_rng(0)
    F = F + 1e-3 * np.abs(F).max(axis=(1, 2), keepdims=True) * rng.normal(size=F.shape)   # noisy
    cands = np.linspace(400.0, 600.0, 21)
    v = V.votes(F, cands, tau=0.1)
    k = rng.uniform(0.1, 10.0, len(F)) * rng.choice([-1.0, 1.0], len(F))
    np.testing.assert_allclose(V.votes(F * k[:, None, None], cands, tau=0.1), v, rtol=1e-10)
    np.testing.assert_allclose(V.votes(np.transpose(F, (0, 2, 1)), cands, tau=0.1), v, rtol=1e-10)


def test_two_cameras_known_side_fixes_the_other():
    # cameras 0..63 have f = 500, the others f = 800; pairs that join the two groups, with the
    # 800 side given as known, vote for the 500 camera; the first image of a pair is side 1
    sc_F, ci, cj, n = _scene_F(np.where(np.arange(128) < 64, 500.0, 800.0), seed=3)
    a = ci < 64
    b = cj < 64
    mixed = a != b
    F = sc_F[mixed]
    k1 = np.where(a[mixed], 0.0, 800.0)        # side 1 is the 500 camera -> candidate
    k2 = np.where(b[mixed], 0.0, 800.0)
    cands = np.linspace(300.0, 900.0, 61)
    f_hat, v = V.estimate(F, cands, 0.05, k1, k2)
    assert f_hat == 500.0 and v.max() == pytest.approx(len(F), rel=1e-9)
    # with the known side misreported the vote no longer reaches the number of pairs
    _, v_bad = V.estimate(F, cands, 0.05, np.where(k1 > 0, 700.0, 0.0), np.where(k2 > 0, 700.0, 0.0))
    assert v_bad.max() < 0.9 * len(F)


def test_rank_one_pairs_contribute_nothing():
    F = np.zeros((3, 3, 3))
    F[:, 0, 0] = 1.0                            # rank 1: lambda_2 = 0
    assert V.votes(F, [500.0], 0.1)[0] == 0.0
