"""The seeded input generators deliver what the design notes state (no method arithmetic is
involved): sizes, outlier fractions, match-score distributions and the relative-pose inputs of
the global stages."""
import numpy as np
import pytest

import oracle as O
import scenegen


def test_scene_sizes_and_outlier_fractions():
    for name, frac in (("ring16", 0.10), ("sphere128", 0.15), ("sphere128_o30", 0.30)):
        sc = scenegen.make_scene(name, seed=0)
        out = sc.outlier.numpy()
        assert abs(out.mean() - frac) < 0.01, (name, out.mean())
        assert sc.n_pp == len(out) == sc.x1.shape[0] == sc.x2.shape[0]
        # every pair has point pairs, every camera takes part in a pair
        assert np.bincount(sc.pair_id.numpy(), minlength=sc.n_pairs).min() > 0
        assert set(np.concatenate([sc.cam_i.numpy(), sc.cam_j.numpy()])) == set(range(sc.n_cams))


def test_match_scores_overlap_but_separate_on_average():
    sc = scenegen.make_scene("sphere128", seed=1)
    s, out = sc.score.numpy(), sc.outlier.numpy()
    # Beta(4, 2) for inliers (mean 2/3), Beta(2, 3) for outliers (mean 2/5)
    assert abs(s[~out].mean() - 2 / 3) < 0.01 and abs(s[out].mean() - 0.4) < 0.01
    assert (s[out] > 0.5).mean() > 0.2 and (s[~out] < 0.5).mean() > 0.1


def test_initial_perturbation_sizes():
    sc = scenegen.make_scene("sphere128", seed=2)
    R0, R = sc.R_init.numpy(), sc.R_gt.numpy()
    # every camera turned by exactly 5 degrees about a random axis
    raw = np.degrees(np.arccos(np.clip((np.einsum("nab,nab->n", R0, R) - 1) / 2, -1, 1)))
    np.testing.assert_allclose(raw, 5.0, atol=1e-9)
    # centres moved by 10% of their distance to the scene centre
    C0 = O.centres_from_poses(R0, sc.t_init.numpy())
    C = O.centres_from_poses(R, sc.t_gt.numpy())
    np.testing.assert_allclose(np.linalg.norm(C0 - C, axis=1), 0.1 * np.linalg.norm(C, axis=1), rtol=1e-9)


def test_relative_rotations_noise_and_wrong_pairs():
    sc = scenegen.make_scene("sphere128", seed=3)
    R = sc.R_gt.numpy()
    ci, cj = sc.cam_i.numpy(), sc.cam_j.numpy()
    Rrel, out = scenegen.relative_rotations(sc, 1.0, 0.05, 0)
    true = np.einsum("nab,ncb->nac", R[cj], R[ci])
    ang = np.degrees(np.arccos(np.clip((np.einsum("nab,nab->n", Rrel, true) - 1) / 2, -1, 1)))
    np.testing.assert_allclose(np.einsum("nba,nbc->nac", Rrel, Rrel), np.tile(np.eye(3), (len(ci), 1, 1)), atol=1e-12)
    assert abs(out.mean() - 0.05) < 0.02
    # |N(0, 1 deg)| about the axis: mean sqrt(2/pi) deg
    assert abs(ang[~out].mean() - np.sqrt(2 / np.pi)) < 0.1
    assert ang[out].mean() > 30.0


def test_relative_translations_noise_and_wrong_pairs():
    sc = scenegen.make_scene("sphere128", seed=4)
    R = sc.R_gt.numpy()
    C = O.centres_from_poses(R, sc.t_gt.numpy())
    ci, cj = sc.cam_i.numpy(), sc.cam_j.numpy()
    t, out = scenegen.relative_translations(sc, 1.0, 0.05, 0)
    true = np.einsum("nab,nb->na", R[cj], C[ci] - C[cj])
    true /= np.linalg.norm(true, axis=1, keepdims=True)
    np.testing.assert_allclose(np.linalg.norm(t, axis=1), 1.0, atol=1e-12)
    ang = np.degrees(np.arccos(np.clip((t * true).sum(1), -1, 1)))
    assert abs(out.mean() - 0.05) < 0.02
    assert ang[~out].max() < 5.0 and ang[out].mean() > 30.0
