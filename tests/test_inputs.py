"""The seeded input generators keep their contract (no method arithmetic is involved): every
scene has the outlier fraction its configuration names, every image pair has point pairs and
every camera takes part in a pair; match scores follow Beta(4, 2) for inliers and Beta(2, 3) for
outliers; initial poses are turned by exactly 5 degrees and moved by 10% of the stated distance;
the closed trajectory closes on itself and links every lap to the others; and the relative
rotations and translations handed to the global stages carry the stated noise and wrong-pair
fraction."""
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


def test_loop_scene_closes_and_links_laps():
    # a reduced copy of the 1,000-camera closed trajectory (same layout and view graph, fewer
    # points and matches so that it builds in seconds on the CPU)
    sc = scenegen.make_scene("loop1000_o30", seed=0, n_pts=20_000, counts=("lognormal", 60.0, 0.9, 400))
    n = sc.n_cams
    R = sc.R_gt.numpy()
    C = O.centres_from_poses(R, sc.t_gt.numpy())
    ci, cj = sc.cam_i.numpy(), sc.cam_j.numpy()
    assert n == 1000 and (ci < cj).all() and len(set(zip(ci, cj))) == len(ci)
    assert abs(sc.outlier.numpy().mean() - 0.30) < 0.01
    assert np.bincount(sc.pair_id.numpy(), minlength=sc.n_pairs).min() > 0
    # the path closes: the last camera is as close to the first as neighbours are to each other
    step = np.linalg.norm(np.diff(C, axis=0), axis=1)
    assert np.linalg.norm(C[-1] - C[0]) < 2 * step.max()
    # every camera looks at the point cloud: its optical axis passes within 1 of the origin
    z = R[:, 2, :]                                    # viewing direction in world coordinates
    miss = np.linalg.norm(np.cross(z, -C), axis=1)   # distance of the origin from the axis
    assert (miss < 1.0).all()
    # 8 neighbours along the path and 12 views of other laps (more than a quarter lap away
    # along the path) for every camera
    steps = np.abs(ci - cj)
    steps = np.minimum(steps, n - steps)
    far = steps > n // (4 * 20)
    deg_far = np.bincount(np.concatenate([ci[far], cj[far]]), minlength=n)
    assert deg_far.min() >= 12 and far.mean() > 0.4
    assert ((steps <= 4) | far).all()
    # the height sweeps +-70 degrees of elevation, so the laps cover the view sphere's band
    elev = np.degrees(np.arcsin(C[:, 2] / np.linalg.norm(C, axis=1)))
    assert elev.min() < -60 and elev.max() > 60
    # initial centres moved by 10% of the median pair baseline
    base = np.median(np.linalg.norm(C[ci] - C[cj], axis=1))
    C0 = O.centres_from_poses(sc.R_init.numpy(), sc.t_init.numpy())
    np.testing.assert_allclose(np.linalg.norm(C0 - C, axis=1), 0.1 * base, rtol=1e-9)


def test_fundamental_matrices_annihilate_true_matches():
    # noise-free matches of a noise-free scene satisfy x2^T F x1 = 0 in pixels from the image
    # centre, and the wrong-pair fraction is as asked
    sc = scenegen.make_scene("ring16", seed=3, sigma_px=0.0, outlier=0.0)
    F, wrong = scenegen.fundamental_matrices(sc, noise=0.0, wrong_frac=0.0)
    assert not wrong.any()
    p1 = np.concatenate([sc.x1.numpy().astype(np.float64) * sc.f, np.ones((sc.n_pp, 1))], 1)
    p2 = np.concatenate([sc.x2.numpy().astype(np.float64) * sc.f, np.ones((sc.n_pp, 1))], 1)
    Fp = F[sc.pair_id.numpy()]
    r = np.einsum("pa,pab,pb->p", p2, Fp, p1) / (np.linalg.norm(Fp, axis=(1, 2)) * sc.f * sc.f)
    assert np.abs(r).max() < 1e-6
    _, wrong = scenegen.fundamental_matrices(scenegen.make_scene("sphere128", seed=3), wrong_frac=0.1)
    assert abs(wrong.mean() - 0.1) < 0.03
