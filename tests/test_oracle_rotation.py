"""Pins of the global-rotation oracle (Eq. fastmap-rotation-objective, the 6D representation and
the column-wise initialisation) against facts that do not restate its formulas."""
import numpy as np
import pytest

import oracle as O
from oracle import rotation as G
import scenegen


def _relative(name="ring16", seed=0, noise_deg=0.0):
    sc = scenegen.make_scene(name, seed=seed)
    R = sc.R_gt.numpy()
    ci, cj = sc.cam_i.numpy(), sc.cam_j.numpy()
    Rrel = np.einsum("nab,ncb->nac", R[cj], R[ci])          # R_j R_i^T
    if noise_deg > 0:
        rng = np.random.default_rng(seed + 1)
        for p in range(len(ci)):
            w = rng.normal(size=3)
            w *= np.radians(noise_deg) / np.linalg.norm(w)
            Rrel[p] = O.expmap(w) @ Rrel[p]
    return R, ci, cj, Rrel


def _random_rotations(n, rng):
    return np.stack([O.expmap(rng.normal(size=3)) for _ in range(n)])


def test_true_columns_are_in_the_null_space_of_the_connection_matrix():
    R, ci, cj, Rrel = _relative()
    A = G.connection_matrix(R.shape[0], ci, cj, Rrel)
    for k in range(3):
        v = R[:, :, k].reshape(-1)
        assert np.abs(A @ v).max() < 1e-12


def test_initialisation_is_exact_on_noise_free_relative_rotations():
    R, ci, cj, Rrel = _relative("sphere128")
    Ri = G.initial_rotations(R.shape[0], ci, cj, Rrel)
    # gauge: camera 0 is the identity, so the answer is R_k R_0^T
    want = np.einsum("nab,cb->nac", R, R[0])
    assert np.abs(Ri - want).max() < 1e-9


def test_initialisation_returns_rotations_on_noisy_input():
    # with inconsistent relative rotations the least-squares columns are not orthogonal by
    # themselves; the result must still be a proper rotation per camera, close to the truth
    R, ci, cj, Rrel = _relative("sphere128", noise_deg=3.0)
    Ri = G.initial_rotations(R.shape[0], ci, cj, Rrel)
    eye = np.tile(np.eye(3), (R.shape[0], 1, 1))
    np.testing.assert_allclose(np.einsum("nba,nbc->nac", Ri, Ri), eye, atol=1e-12)
    np.testing.assert_allclose(np.linalg.det(Ri), 1.0, atol=1e-12)
    assert O.rotation_error_deg(Ri, R).mean() < 3.0


def test_six_d_round_trip_and_orthonormality():
    rng = np.random.default_rng(0)
    Rs = _random_rotations(20, rng)
    np.testing.assert_allclose(G.rot_from_6d(G.six_d_from_rot(Rs)), Rs, atol=1e-13)
    a = rng.normal(size=(20, 6))
    Rr = G.rot_from_6d(a)
    np.testing.assert_allclose(np.einsum("nba,nbc->nac", Rr, Rr), np.tile(np.eye(3), (20, 1, 1)), atol=1e-13)
    np.testing.assert_allclose(np.linalg.det(Rr), 1.0, atol=1e-13)


def test_zero_loss_at_truth_and_gauge_invariance():
    R, ci, cj, Rrel = _relative()
    assert G.loss_grad_R(R, ci, cj, Rrel)[0] < 1e-6      # arccos near 1 amplifies rounding
    rng = np.random.default_rng(1)
    Rn = _random_rotations(R.shape[0], rng)
    Q = O.expmap(np.array([0.3, -0.2, 0.5]))
    l1 = G.loss_grad_R(Rn, ci, cj, Rrel)[0]
    assert G.loss_grad_R(Rn @ Q, ci, cj, Rrel)[0] == pytest.approx(l1, rel=1e-12)


def test_single_pair_geodesic_closed_form():
    th = 0.7
    Rj = O.expmap(np.array([0.0, 0.0, th]))
    loss, _ = G.loss_grad_R(np.stack([np.eye(3), Rj]), [0], [1], [np.eye(3)])
    assert loss == pytest.approx(th, rel=1e-12)


def test_gradient_central_differences_through_6d():
    R, ci, cj, Rrel = _relative(noise_deg=5.0)
    rng = np.random.default_rng(2)
    a = G.six_d_from_rot(_random_rotations(R.shape[0], rng)) + 0.1 * rng.normal(size=(R.shape[0], 6))
    _, g = G.loss_grad_6d(a, ci, cj, Rrel)
    h = 1e-6
    for k, q in [(0, 0), (1, 4), (5, 2), (9, 5), (15, 3)]:
        ap, am = a.copy(), a.copy()
        ap[k, q] += h
        am[k, q] -= h
        fd = (G.loss_grad_6d(ap, ci, cj, Rrel)[0] - G.loss_grad_6d(am, ci, cj, Rrel)[0]) / (2 * h)
        assert g[k, q] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_geodesic_refinement_removes_the_pull_of_wrong_pairs():
    # 5% of the relative rotations replaced by wrong ones: the least-squares initialisation is
    # pulled by them; the robust geodesic objective is not
    R, ci, cj, Rrel = _relative("sphere128", noise_deg=0.5)
    rng = np.random.default_rng(7)
    for p in np.nonzero(rng.random(len(ci)) < 0.05)[0]:
        Rrel[p] = O.expmap(rng.normal(size=3)) @ Rrel[p]
    Ri = G.initial_rotations(R.shape[0], ci, cj, Rrel)
    a, loss = G.adam(G.six_d_from_rot(Ri), ci, cj, Rrel, 300, 1e-3)
    e0 = O.rotation_error_deg(Ri, R).mean()
    e1 = O.rotation_error_deg(G.rot_from_6d(a), R).mean()
    assert loss < G.loss_grad_R(Ri, ci, cj, Rrel)[0]
    assert e0 > 1.0 and e1 < 0.25 * e0
