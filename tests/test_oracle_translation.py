"""Pins of the global-translation oracle (Eq. fastmap-global-translation-objective and the
multiple-initialisation merge) against facts that do not restate its formulas."""
import numpy as np
import pytest

import oracle as O
from oracle import translation as T
import scenegen


def _exact_directions(name="ring16", seed=0):
    sc = scenegen.make_scene(name, seed=seed)
    R = sc.R_gt.numpy()
    C = O.centres_from_poses(R, sc.t_gt.numpy())
    ci, cj = sc.cam_i.numpy(), sc.cam_j.numpy()
    # unit relative translation of each pair in camera j's frame, from the true poses
    t = np.stack([R[j] @ (C[i] - C[j]) for i, j in zip(ci, cj)])
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    return R, C, ci, cj, t


def test_direction_is_the_world_baseline():
    R, C, ci, cj, t = _exact_directions()
    o = T.relative_directions(R, t, cj)
    want = (C[cj] - C[ci]) / np.linalg.norm(C[cj] - C[ci], axis=1, keepdims=True)
    np.testing.assert_allclose(o, want, atol=1e-14)


def test_zero_loss_and_a_minimum_at_true_centres():
    # the L1 objective is not differentiable at its zero: check the value and that every
    # small move away from the truth (other than a similarity) increases it
    R, C, ci, cj, t = _exact_directions()
    oij = T.relative_directions(R, t, cj)
    loss, _ = T.loss_grad(C, ci, cj, oij)
    assert loss < 1e-14
    rng = np.random.default_rng(2)
    for _ in range(5):
        moved = C + 1e-4 * rng.normal(size=C.shape)
        assert T.loss_grad(moved, ci, cj, oij)[0] > 1e-6


def test_single_pair_closed_form():
    # o_i = 0, o_j = e_x, target e_y: r = (1, -1, 0), L = 2; the subgradient (1, -1, 0) projected
    # orthogonally to e_x is (0, -1, 0)
    o = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    loss, g = T.loss_grad(o, [0], [1], [[0.0, 1.0, 0.0]])
    assert loss == pytest.approx(2.0)
    np.testing.assert_allclose(g, [[0.0, 1.0, 0.0], [0.0, -1.0, 0.0]], atol=1e-15)


def test_similarity_invariance_and_gauge_identities():
    R, C, ci, cj, t = _exact_directions()
    oij = T.relative_directions(R, t, cj)
    rng = np.random.default_rng(3)
    o = rng.normal(size=C.shape)
    loss, g = T.loss_grad(o, ci, cj, oij)
    for s, d in [(2.5, np.array([1.0, -2.0, 0.5])), (0.01, np.zeros(3))]:
        assert T.loss_grad(s * o + d, ci, cj, oij)[0] == pytest.approx(loss, rel=1e-12)
    # translation invariance: the gradient sums to zero; scale invariance: orthogonal to o
    assert np.abs(g.sum(0)).max() < 1e-14
    assert abs((g * o).sum()) < 1e-14


def test_gradient_central_differences():
    R, C, ci, cj, t = _exact_directions()
    oij = T.relative_directions(R, t, cj)
    rng = np.random.default_rng(5)
    o = rng.normal(size=C.shape)
    _, g = T.loss_grad(o, ci, cj, oij)
    h = 1e-6
    for k, a in [(0, 0), (3, 1), (7, 2), (15, 0)]:
        op, om = o.copy(), o.copy()
        op[k, a] += h
        om[k, a] -= h
        fd = (T.loss_grad(op, ci, cj, oij)[0] - T.loss_grad(om, ci, cj, oij)[0]) / (2 * h)
        assert g[k, a] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_normalize_removes_translation_and_scale():
    rng = np.random.default_rng(1)
    o = rng.normal(size=(10, 3))
    n = T.normalize(o)
    np.testing.assert_allclose(n.mean(0), 0.0, atol=1e-15)
    assert np.linalg.norm(n, axis=1).mean() == pytest.approx(1.0)
    np.testing.assert_allclose(T.normalize(3.0 * o + 7.0), n, atol=1e-13)


def test_camera_losses_by_brute_force():
    # a camera's loss is the mean L1 term over every pair it belongs to, as first or second image
    R, C, ci, cj, t = _exact_directions()
    oij = T.relative_directions(R, t, cj)
    rng = np.random.default_rng(4)
    o = C + 0.2 * rng.normal(size=C.shape)
    terms = []
    for i, j, d in zip(ci, cj, oij):
        u = o[j] - o[i]
        terms.append(np.abs(u / np.linalg.norm(u) - d).sum())
    want = np.zeros(len(C))
    for k in range(len(C)):
        mine = [terms[p] for p in range(len(ci)) if ci[p] == k or cj[p] == k]
        want[k] = np.mean(mine) if mine else 0.0
    np.testing.assert_allclose(T.camera_losses(o, ci, cj, oij), want, rtol=1e-13)


def test_merge_takes_each_camera_from_its_best_run():
    R, C, ci, cj, t = _exact_directions()
    oij = T.relative_directions(R, t, cj)
    a = 2.0 * C + 1.0
    a[3] += np.array([0.5, 0.0, 0.0])        # camera 3 wrong in run a
    b = 0.5 * C - 2.0
    b[5] += np.array([0.0, 0.3, 0.0])        # camera 5 wrong in run b
    la, lb = T.camera_losses(a, ci, cj, oij), T.camera_losses(b, ci, cj, oij)
    assert la[3] > lb[3] and lb[5] > la[5]
    merged = T.merge([a, b], [la, lb])
    np.testing.assert_array_equal(merged[3], T.normalize(b)[3])
    np.testing.assert_array_equal(merged[5], T.normalize(a)[5])


def test_random_initialisations_recover_the_centres():
    R, C, ci, cj, t = _exact_directions("ring16")
    oij = T.relative_directions(R, t, cj)
    inits = np.random.default_rng(0).normal(size=(3,) + C.shape)
    o, loss = T.solve(inits, ci, cj, oij, 500, 500, 0.01)
    err = np.linalg.norm(T.normalize(o) - T.normalize(C), axis=1)
    # Adam with a constant step size hovers within about one step of the optimum
    assert err.max() < 0.01
    assert loss < 0.01
