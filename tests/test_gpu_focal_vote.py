"""Focal-length vote on the GPU (fm_focal_vote, Sec. "Intrinsics Estimation", Eq.
fastmap-focal-vote) against the FP64 oracle on the same fundamental matrices.

Tolerance, from the arithmetic: each term exp((1 - r)/tau) is computed in FP32 from a ratio r
whose FP32 error is a few 1e-7 relative (Jacobi rotations keep nearly equal eigenvalues
accurate), so a term carries a relative error of about 1e-6 / tau plus the FP32 exponential;
with tau >= 0.05 every vote is held to 1e-4 relative (plus 1e-6 of the number of pairs for
votes near zero), and the winning candidate must be the oracle's unless the oracle's two best
votes lie within that tolerance of each other.
"""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import focal_vote as V
import scenegen
import paper_2605_18052_gb300 as fm
from paper_2605_18052_gb300 import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    build.build()
    fm.load_library()


def _noisy_F(name, seed, f_cam=None, noise=1e-3, wrong=0.1, **kw):
    sc = scenegen.make_scene(name, seed=seed, **kw)
    R = sc.R_gt.numpy()
    C = O.centres_from_poses(R, sc.t_gt.numpy())
    ci, cj = sc.cam_i.numpy(), sc.cam_j.numpy()
    f = np.full(sc.n_cams, 500.0) if f_cam is None else f_cam
    F = V.fundamental_from_poses(R, C, ci, cj, f)
    # noise and wrong pairs in calibrated coordinates (where every entry has the same scale),
    # then back to pixels: F = K_j^-T E K_i^-1
    si = np.stack([f[ci], f[ci], np.ones(len(ci))], 1)
    sj = np.stack([f[cj], f[cj], np.ones(len(cj))], 1)
    E = sj[:, :, None] * F * si[:, None, :]
    rng = np.random.default_rng(seed)
    E = E + noise * rng.normal(size=E.shape)
    bad = rng.random(len(E)) < wrong                  # pairs with a wrong fundamental matrix
    E[bad] = rng.normal(size=(int(bad.sum()), 3, 3))
    return E / (sj[:, :, None] * si[:, None, :]), ci, cj


def _check(v_gpu, v_or, B, cands):
    np.testing.assert_allclose(v_gpu, v_or, rtol=1e-4, atol=1e-6 * B)
    top = np.sort(v_or)[-2:]
    if len(top) == 1 or top[1] - top[0] > 2e-4 * top[1]:
        assert cands[int(np.argmax(v_gpu))] == cands[int(np.argmax(v_or))]


@pytest.mark.parametrize("tau", [0.05, 0.2])
def test_focal_vote_matches_oracle(tau):
    F, _, _ = _noisy_F("sphere128", 0)
    cands = np.linspace(300.0, 800.0, 101)
    v_gpu = fm.focal_vote(F, cands, tau)
    v_or = V.votes(F, cands, tau)
    _check(v_gpu, v_or, len(F), cands)
    assert abs(cands[int(np.argmax(v_gpu))] - 500.0) <= 10.0
    # bit-reproducible
    np.testing.assert_array_equal(fm.focal_vote(F, cands, tau), v_gpu)


def test_focal_vote_with_known_sides():
    f_cam = np.where(np.arange(128) < 64, 500.0, 800.0)
    F, ci, cj = _noisy_F("sphere128", 1, f_cam)
    a, b = ci < 64, cj < 64
    mixed = a != b
    k1 = np.where(a[mixed], 0.0, 800.0)
    k2 = np.where(b[mixed], 0.0, 800.0)
    cands = np.linspace(300.0, 900.0, 61)
    v_gpu = fm.focal_vote(F[mixed], cands, 0.05, k1, k2)
    v_or = V.votes(F[mixed], cands, 0.05, k1, k2)
    _check(v_gpu, v_or, int(mixed.sum()), cands)
    assert abs(cands[int(np.argmax(v_gpu))] - 500.0) <= 10.0


def test_focal_vote_ragged_and_degenerate():
    # pair counts that are not a multiple of the block, candidate counts that are not a multiple
    # of the chunk, one candidate, one pair, and rank-1 pairs that contribute nothing
    F, _, _ = _noisy_F("ring16", 2, wrong=0.0)
    for B, nc in ((1, 1), (7, 3), (len(F), 17)):
        cands = np.linspace(420.0, 580.0, nc)
        v_gpu = fm.focal_vote(F[:B], cands, 0.1)
        _check(v_gpu, V.votes(F[:B], cands, 0.1), B, cands)
    R1 = np.zeros((5, 3, 3))
    R1[:, 0, 0] = 1.0
    np.testing.assert_array_equal(fm.focal_vote(R1, [500.0, 600.0], 0.1), 0.0)


def test_focal_vote_rejects_bad_arguments():
    F = np.eye(3)[None].repeat(2, 0)
    for kw in (dict(tau=0.0), dict(tau=float("nan"))):
        with pytest.raises(fm.FastMapError):
            fm.focal_vote(F, [500.0], **kw)
    with pytest.raises(fm.FastMapError):
        fm.focal_vote(F, [-1.0], 0.1)
    with pytest.raises(fm.FastMapError):
        fm.focal_vote(np.zeros((1, 3, 3)), [500.0], 0.1)
    with pytest.raises(fm.FastMapError):
        fm.focal_vote(F, [500.0], 0.1, f1_known=[500.0, -2.0])
