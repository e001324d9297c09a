"""The global translation kernels (fm_translation_*) against the FP64 oracle on the same inputs.

Tolerances: per-pair terms are FP32 computed from the FP64 difference of two centres (unit
vectors, errors of a few 1e-7), per-camera sums FP32 over a few dozen pairs, loss FP64:
loss relative 1e-5, gradient 1e-4 of its largest component (a subgradient component could
differ where a residual component lies within FP32 rounding of 0; random centres keep every
component far from it). Adam runs from random centres follow the oracle closely while the
residuals stay away from 0 (the first iterations): 20 steps agree within 1e-3 of a step.
"""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import translation as T
import scenegen
import paper_2605_18052_gb300 as fm
from paper_2605_18052_gb300 import build
from paper_2605_18052_gb300 import translation as gtr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    build.build()
    fm.load_library()


def _inputs(name="ring16", noise_deg=1.0, outliers=0.05, seed=0):
    sc = scenegen.make_scene(name, seed=seed)
    R = sc.R_gt.numpy()
    C = O.centres_from_poses(R, sc.t_gt.numpy())
    t, _ = scenegen.relative_translations(sc, noise_deg, outliers, seed)
    return R, C, sc.cam_i.numpy(), sc.cam_j.numpy(), t


@pytest.mark.parametrize("name", ["ring16", "sphere128"])
def test_loss_grad_and_camera_losses_match_oracle(name):
    R, C, ci, cj, t = _inputs(name)
    oij = T.relative_directions(R, t, cj)
    inits = np.random.default_rng(1).normal(size=(3, C.shape[0], 3))
    with fm.Translation(R, ci, cj, t, inits) as tr:
        loss, g, cl = tr.loss_grad()
    for r in range(3):
        l_o, g_o = T.loss_grad(inits[r], ci, cj, oij)
        assert loss[r] == pytest.approx(l_o, rel=1e-5)
        assert np.abs(g[r] - g_o).max() <= 1e-4 * np.abs(g_o).max()
        np.testing.assert_allclose(cl[r], T.camera_losses(inits[r], ci, cj, oij), rtol=1e-5, atol=1e-7)


@pytest.mark.parametrize("use_graph", [1, 0])
def test_adam_steps_match_oracle(use_graph):
    R, C, ci, cj, t = _inputs("ring16")
    oij = T.relative_directions(R, t, cj)
    inits = np.random.default_rng(2).normal(size=(2, C.shape[0], 3))
    lr = 1e-2
    with fm.Translation(R, ci, cj, t, inits, fm.translation_options(lr=lr, use_graph=use_graph)) as tr:
        tr.step(20)
        o_g = tr.centres()
    for r in range(2):
        o_o, _ = T.adam(inits[r], ci, cj, oij, 20, lr)
        assert np.abs(o_g[r] - o_o).max() < 1e-3 * lr


def test_merge_matches_oracle_on_constructed_runs():
    R, C, ci, cj, t = _inputs("ring16", noise_deg=0.0, outliers=0.0)
    oij = T.relative_directions(R, t, cj)
    a = 2.0 * C + 1.0
    a[3] += np.array([0.5, 0.0, 0.0])
    b = 0.5 * C - 2.0
    b[5] += np.array([0.0, 0.3, 0.0])
    with fm.Translation(R, ci, cj, t, np.stack([a, b])) as tr:
        tr.merge()
        assert tr.n_runs == 1
        merged = tr.centres()[0]
    want = T.merge([a, b], [T.camera_losses(a, ci, cj, oij), T.camera_losses(b, ci, cj, oij)])
    np.testing.assert_allclose(merged, want, rtol=0, atol=1e-12)


def test_random_starts_recover_the_centres():
    R, C, ci, cj, t = _inputs("sphere128", noise_deg=0.5, outliers=0.05)
    o, loss = gtr.solve(R, ci, cj, t, n_runs=4, iters=600, final_iters=600, lr=1e-2, final_lr=2e-3, seed=3)
    err = np.linalg.norm(o - T.normalize(C), axis=1)
    # the noise (0.5 deg per pair, 5% wrong pairs) limits the accuracy, not the optimiser
    assert np.median(err) < 0.01
    assert np.quantile(err, 0.95) < 0.05


def test_degenerate_centres_are_reported():
    R, C, ci, cj, t = _inputs("ring16")
    o = np.random.default_rng(4).normal(size=(1, C.shape[0], 3))
    o[0, cj[0]] = o[0, ci[0]]
    with fm.Translation(R, ci, cj, t, o) as tr:
        with pytest.raises(fm.FastMapError) as ei:
            tr.loss_grad()
        assert ei.value.status == -4
