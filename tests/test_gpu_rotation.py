"""The global rotation kernels (fm_rotation_*) against the FP64 oracle on the same inputs.

Everything on both sides is FP64 except the GPU's Adam moments (FP32). The initialisation
solves the same anchored least-squares systems (conjugate gradients to a relative residual of
1e-9 on the GPU, a direct sparse solve in the oracle): rotations agree to 1e-6. Loss and
gradient agree to 1e-10 relative (summation order only); 50 Adam steps agree to 1e-3 of a step.
"""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import rotation as G
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


def _relative(name, noise_deg=0.0, outliers=0.0, seed=0):
    sc = scenegen.make_scene(name, seed=seed)
    R = sc.R_gt.numpy()
    ci, cj = sc.cam_i.numpy(), sc.cam_j.numpy()
    Rrel = np.einsum("nab,ncb->nac", R[cj], R[ci])
    rng = np.random.default_rng(seed + 11)
    if noise_deg > 0:
        for p in range(len(ci)):
            w = rng.normal(size=3)
            Rrel[p] = O.expmap(w * np.radians(noise_deg) / np.linalg.norm(w)) @ Rrel[p]
    if outliers > 0:
        for p in np.nonzero(rng.random(len(ci)) < outliers)[0]:
            Rrel[p] = O.expmap(rng.normal(size=3)) @ Rrel[p]
    return R, ci, cj, Rrel


@pytest.mark.parametrize("name,noise,outl", [("ring16", 0.0, 0.0), ("sphere128", 0.0, 0.0),
                                             ("sphere128", 2.0, 0.05)])
def test_initialisation_matches_oracle(name, noise, outl):
    R, ci, cj, Rrel = _relative(name, noise, outl)
    with fm.Rotation(ci, cj, Rrel, R.shape[0]) as rp:
        iters, resid = rp.initialize()
        Rg = rp.rotations()
    Ro = G.initial_rotations(R.shape[0], ci, cj, Rrel)
    assert resid <= 1e-9 and iters > 0
    assert np.abs(Rg - Ro).max() < 1e-6
    if noise == 0.0:
        assert np.abs(Rg - np.einsum("nab,cb->nac", R, R[0])).max() < 1e-6


def test_loss_and_gradient_match_oracle():
    R, ci, cj, Rrel = _relative("sphere128", 3.0)
    rng = np.random.default_rng(5)
    a = G.six_d_from_rot(R) + 0.2 * rng.normal(size=(R.shape[0], 6))
    with fm.Rotation(ci, cj, Rrel, R.shape[0]) as rp:
        rp.set_params(a)
        loss, g = rp.loss_grad()
        Rg = rp.rotations()
    l_o, g_o = G.loss_grad_6d(a, ci, cj, Rrel)
    assert loss == pytest.approx(l_o, rel=1e-10)
    assert np.abs(g - g_o).max() <= 1e-9 * np.abs(g_o).max()
    np.testing.assert_allclose(Rg, G.rot_from_6d(a), atol=1e-14)


@pytest.mark.parametrize("use_graph", [1, 0])
def test_adam_steps_match_oracle(use_graph):
    R, ci, cj, Rrel = _relative("sphere128", 2.0, 0.05)
    Ro = G.initial_rotations(R.shape[0], ci, cj, Rrel)
    lr = 1e-3
    with fm.Rotation(ci, cj, Rrel, R.shape[0], fm.rotation_options(lr=lr, use_graph=use_graph)) as rp:
        rp.set_rotations(Ro)
        rp.step(50)
        a_g = rp.params()
    a_o, _ = G.adam(G.six_d_from_rot(Ro), ci, cj, Rrel, 50, lr)
    assert np.abs(a_g - a_o).max() < 1e-3 * lr


def test_refinement_removes_the_pull_of_wrong_pairs():
    R, ci, cj, Rrel = _relative("sphere128", 0.5, 0.05, seed=1)
    with fm.Rotation(ci, cj, Rrel, R.shape[0], fm.rotation_options(lr=1e-3)) as rp:
        rp.initialize()
        e0 = O.rotation_error_deg(rp.rotations(), R).mean()
        rp.step(300)
        e1 = O.rotation_error_deg(rp.rotations(), R).mean()
    assert e0 > 1.0 and e1 < 0.25 * e0
