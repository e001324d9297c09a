"""The pre-aggregated quadratic form (fm_preaggregate / fm_irls_preaggregate / fm_loss_grad_quadratic
/ fm_step_quadratic) against the oracle's IRLS objective, which it must reproduce for fixed
weights at any poses, not only at the anchor where the form was collected.

Tolerances are those of the streaming path (loss relative 1e-4, gradient 1e-4 of its largest
component): the form's sums are FP32 like the streaming pass's, and anchoring keeps the large
second moments W out of the loss except through the step d = e - e0, so no cancellation beyond
the streaming pass's enters.
"""
import numpy as np
import pytest
import torch

import oracle as O
import scenegen
from bounds import assert_grad_close
import paper_2605_18052_gb300 as fm
from paper_2605_18052_gb300 import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    build.build()
    fm.load_library()


def _oracle_inputs(sc, storage):
    prob = O.Problem.from_scene(sc)
    if storage == "fp16":
        _, d1, d2 = O.fp16_centroid_storage(prob, sc.x1.numpy(), sc.x2.numpy())
        prob = O.Problem(sc.n_cams, prob.cam_i, prob.cam_j, prob.pair_id, d1, d2)
    return prob


def _gpu_problem(sc, R, t, **opt):
    return fm.Problem(R, t, sc.cam_i, sc.cam_j, sc.pair_id, sc.x1, sc.x2, options=fm.default_options(**opt))


def _assert_grad_close(g, ref, tol=1e-4):
    assert_grad_close(g, ref, tol)


def _moved(R, c, seed, deg, frac):
    """Poses moved by random rotations of up to `deg` degrees and centre steps of `frac` of
    the scene's spread: about what one round of iterations moves them."""
    rng = np.random.default_rng(seed)
    phi = rng.normal(size=(R.shape[0], 3))
    phi *= np.radians(deg) * rng.uniform(0, 1, (R.shape[0], 1)) / np.linalg.norm(phi, axis=1, keepdims=True)
    R1 = np.stack([O.expmap(p) @ r for p, r in zip(phi, R)])
    c1 = c + frac * c.std(0) * rng.normal(size=c.shape)
    return R1, c1


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
@pytest.mark.parametrize("name", ["ring16", "sphere128"])
def test_quadratic_loss_grad_matches_oracle_away_from_anchor(name, storage):
    sc = scenegen.make_scene(name, seed=3)
    R0, t0 = sc.R_init.numpy(), sc.t_init.numpy()
    c0 = O.centres_from_poses(R0, t0)
    prob = _oracle_inputs(sc, storage)
    rng = np.random.default_rng(4)
    w32 = rng.uniform(0.0, 50.0, sc.n_pp).astype(np.float32)
    w = O.quantize_weights_fp16(w32, 1e-6) if storage == "fp16" else w32.astype(np.float64)
    with _gpu_problem(sc, R0, t0, storage=storage) as gp:
        gp.set_weights(w32)
        gp.preaggregate()
        # at the anchor
        l_q, g_q = gp.loss_grad_quadratic()
        l_or, g_or = O.loss_grad(prob, R0, c0, w)
        assert l_q == pytest.approx(l_or, rel=1e-4)
        _assert_grad_close(g_q, g_or)
        # away from it: the form is exact for any poses
        for k, (deg, frac) in enumerate([(0.5, 0.02), (3.0, 0.1)]):
            R1, c1 = _moved(R0, c0, 10 + k, deg, frac)
            gp.set_params(R1, c1)
            l_q, g_q = gp.loss_grad_quadratic()
            l_s, g_s = gp.loss_grad()          # the streaming pass, same weights
            l_or, g_or = O.loss_grad(prob, R1, c1, w)
            assert l_q == pytest.approx(l_or, rel=1e-4)
            _assert_grad_close(g_q, g_or)
            assert l_q == pytest.approx(l_s, rel=1e-4)
            _assert_grad_close(g_q, g_s)


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_fused_reweighting_writes_the_irls_weights(storage):
    # same arithmetic as fm_irls_weights: identical weights and count, bit for bit
    sc = scenegen.make_scene("sphere128", seed=1)
    R0, t0 = sc.R_init.numpy(), sc.t_init.numpy()
    for tau in (0.02, float("inf")):
        with _gpu_problem(sc, R0, t0, storage=storage) as gp:
            k1 = gp.irls_weights(tau)
            w1 = gp.get_weights()
            l1, g1 = gp.loss_grad()
        with _gpu_problem(sc, R0, t0, storage=storage) as gp:
            k2 = gp.irls_preaggregate(tau)
            w2 = gp.get_weights()
            l2, g2 = gp.loss_grad_quadratic()
        assert k1 == k2
        np.testing.assert_array_equal(w1, w2)
        assert l2 == pytest.approx(l1, rel=1e-4)
        _assert_grad_close(g2, g1)


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_quadratic_steps_match_oracle(storage):
    sc = scenegen.make_scene("ring16", seed=6)
    R0, t0 = sc.R_init.numpy(), sc.t_init.numpy()
    c0 = O.centres_from_poses(R0, t0)
    prob = _oracle_inputs(sc, storage)
    w = O.irls_weights(O.residuals(prob, R0, c0), 0.05, 1e-6)[0]
    wq = O.quantize_weights_fp16(w, 1e-6) if storage == "fp16" else w.astype(np.float32).astype(np.float64)
    lr_r, lr_c = 5e-3, 5e-3 * 3.0
    with _gpu_problem(sc, R0, t0, storage=storage, lr_rot=lr_r, lr_c=lr_c) as gp:
        gp.set_weights(w.astype(np.float32))
        gp.preaggregate()
        gp.step_quadratic(25)
        R_g, t_g = gp.get_poses()
        _, _, steps = gp.get_state()
        loss_last = gp.last_loss()
    assert steps == 25
    R_o, c_o = R0.copy(), c0.copy()
    m = np.zeros((sc.n_cams, 6))
    v = np.zeros((sc.n_cams, 6))
    for k in range(25):
        l_o, g = O.loss_grad(prob, R_o, c_o, wq)
        O.adam_step(R_o, c_o, g, m, v, k + 1, lr_r, lr_c)
    ang = np.degrees(np.arccos(np.clip((np.einsum("nab,nab->n", R_g, R_o) - 1) / 2, -1, 1)))
    c_g = O.centres_from_poses(R_g, t_g)
    print("loss", loss_last, l_o, "ang", ang.max() / np.degrees(lr_r), "c", np.abs(c_g - c_o).max() / lr_c)
    assert ang.max() < 0.02 * np.degrees(lr_r)
    assert np.abs(c_g - c_o).max() < 0.02 * lr_c
    assert loss_last == pytest.approx(l_o, rel=1e-3)


def test_quadratic_graph_and_eager_agree():
    sc = scenegen.make_scene("ring16", seed=7)
    R0, t0 = sc.R_init.numpy(), sc.t_init.numpy()
    res = []
    for use_graph in (1, 0):
        with _gpu_problem(sc, R0, t0, use_graph=use_graph) as gp:
            gp.irls_preaggregate(0.1)
            gp.step_quadratic(11)
            res.append(gp.get_params())
    np.testing.assert_array_equal(res[0][0], res[1][0])
    np.testing.assert_array_equal(res[0][1], res[1][1])


def test_quadratic_refine_reaches_the_streaming_accuracy():
    from paper_2605_18052_gb300 import learned
    sc = scenegen.make_scene("sphere128", seed=4)
    R0, t0 = sc.R_init.numpy(), sc.t_init.numpy()
    Rg = sc.R_gt.numpy()
    sch = learned.default_schedule(sc, rounds=20)
    errs = []
    for quadratic in (False, True):
        with fm.Problem(R0, t0, sc.cam_i, sc.cam_j, sc.pair_id, sc.x1, sc.x2, options=sch.options()) as gp:
            fm.refine(gp, sch, quadratic=quadratic)
            R, _ = gp.get_poses()
        errs.append(O.rotation_error_deg(R, Rg).mean())
    e0 = O.rotation_error_deg(R0, Rg).mean()
    e_s, e_q = errs
    assert e_q < 0.5 * e0
    assert e_q <= 1.3 * e_s + 0.02 and e_s <= 1.3 * e_q + 0.02, (e_s, e_q)


def test_stale_or_missing_form_is_rejected():
    sc = scenegen.make_scene("ring16", seed=8)
    R0, t0 = sc.R_init.numpy(), sc.t_init.numpy()
    with _gpu_problem(sc, R0, t0) as gp:
        with pytest.raises(fm.FastMapError):
            gp.step_quadratic(1)
        gp.preaggregate()
        gp.step_quadratic(1)
        gp.irls_weights(0.1)                 # new weights: the form is stale
        with pytest.raises(fm.FastMapError):
            gp.loss_grad_quadratic()
        gp.irls_preaggregate(0.1)
        gp.loss_grad_quadratic()
    with _gpu_problem(sc, R0, t0, loss="l1") as gp:
        with pytest.raises(fm.FastMapError):
            gp.preaggregate()
