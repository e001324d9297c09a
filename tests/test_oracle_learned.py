"""Pins for the oracle of the learned inlier-weight variant (no GPU)."""
import numpy as np
import pytest
import torch

from oracle import learned as L


def test_bf16_rounding_matches_library_conversion():
    x = np.random.default_rng(0).normal(0, 30, 5000).astype(np.float32)
    x[:4] = [0.0, -0.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8]   # ties go to even
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(L.bf16_round(x).astype(np.float32), ref)


def test_flat_layout_round_trip_and_size():
    p = L.init_params(3)
    v = L.flatten(p)
    assert v.shape == (1377,)
    q = L.unflatten(v)
    for k in p:
        np.testing.assert_array_equal(p[k], q[k])


@pytest.mark.parametrize("quant", [False, True])
def test_cross_entropy_gradient_central_differences(quant):
    rng = np.random.default_rng(1)
    X = rng.normal(size=(64, 8))
    y = (rng.random(64) < 0.4).astype(np.float64)
    p = L.init_params(2)
    for k in p:
        p[k] = p[k] + 0.1 * rng.normal(size=p[k].shape)
    if quant:
        # with inputs and weights on the BF16 grid and the hidden roundings passed straight
        # through, the gradient must be that of the unrounded-activation network
        X = L.bf16_round(X)
        p = L.quantized(p)
    fn = L.bce_loss_grad
    loss, g = fn(p, X, y)
    v = L.flatten(p)
    gv = L.flatten(g)
    h = 1e-6
    for q in rng.choice(len(v), 40, replace=False):
        vp, vm = v.copy(), v.copy()
        vp[q] += h
        vm[q] -= h
        fd = (fn(L.unflatten(vp), X, y)[0] - fn(L.unflatten(vm), X, y)[0]) / (2 * h)
        assert abs(fd - gv[q]) <= 1e-6 * max(1.0, abs(gv).max())


def test_bf16_forward_close_to_exact_forward():
    rng = np.random.default_rng(4)
    X = rng.normal(size=(2000, 8))
    p = L.init_params(5)
    assert np.abs(L.forward_bf16(p, X) - L.forward(p, X)).max() < 0.05


def test_features_closed_form():
    # two image pairs; pair 0: |e| = 1e-3, 1e-2; pair 1: |e| = 0.1
    e = np.array([1e-3, 1e-2, 0.1])
    ep = np.array([2e-3, 1e-2, 0.05])
    score = np.array([0.9, 0.1, 0.5])
    pid = np.array([0, 0, 1])
    f = L.features(e, ep, score, pid, 2, 0.02, 3)
    le = np.log(e + 1e-6)
    lp = np.log(ep + 1e-6)
    m0 = (le[0] + le[1]) / 2
    np.testing.assert_allclose(f[:, 0], le - np.log(0.02))
    np.testing.assert_allclose(f[:, 1], [le[0] - m0, le[1] - m0, 0.0], atol=1e-15)
    np.testing.assert_allclose(f[:, 2], lp - le)
    np.testing.assert_allclose(f[:, 3], score)
    np.testing.assert_allclose(f[:, 4], [1.0, 1.0, 0.0])
    np.testing.assert_allclose(f[:, 5], [np.log(2) / 10, np.log(2) / 10, 0.0])
    np.testing.assert_allclose(f[:, 6], 0.3)
    np.testing.assert_allclose(f[:, 7], lp - np.log(0.02))


def test_adam_first_step_closed_form():
    p = {"W1": np.ones((8, 32)), "b1": np.zeros(32), "W2": np.zeros((32, 32)), "b2": np.zeros(32),
         "W3": np.zeros((32, 1)), "b3": np.zeros(1)}
    g = {k: np.full_like(v, -2.0) for k, v in p.items()}
    m, v = L.adam_init(p)
    L.adam_update(p, g, m, v, 1, 0.01)
    np.testing.assert_allclose(p["W1"], 1.01, rtol=1e-6)
    np.testing.assert_allclose(p["b3"], 0.01, rtol=1e-6)


def test_learned_weights_definition():
    p = L.init_params(0)
    e = np.array([1e-7, 1e-3, 0.5])
    f = np.zeros((3, 8))
    w, prob = L.learned_weights(p, e, f, 1e-6, tau_cap=0.1)
    np.testing.assert_allclose(w[:2], prob[:2] / np.array([1e-6, 1e-3]))
    assert w[2] == 0.0
