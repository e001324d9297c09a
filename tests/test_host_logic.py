"""Host-side control flow of the package, without a GPU: the round loops drive the library's
entry points in the order and with the arguments the schedule fixes, the schedule follows the
threshold rule of the oracle, and the evaluation metrics agree with the oracle's."""
import numpy as np
import pytest

import oracle as O
import scenegen
from paper_2605_18052_gb300 import learned, metrics
from paper_2605_18052_gb300.refine import Schedule, refine


class Recorder:
    """Stands in for binding.Problem and records the calls a round loop makes."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def call(*args):
            self.calls.append((name, *args))
            return 0
        return call


def _schedule():
    return Schedule(rounds=5, iters_per_round=7, tau0=0.3, tau_min=0.02, tau_factor=0.5, decay=0.9,
                    lr_rot=2e-3, lr_c=5e-2, delta=1e-4, beta2=0.99)


@pytest.mark.parametrize("quadratic", [False, True])
def test_refine_drives_one_reweighting_and_iters_per_round(quadratic):
    sch = _schedule()
    seen = []
    p = refine(Recorder(), sch, callback=lambda r, prob: seen.append(r), first_round=1, quadratic=quadratic)
    per_round = 3 if quadratic else 2
    assert len(p.calls) == per_round * 4 and seen == [1, 2, 3, 4]
    for k, r in enumerate(range(1, 5)):
        c = p.calls[per_round * k: per_round * (k + 1)]
        assert c[0] == ("set_learning_rate", pytest.approx(2e-3 * 0.9 ** r), pytest.approx(5e-2 * 0.9 ** r))
        tau = O.threshold_schedule(r, 0.3, 0.02, 0.5)
        if quadratic:
            assert c[1] == ("irls_preaggregate", pytest.approx(tau)) and c[2] == ("step_quadratic", 7)
        else:
            assert c[1] == ("step_irls", pytest.approx(tau), 7)


def test_refine_streaming_round_is_one_fused_call():
    p = refine(Recorder(), _schedule())
    names = [c[0] for c in p.calls]
    assert names == ["set_learning_rate", "step_irls"] * 5


@pytest.mark.parametrize("quadratic", [False, True])
def test_refine_learned_reweights_with_the_network_every_round(quadratic):
    sch = _schedule()
    net = object()
    p = learned.refine_learned(Recorder(), net, sch, quadratic=quadratic)
    assert p.calls[0] == ("reset_history",)
    body = p.calls[1:]
    per_round = 4 if quadratic else 2
    assert len(body) == per_round * sch.rounds
    for r in range(sch.rounds):
        c = body[per_round * r: per_round * (r + 1)]
        tau = O.threshold_schedule(r, 0.3, 0.02, 0.5)
        assert c[0] == ("set_learning_rate", pytest.approx(2e-3 * 0.9 ** r), pytest.approx(5e-2 * 0.9 ** r))
        if quadratic:
            assert c[1][0] == "learned_weights" and c[1][1] is net
            assert c[1][2:] == (pytest.approx(tau), pytest.approx(tau), r)
            assert c[2] == ("preaggregate",) and c[3] == ("step_quadratic", 7)
        else:   # the learned reweighting fused into the round's first pass
            assert c[1][0] == "step_learned" and c[1][1] is net
            assert c[1][2:] == (pytest.approx(tau), pytest.approx(tau), r, 7)
    # a resumed run keeps the residual history
    p = learned.refine_learned(Recorder(), net, sch, first_round=2)
    assert [c[0] for c in p.calls[:2]] == ["set_learning_rate", "step_learned"]


def test_schedule_threshold_matches_the_oracle_rule():
    sch = _schedule()
    for r in range(12):
        assert sch.tau(r) == O.threshold_schedule(r, sch.tau0, sch.tau_min, sch.tau_factor)


def test_default_schedule_from_the_scene():
    sc = scenegen.make_scene("ring16", seed=0)
    sch = learned.default_schedule(sc, 9)
    C = O.centres_from_poses(sc.R_gt.numpy(), sc.t_gt.numpy())
    ci, cj = sc.cam_i.numpy(), sc.cam_j.numpy()
    base = np.median(np.linalg.norm(C[ci] - C[cj], axis=1))
    assert sch.rounds == 9 and sch.iters_per_round == 25
    assert sch.delta == pytest.approx(sc.sigma_px / sc.f) and sch.tau_min == pytest.approx(4 * sc.sigma_px / sc.f)
    assert sch.lr_c == pytest.approx(1e-2 * base, rel=1e-12)


def test_metrics_agree_with_the_oracle():
    rng = np.random.default_rng(0)
    sc = scenegen.make_scene("ring16", seed=1)
    Rg, tg = sc.R_gt.numpy(), sc.t_gt.numpy()
    R = np.einsum("nab,nbc->nac", np.stack([O.expmap(0.05 * rng.normal(size=3)) for _ in range(sc.n_cams)]), Rg)
    t = tg + 0.05 * rng.normal(size=tg.shape)
    np.testing.assert_allclose(metrics.rotation_error_deg(R, Rg), O.rotation_error_deg(R, Rg), atol=1e-9)
    ci, cj = sc.cam_i.numpy(), sc.cam_j.numpy()
    np.testing.assert_allclose(
        metrics.translation_error_deg(R, t, Rg, tg, ci, cj),
        O.translation_error_deg(R, O.centres_from_poses(R, t), Rg, O.centres_from_poses(Rg, tg), ci, cj), atol=1e-9)
