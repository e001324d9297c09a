"""IRLS epipolar adjustment driver (Sec. "Epipolar Adjustment"): host control flow only.

Each round reweights the point pairs at the current poses with a filtering threshold that
starts large and shrinks by a constant factor every round down to a floor, then runs a fixed
number of Adam iterations on the reweighted objective. All per-point-pair work happens inside the library
calls (fm_step_irls: the reweighting fused into the round's first pass over the point pairs).

With `quadratic=True` a round makes one pass over the point pairs (reweighting and the
per-image-pair quadratic form of the reweighted objective, fm_irls_preaggregate) and its
iterations evaluate the objective from the form alone (fm_step_quadratic). With the weights
fixed the objective is exactly quadratic in each essential matrix, so both modes follow the
same trajectory up to FP32 rounding.
"""
from __future__ import annotations

import dataclasses


@dataclasses.dataclass
class Schedule:
    rounds: int = 8
    iters_per_round: int = 25
    tau0: float = 0.5         # initial filtering threshold (normalized epipolar error)
    tau_min: float = 0.004    # threshold floor
    tau_factor: float = 0.8   # threshold factor per round
    decay: float = 0.95       # learning-rate factor per round
    lr_rot: float = 1e-2      # radians
    lr_c: float = 1e-2        # scene units (scale with the typical baseline)
    delta: float = 1e-6       # IRLS weight floor: w = 1/max(|eps|, delta) (a problem option)
    beta2: float = 0.999      # Adam second-moment decay (a problem option)

    def tau(self, r: int) -> float:
        return max(self.tau_min, self.tau0 * self.tau_factor ** r)

    def options(self, **kw):
        """Problem options carrying this schedule's step sizes, weight floor and Adam beta2."""
        from .binding import default_options
        base = dict(lr_rot=self.lr_rot, lr_c=self.lr_c, delta=self.delta, beta2=self.beta2)
        base.update(kw)
        return default_options(**base)


def refine(problem, schedule: Schedule, callback=None, first_round: int = 0, quadratic: bool = False):
    """Run `schedule` on `problem` (a binding.Problem). callback(r, problem) after each round."""
    for r in range(first_round, schedule.rounds):
        s = schedule.decay ** r
        problem.set_learning_rate(schedule.lr_rot * s, schedule.lr_c * s)
        if quadratic:
            problem.irls_preaggregate(schedule.tau(r))
            problem.step_quadratic(schedule.iters_per_round)
        else:
            problem.step_irls(schedule.tau(r), schedule.iters_per_round)
        if callback is not None:
            callback(r, problem)
    return problem
