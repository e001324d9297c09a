"""IRLS epipolar adjustment driver (Sec. "Epipolar Adjustment"): host control flow only.

Each round reweights the point pairs at the current poses with a filtering threshold that
starts large and shrinks by a constant factor every round down to a floor, then runs a fixed
number of Adam iterations on the reweighted objective. All per-point-pair work happens inside the library
calls (fm_irls_weights, fm_step).
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

    def tau(self, r: int) -> float:
        return max(self.tau_min, self.tau0 * self.tau_factor ** r)


def refine(problem, schedule: Schedule, callback=None, first_round: int = 0):
    """Run `schedule` on `problem` (a binding.Problem). callback(r, problem) after each round."""
    for r in range(first_round, schedule.rounds):
        problem.irls_weights(schedule.tau(r))
        s = schedule.decay ** r
        problem.set_learning_rate(schedule.lr_rot * s, schedule.lr_c * s)
        problem.step(schedule.iters_per_round)
        if callback is not None:
            callback(r, problem)
    return problem
