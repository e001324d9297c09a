"""Learned inlier weights: training data from the method's own IRLS runs, training with the
library's kernels, and the refinement loop that uses the network for reweighting.

Host control flow only: every per-point-pair pass (features, MLP inference, losses, training
forward/backward) runs in libfastmap's kernels (fm_collect_features, fm_learned_weights,
fm_mlp_train_step); PyTorch only holds device buffers and samples rows.
"""
from __future__ import annotations

import numpy as np
import torch

from .binding import Mlp
from .refine import Schedule

N_FEAT, HIDDEN = 8, 32


def init_params(seed: int = 0) -> np.ndarray:
    """He-initialised parameters in the library's flat layout (W1, b1, W2, b2, W3, b3)."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, np.sqrt(2.0 / N_FEAT), N_FEAT * HIDDEN), np.zeros(HIDDEN),
             rng.normal(0, np.sqrt(2.0 / HIDDEN), HIDDEN * HIDDEN), np.zeros(HIDDEN),
             rng.normal(0, np.sqrt(1.0 / HIDDEN), HIDDEN), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def collect_training_data(problem, schedule: Schedule, collect_rounds: int, per_round: int,
                          generator: torch.Generator):
    """Run plain IRLS for `schedule.rounds` rounds; during the first `collect_rounds` rounds
    keep the features of `per_round` random point pairs; label them with the IRLS mask at the
    converged poses (|eps| <= tau_min). Returns CUDA tensors (features bf16 n x 8, labels f32)."""
    n = problem.n_pp
    feats = torch.empty(n, N_FEAT, dtype=torch.bfloat16, device="cuda")
    rows, idxs = [], []
    problem.reset_history()
    for r in range(schedule.rounds):
        if r < collect_rounds:
            problem.collect_features(schedule.tau(r), r, feats)
            idx = torch.randint(0, n, (per_round,), device="cuda", generator=generator)
            rows.append(feats[idx].clone())
            idxs.append(idx)
        problem.irls_weights(schedule.tau(r))
        s = schedule.decay ** r
        problem.set_learning_rate(schedule.lr_rot * s, schedule.lr_c * s)
        problem.step(schedule.iters_per_round)
    problem.irls_weights(schedule.tau_min)
    mask = torch.from_numpy(problem.get_weights() > 0).to("cuda")
    X = torch.cat(rows)
    Y = torch.cat([mask[i] for i in idxs]).to(torch.float32)
    return X, Y


def train(net: Mlp, X: torch.Tensor, Y: torch.Tensor, steps: int, batch: int, lr: float,
          generator: torch.Generator, log_every: int = 0):
    """Minibatch Adam on the cross-entropy; returns the losses that were read back."""
    losses = []
    n = Y.numel()
    for it in range(steps):
        idx = torch.randint(0, n, (batch,), device="cuda", generator=generator)
        want = log_every > 0 and (it % log_every == 0 or it == steps - 1)
        loss = net.train_step(X[idx].contiguous(), Y[idx].contiguous(), lr, want_loss=want)
        if want:
            losses.append((it, loss))
    return losses


def refine_learned(problem, net: Mlp, schedule: Schedule, callback=None, first_round: int = 0):
    """The IRLS loop with learned reweighting: w = p / max(|eps|, delta) for |eps| <= tau_r."""
    if first_round == 0:
        problem.reset_history()
    for r in range(first_round, schedule.rounds):
        tau = schedule.tau(r)
        problem.learned_weights(net, tau, tau, r)
        s = schedule.decay ** r
        problem.set_learning_rate(schedule.lr_rot * s, schedule.lr_c * s)
        problem.step(schedule.iters_per_round)
        if callback is not None:
            callback(r, problem)
    return problem
