"""Global translation driver (Sec. "Global Translation"): host control flow over the
fm_translation_* kernels. Random initial centres are drawn here (seeded) and passed to the
library, which advances all runs together, merges them and runs the final optimisation."""
from __future__ import annotations

import numpy as np

from .binding import Translation, translation_options


def solve(R, cam_i, cam_j, t_rel, n_runs: int = 8, iters: int = 1000, final_iters: int = 1000,
          lr: float = 1e-2, final_lr: float | None = None, seed: int = 0, use_graph: bool = True):
    """Centres (n_cams, 3), normalised to zero mean and unit mean norm, and the final loss."""
    n_cams = np.asarray(R).reshape(-1, 9).shape[0]
    rng = np.random.default_rng(seed)
    inits = rng.normal(size=(n_runs, n_cams, 3))
    with Translation(R, cam_i, cam_j, t_rel, inits, translation_options(lr=lr, use_graph=1 if use_graph else 0)) as tr:
        tr.step(iters)
        tr.merge()
        if final_lr is not None:
            tr.set_learning_rate(final_lr)
        tr.step(final_iters)
        o = tr.centres()[0]
        loss = tr.loss_grad()[0][0]
    o = o - o.mean(0)
    return o / np.linalg.norm(o, axis=1).mean(), float(loss)
