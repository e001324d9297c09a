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


def refine_learned(problem, net: Mlp, schedule: Schedule, callback=None, first_round: int = 0,
                   quadratic: bool = False):
    """The IRLS loop with learned reweighting: w = p / max(|eps|, delta) for |eps| <= tau_r.
    quadratic: iterate on the pre-aggregated quadratic form of each round's objective."""
    if first_round == 0:
        problem.reset_history()
    for r in range(first_round, schedule.rounds):
        tau = schedule.tau(r)
        s = schedule.decay ** r
        problem.set_learning_rate(schedule.lr_rot * s, schedule.lr_c * s)
        if quadratic:
            problem.learned_weights(net, tau, tau, r)
            problem.preaggregate()
            problem.step_quadratic(schedule.iters_per_round)
        else:   # the reweighting fused into the round's first pass (fm_step_learned)
            problem.step_learned(net, tau, tau, r, schedule.iters_per_round)
        if callback is not None:
            callback(r, problem)
    return problem


# ---- training on the method's own converged runs ------------------------------------------------
def default_schedule(sc, rounds: int, iters: int = 25) -> Schedule:
    """The reweighting schedule used for both arms. The thesis fixes none of these values:
    the threshold starts at 0.1 (about the 60th percentile of |eps| at poses 5 degrees off,
    so most outlier matches are filtered from the first round) and shrinks by 0.8 per round
    to 4 sigma/f; the weight floor delta is the noise level sigma/f (below it the L1
    approximation z^2/|z^| would pin a pair to its current residual); Adam step sizes
    3e-3 rad and 1e-2 of the median baseline, decayed by 0.985 per round, beta2 = 0.99."""
    R, t = sc.R_gt.double(), sc.t_gt.double()
    C = -(R.transpose(1, 2) @ t[:, :, None])[:, :, 0]
    base = float((C[sc.cam_i.long()] - C[sc.cam_j.long()]).norm(dim=1).median())
    noise = sc.sigma_px / sc.f
    return Schedule(rounds=rounds, iters_per_round=iters, tau0=0.1, tau_min=4 * noise,
                    tau_factor=0.8, decay=0.985, lr_rot=3e-3, lr_c=1e-2 * base, delta=noise, beta2=0.99)


def train_from_scenes(config: str, seeds, rounds: int, collect_rounds: int, per_round: int,
                      steps: int, batch: int, lr: float, seed: int = 0, log=print):
    """Collect training data from plain-IRLS runs on seeded scenes of `config` and train a
    network with the library's kernels. Returns the trained parameters (flat float32)."""
    import scenegen
    from .binding import Problem
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    Xs, Ys = [], []
    for k, s in enumerate(seeds):
        sc = scenegen.make_scene(config, seed=int(s), device="cuda")
        sch = default_schedule(sc, rounds)
        with Problem(sc.R_init.cpu(), sc.t_init.cpu(), sc.cam_i.cpu(), sc.cam_j.cpu(), sc.pair_id,
                     sc.x1, sc.x2, options=sch.options()) as gp:
            gp.set_scores(sc.score)
            X, Y = collect_training_data(gp, sch, collect_rounds, per_round, gen)
        Xs.append(X)
        Ys.append(Y)
        if log and (k % 20 == 0 or k == len(seeds) - 1):
            log(f"scene {k + 1}/{len(seeds)} seed {s}: {sc.n_pp} point pairs, inlier labels {float(Y.mean()):.3f}")
        del sc
        torch.cuda.empty_cache()
    X = torch.cat(Xs)
    Y = torch.cat(Ys)
    net = Mlp(init_params(seed))
    losses = train(net, X, Y, steps, batch, lr, gen, log_every=max(1, steps // 10))
    if log:
        log("training losses: " + ", ".join(f"{it}:{l:.4f}" for it, l in losses))
    out = net.params()
    net.close()
    return out, X.shape[0], losses


def time_to_accuracy(sc, arm: str, net: Mlp | None = None, storage: str = "fp16", max_rounds: int = 80,
                     threshold_deg: float = 0.1, thresholds=(2.0, 1.0, 0.5, 0.25, 0.1), schedule=None):
    """Device time of the refinement loop until the mean rotation error (after global
    alignment) is <= threshold_deg, and the time at which each of `thresholds` was first
    reached. The error is checked after every round and the check is not timed.
    arm: "irls" (plain reweighting) or "learned", each optionally with the suffix "_quad"
    (iterations on the pre-aggregated quadratic form). `schedule` replaces the default schedule
    (its rounds are ignored in favour of max_rounds). Returns a dict."""
    from . import metrics
    from .binding import Problem
    sch = default_schedule(sc, max_rounds) if schedule is None else schedule
    Rg = sc.R_gt.cpu().numpy()
    stream = torch.cuda.current_stream()
    total_ms, hist, first = 0.0, [], {}
    with Problem(sc.R_init.cpu(), sc.t_init.cpu(), sc.cam_i.cpu(), sc.cam_j.cpu(), sc.pair_id, sc.x1, sc.x2,
                 options=sch.options(storage=storage)) as gp:
        gp.set_scores(sc.score)
        gp.reset_history()
        for r in range(max_rounds):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            tau = sch.tau(r)
            s = sch.decay ** r
            gp.set_learning_rate(sch.lr_rot * s, sch.lr_c * s)
            if arm == "irls":
                gp.step_irls(tau, sch.iters_per_round)
            elif arm == "irls_quad":
                gp.irls_preaggregate(tau)
                gp.step_quadratic(sch.iters_per_round)
            elif arm == "learned":
                gp.step_learned(net, tau, tau, r, sch.iters_per_round)
            elif arm == "learned_quad":
                gp.learned_weights(net, tau, tau, r)
                gp.preaggregate()
                gp.step_quadratic(sch.iters_per_round)
            else:
                raise ValueError(f"unknown arm {arm!r}")
            e1.record(stream)
            torch.cuda.synchronize()
            total_ms += e0.elapsed_time(e1)
            R, _ = gp.get_poses()
            err = float(metrics.rotation_error_deg(R, Rg).mean())
            hist.append(err)
            for th in thresholds:
                if err <= th and th not in first:
                    first[th] = (total_ms, r + 1)
            if err <= threshold_deg:
                break
    done = hist[-1] <= threshold_deg
    return {"reached": done, "ms": total_ms, "rounds": len(hist), "final_deg": hist[-1], "history_deg": hist,
            "ms_to": {str(th): (round(first[th][0], 3) if th in first else None) for th in thresholds},
            "rounds_to": {str(th): (first[th][1] if th in first else None) for th in thresholds}}


def _main():
    import argparse
    import os
    ap = argparse.ArgumentParser(description="train the inlier-weight MLP on converged IRLS runs")
    ap.add_argument("--config", default="sphere128")
    ap.add_argument("--scenes", type=int, default=200)
    ap.add_argument("--first-seed", type=int, default=1000)
    ap.add_argument("--rounds", type=int, default=40)
    ap.add_argument("--collect-rounds", type=int, default=6)
    ap.add_argument("--per-round", type=int, default=8192)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=16384)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "mlp_inlier.npy"))
    a = ap.parse_args()
    params, n, losses = train_from_scenes(a.config, range(a.first_seed, a.first_seed + a.scenes), a.rounds,
                                          a.collect_rounds, a.per_round, a.steps, a.batch, a.lr)
    os.makedirs(os.path.dirname(a.out), exist_ok=True)
    np.save(a.out, params)
    print(f"saved {a.out}: {params.shape[0]} parameters trained on {n} samples")


if __name__ == "__main__":
    _main()
