"""Benchmark of the epipolar-adjustment hot path on GB300.

One step = one IRLS round of the method: reweighting with filtering at the current poses
followed by `--iters` optimiser iterations (loss + analytic gradient over every point pair,
per-camera gradient, Adam + exponential map), all on the GPU (fm_step_irls: the reweighting
is fused into the round's first pass).

Default workload: the 4,000-camera trajectory scene (~1.5e8 point pairs, ~5e4 image pairs,
Pareto match counts, 25% outliers), FP16 centroid-offset storage, FP32 arithmetic. The
inputs (>1 GB) are larger than L2, so no flush is needed between timed iterations.

Prints one JSON line. `value` counts point pairs evaluated by loss+gradient passes per second
(G point-pairs/s); the reweighting pass of each round is inside the timed region but not
counted. `--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "G point-pairs/s epipolar loss+grad (% HBM peak); time to rot err<0.1° learned vs IRLS"
UNIT = "G point-pairs/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="traj4000")
    ap.add_argument("--storage", default="fp16", choices=["fp16", "fp32"])
    ap.add_argument("--iters", type=int, default=25, help="optimiser iterations per IRLS round")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-tta", action="store_true", help="skip the time-to-accuracy comparison")
    ap.add_argument("--no-quad", action="store_true", help="skip the quadratic-form timing")
    ap.add_argument("--no-translation", action="store_true", help="skip the global-translation timing")
    ap.add_argument("--no-focal", action="store_true", help="skip the focal refinement and focal vote timings")
    ap.add_argument("--no-passes", action="store_true", help="skip the once-per-round pass timings")
    ap.add_argument("--no-configs", action="store_true", help="skip the other workloads")
    ap.add_argument("--clocks-csv", default=None, help="keep nvidia-smi's clock samples in this file")
    ap.add_argument("--shard", action="store_true",
                    help="split one problem across the ranks (whole image pairs per rank, one NCCL "
                         "all-reduce of the gradient per iteration, strong scaling) instead of replicas")
    ap.add_argument("--tta-config", default="loop1000_o30")
    ap.add_argument("--tta-rounds", type=int, default=120)
    ap.add_argument("--tta-rounds-large", type=int, default=80,
                    help="round limit of the learned-vs-IRLS comparison on the benchmark workload")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# the sources a kernel's code comes from; a committed traffic figure is used only while their
# combined hash matches the one recorded with it
KERNEL_SOURCES = {
    "stream_loss": ("fm_kernels.cu", "fm_walk.cuh", "fm_internal.cuh"),
    "stream_reweight": ("fm_kernels.cu", "fm_walk.cuh", "fm_internal.cuh"),
    "quad_accumulate": ("fm_quad.cu", "fm_walk.cuh", "fm_internal.cuh"),
    "learned_loss": ("fm_mlp.cu", "fm_tcgen05.cuh", "fm_walk.cuh", "fm_internal.cuh"),
}


def kernel_source_hash(kernel: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2605_18052_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_tag: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current
    kernel sources (the summary records their hash); else None."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    h = kernel_source_hash(kernel_tag.split("_fp")[0])
    for line in open(path):
        parts = line.split()
        if len(parts) >= 3 and parts[0] == kernel_tag and parts[1] == h:
            return float(parts[2])
    return None


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs.

    The sampler is started before the timed region and waits (at most 3 s) for nvidia-smi's
    first line; only lines written after that count, so every sample is taken while timed
    work runs. The raw samples go to `path` (a temporary file unless --clocks-csv names one).
    """

    def __init__(self, index: int, path: str | None = None):
        import tempfile
        self.index = index
        self.proc = None
        self.skip = 0
        self.path = path or os.path.join(tempfile.gettempdir(), f"fm_bench_clocks_rank{index}_{os.getpid()}.csv")

    def _lines(self) -> int:
        try:
            with open(self.path) as f:
                return sum(1 for _ in f)
        except OSError:
            return 0

    def __enter__(self):
        os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return self
        t0 = time.perf_counter()
        while self._lines() == 0 and self.proc.poll() is None and time.perf_counter() - t0 < 3.0:
            time.sleep(0.02)
        self.skip = self._lines()   # written before the timed region started
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            lines = fh.readlines()

        def parse(rows):
            sm, mx, reasons = [], None, set()
            for line in rows:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx = float(f[2])
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
            return sm, mx, reasons

        sm, mx, reasons = parse(lines[self.skip:])
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
               "reasons": sorted(reasons), "samples": len(sm)}
        if not sm:   # region shorter than the 200 ms period: the sample just before it
            sm, mx, reasons = parse(lines[:self.skip][-1:])
            out.update({"sm_mhz": sm[0] if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                        "note": "timed region shorter than the sampling period; sample taken just before it"})
        return out


def schedule_for(sc, iters):
    from paper_2605_18052_gb300.learned import default_schedule
    return default_schedule(sc, max(1, sc.iters // iters), iters)


def _speedups(res, a, b):
    """Wall-time ratio a / b at every threshold both arms reached."""
    out = {}
    for th, ta in res[a]["ms_to"].items():
        tb = res[b]["ms_to"].get(th)
        out[th] = round(ta / tb, 3) if ta is not None and tb is not None and tb > 0 else None
    return out


def time_to_accuracy_section(args, bench_scene=None):
    """Learned vs plain IRLS: device time of the round loop until the mean rotation error is
    <= 0.1 deg (and the times to 2, 1, 0.5, 0.25 deg), each arm with the streaming iterations and
    with the pre-aggregated quadratic form, on
      (1) the 1,000-camera closed trajectory with 30% outliers (the evaluation scene of the
          learned-weight workload; the network never saw it: it was trained on 128-camera spheres),
      (2) the 1,000-camera open trajectory with 30% outliers (0.1 deg lies beyond what its
          objective determines; reported at the thresholds both arms reach),
      (3) a held-out 128-camera sphere with 30% outliers (the network's training shape, seeds
          outside the training seeds 1000-1199),
      (4) the benchmark's 4,000-camera scene: the learned arm on FP16 storage against the plain
          FP32 IRLS loop, and the same on the 4,000-camera closed trajectory."""
    import numpy as np
    import torch
    import scenegen
    from paper_2605_18052_gb300 import Mlp, learned
    path = os.path.join(ROOT, "paper_2605_18052_gb300", "data", "mlp_inlier.npy")
    if not os.path.exists(path):
        return {"unavailable": "no trained network (python -m paper_2605_18052_gb300.learned)"}
    net = Mlp(np.load(path))
    out = {"threshold_deg": 0.1, "storage": args.storage}

    def arm_result(sc, arm, storage, rounds):
        r = learned.time_to_accuracy(sc, arm, net if arm.startswith("learned") else None, storage, rounds)
        res = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items() if k != "history_deg"}
        res["storage"] = storage
        res["ms_per_round"] = round(r["ms"] / max(1, r["rounds"]), 4)
        res["history_deg_every_5"] = [round(x, 4) for x in r["history_deg"][::5]]
        return res

    for cfg, seed, rounds in ((args.tta_config, args.seed, args.tta_rounds), ("traj1000_o30", 0, 120),
                              ("sphere128_o30", 8, 80)):
        sc = scenegen.make_scene(cfg, seed=seed, device="cuda")
        torch.cuda.empty_cache()
        res = {"scene": f"{cfg} seed {seed}: {sc.n_cams} cameras, {sc.n_pp} point pairs", "max_rounds": rounds}
        for arm in ("irls", "learned", "irls_quad", "learned_quad"):
            res[arm] = arm_result(sc, arm, args.storage, rounds)
        for a, b in (("irls", "learned"), ("irls_quad", "learned_quad"), ("irls", "learned_quad")):
            res[f"speedup_{b}_over_{a}"] = (res[a]["ms"] / res[b]["ms"]
                                            if res[a]["reached"] and res[b]["reached"] else None)
            res[f"speedup_{b}_over_{a}_at"] = _speedups(res, a, b)
        out[cfg] = res
        del sc
        torch.cuda.empty_cache()
    if bench_scene is not None:
        sc = bench_scene
        rounds = args.tta_rounds_large
        res = {"scene": f"{args.config} seed {args.seed}: {sc.n_cams} cameras, {sc.n_pp} point pairs",
               "max_rounds": rounds,
               "irls_fp32": arm_result(sc, "irls", "fp32", rounds),
               "learned_fp16": arm_result(sc, "learned", "fp16", rounds)}
        res["speedup_learned_fp16_over_irls_fp32_at"] = _speedups(res, "irls_fp32", "learned_fp16")
        out[args.config] = res
        # the same comparison at the same size on the closed trajectory (4,000 cameras in 40 laps),
        # where the objective's minimum lies near the truth and 0.1 deg is within reach
        if args.config != "loop4000":
            sc = scenegen.make_scene("loop4000", seed=args.seed, device="cuda")
            torch.cuda.empty_cache()
            res = {"scene": f"loop4000 seed {args.seed}: {sc.n_cams} cameras, {sc.n_pp} point pairs",
                   "max_rounds": rounds,
                   "irls_fp32": arm_result(sc, "irls", "fp32", rounds),
                   "learned_fp16": arm_result(sc, "learned", "fp16", rounds)}
            res["speedup_learned_fp16_over_irls_fp32"] = (
                res["irls_fp32"]["ms"] / res["learned_fp16"]["ms"]
                if res["irls_fp32"]["reached"] and res["learned_fp16"]["reached"] else None)
            res["speedup_learned_fp16_over_irls_fp32_at"] = _speedups(res, "irls_fp32", "learned_fp16")
            out["loop4000"] = res
            del sc
            torch.cuda.empty_cache()
    net.close()
    return out


def translation_section(sc, stream, runs: int = 8, iters: int = 1000, final_iters: int = 1000):
    """Global translation (centres from unit relative translations, rotations fixed) on the
    scene's image pairs: 1 deg noise per pair, 5% wrong pairs; `runs` random starts advanced
    together, merged, then one final run."""
    import numpy as np
    import torch
    import scenegen
    import paper_2605_18052_gb300 as fm
    R = sc.R_gt.cpu().numpy()
    t_rel, _ = scenegen.relative_translations(sc, 1.0, 0.05, 0)
    inits = np.random.default_rng(0).normal(size=(runs, sc.n_cams, 3))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    with fm.Translation(R, sc.cam_i.cpu().numpy(), sc.cam_j.cpu().numpy(), t_rel, inits,
                        fm.translation_options(lr=1e-2), stream=stream.cuda_stream) as tr:
        tr.step(16)                       # warm-up (graph build)
        tr.set_centres(inits)
        torch.cuda.synchronize()
        ev[0].record(stream)
        tr.step(iters)
        ev[1].record(stream)
        tr.merge()
        tr.set_learning_rate(2e-3)
        ev[2].record(stream)
        tr.step(final_iters)
        ev[3].record(stream)
        o = tr.centres()[0]
    torch.cuda.synchronize()
    C = -(sc.R_gt.double().transpose(1, 2) @ sc.t_gt.double()[:, :, None])[:, :, 0].cpu().numpy()

    def norm(x):
        x = x - x.mean(0)
        return x / np.linalg.norm(x, axis=1).mean()

    err = np.linalg.norm(norm(o) - norm(C), axis=1)
    runs_ms = ev[0].elapsed_time(ev[1])
    final_ms = ev[2].elapsed_time(ev[3])
    # the same solve on the 128-camera sphere scene, where random starts reach the centres
    from paper_2605_18052_gb300 import translation as gtr
    sp = scenegen.make_scene("sphere128", seed=0)
    t_sp, _ = scenegen.relative_translations(sp, 1.0, 0.05, 0)
    o_sp, _ = gtr.solve(sp.R_gt.numpy(), sp.cam_i.numpy(), sp.cam_j.numpy(), t_sp, n_runs=runs, iters=iters,
                        final_iters=final_iters, lr=1e-2, final_lr=2e-3)
    C_sp = -(sp.R_gt.double().transpose(1, 2) @ sp.t_gt.double()[:, :, None])[:, :, 0].numpy()
    err_sp = np.linalg.norm(o_sp - norm(C_sp), axis=1)
    # and on the 1,000-camera closed trajectory (only its cameras and image pairs matter here):
    # random starts unfold there, but the 20 laps need more and larger steps than the sphere
    lp = scenegen.make_scene("loop1000", seed=0, n_pts=20_000, counts=("lognormal", 60.0, 0.9, 400))
    t_lp, _ = scenegen.relative_translations(lp, 1.0, 0.05, 0)
    lp_iters, lp_final = 4 * iters, 2 * final_iters
    o_lp, _ = gtr.solve(lp.R_gt.numpy(), lp.cam_i.numpy(), lp.cam_j.numpy(), t_lp, n_runs=runs, iters=lp_iters,
                        final_iters=lp_final, lr=3e-2, final_lr=3e-3)
    C_lp = -(lp.R_gt.double().transpose(1, 2) @ lp.t_gt.double()[:, :, None])[:, :, 0].numpy()
    err_lp = np.linalg.norm(o_lp - norm(C_lp), axis=1)
    return {"pairs": sc.n_pairs, "cameras": sc.n_cams, "runs": runs, "iters": iters, "final_iters": final_iters,
            "iteration_us_all_runs": runs_ms / iters * 1e3, "iteration_us_final": final_ms / final_iters * 1e3,
            "pair_terms_per_s": runs * sc.n_pairs * iters / (runs_ms * 1e-3),
            "solve_ms": runs_ms + ev[1].elapsed_time(ev[2]) + final_ms,
            "median_centre_error": float(np.median(err)), "p95_centre_error": float(np.quantile(err, 0.95)),
            "sphere128_median_centre_error": float(np.median(err_sp)),
            "sphere128_p95_centre_error": float(np.quantile(err_sp, 0.95)),
            "loop1000_median_centre_error": float(np.median(err_lp)),
            "loop1000_p95_centre_error": float(np.quantile(err_lp, 0.95)),
            "loop1000_iters": [lp_iters, lp_final], "loop1000_lr": [3e-2, 3e-3],
            "note": "centre errors after normalising both to zero mean and unit mean norm; on the "
                    "4,000-camera open trajectory (a chain of overlapping views) random starts do not "
                    "unfold within the iteration budget, on the 128-camera sphere and the 1,000-camera "
                    "closed trajectory (4x the runs' iterations at 3x the step size) they do"}


def rotation_section(sc, stream, iters: int = 500):
    """Global rotation on the scene's image pairs (relative rotations with 1 deg noise; pairs
    with wrong relative rotations are filtered upstream in the pipeline): column-wise
    initialisation (conjugate gradients), then `iters` Adam steps on the geodesic objective.
    The robustness to wrong pairs is shown on the 128-camera sphere with 5% of them."""
    import numpy as np
    import torch
    import scenegen
    import paper_2605_18052_gb300 as fm
    from paper_2605_18052_gb300 import metrics

    def run(scene, outliers, timed):
        Rrel, _ = scenegen.relative_rotations(scene, 1.0, outliers, 0)
        Rg = scene.R_gt.cpu().numpy()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        with fm.Rotation(scene.cam_i.cpu().numpy(), scene.cam_j.cpu().numpy(), Rrel, scene.n_cams,
                         fm.rotation_options(lr=1e-3), stream=stream.cuda_stream) as rp:
            if timed:
                rp.initialize()             # warm-up
                rp.step(16)
            torch.cuda.synchronize()
            ev[0].record(stream)
            cg_iters, cg_res = rp.initialize()
            ev[1].record(stream)
            e0 = float(metrics.rotation_error_deg(rp.rotations(), Rg).mean())
            torch.cuda.synchronize()
            ev[2].record(stream)
            rp.step(iters)
            ev[3].record(stream)
            R1 = rp.rotations()
        torch.cuda.synchronize()
        e1 = float(metrics.rotation_error_deg(R1, Rg).mean())
        it_ms = ev[2].elapsed_time(ev[3])
        return {"pairs": scene.n_pairs, "cameras": scene.n_cams, "wrong_pairs": outliers,
                "init_ms": ev[0].elapsed_time(ev[1]), "cg_iterations": cg_iters,
                "cg_relative_residual": cg_res, "init_rotation_error_deg": e0, "iters": iters,
                "iteration_us": it_ms / iters * 1e3, "pair_terms_per_s": scene.n_pairs * iters / (it_ms * 1e-3),
                "refined_rotation_error_deg": e1}

    out = run(sc, 0.0, True)
    out["sphere128_5pct_wrong_pairs"] = run(scenegen.make_scene("sphere128", seed=0), 0.05, False)
    # the 1,000-camera closed trajectory (only its cameras and image pairs matter here), whose
    # loop closures pin the rotations the open chain leaves loose
    lp = scenegen.make_scene("loop1000", seed=0, n_pts=20_000, counts=("lognormal", 60.0, 0.9, 400))
    out["loop1000"] = run(lp, 0.0, False)
    out["loop1000_5pct_wrong_pairs"] = run(lp, 0.05, False)
    return out


def focal_section(args, sc, sch, stream, n_pp: int, pose_only_ms: float):
    """The benchmark's step with refine_focal=1 on a second problem over the same point pairs."""
    import torch
    import paper_2605_18052_gb300 as fm
    gf = fm.Problem(sc.R_init.cpu(), sc.t_init.cpu(), sc.cam_i.cpu(), sc.cam_j.cpu(), sc.pair_id,
                    sc.x1, sc.x2, options=sch.options(storage=args.storage, refine_focal=1))
    try:
        for r in range(args.warmup):
            gf.step_irls(sch.tau(r % sch.rounds), args.iters)
        gf.synchronize()
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for k in range(args.steps):
            gf.step_irls(sch.tau((args.warmup + k) % sch.rounds), args.iters)
        f1.record(stream)
        torch.cuda.synchronize()
        f_ms = f0.elapsed_time(f1) / args.steps
        s = gf.focal_scales()
    finally:
        gf.close()
    return {"value": float(n_pp) * args.iters / (f_ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": f_ms,
            "time_vs_pose_only": f_ms / pose_only_ms,
            "scales_min_max": [float(s.min()), float(s.max())],
            "note": "same step (1 fused IRLS round + iters iterations) with the focal scales s_k optimised "
                    "with the poses; the point pairs are those of the pose-only line"}


# algorithmic bytes per point pair of each timed pass, by storage (reads + writes)
PASS_BYTES = {
    "stream_loss": {"fp16": 10, "fp32": 20},        # keypoints + weight
    "stream_reweight": {"fp16": 10, "fp32": 20},    # keypoints in, weight out
    "quad_accumulate": {"fp16": 10, "fp32": 20},    # keypoints in, weight out
    "learned_loss": {"fp16": 16, "fp32": 26},       # keypoints, score, history in; weight, history out
    "pair_stats": {"fp16": 8, "fp32": 16},          # keypoints
}
# FP32 FMA-pipe operations per point pair of the form pass (9 residual, ~5 weight, 10 monomial
# products, 46 multiply-adds into the sums); the pipe's peak is 152 SMs x 128 lanes x clock
QUAD_FMA_OPS = 66
FP32_LANES = 152 * 128


def pass_entry(name, storage, config, n_pp, ms, launches, peak, sm_mhz):
    if not launches:
        return {"unavailable": "no timed launches"}
    us = ms / launches * 1e3
    gbs = n_pp * PASS_BYTES[name][storage] / (us * 1e-6) / 1e9
    e = {"us_per_launch": us, "launches": launches, "bytes_per_point_pair": PASS_BYTES[name][storage],
         "achieved_gbs": gbs, "hbm_frac": gbs / peak, "g_point_pairs_per_s": n_pp / (us * 1e-6) / 1e9}
    if name in KERNEL_SOURCES:   # DRAM bytes per launch from the committed ncu summary, if current
        e["traffic"] = profiled_traffic(f"{name}_{storage}_{config}")
    if name == "quad_accumulate":
        t = n_pp * QUAD_FMA_OPS / (us * 1e-6) / 1e12
        pk = FP32_LANES * (sm_mhz or 2070.0) * 1e6 / 1e12
        e.update({"fma_ops_per_point_pair": QUAD_FMA_OPS, "achieved_tfma_s": t, "fp32_pipe_peak_tfma_s": pk,
                  "fp32_pipe_frac": t / pk})
    return e


def passes_section(args, gp, sc, sch, n_pp, peak, sm_mhz, reweight_timed):
    """CUDA-event times of the once-per-round passes on the benchmark workload, against the HBM
    roofline (and the FP32 pipe for the form pass)."""
    import numpy as np
    from paper_2605_18052_gb300 import Mlp, binding
    out = {"stream_reweight": pass_entry("stream_reweight", args.storage, args.config, n_pp, *reweight_timed, peak,
                                         sm_mhz)}
    gp.enable_kernel_timing(True)
    for k in range(args.steps // 4 + 3):
        gp.irls_preaggregate(sch.tau(k % sch.rounds))
    gp.synchronize()
    gp.pass_time(binding.PASS_QUAD_ACCUMULATE)      # drop the warm-up launches
    for k in range(args.steps // 4):
        gp.irls_preaggregate(sch.tau(k % sch.rounds))
    out["quad_accumulate"] = pass_entry("quad_accumulate", args.storage, args.config, n_pp,
                                        *gp.pass_time(binding.PASS_QUAD_ACCUMULATE), peak, sm_mhz)
    path = os.path.join(ROOT, "paper_2605_18052_gb300", "data", "mlp_inlier.npy")
    if os.path.exists(path):
        net = Mlp(np.load(path))
        gp.set_scores(sc.score)
        gp.reset_history()
        for r in range(3):
            gp.step_learned(net, sch.tau(r), sch.tau(r), r, 1)
        gp.synchronize()
        gp.pass_time(binding.PASS_LEARNED_LOSS)
        gp.pass_time(binding.PASS_PAIR_STATS)
        for r in range(3, 3 + args.steps // 4):
            gp.step_learned(net, sch.tau(r), sch.tau(r), r, 1)
        out["learned_loss"] = pass_entry("learned_loss", args.storage, args.config, n_pp,
                                         *gp.pass_time(binding.PASS_LEARNED_LOSS), peak, sm_mhz)
        out["pair_stats"] = pass_entry("pair_stats", args.storage, args.config, n_pp,
                                       *gp.pass_time(binding.PASS_PAIR_STATS), peak, sm_mhz)
        net.close()
    gp.enable_kernel_timing(False)
    out["note"] = ("each pass timed alone with CUDA events on the problem's stream (no overlap with its "
                   "neighbours); bytes are algorithmic (reads + writes per point pair)")
    return out


def configs_section(args, peak, bench_scene=None):
    """The other workloads of the benchmark: microseconds per iteration of one IRLS round and the
    loss+gradient pass against the HBM roofline. ring16 and sphere128 fit in L2 (129 MB): their
    rates are L2-resident, not HBM figures."""
    import torch
    import scenegen
    import paper_2605_18052_gb300 as fm
    l2_bytes = 129e6
    out = {}
    cases = [("ring16", "fp32"), ("sphere128", "fp32"), ("traj1000", "fp16"), ("traj1000", "fp32")]
    if bench_scene is not None:
        cases.append((args.config, "fp32" if args.storage == "fp16" else "fp16"))
    scenes = {}
    for cfg, storage in cases:
        sc = bench_scene if (cfg == args.config and bench_scene is not None) else scenes.get(cfg)
        if sc is None:
            sc = scenegen.make_scene(cfg, seed=0, device="cuda")
            scenes = {cfg: sc}
            torch.cuda.empty_cache()
        sch = schedule_for(sc, args.iters)
        with fm.Problem(sc.R_init.cpu(), sc.t_init.cpu(), sc.cam_i.cpu(), sc.cam_j.cpu(), sc.pair_id, sc.x1, sc.x2,
                        options=sch.options(storage=storage)) as gp:
            info = gp.info()
            for r in range(3):
                gp.step_irls(sch.tau(r), args.iters)
            gp.synchronize()
            stream = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            steps = max(5, args.steps // 5)
            torch.cuda.synchronize()
            e0.record(stream)
            for r in range(steps):
                gp.step_irls(sch.tau((3 + r) % sch.rounds), args.iters)
            e1.record(stream)
            torch.cuda.synchronize()
            round_ms = e0.elapsed_time(e1) / steps
            gp.enable_kernel_timing(True)
            for r in range(steps):
                gp.step_irls(sch.tau((3 + r) % sch.rounds), args.iters)
            k_ms, k_n = gp.kernel_time()
            gp.enable_kernel_timing(False)
        n_pp = info["n_pp"]
        bytes_pass = info["stream_bytes"]
        us = k_ms / max(1, k_n) * 1e3
        gbs = bytes_pass / (us * 1e-6) / 1e9
        resident = bytes_pass < l2_bytes
        out[f"{cfg}_{storage}"] = {
            "workload": f"{cfg}: {sc.n_cams} cameras, {sc.n_pairs} image pairs, {n_pp} point pairs",
            "storage": storage, "us_per_iteration": round_ms / args.iters * 1e3,
            "g_point_pairs_per_s": n_pp * args.iters / (round_ms * 1e-3) / 1e9,
            "stream_loss_us": us, "stream_loss_gbs": gbs,
            "hbm_frac": None if resident else gbs / peak,
            "l2_resident": resident,
            "note": "L2-resident: not an HBM number" if resident else "inputs larger than L2"}
    return out


def focal_vote_section(sc, n_cand: int = 256, tau: float = 0.05):
    """The focal-length vote (fm_focal_vote) over the scene's image pairs: fundamental matrices
    from the true poses with 1e-3 calibrated noise and 10% wrong pairs, f = 500 px, candidates
    300..800 px. Reports the kernels' device time and candidate-pair terms per second."""
    import numpy as np
    import scenegen
    import paper_2605_18052_gb300 as fm
    F, _ = scenegen.fundamental_matrices(sc, 1e-3, 0.1, 0)
    cands = np.linspace(300.0, 800.0, n_cand)
    fm.focal_vote(F, cands, tau)                       # warm-up
    times = []
    for _ in range(5):
        v, ms = fm.focal_vote(F, cands, tau, timed=True)
        times.append(ms)
    ms = sorted(times)[len(times) // 2]
    terms = len(F) * n_cand
    return {"pairs": len(F), "candidates": n_cand, "tau": tau, "ms": ms,
            "g_terms_per_s": terms / (ms * 1e-3) / 1e9, "estimate_px": float(cands[int(np.argmax(v))]),
            "true_px": 500.0,
            "note": "one term = E = K2^T F K1, E^T E, four Jacobi sweeps, ratio, exp (about 300 FP32 "
                    "operations); ALU-bound"}


def oracle_sample(sc):
    """The CPU baseline's sample: the first whole image pairs up to 4 M point pairs, as an
    oracle problem, with the initial poses."""
    import numpy as np
    import oracle as O
    cnt = np.bincount(sc.pair_id.cpu().numpy(), minlength=sc.n_pairs)
    target = 4_000_000
    nb = int(np.searchsorted(np.cumsum(cnt), target)) + 1
    nb = min(nb, sc.n_pairs)
    npp = int(cnt[:nb].sum())
    pid = sc.pair_id[:npp].cpu().numpy()
    prob = O.Problem(sc.n_cams, sc.cam_i.cpu().numpy(), sc.cam_j.cpu().numpy(), pid,
                     sc.x1[:npp].cpu().numpy(), sc.x2[:npp].cpu().numpy())
    R0 = sc.R_init.cpu().numpy()
    c0 = O.centres_from_poses(R0, sc.t_init.cpu().numpy())
    return prob, R0, c0, nb, npp


def cpu_oracle_rate(sc, seconds: float, sample=None):
    """FP64 oracle loss+gradient on a bounded sample of whole image pairs (1 thread)."""
    import numpy as np
    import oracle as O
    prob, R0, c0, nb, npp = sample if sample is not None else oracle_sample(sc)
    w = np.ones(npp)
    evals = 0
    t0 = time.perf_counter()
    while True:
        O.loss_grad(prob, R0, c0, w)
        evals += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return evals * npp / el / 1e9, f"first {nb} image pairs ({npp} point pairs), {evals} loss+grad evaluations"


def _oracle_worker(args):
    """One process of the all-cores CPU baseline: the oracle's loss+gradient on its share of
    the sample, repeated for `seconds`; returns point pairs evaluated and the elapsed time."""
    n_cams, ci, cj, pid, x1, x2, R0, c0, seconds = args
    import numpy as np
    import oracle as O
    prob = O.Problem(n_cams, ci, cj, pid, x1, x2)
    w = np.ones(pid.shape[0])
    evals = 0
    t0 = time.perf_counter()
    while True:
        O.loss_grad(prob, R0, c0, w)
        evals += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return evals * pid.shape[0], el


def cpu_oracle_rate_all_cores(sc, seconds: float):
    """The same oracle, one process per host core, each on a disjoint block of whole image
    pairs of the same sample (processes started with spawn: this runs after CUDA work)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import numpy as np
    cores = os.cpu_count() or 1
    cnt = np.bincount(sc.pair_id.cpu().numpy(), minlength=sc.n_pairs)
    target = 4_000_000
    nb = min(int(np.searchsorted(np.cumsum(cnt), target)) + 1, sc.n_pairs)
    off = np.concatenate([[0], np.cumsum(cnt[:nb])])
    cuts = np.linspace(0, nb, cores + 1).astype(int)
    pid_all = sc.pair_id.cpu().numpy()
    x1_all, x2_all = sc.x1.cpu().numpy(), sc.x2.cpu().numpy()
    ci_all, cj_all = sc.cam_i.cpu().numpy(), sc.cam_j.cpu().numpy()
    R0 = sc.R_init.cpu().numpy()
    c0 = -(np.einsum("nba,nb->na", R0, sc.t_init.cpu().numpy()))
    jobs = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        if b <= a:
            continue
        lo, hi = int(off[a]), int(off[b])
        jobs.append((sc.n_cams, ci_all[a:b], cj_all[a:b], pid_all[lo:hi] - a, x1_all[lo:hi], x2_all[lo:hi],
                     R0, c0, seconds))
    with cf.ProcessPoolExecutor(max_workers=len(jobs), mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_oracle_worker, jobs))
    pp = sum(r[0] for r in res)
    el = max(r[1] for r in res)
    return pp / el / 1e9, len(jobs)


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part", "processor\t")) and ":" in line:
                    v = line.split(":", 1)[1].strip()
                    if v and not v.isdigit():
                        import platform
                        return f"{platform.machine()} {v}"
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def bench_config(args, sc, world: int) -> dict:
    """The workload description both arms report."""
    return {"workload": f"{args.config}: {sc.n_cams} cameras, {sc.n_pairs} image pairs, {sc.n_pp} point pairs",
            "storage": args.storage, "iters_per_step": args.iters,
            "step": "1 IRLS round: reweighting (fused into the first pass) + iters x (loss+grad, Adam)",
            "l2": "inputs larger than L2 (no flush needed)",
            "parallelism": f"replicas x{world}"}


def run_reference(args, rank):
    import torch
    import scenegen
    if rank != 0:
        return
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    sc = scenegen.make_scene(args.config, seed=args.seed, device=dev).to("cpu")
    # about 6 x --cpu-seconds of oracle work over the whole run (a minute by default)
    per_step = 6.0 * args.cpu_seconds / max(1, args.steps + args.warmup)
    vals = []
    sample = ""
    prepared = oracle_sample(sc)
    for k in range(args.warmup + args.steps):
        v, sample = cpu_oracle_rate(sc, per_step if k >= args.warmup else min(0.5, per_step), prepared)
        if k >= args.warmup:
            vals.append(v)
    value = statistics.median(vals)
    npp_total = sc.n_pp
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": args.iters * npp_total / (value * 1e9) * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded scene generator)",
           "config": bench_config(args, sc, args.gpus),
           "implementation": "FP64 CPU oracle (plain C loops), 1 thread, on a bounded sample of the workload",
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                            "seconds_per_iteration": npp_total / (value * 1e9)},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_sharded(args, rank, world, local):
    """One problem split across the ranks: rank r holds the point pairs of a contiguous range of
    whole image pairs (balanced by point-pair count) and a replica of all poses; every iteration
    is fm_loss_grad_device on its shard into one device buffer, an in-place NCCL all-reduce of
    that buffer, and fm_apply_gradient from it (the device data plane of shard.py). A step is
    one IRLS round (local reweighting + iters iterations); total work is fixed (strong scaling)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    import scenegen
    import paper_2605_18052_gb300 as fm
    from paper_2605_18052_gb300 import shard

    sc = scenegen.make_scene(args.config, seed=args.seed, device="cuda")
    torch.cuda.empty_cache()
    sch = schedule_for(sc, args.iters)
    counts = torch.bincount(sc.pair_id.long(), minlength=sc.n_pairs).cpu().numpy()
    b, e = shard.partition_pairs(counts, world)[rank]
    lo, hi = shard.shard_point_pairs(sc.pair_id.cpu().numpy(), b, e)
    if hi <= lo:
        raise SystemExit(f"rank {rank} received no point pairs (more ranks than image pairs)")
    opt = sch.options(storage=args.storage, z_total=sc.n_pp)
    gp = fm.Problem(sc.R_init.cpu(), sc.t_init.cpu(), sc.cam_i[b:e].cpu(), sc.cam_j[b:e].cpu(),
                    (sc.pair_id[lo:hi] - b).contiguous(), sc.x1[lo:hi].contiguous(), sc.x2[lo:hi].contiguous(),
                    options=opt)
    adj = shard.ShardedAdjustment(shard.DeviceGpuShard(gp))

    def one_step(r):
        s = sch.decay ** (r % sch.rounds)
        adj.round(sch.tau(r % sch.rounds), args.iters, sch.lr_rot * s, sch.lr_c * s)

    for r in range(args.warmup):
        one_step(r)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local, args.clocks_csv) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for k in range(args.steps):
            one_step(args.warmup + k)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = torch.tensor([ev0.elapsed_time(ev1)], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(ms, op=dist.ReduceOp.MAX)
        dist.barrier()
    ms_max = float(ms.item())
    value = float(sc.n_pp) * args.iters * args.steps / (ms_max * 1e-3) / 1e9
    R_out, _ = gp.get_poses()
    gp.close()
    if rank == 0:
        from paper_2605_18052_gb300 import metrics
        err = float(metrics.rotation_error_deg(R_out, sc.R_gt.cpu().numpy()).mean())
        cfg = bench_config(args, sc, world)
        cfg["parallelism"] = f"image-pair shards x{world}"
        cfg["step"] = "1 IRLS round: local reweighting + iters x (shard loss+grad, all-reduce, Adam)"
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
               "scaling": "strong", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic (seeded scene generator; every rank builds the same scene and keeps its shard)",
               "config": cfg, "roofline": None, "cpu_baseline": None, "e2e": None,
               "gpu_launches": args.steps * (1 + 2 + 6 * args.iters),
               "shard": {"pairs": [b, e], "point_pairs": hi - lo,
                         "mean_rotation_error_deg_after": err},
               "clocks": clk.summary(),
               "note": "roofline, CPU baseline and end-to-end figures are reported by the replica mode"}
        print(json.dumps(out))


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import numpy as np
    import torch
    import torch.distributed as dist
    import scenegen
    import paper_2605_18052_gb300 as fm
    from paper_2605_18052_gb300 import build as fm_build

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        fm_build.build()
    if world > 1:
        dist.barrier()
    fm.load_library()
    if args.shard:
        run_sharded(args, rank, world, local)
        if world > 1:
            dist.destroy_process_group()
        return

    # each rank: its own seeded scene (weak scaling: replicas, no data-path collective)
    sc = scenegen.make_scene(args.config, seed=args.seed + rank, device="cuda")
    torch.cuda.empty_cache()   # drop the generator's temporaries
    sch = schedule_for(sc, args.iters)
    opt = sch.options(storage=args.storage)
    stream = torch.cuda.current_stream()
    gp = fm.Problem(sc.R_init.cpu(), sc.t_init.cpu(), sc.cam_i.cpu(), sc.cam_j.cpu(), sc.pair_id,
                    sc.x1, sc.x2, options=opt)
    info = gp.info()
    n_pp = info["n_pp"]

    def one_step(r):
        gp.step_irls(sch.tau(r % sch.rounds), args.iters)

    for r in range(args.warmup):
        one_step(r)
    gp.synchronize()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local, args.clocks_csv) as clk:
        # timed region: the production path (CUDA graphs of chained iterations)
        torch.cuda.synchronize()
        ev0.record(stream)
        for k in range(args.steps):
            one_step(args.warmup + k)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        # second timed region, same steps, with CUDA events around every launch of the
        # streaming kernel on the problem's stream (eager launches): its mean duration
        gp.enable_kernel_timing(True)
        for k in range(args.steps):
            one_step(args.warmup + args.steps + k)
        kern_ms, kern_n = gp.kernel_time()
        reweight_timed = gp.pass_time(fm.binding.PASS_STREAM_REWEIGHT)
        gp.enable_kernel_timing(False)
        torch.cuda.synchronize()
    t_local = torch.tensor([ms], dtype=torch.float64, device="cuda")
    pp_local = torch.tensor([float(n_pp) * args.iters * args.steps], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t_local, op=dist.ReduceOp.MAX)
        dist.all_reduce(pp_local, op=dist.ReduceOp.SUM)
    ms_max = float(t_local.item())
    value = float(pp_local.item()) / (ms_max * 1e-3) / 1e9

    # roofline of the dominant kernel (loss+gradient stream)
    bytes_per_launch = info["stream_bytes"]
    avg_launch_s = kern_ms * 1e-3 / max(1, kern_n)
    achieved = bytes_per_launch / avg_launch_s / 1e9
    peak, peak_kind = peaks()
    tag = f"stream_loss_{args.storage}_{args.config}"
    traffic = profiled_traffic(tag)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": f"k_stream_loss<{args.storage.upper()}, IRLS>",
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs burst copy)" if peak_kind == "measured" else "fallback 6.8 TB/s",
                "bytes_per_launch": bytes_per_launch, "avg_launch_us": avg_launch_s * 1e6}
    # global translation stage on the same scene's image pairs (8 runs from random centres),
    # global rotation stage on them (initialisation + refinement)
    trans = rot = None
    if rank == 0 and not args.no_translation:
        trans = translation_section(sc, stream)
        rot = rotation_section(sc, stream)

    clocks = clk.summary()
    passes = configs = None
    if rank == 0 and not args.no_passes:
        try:
            passes = passes_section(args, gp, sc, sch, n_pp, peak, clocks.get("sm_mhz"), reweight_timed)
        except Exception as e:   # recorded; the main line stands
            passes = {"unavailable": f"{type(e).__name__}: {str(e)[:300]}"}

    # per step: 3 launches per iteration (the first one's pass fused with the reweighting), one
    # finalize after the fused iteration and one per graph launch of the rest (graphs of 8
    # chained iterations, then single iterations)
    rest = args.iters - 1
    launches = args.steps * (3 * args.iters + 1 + rest // 8 + rest % 8)

    # the same rounds on the pre-aggregated quadratic form: one pass over the point pairs per
    # round (reweighting fused with the form), iterations in O(image pairs)
    quad = None
    if not args.no_quad:
        def quad_round(r):
            gp.irls_preaggregate(sch.tau(r % sch.rounds))
            gp.step_quadratic(args.iters)
        for r in range(args.warmup):
            quad_round(r)
        torch.cuda.synchronize()
        q0 = torch.cuda.Event(enable_timing=True)
        q1 = torch.cuda.Event(enable_timing=True)
        q2 = torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        for k in range(args.steps):
            quad_round(args.warmup + k)
        q1.record(stream)
        for k in range(args.steps):
            gp.step_quadratic(args.iters)
        q2.record(stream)
        torch.cuda.synchronize()
        q_ms = q0.elapsed_time(q1) / args.steps
        it_us = q1.elapsed_time(q2) / args.steps / args.iters * 1e3
        quad = {"ms_per_step": q_ms, "iteration_us": it_us,
                "reweight_and_form_ms": q_ms - it_us * args.iters * 1e-3,
                "equivalent_value": float(n_pp) * args.iters / (q_ms * 1e-3) / 1e9, "unit": UNIT,
                "form_pass_traffic": profiled_traffic(f"quad_accumulate_{args.storage}_{args.config}"),
                "note": "same step (1 reweighting round + iters iterations) with the gradient taken from the "
                        "per-image-pair quadratic form; equivalent_value counts the point pairs the "
                        "streaming path would have read"}

    # the same rounds with the focal lengths refined together with the poses (F = S_j E S_i):
    # the streaming pass reads the same bytes, the camera step also moves rho_k = log s_k
    focal = None
    if not args.no_focal:
        try:
            focal = focal_section(args, sc, sch, stream, n_pp, ms_max / args.steps)
        except Exception as e:   # recorded; the main line stands
            focal = {"unavailable": f"{type(e).__name__}: {str(e)[:200]}"}

    # end to end through the public API with pinned host buffers: create + full schedule + poses
    e2e = None
    if not args.no_e2e:
        h = {k: getattr(sc, k).cpu().pin_memory() for k in ("pair_id", "x1", "x2")}
        Rh, th = sc.R_init.cpu(), sc.t_init.cpu()
        cih, cjh = sc.cam_i.cpu(), sc.cam_j.cpu()
        del gp
        torch.cuda.synchronize()
        times, parts = [], []
        for k in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            jp = fm.Problem(Rh, th, cih, cjh, h["pair_id"], h["x1"], h["x2"], options=opt)
            t1 = time.perf_counter()
            fm.refine(jp, sch)
            R_out, t_out = jp.get_poses()
            t2 = time.perf_counter()
            jp.close()
            t3 = time.perf_counter()
            times.append(t3 - t0)
            parts.append((t1 - t0, t2 - t1, t3 - t2))
        t_job = statistics.median(times[1:])
        e2e_pp = float(n_pp) * sch.rounds * sch.iters_per_round
        e2e = {"value": e2e_pp / t_job / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(n_pp * (4 + 8 + 8) + sc.n_cams * 12 * 8 + sc.n_pairs * 8),
               "d2h_bytes_per_step": int(sc.n_cams * 12 * 8),
               "job": f"fm_create_problem from pinned host buffers + {sch.rounds} rounds x {sch.iters_per_round} iterations + fm_get_poses",
               "seconds_per_job": t_job,
               "seconds_create_refine_destroy": [round(statistics.median(x[i] for x in parts[1:]), 5) for i in range(3)]}

    tta = None
    if rank == 0 and not args.no_tta:
        try:
            tta = time_to_accuracy_section(args, sc)
        except Exception as e:   # recorded; the main line stands
            tta = {"unavailable": f"{type(e).__name__}: {str(e)[:300]}"}

    if rank == 0 and not args.no_configs:
        try:
            configs = configs_section(args, peak, sc)
        except Exception as e:   # recorded; the main line stands
            configs = {"unavailable": f"{type(e).__name__}: {str(e)[:300]}"}

    focal_vote = None
    if rank == 0 and not args.no_focal:
        try:
            focal_vote = focal_vote_section(sc)
        except Exception as e:
            focal_vote = {"unavailable": f"{type(e).__name__}: {str(e)[:300]}"}

    cpu = None
    if rank == 0 and not args.no_cpu:
        v, sample = cpu_oracle_rate(sc, args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
               "seconds_per_iteration": n_pp / (v * 1e9),
               "host_cores": os.cpu_count(), "cpu_model": cpu_model()}
        try:
            va, procs = cpu_oracle_rate_all_cores(sc, args.cpu_seconds)
            cpu["all_cores"] = {"value": va, "unit": UNIT, "cores": procs,
                                "seconds_per_iteration": n_pp / (va * 1e9),
                                "sample": "the same image pairs split into one block per process"}
        except Exception as e:   # a host that cannot start processes keeps the 1-thread figure
            cpu["all_cores"] = {"unavailable": str(e)[:200]}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic (seeded scene generator, trajectory scene shaped like the paper's large scenes)",
               "config": bench_config(args, sc, world),
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
               "time_to_accuracy": tta, "quadratic_path": quad, "global_translation": trans,
               "global_rotation": rot, "focal_refinement": focal, "focal_vote": focal_vote,
               "passes": passes, "configs": configs,
               "clocks": clocks, "hbm_frac_of_step": value * 1e9 * bytes_per_launch / n_pp / 1e9 / peak}
        print(json.dumps(out))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
