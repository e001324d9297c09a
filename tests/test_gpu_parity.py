"""Parity of the CUDA path (through the C ABI) against the FP64 oracle on identical inputs.

Tolerances:
  * loss: relative 1e-4 (FP32 per-point-pair terms summed per warp range and then in FP64).
  * gradient: max |g_gpu - g_oracle| <= 1e-4 * max |g_oracle| over the whole (n_cams x 6)
    gradient, and per camera and block (rotation, centre) |dg_k| <= 1e-4 |g_k| + 1e-7 max |g|
    (tests/bounds.py states why: the FP32 pair sums carry about 1e-7 of their gross magnitude,
    so a component that cancels to near zero cannot be held to a purely relative bound); for the
    L1 objective plus the largest change of the sign decisions within the residual bound.
  * residuals: absolute 2e-6 in normalized units (FP32 forward error of a 3x3 bilinear form
    with |E| <= 1, |x| <= 1: about 12 roundings of terms <= 3, i.e. < 12 * 2^-24 * 3).
  * IRLS mask: identical except where the oracle's |eps| is within that residual bound of
    the threshold; weights: relative (bound / max(|eps|, delta)) + 2^-22 (+ 2^-11 for FP16).
Inputs for the FP16 path are the oracle's own restatement of the storage rule (centroid by
exact integer sums, FP16 offsets), never values read back from the GPU.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
import scenegen
from bounds import assert_grad_close, l1_flip_allowance
import paper_2605_18052_gb300 as fm
from paper_2605_18052_gb300 import build

pytestmark = pytest.mark.gpu

RESID_ATOL = 2e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    build.build()
    fm.load_library()


def _scene(name="ring16", seed=0, **kw):
    return scenegen.make_scene(name, seed=seed, **kw)


def _oracle_inputs(sc, storage, delta=1e-6):
    """Oracle problem on exactly the inputs the GPU path computes with."""
    prob = O.Problem.from_scene(sc)
    if storage == "fp16":
        _, d1, d2 = O.fp16_centroid_storage(prob, sc.x1.numpy(), sc.x2.numpy())
        prob = O.Problem(sc.n_cams, prob.cam_i, prob.cam_j, prob.pair_id, d1, d2)
    return prob


def _assert_grad_close(g, ref, tol=1e-4, allowance=None):
    assert_grad_close(g, ref, tol, allowance=allowance)


def _gpu_problem(sc, R, t, **opt):
    return fm.Problem(R, t, sc.cam_i, sc.cam_j, sc.pair_id, sc.x1, sc.x2,
                      options=fm.default_options(**opt))


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
@pytest.mark.parametrize("loss", ["irls", "l1"])
@pytest.mark.parametrize("name", ["ring16", "sphere128"])
def test_loss_grad_parity(name, loss, storage):
    sc = _scene(name)
    R0, t0 = sc.R_init.numpy(), sc.t_init.numpy()
    c0 = O.centres_from_poses(R0, t0)
    prob = _oracle_inputs(sc, storage)
    rng = np.random.default_rng(1)
    with _gpu_problem(sc, R0, t0, storage=storage, loss=loss) as gp:
        w = None
        if loss == "irls":
            w32 = rng.uniform(0.0, 50.0, sc.n_pp).astype(np.float32)
            gp.set_weights(w32)
            w = O.quantize_weights_fp16(w32, 1e-6) if storage == "fp16" else w32.astype(np.float64)
        l_gpu, g_gpu = gp.loss_grad()
    l_or, g_or = O.loss_grad(prob, R0, c0, w, loss)
    assert l_gpu == pytest.approx(l_or, rel=1e-4)
    allow = l1_flip_allowance(prob, R0, c0, O.residuals(prob, R0, c0), RESID_ATOL) if loss == "l1" else None
    _assert_grad_close(g_gpu, g_or, allowance=allow)


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_residual_parity_elementwise(storage):
    sc = _scene("sphere128")
    R0, t0 = sc.R_init.numpy(), sc.t_init.numpy()
    prob = _oracle_inputs(sc, storage)
    with _gpu_problem(sc, R0, t0, storage=storage) as gp:
        e_gpu = gp.residuals().astype(np.float64)
    e_or = O.residuals(prob, R0, O.centres_from_poses(R0, t0))
    assert np.abs(e_gpu - e_or).max() <= RESID_ATOL


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_irls_weights_parity(storage):
    sc = _scene("sphere128", seed=1)
    R0, t0 = sc.R_init.numpy(), sc.t_init.numpy()
    prob = _oracle_inputs(sc, storage)
    e_or = O.residuals(prob, R0, O.centres_from_poses(R0, t0))
    delta = 1e-6
    for tau in (0.02, math.inf):
        w_or, kept_or = O.irls_weights(e_or, tau, delta)
        with _gpu_problem(sc, R0, t0, storage=storage) as gp:
            kept = gp.irls_weights(tau)
            w_gpu = gp.get_weights().astype(np.float64)
        a = np.abs(e_or)
        undecided = np.abs(a - tau) <= RESID_ATOL
        mask_gpu, mask_or = w_gpu > 0, w_or > 0
        assert np.array_equal(mask_gpu[~undecided], mask_or[~undecided])
        assert abs(kept - kept_or) <= undecided.sum()
        both = mask_gpu & mask_or
        rel = np.abs(w_gpu[both] - w_or[both]) / w_or[both]
        bound = RESID_ATOL / np.maximum(a[both], delta) + 2.0 ** -22
        if storage == "fp16":
            bound += 2.0 ** -11
        assert (rel <= bound).all()


def test_unsorted_input_matches_sorted():
    sc = _scene("ring16", seed=2)
    R0, t0 = sc.R_init.numpy(), sc.t_init.numpy()
    perm = np.random.default_rng(3).permutation(sc.n_pp)
    for storage in ("fp32", "fp16"):
        with _gpu_problem(sc, R0, t0, storage=storage) as gs:
            e_s = gs.residuals()
            l_s, g_s = gs.loss_grad()
            assert gs.info()["input_was_sorted"] == 1
        with fm.Problem(R0, t0, sc.cam_i, sc.cam_j, sc.pair_id[perm], sc.x1[perm], sc.x2[perm],
                        options=fm.default_options(storage=storage)) as gu:
            assert gu.info()["input_was_sorted"] == 0
            e_u = gu.residuals()
            l_u, g_u = gu.loss_grad()
            w = np.random.default_rng(4).uniform(0, 3, sc.n_pp).astype(np.float32)
            gu.set_weights(w)
            np.testing.assert_array_equal(gu.get_weights(), w if storage == "fp32"
                                          else O.quantize_weights_fp16(w, 1e-6).astype(np.float32))
        # residuals are per point pair: identical bits, returned in input order
        np.testing.assert_array_equal(e_u, e_s[perm])
        assert l_u == pytest.approx(l_s, rel=1e-6)
        _assert_grad_close(g_u, g_s, 1e-5)


def _ragged_problem(sizes, n_cams=4, seed=0):
    """Pairs with the given point-pair counts, cycling over camera pairs, all noise-free
    projections of random points (so the layout's boundaries, not the data, are tested)."""
    rng = np.random.default_rng(seed)
    sc = _scene("ring16", seed=seed, sigma_px=0.0, outlier=0.0)
    R, t = sc.R_gt.numpy()[:n_cams], sc.t_gt.numpy()[:n_cams]
    C = O.centres_from_poses(R, t)
    pairs = [(i, j) for i in range(n_cams) for j in range(i + 1, n_cams)]
    cam_i, cam_j, pid, x1, x2 = [], [], [], [], []
    for n, m in enumerate(sizes):
        i, j = pairs[n % len(pairs)]
        cam_i.append(i)
        cam_j.append(j)
        X = rng.normal(0, 0.4, (m, 3))
        for k, xs in ((i, x1), (j, x2)):
            Xc = (R[k] @ (X - C[k]).T).T
            xs.append(Xc[:, :2] / Xc[:, 2:3] + rng.normal(0, 0.002, (m, 2)))
        pid.append(np.full(m, n, np.int32))
    return (R, t, np.array(cam_i, np.int32), np.array(cam_j, np.int32), np.concatenate(pid),
            np.concatenate(x1).astype(np.float32), np.concatenate(x2).astype(np.float32))


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
@pytest.mark.parametrize("sizes", [
    [1],                                         # one point pair in total
    [1, 1, 1],                                   # every pair a single point pair
    [2047, 2049, 1, 3, 4096, 5000, 1, 65, 63],   # pairs across warp-range boundaries
    [2048, 2048, 1, 4095],                       # pairs ending exactly on range boundaries
    [12345],                                     # a pair longer than several ranges
    list(range(1, 200)),                         # many short pairs inside one range
])
def test_ragged_layouts(sizes, storage):
    R, t, ci, cj, pid, x1, x2 = _ragged_problem(sizes)
    rng = np.random.default_rng(5)
    R1 = np.array([O.expmap(rng.normal(0, 0.03, 3)) @ r for r in R])
    c1 = O.centres_from_poses(R, t) + rng.normal(0, 0.05, (len(R), 3))
    t1 = O.poses_from_centres(R1, c1)
    prob = O.Problem(len(R), ci, cj, pid, x1, x2)
    if storage == "fp16":
        _, d1, d2 = O.fp16_centroid_storage(prob, x1, x2)
        prob = O.Problem(len(R), ci, cj, pid, d1, d2)
    w = rng.uniform(0.5, 2.0, len(pid)).astype(np.float32)
    wq = O.quantize_weights_fp16(w, 1e-6) if storage == "fp16" else w.astype(np.float64)
    with fm.Problem(R1, t1, ci, cj, pid, x1, x2, options=fm.default_options(storage=storage)) as gp:
        gp.set_weights(w)
        l_gpu, g_gpu = gp.loss_grad()
        e_gpu = gp.residuals()
    l_or, g_or = O.loss_grad(prob, R1, c1, wq)
    assert l_gpu == pytest.approx(l_or, rel=1e-4)
    _assert_grad_close(g_gpu, g_or)
    assert np.abs(e_gpu - O.residuals(prob, R1, c1)).max() <= RESID_ATOL


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_optimizer_steps_match_oracle(storage):
    # K Adam iterations from the same poses with the same weights
    sc = _scene("ring16", seed=6)
    R0, t0 = sc.R_init.numpy(), sc.t_init.numpy()
    c0 = O.centres_from_poses(R0, t0)
    prob = _oracle_inputs(sc, storage)
    w = O.irls_weights(O.residuals(prob, R0, c0), 0.05, 1e-6)[0]
    wq = O.quantize_weights_fp16(w, 1e-6) if storage == "fp16" else w.astype(np.float32).astype(np.float64)
    lr_r, lr_c = 5e-3, 5e-3 * 3.0
    with _gpu_problem(sc, R0, t0, storage=storage, lr_rot=lr_r, lr_c=lr_c) as gp:
        gp.set_weights(w.astype(np.float32))
        gp.step(25)
        R_g, t_g = gp.get_poses()
        _, _, steps = gp.get_state()
    assert steps == 25
    R_o, c_o = R0.copy(), c0.copy()
    m = np.zeros((sc.n_cams, 6))
    v = np.zeros((sc.n_cams, 6))
    for k in range(25):
        _, g = O.loss_grad(prob, R_o, c_o, wq)
        O.adam_step(R_o, c_o, g, m, v, k + 1, lr_r, lr_c)
    ang = np.degrees(np.arccos(np.clip((np.einsum("nab,nab->n", R_g, R_o) - 1) / 2, -1, 1)))
    c_g = O.centres_from_poses(R_g, t_g)
    # 25 steps of at most lr each: the paths agree to a small fraction of one step
    assert ang.max() < 0.02 * np.degrees(lr_r)
    assert np.abs(c_g - c_o).max() < 0.02 * lr_c


def test_refine_schedule_matches_oracle_accuracy():
    sc = _scene("ring16", seed=0)
    R0, t0 = sc.R_init.numpy(), sc.t_init.numpy()
    Rg = sc.R_gt.numpy()
    cg = O.centres_from_poses(Rg, sc.t_gt.numpy())
    prob = O.Problem.from_scene(sc)
    base = float(np.median(np.linalg.norm(cg[prob.cam_i] - cg[prob.cam_j], axis=1)))
    sch = fm.Schedule(rounds=12, iters_per_round=25, tau0=0.5, tau_min=4 * sc.sigma_px / sc.f,
                      tau_factor=0.8, decay=0.95, lr_rot=1e-2, lr_c=1e-2 * base)
    with _gpu_problem(sc, R0, t0) as gp:
        fm.refine(gp, sch)
        R_g, t_g = gp.get_poses()
    R_o, c_o, _ = O.refine(prob, R0, O.centres_from_poses(R0, t0), sch.rounds, sch.iters_per_round,
                           sch.tau0, sch.tau_min, 1e-6, sch.lr_rot, sch.lr_c, sch.decay,
                           tau_factor=sch.tau_factor)
    e_g = O.rotation_error_deg(R_g, Rg).mean()
    e_o = O.rotation_error_deg(R_o, Rg).mean()
    e0 = O.rotation_error_deg(R0, Rg).mean()
    # Over many rounds the two trajectories are not comparable point by point: mask decisions
    # at the filtering threshold and Adam's sign-like normalisation of near-zero gradient
    # components amplify rounding differences (the 25-step test above is the pointwise
    # check). Both loops must reach the same accuracy.
    assert e_g < 0.5 * e0
    assert e_g <= 1.3 * e_o + 0.02 and e_o <= 1.3 * e_g + 0.02, (e_g, e_o)


def test_determinism_and_resume_bit_exact():
    sc = _scene("sphere128", seed=2)
    R0, t0 = sc.R_init.numpy(), sc.t_init.numpy()
    outs = []
    for _ in range(2):
        with _gpu_problem(sc, R0, t0) as gp:
            gp.irls_weights(0.05)
            gp.step(10)
            l, g = gp.loss_grad()
            outs.append((l, g, *gp.get_poses()))
    assert outs[0][0] == outs[1][0]
    for a, b in zip(outs[0][1:], outs[1][1:]):
        np.testing.assert_array_equal(a, b)
    # checkpoint after 5 iterations, resume in a fresh problem
    with _gpu_problem(sc, R0, t0) as gp:
        gp.irls_weights(0.05)
        gp.step(5)
        R5, c5 = gp.get_params()
        m, v, s = gp.get_state()
        w = gp.get_weights()
        gp.step(5)
        Ra, ca = gp.get_params()
    with _gpu_problem(sc, R0, t0) as gp:
        gp.set_params(R5, c5)
        gp.set_weights(w)
        gp.set_state(m, v, s)
        gp.step(5)
        Rb, cb = gp.get_params()
    np.testing.assert_array_equal(Ra, Rb)
    np.testing.assert_array_equal(ca, cb)


def test_graph_and_eager_iterations_agree():
    sc = _scene("ring16", seed=7)
    R0, t0 = sc.R_init.numpy(), sc.t_init.numpy()
    res = []
    for use_graph in (1, 0):
        with _gpu_problem(sc, R0, t0, use_graph=use_graph) as gp:
            gp.step(7)
            res.append(gp.get_poses())
    np.testing.assert_array_equal(res[0][0], res[1][0])
    np.testing.assert_array_equal(res[0][1], res[1][1])


def test_kernel_timing_counts_launches():
    sc = _scene("ring16", seed=8)
    with _gpu_problem(sc, sc.R_init.numpy(), sc.t_init.numpy()) as gp:
        gp.enable_kernel_timing(True)
        gp.step(6)
        ms, n = gp.kernel_time()
    assert n == 6 and ms > 0


def test_invalid_inputs_are_rejected():
    R, t, ci, cj, pid, x1, x2 = _ragged_problem([10, 10, 10])
    bad = [
        dict(pid=np.where(pid == 2, 3, pid).astype(np.int32)),   # pair index out of range
        dict(pid=np.where(pid == 1, 0, pid).astype(np.int32)),   # pair 1 left empty
        dict(x1=np.where(np.arange(len(pid))[:, None] == 4, np.nan, x1).astype(np.float32)),
        dict(x2=np.full_like(x2, 9.0)),                          # |coordinate| > 8
    ]
    for b in bad:
        with pytest.raises(fm.FastMapError) as ei:
            fm.Problem(R, t, ci, cj, b.get("pid", pid), b.get("x1", x1), b.get("x2", x2))
        assert ei.value.status == -1
    with fm.Problem(R, t, ci, cj, pid, x1, x2) as gp:
        with pytest.raises(fm.FastMapError):
            gp.set_weights(np.full(len(pid), -1.0, np.float32))
        gp.set_weights(np.ones(len(pid), np.float32))
        # two cameras at the same centre: zero-length relative translation on the device
        R2, t2 = R.copy(), t.copy()
        C = O.centres_from_poses(R2, t2)
        C[1] = C[0]
        gp.set_poses(R2, O.poses_from_centres(R2, C))
        with pytest.raises(fm.FastMapError) as ei:
            gp.loss_grad()
        assert ei.value.status == -4
        gp.set_poses(R, t)   # recovers
        gp.loss_grad()


def test_two_shards_on_one_gpu_sum_to_the_whole_problem():
    from paper_2605_18052_gb300.shard import partition_pairs, shard_point_pairs
    sc = _scene("sphere128", seed=9)
    R0, t0 = sc.R_init.numpy(), sc.t_init.numpy()
    pid = sc.pair_id.numpy()
    counts = np.bincount(pid, minlength=sc.n_pairs)
    ci, cj = sc.cam_i.numpy(), sc.cam_j.numpy()
    x1, x2 = sc.x1.numpy(), sc.x2.numpy()
    shards = []
    for b, e in partition_pairs(counts, 2):
        lo, hi = shard_point_pairs(pid, b, e)
        shards.append(fm.Problem(R0, t0, ci[b:e], cj[b:e], pid[lo:hi] - b, x1[lo:hi], x2[lo:hi],
                                 options=fm.default_options(z_total=sc.n_pp)))
    with _gpu_problem(sc, R0, t0) as whole:
        l_w, g_w = whole.loss_grad()
        parts = [s.loss_grad() for s in shards]
        assert sum(p[0] for p in parts) == pytest.approx(l_w, rel=1e-6)
        _assert_grad_close(sum(p[1] for p in parts), g_w, 1e-5)
        # ten replicated steps with the summed gradient follow the unsharded loop
        for _ in range(10):
            g = sum(s.loss_grad()[1] for s in shards)
            for s in shards:
                s.apply_gradient(g)
            whole.step(1)
        Rw, tw = whole.get_poses()
        R0s, t0s = shards[0].get_poses()
        R1s, _ = shards[1].get_poses()
    np.testing.assert_array_equal(R0s, R1s)
    # the summed gradient differs from the whole problem's in its last bits, and Adam's
    # normalisation turns a last-bit difference of a near-zero component into a visible step
    # difference; as for the oracle comparison, the paths agree to a small fraction of one step
    # (lr_rot = 1e-2 rad by default)
    ang = np.degrees(np.arccos(np.clip((np.einsum("nab,nab->n", Rw, R0s) - 1) / 2, -1, 1)))
    assert ang.max() < 0.02 * np.degrees(1e-2)
    for s in shards:
        s.close()


def test_apply_gradient_is_the_optimiser_step():
    # fm_apply_gradient with the problem's own gradient takes the same step as fm_step, bit for
    # bit: the FP64 gradient rounds to the FP32 value the camera step uses (hi of its
    # compensated hi + lo sum), and both run the same update
    sc = _scene("sphere128", seed=10)
    R0, t0 = sc.R_init.numpy(), sc.t_init.numpy()
    with _gpu_problem(sc, R0, t0) as a, _gpu_problem(sc, R0, t0) as b:
        a.irls_weights(0.05)
        b.irls_weights(0.05)
        for _ in range(10):
            a.apply_gradient(a.loss_grad()[1])
            b.step(1)
        Ra, ta = a.get_poses()
        Rb, tb = b.get_poses()
        assert a.get_state()[2] == b.get_state()[2] == 10
        np.testing.assert_array_equal(Ra, Rb)
        np.testing.assert_array_equal(ta, tb)
        assert a.loss_grad()[0] == b.loss_grad()[0]


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
@pytest.mark.parametrize("tau", [0.05, math.inf])
def test_fused_reweighting_round_is_bit_identical(storage, tau):
    # fm_step_irls = fm_irls_weights + fm_step with the reweighting inside the first pass
    sc = _scene("sphere128", seed=3)
    R0, t0 = sc.R_init.numpy(), sc.t_init.numpy()
    res = []
    for fused in (False, True):
        with _gpu_problem(sc, R0, t0, storage=storage) as gp:
            if fused:
                kept = gp.step_irls(tau, 9, count=True)
            else:
                kept = gp.irls_weights(tau)
                gp.step(9)
            res.append((kept, gp.get_weights(), gp.get_params(), gp.last_loss(), gp.get_state()[2]))
    (k0, w0, p0, l0, s0), (k1, w1, p1, l1, s1) = res
    assert k0 == k1 and s0 == s1 == 9 and l0 == l1
    np.testing.assert_array_equal(w0, w1)
    np.testing.assert_array_equal(p0[0], p1[0])
    np.testing.assert_array_equal(p0[1], p1[1])
