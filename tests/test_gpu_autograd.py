"""The torch.autograd.Function form of the objective: forward = one fused loss/adjoint pass,
backward = the stashed per-camera gradient (or a recomputed pass), checked against the C ABI,
through a rotation parameterisation, and on the 1,000-camera trajectory scene (FP16 storage)
against the oracle's analytic gradient and against FP64 central differences of the oracle
loss on 32 random cameras."""
import numpy as np
import pytest
import torch

import oracle as O
import scenegen
import paper_2605_18052_gb300 as fm
from paper_2605_18052_gb300 import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    build.build()
    fm.load_library()


def _torch_exp(phi):
    """Rodrigues in torch (test-side parameterisation only)."""
    th = torch.linalg.norm(phi, dim=1, keepdim=True).clamp_min(1e-30)[..., None]
    K = torch.zeros(phi.shape[0], 3, 3, dtype=phi.dtype, device=phi.device)
    K[:, 0, 1], K[:, 0, 2], K[:, 1, 2] = -phi[:, 2], phi[:, 1], -phi[:, 0]
    K = K - K.transpose(1, 2)
    eye = torch.eye(3, dtype=phi.dtype, device=phi.device)
    return eye + torch.sin(th) / th * K + (1 - torch.cos(th)) / th ** 2 * (K @ K)


def test_autograd_matches_c_abi_and_parameterisation():
    sc = scenegen.make_scene("ring16", seed=11)
    R0, t0 = sc.R_init.numpy(), sc.t_init.numpy()
    c0 = O.centres_from_poses(R0, t0)
    w = np.random.default_rng(0).uniform(0, 10, sc.n_pp).astype(np.float32)
    with fm.Problem(R0, t0, sc.cam_i, sc.cam_j, sc.pair_id, sc.x1, sc.x2) as gp:
        gp.set_weights(w)
        l_ref, g_ref = gp.loss_grad()
        dev = torch.device("cuda")
        phi = torch.zeros(sc.n_cams, 3, dtype=torch.float64, device=dev, requires_grad=True)
        c = torch.tensor(c0, device=dev, requires_grad=True)
        Rb = torch.tensor(R0, device=dev)
        for recompute in (False, True):
            phi.grad = None
            c.grad = None
            loss = fm.epipolar_loss(gp, _torch_exp(phi) @ Rb, c, recompute=recompute)
            (3.0 * loss).backward()
            assert loss.item() == pytest.approx(l_ref, rel=1e-12)
            # at phi = 0 the exponential map's Jacobian is the identity
            np.testing.assert_allclose(phi.grad.cpu().numpy(), 3.0 * g_ref[:, :3], rtol=1e-9,
                                       atol=1e-12 * np.abs(g_ref).max())
            np.testing.assert_allclose(c.grad.cpu().numpy(), 3.0 * g_ref[:, 3:], rtol=1e-12, atol=0)


def _sub_problem(prob, cams, n_total):
    """Point pairs of the pairs touching any camera in `cams` (losses rescaled to the full Z)."""
    pairs = np.flatnonzero(np.isin(prob.cam_i, cams) | np.isin(prob.cam_j, cams))
    sel = np.isin(prob.pair_id, pairs)
    remap = -np.ones(prob.n_pairs, np.int64)
    remap[pairs] = np.arange(len(pairs))
    sub = O.Problem(prob.n_cams, prob.cam_i[pairs], prob.cam_j[pairs], remap[prob.pair_id[sel]],
                    prob.x1[sel], prob.x2[sel])
    return sub, sel, sub.n_pp / n_total


def test_fd_on_32_cameras_of_the_1000_camera_scene():
    sc = scenegen.make_scene("traj1000", seed=0, device="cuda")
    torch.cuda.empty_cache()
    R0 = sc.R_init.cpu().numpy()
    c0 = O.centres_from_poses(R0, sc.t_init.cpu().numpy())
    rng = np.random.default_rng(1)
    w = rng.uniform(0.0, 5.0, sc.n_pp).astype(np.float32)
    gp = fm.Problem(sc.R_init.cpu(), sc.t_init.cpu(), sc.cam_i.cpu(), sc.cam_j.cpu(), sc.pair_id,
                    sc.x1, sc.x2, options=fm.default_options(storage="fp16"))
    gp.set_weights(w)
    R = torch.tensor(R0, device="cuda", requires_grad=True)
    c = torch.tensor(c0, device="cuda", requires_grad=True)
    loss = fm.epipolar_loss(gp, R, c)
    loss.backward()
    Rn = R.detach().cpu().numpy()
    gR = R.grad.cpu().numpy()
    M = np.einsum("nab,ncb->nac", gR, Rn)  # 0.5 [g_phi]_x
    g_phi = np.stack([M[:, 2, 1] - M[:, 1, 2], M[:, 0, 2] - M[:, 2, 0], M[:, 1, 0] - M[:, 0, 1]], 1)
    g_gpu = np.concatenate([g_phi, c.grad.cpu().numpy()], 1)
    gp.close()

    # oracle on the exact (dequantized FP16) inputs and quantized weights
    x1 = sc.x1.cpu().numpy()
    x2 = sc.x2.cpu().numpy()
    base = O.Problem(sc.n_cams, sc.cam_i.cpu().numpy(), sc.cam_j.cpu().numpy(), sc.pair_id.cpu().numpy(), x1, x2)
    _, d1, d2 = O.fp16_centroid_storage(base, x1, x2)
    prob = O.Problem(sc.n_cams, base.cam_i, base.cam_j, base.pair_id, d1, d2)
    wq = O.quantize_weights_fp16(w, 1e-6)
    l_or, g_or = O.loss_grad(prob, R0, c0, wq)
    assert loss.item() == pytest.approx(l_or, rel=1e-4)
    assert np.abs(g_gpu - g_or).max() <= 1e-4 * np.abs(g_or).max()

    # FP64 central differences of the oracle loss on 32 random cameras; only the pairs that
    # touch camera k change, so the difference is taken on that sub-problem
    for k in rng.choice(sc.n_cams, 32, replace=False):
        sub, sel, frac = _sub_problem(prob, [k], prob.n_pp)
        ws = wq[sel]
        fd = np.zeros(6)
        for q in range(6):
            Rp, Rm, cp, cm = R0.copy(), R0.copy(), c0.copy(), c0.copy()
            h = 1e-6
            if q < 3:
                e = np.zeros(3)
                e[q] = h
                Rp[k] = O.expmap(e) @ R0[k]
                Rm[k] = O.expmap(-e) @ R0[k]
            else:
                cp[k, q - 3] += h
                cm[k, q - 3] -= h
            fd[q] = (O.loss_grad(sub, Rp, cp, ws)[0] - O.loss_grad(sub, Rm, cm, ws)[0]) / (2 * h) * frac
        assert np.abs(g_gpu[k] - fd).max() <= 1e-4 * np.abs(fd).max() + 1e-9 * np.abs(g_or).max(), (k, g_gpu[k], fd)
