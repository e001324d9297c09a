"""fm_loss_grad_noalloc: loss and gradient for callers that cannot call cudaMalloc (device
memory owned by another memory manager, or a loop that cannot afford cudaMalloc's implicit
device synchronisation). Its intermediates live in a fixed __device__ array of the library.

Checked through the C ABI against the FP64 oracle and against the existing entry point
(fm_create_problem + fm_loss_grad) with the parity tolerance of the other tests (loss relative
1e-4; gradient within 1e-4 of its largest entry and per camera, tests/bounds.py), on two calls
in a row of different sizes (stale scratch from the first call must not leak into the second),
plus: a repeated call is bit-identical, device free memory does not change across a call,
sizes beyond the limits are refused, and invalid device data (offsets that do not rise, a pair
of one camera with itself, a coordinate beyond 8, a negative weight) is refused with FM_EINVAL
after which a valid call still gives the right result from the shared array.
This file is collected after the other parity files (only the full-size checks follow), so a
run that stops at the first failure has run them first.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
import scenegen
from bounds import assert_grad_close
import paper_2605_18052_gb300 as fm
from paper_2605_18052_gb300 import binding, build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    build.build()
    return binding.load_library()


def _inputs(sc, mode, seed):
    rng = np.random.default_rng(seed)
    R = sc.R_init.numpy()
    t = sc.t_init.numpy()
    w = rng.uniform(0.0, 20.0, sc.n_pp).astype(np.float32)
    dev = torch.device("cuda")
    c = -np.einsum("nba,nb->na", R, t)
    pid = sc.pair_id.long()
    off = torch.zeros(sc.n_pairs + 1, dtype=torch.int32)
    off[1:] = torch.cumsum(torch.bincount(pid, minlength=sc.n_pairs), 0).to(torch.int32)
    d = {
        "R": torch.as_tensor(R.reshape(-1, 9), dtype=torch.float64, device=dev).contiguous(),
        "c": torch.as_tensor(c, dtype=torch.float64, device=dev).contiguous(),
        "ci": sc.cam_i.to(dev).contiguous(), "cj": sc.cam_j.to(dev).contiguous(),
        "off": off.to(dev), "kp": torch.cat([sc.x1, sc.x2], 1).to(dev).contiguous(),
        "w": torch.as_tensor(w, device=dev), "loss": torch.zeros(1, dtype=torch.float64, device=dev),
        "grad": torch.zeros(sc.n_cams * 6, dtype=torch.float64, device=dev),
    }
    return R, t, w, d


def _status(lib, sc, d, mode):
    P = lambda x: ctypes.c_void_p(x.data_ptr())
    return lib.fm_loss_grad_noalloc(sc.n_cams, P(d["R"]), P(d["c"]), sc.n_pairs, P(d["ci"]), P(d["cj"]),
                                    P(d["off"]), sc.n_pp, P(d["kp"]), P(d["w"]), mode, P(d["loss"]),
                                    P(d["grad"]), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _call(lib, sc, d, mode):
    st = _status(lib, sc, d, mode)
    assert st == 0, lib.fm_last_error().decode()
    return float(d["loss"].item()), d["grad"].cpu().numpy().reshape(-1, 6)


def _oracle(sc, R, t, w, mode):
    prob = O.Problem.from_scene(sc)
    c = O.centres_from_poses(R, t)
    if mode == fm.FM_LOSS_IRLS:
        return O.loss_grad(prob, R, c, w.astype(np.float64), "irls")
    return O.loss_grad(prob, R, c, None, "l1")


def _reference(sc, R, t, w, mode):
    with fm.Problem(R, t, sc.cam_i, sc.cam_j, sc.pair_id, sc.x1, sc.x2,
                    options=fm.default_options(loss=mode)) as gp:
        if mode == fm.FM_LOSS_IRLS:
            gp.set_weights(w)
        return gp.loss_grad()


def _close(l, g, l_ref, g_ref):
    assert l == pytest.approx(l_ref, rel=1e-4)
    assert_grad_close(g, g_ref)


def test_noalloc_matches_loss_grad_on_two_calls(lib):
    big = scenegen.make_scene("sphere128", seed=3)
    small = scenegen.make_scene("ring16", seed=4)
    R1, t1, w1, d1 = _inputs(big, fm.FM_LOSS_IRLS, 1)
    R2, t2, w2, d2 = _inputs(small, fm.FM_LOSS_L1, 2)
    ref1 = _reference(big, R1, t1, w1, fm.FM_LOSS_IRLS)
    ref2 = _reference(small, R2, t2, w2, fm.FM_LOSS_L1)
    torch.cuda.synchronize()

    l1, g1 = _call(lib, big, d1, fm.FM_LOSS_IRLS)        # first call on this device
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    l2, g2 = _call(lib, small, d2, fm.FM_LOSS_L1)        # second call, smaller problem
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    _close(l1, g1, *ref1)
    _close(l2, g2, *ref2)
    _close(l1, g1, *_oracle(big, R1, t1, w1, fm.FM_LOSS_IRLS))
    _close(l2, g2, *_oracle(small, R2, t2, w2, fm.FM_LOSS_L1))
    assert free_after == free_before

    l3, g3 = _call(lib, small, d2, fm.FM_LOSS_L1)        # same inputs again: same bits
    assert l3 == l2
    np.testing.assert_array_equal(g3, g2)


def test_noalloc_refuses_sizes_beyond_its_limits(lib):
    z = ctypes.c_void_p(16)   # never dereferenced: sizes are checked first
    cases = [(4097, 10, 100), (2, 32769, 40000), (2, 1, (1 << 26) + 1), (1, 1, 1)]
    for n_cams, n_pairs, n_pp in cases:
        st = lib.fm_loss_grad_noalloc(n_cams, z, z, n_pairs, z, z, z, n_pp, z, None, 0, z, z, None)
        assert st == -1
        assert "fm_loss_grad_noalloc" in lib.fm_last_error().decode()


def test_noalloc_refuses_invalid_device_data_then_recovers(lib):
    # each case corrupts one device input (all reads stay inside the caller's buffers), is
    # refused with FM_EINVAL, and the valid call that follows still matches the oracle
    sc = scenegen.make_scene("ring16", seed=6)
    R, t, w, d = _inputs(sc, fm.FM_LOSS_IRLS, 3)
    ref = _oracle(sc, R, t, w, fm.FM_LOSS_IRLS)

    def corrupt(key, index, value, col=None):
        saved = d[key].clone()
        if col is None:
            d[key][index] = value
        else:
            d[key][index, col] = value
        st = _status(lib, sc, d, fm.FM_LOSS_IRLS)
        msg = lib.fm_last_error().decode()
        d[key].copy_(saved)
        return st, msg

    cases = [("off", 3, int(d["off"][2].item()), None),          # offsets do not rise
             ("cj", 5, int(d["ci"][5].item()), None),             # cam_i == cam_j
             ("ci", 0, sc.n_cams, None),                          # camera index out of range
             ("kp", 7, 9.0, 2),                                   # |coordinate| > 8
             ("kp", 11, float("nan"), 0),                         # non-finite coordinate
             ("w", 13, -1.0, None)]                               # negative weight
    for key, index, value, col in cases:
        st, msg = corrupt(key, index, value, col)
        assert st == -1, (key, index, value, msg)
        assert "fm_loss_grad_noalloc" in msg
        l, g = _call(lib, sc, d, fm.FM_LOSS_IRLS)
        _close(l, g, *ref)
