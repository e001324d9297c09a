"""ctypes binding of libfastmap (include/fastmap.h): argument marshalling only.

Every computation runs in the library's CUDA kernels. If the library is missing this module
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfastmap.so")

FM_STORE_FP32, FM_STORE_FP16 = 0, 1
FM_LOSS_IRLS, FM_LOSS_L1 = 0, 1
# timed passes (fm_pass_time)
PASS_STREAM_LOSS, PASS_STREAM_REWEIGHT, PASS_QUAD_ACCUMULATE, PASS_LEARNED_LOSS, PASS_PAIR_STATS = range(5)

EXPORTED = [
    "fm_default_options", "fm_create_problem", "fm_destroy_problem", "fm_problem_info",
    "fm_get_poses", "fm_set_poses", "fm_get_params", "fm_set_params", "fm_set_params_device", "fm_set_weights", "fm_get_weights", "fm_irls_weights",
    "fm_loss_grad", "fm_loss_grad_device", "fm_residuals", "fm_step", "fm_step_irls", "fm_last_loss",
    "fm_set_learning_rate", "fm_reset_optimizer", "fm_get_state", "fm_set_state",
    "fm_synchronize", "fm_apply_gradient", "fm_enable_kernel_timing", "fm_kernel_time", "fm_pass_time",
    "fm_loss_grad_noalloc",
    "fm_status_string", "fm_last_error", "fm_mlp_num_params", "fm_mlp_create", "fm_mlp_destroy",
    "fm_mlp_get_params", "fm_mlp_set_params", "fm_mlp_train_step", "fm_mlp_gradient", "fm_mlp_forward",
    "fm_set_scores", "fm_collect_features", "fm_learned_weights", "fm_step_learned", "fm_reset_history",
    "fm_preaggregate", "fm_irls_preaggregate", "fm_loss_grad_quadratic", "fm_step_quadratic",
    "fm_set_focal_learning_rate", "fm_get_focal_scales", "fm_set_focal_scales", "fm_get_focal_gradient",
    "fm_translation_default_options", "fm_translation_create", "fm_translation_destroy",
    "fm_translation_num_runs", "fm_translation_loss_grad", "fm_translation_step", "fm_translation_merge",
    "fm_translation_set_learning_rate", "fm_translation_get_centres", "fm_translation_set_centres",
    "fm_rotation_default_options", "fm_rotation_create", "fm_rotation_destroy", "fm_rotation_initialize",
    "fm_rotation_loss_grad", "fm_rotation_step", "fm_rotation_set_learning_rate", "fm_rotation_get_rotations",
    "fm_rotation_get_params", "fm_rotation_set_rotations", "fm_rotation_set_params", "fm_focal_vote",
]


class FastMapError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int32), ("loss", ctypes.c_int32), ("delta", ctypes.c_double),
                ("lr_rot", ctypes.c_double), ("lr_c", ctypes.c_double), ("beta1", ctypes.c_double),
                ("beta2", ctypes.c_double), ("adam_eps", ctypes.c_double),
                ("use_graph", ctypes.c_int32), ("refine_focal", ctypes.c_int32), ("z_total", ctypes.c_int64)]


class Info(ctypes.Structure):
    _fields_ = [("n_cams", ctypes.c_int32), ("n_pairs", ctypes.c_int32), ("n_pp", ctypes.c_int64),
                ("storage", ctypes.c_int32), ("loss", ctypes.c_int32),
                ("n_warp_ranges", ctypes.c_int64), ("stream_bytes", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("input_was_sorted", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libfastmap.so (built by paper_2605_18052_gb300.build); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FastMapError(-3, f"{path} is missing: build it with paper_2605_18052_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "fm_default_options": (None, [P]),
        "fm_create_problem": (I32, [I32, P, P, I32, P, P, I64, P, P, P, I32, P, P, P]),
        "fm_destroy_problem": (None, [P]),
        "fm_problem_info": (I32, [P, P]),
        "fm_get_poses": (I32, [P, P, P]),
        "fm_set_poses": (I32, [P, P, P]),
        "fm_get_params": (I32, [P, P, P]),
        "fm_set_params": (I32, [P, P, P]),
        "fm_set_params_device": (I32, [P, P, P]),
        "fm_set_weights": (I32, [P, P, I32]),
        "fm_get_weights": (I32, [P, P]),
        "fm_irls_weights": (I32, [P, D, P]),
        "fm_loss_grad": (I32, [P, P, P]),
        "fm_loss_grad_device": (I32, [P, P, P]),
        "fm_residuals": (I32, [P, P]),
        "fm_step": (I32, [P, I32]),
        "fm_step_irls": (I32, [P, D, I32, P]),
        "fm_last_loss": (I32, [P, P]),
        "fm_set_learning_rate": (I32, [P, D, D]),
        "fm_reset_optimizer": (I32, [P]),
        "fm_get_state": (I32, [P, P, P, P]),
        "fm_set_state": (I32, [P, P, P, I64]),
        "fm_synchronize": (I32, [P]),
        "fm_apply_gradient": (I32, [P, P, I32]),
        "fm_enable_kernel_timing": (I32, [P, I32]),
        "fm_kernel_time": (I32, [P, P, P]),
        "fm_pass_time": (I32, [P, I32, P, P]),
        "fm_loss_grad_noalloc": (I32, [I32, P, P, I32, P, P, P, I64, P, P, I32, P, P, P]),
        "fm_mlp_num_params": (I32, []),
        "fm_mlp_create": (I32, [P, P]),
        "fm_mlp_destroy": (None, [P]),
        "fm_mlp_get_params": (I32, [P, P]),
        "fm_mlp_set_params": (I32, [P, P]),
        "fm_mlp_train_step": (I32, [P, P, P, I32, ctypes.c_float, P, P]),
        "fm_mlp_gradient": (I32, [P, P, P, I32, P, P]),
        "fm_mlp_forward": (I32, [P, P, I32, P, P]),
        "fm_set_scores": (I32, [P, P, I32]),
        "fm_collect_features": (I32, [P, D, I32, P]),
        "fm_learned_weights": (I32, [P, P, D, D, I32, P]),
        "fm_step_learned": (I32, [P, P, D, D, I32, I32, P]),
        "fm_reset_history": (I32, [P]),
        "fm_preaggregate": (I32, [P]),
        "fm_irls_preaggregate": (I32, [P, D, P]),
        "fm_loss_grad_quadratic": (I32, [P, P, P]),
        "fm_step_quadratic": (I32, [P, I32]),
        "fm_set_focal_learning_rate": (I32, [P, D]),
        "fm_get_focal_scales": (I32, [P, P]),
        "fm_set_focal_scales": (I32, [P, P]),
        "fm_get_focal_gradient": (I32, [P, P]),
        "fm_translation_default_options": (None, [P]),
        "fm_translation_create": (I32, [I32, P, I32, P, P, P, I32, P, P, P, P]),
        "fm_translation_destroy": (None, [P]),
        "fm_translation_num_runs": (I32, [P]),
        "fm_translation_loss_grad": (I32, [P, P, P, P]),
        "fm_translation_step": (I32, [P, I32]),
        "fm_translation_merge": (I32, [P]),
        "fm_translation_set_learning_rate": (I32, [P, D]),
        "fm_translation_get_centres": (I32, [P, P]),
        "fm_translation_set_centres": (I32, [P, P]),
        "fm_rotation_default_options": (None, [P]),
        "fm_rotation_create": (I32, [I32, I32, P, P, P, P, P, P]),
        "fm_rotation_destroy": (None, [P]),
        "fm_rotation_initialize": (I32, [P, P, P]),
        "fm_rotation_loss_grad": (I32, [P, P, P]),
        "fm_rotation_step": (I32, [P, I32]),
        "fm_rotation_set_learning_rate": (I32, [P, D]),
        "fm_rotation_get_rotations": (I32, [P, P]),
        "fm_rotation_get_params": (I32, [P, P]),
        "fm_rotation_set_rotations": (I32, [P, P]),
        "fm_rotation_set_params": (I32, [P, P]),
        "fm_focal_vote": (I32, [I32, P, P, P, I32, P, D, P, P, P]),
        "fm_status_string": (ctypes.c_char_p, [I32]),
        "fm_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        lib = load_library()
        raise FastMapError(status, lib.fm_last_error().decode() or lib.fm_status_string(status).decode())


def default_options(**kw) -> Options:
    o = Options()
    load_library().fm_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if k == "storage" and isinstance(v, str):
            v = {"fp32": FM_STORE_FP32, "fp16": FM_STORE_FP16}[v]
        if k == "loss" and isinstance(v, str):
            v = {"irls": FM_LOSS_IRLS, "l1": FM_LOSS_L1}[v]
        setattr(o, k, v)
    return o


def _host(a, dtype) -> np.ndarray:
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _is_cuda(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return ctypes.c_void_p(0)


class Problem:
    """One epipolar-adjustment problem held on the GPU (see include/fastmap.h)."""

    def __init__(self, R, t, cam_i, cam_j, pair_id, x1, x2, options: Options | None = None,
                 stream=None):
        lib = load_library()
        R = _host(R, np.float64).reshape(-1, 9)
        t = _host(t, np.float64).reshape(-1, 3)
        ci = _host(cam_i, np.int32)
        cj = _host(cam_j, np.int32)
        self.n_cams = R.shape[0]
        self.n_pairs = ci.shape[0]
        on_dev = _is_cuda(pair_id)
        if on_dev:
            import torch
            pid = pair_id.to(torch.int32).contiguous()
            a = x1.to(torch.float32).contiguous()
            b = x2.to(torch.float32).contiguous()
            self._keep = (pid, a, b)
            ptrs = [ctypes.c_void_p(pid.data_ptr()), ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr())]
            n_pp = pid.numel()
        else:
            pid = _host(pair_id, np.int32)
            a = _host(x1, np.float32)
            b = _host(x2, np.float32)
            ptrs = [_ptr(pid), _ptr(a), _ptr(b)]
            n_pp = pid.shape[0]
        self.n_pp = int(n_pp)
        self.options = options if options is not None else default_options()
        self.stream = stream if stream is not None else _current_stream()
        h = ctypes.c_void_p()
        _check(lib.fm_create_problem(self.n_cams, _ptr(R), _ptr(t), self.n_pairs, _ptr(ci), _ptr(cj),
                                     self.n_pp, *ptrs, 1 if on_dev else 0, ctypes.byref(self.options),
                                     self.stream, ctypes.byref(h)))
        self._h = h
        self._keep = None

    # -- lifecycle -------------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            load_library().fm_destroy_problem(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def info(self) -> dict:
        inf = Info()
        _check(load_library().fm_problem_info(self._h, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in Info._fields_ if f != "reserved"}

    # -- poses, weights, state ----------------------------------------------------------------
    def get_poses(self):
        R = np.empty((self.n_cams, 3, 3))
        t = np.empty((self.n_cams, 3))
        _check(load_library().fm_get_poses(self._h, _ptr(R), _ptr(t)))
        return R, t

    def set_poses(self, R, t):
        R = _host(R, np.float64)
        t = _host(t, np.float64)
        _check(load_library().fm_set_poses(self._h, _ptr(R), _ptr(t)))

    def get_params(self):
        """Exact optimiser parameters (R, camera centres c)."""
        R = np.empty((self.n_cams, 3, 3))
        c = np.empty((self.n_cams, 3))
        _check(load_library().fm_get_params(self._h, _ptr(R), _ptr(c)))
        return R, c

    def set_params(self, R, c):
        R = _host(R, np.float64)
        c = _host(c, np.float64)
        _check(load_library().fm_set_params(self._h, _ptr(R), _ptr(c)))

    def set_params_device(self, R, c):
        """Asynchronous parameter update from contiguous float64 CUDA tensors (N,3,3), (N,3)."""
        _check(load_library().fm_set_params_device(self._h, ctypes.c_void_p(R.data_ptr()),
                                                   ctypes.c_void_p(c.data_ptr())))

    def set_scores(self, score):
        if _is_cuda(score):
            import torch
            score = score.to(torch.float32).contiguous()
            _check(load_library().fm_set_scores(self._h, ctypes.c_void_p(score.data_ptr()), 1))
        else:
            sv = _host(score, np.float32)
            _check(load_library().fm_set_scores(self._h, _ptr(sv), 0))

    def collect_features(self, tau: float, round_index: int, out):
        """Features of every point pair (out: CUDA bfloat16 tensor n_pp x 8, input order)."""
        _check(load_library().fm_collect_features(self._h, float(tau), int(round_index),
                                                  ctypes.c_void_p(out.data_ptr())))

    def learned_weights(self, net: "Mlp", tau: float, tau_cap: float, round_index: int) -> int:
        n = ctypes.c_int64()
        _check(load_library().fm_learned_weights(self._h, net._h, float(tau), float(tau_cap),
                                                 int(round_index), ctypes.byref(n)))
        return n.value

    def step_learned(self, net: "Mlp", tau: float, tau_cap: float, round_index: int, n_iters: int,
                     count: bool = False):
        """One learned IRLS round: the learned reweighting fused into the first of n_iters
        iterations. Returns the number of point pairs with |eps| <= tau_cap if `count`."""
        n = ctypes.c_int64()
        _check(load_library().fm_step_learned(self._h, net._h, float(tau), float(tau_cap), int(round_index),
                                              int(n_iters), ctypes.byref(n) if count else None))
        return n.value if count else None

    def reset_history(self):
        _check(load_library().fm_reset_history(self._h))

    def set_weights(self, w):
        if _is_cuda(w):
            import torch
            w = w.to(torch.float32).contiguous()
            _check(load_library().fm_set_weights(self._h, ctypes.c_void_p(w.data_ptr()), 1))
        else:
            wv = _host(w, np.float32)
            _check(load_library().fm_set_weights(self._h, _ptr(wv), 0))

    def get_weights(self) -> np.ndarray:
        w = np.empty(self.n_pp, np.float32)
        _check(load_library().fm_get_weights(self._h, _ptr(w)))
        return w

    def get_state(self):
        m = np.empty((self.n_cams, 6))
        v = np.empty((self.n_cams, 6))
        s = ctypes.c_int64()
        _check(load_library().fm_get_state(self._h, _ptr(m), _ptr(v), ctypes.byref(s)))
        return m, v, s.value

    def set_state(self, m, v, step: int):
        m = _host(m, np.float64)
        v = _host(v, np.float64)
        _check(load_library().fm_set_state(self._h, _ptr(m), _ptr(v), int(step)))

    def reset_optimizer(self):
        _check(load_library().fm_reset_optimizer(self._h))

    def set_learning_rate(self, lr_rot: float, lr_c: float):
        _check(load_library().fm_set_learning_rate(self._h, float(lr_rot), float(lr_c)))

    # -- compute -----------------------------------------------------------------------------------
    def irls_weights(self, tau: float) -> int:
        n = ctypes.c_int64()
        _check(load_library().fm_irls_weights(self._h, float(tau), ctypes.byref(n)))
        return n.value

    def loss_grad(self):
        loss = ctypes.c_double()
        g = np.empty((self.n_cams, 6))
        _check(load_library().fm_loss_grad(self._h, ctypes.byref(loss), _ptr(g)))
        return loss.value, g

    def loss_grad_device(self, loss_out, grad_out):
        """Asynchronous loss/gradient into device tensors (float64, sizes 1 and n_cams*6)."""
        _check(load_library().fm_loss_grad_device(
            self._h, ctypes.c_void_p(loss_out.data_ptr()) if loss_out is not None else None,
            ctypes.c_void_p(grad_out.data_ptr()) if grad_out is not None else None))

    def residuals(self) -> np.ndarray:
        e = np.empty(self.n_pp, np.float32)
        _check(load_library().fm_residuals(self._h, _ptr(e)))
        return e

    def apply_gradient(self, grad):
        """One Adam step with a gradient computed elsewhere (n_cams x 6 float64, host or CUDA)."""
        if _is_cuda(grad):
            import torch
            g = grad.to(torch.float64).contiguous()
            _check(load_library().fm_apply_gradient(self._h, ctypes.c_void_p(g.data_ptr()), 1))
        else:
            g = _host(grad, np.float64)
            _check(load_library().fm_apply_gradient(self._h, _ptr(g), 0))

    def step(self, n_iters: int = 1):
        _check(load_library().fm_step(self._h, int(n_iters)))

    def step_irls(self, tau: float, n_iters: int, count: bool = False):
        """One IRLS round: reweighting at threshold tau fused into the first of n_iters
        iterations. Returns the number of kept point pairs if `count` (synchronises)."""
        n = ctypes.c_int64()
        _check(load_library().fm_step_irls(self._h, float(tau), int(n_iters), ctypes.byref(n) if count else None))
        return n.value if count else None

    # focal refinement (scales s_k = f0_k / f_k of the normalised keypoints)
    def focal_scales(self) -> np.ndarray:
        out = np.empty(self.n_cams)
        _check(load_library().fm_get_focal_scales(self._h, _ptr(out)))
        return out

    def set_focal_scales(self, s):
        s = np.ascontiguousarray(_host(s, np.float64).reshape(self.n_cams))
        _check(load_library().fm_set_focal_scales(self._h, _ptr(s)))

    def focal_gradient(self) -> np.ndarray:
        out = np.empty(self.n_cams)
        _check(load_library().fm_get_focal_gradient(self._h, _ptr(out)))
        return out

    def set_focal_learning_rate(self, lr: float):
        _check(load_library().fm_set_focal_learning_rate(self._h, float(lr)))

    # pre-aggregated quadratic form of the IRLS objective (fixed weights)
    def preaggregate(self):
        """Collect the per-image-pair quadratic form at the current poses and weights."""
        _check(load_library().fm_preaggregate(self._h))

    def irls_preaggregate(self, tau: float) -> int:
        """IRLS reweighting at threshold tau and the quadratic form, in one pass."""
        n = ctypes.c_int64()
        _check(load_library().fm_irls_preaggregate(self._h, float(tau), ctypes.byref(n)))
        return n.value

    def loss_grad_quadratic(self):
        loss = ctypes.c_double()
        g = np.empty((self.n_cams, 6))
        _check(load_library().fm_loss_grad_quadratic(self._h, ctypes.byref(loss), _ptr(g)))
        return loss.value, g

    def step_quadratic(self, n_iters: int = 1):
        _check(load_library().fm_step_quadratic(self._h, int(n_iters)))

    def last_loss(self) -> float:
        loss = ctypes.c_double()
        _check(load_library().fm_last_loss(self._h, ctypes.byref(loss)))
        return loss.value

    def synchronize(self):
        _check(load_library().fm_synchronize(self._h))

    def enable_kernel_timing(self, enable: bool = True):
        _check(load_library().fm_enable_kernel_timing(self._h, 1 if enable else 0))

    def kernel_time(self):
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        _check(load_library().fm_kernel_time(self._h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def pass_time(self, which: int):
        """(summed ms, launches) of one timed pass (PASS_*) since the last call; resets it."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        _check(load_library().fm_pass_time(self._h, int(which), ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value


class TranslationOptions(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("adam_eps", ctypes.c_double), ("use_graph", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def translation_options(**kw) -> TranslationOptions:
    o = TranslationOptions()
    load_library().fm_translation_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Translation:
    """Global translation stage on the GPU (fm_translation_*): camera centres from unit
    relative translations with the rotations fixed, several runs from given initial centres,
    their merge and the final run."""

    def __init__(self, R, cam_i, cam_j, t_rel, o_init, options: TranslationOptions | None = None, stream=None):
        lib = load_library()
        R = _host(R, np.float64).reshape(-1, 9)
        ci = _host(cam_i, np.int32).reshape(-1)
        cj = _host(cam_j, np.int32).reshape(-1)
        t = _host(t_rel, np.float64).reshape(-1, 3)
        o0 = _host(o_init, np.float64)
        self.n_cams, self.n_pairs = R.shape[0], ci.shape[0]
        o0 = o0.reshape(-1, self.n_cams, 3)
        h = ctypes.c_void_p()
        _check(lib.fm_translation_create(self.n_cams, _ptr(R), self.n_pairs, _ptr(ci), _ptr(cj), _ptr(t),
                                         o0.shape[0], _ptr(np.ascontiguousarray(o0)),
                                         ctypes.byref(options) if options is not None else None,
                                         stream if stream is not None else _current_stream(), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load_library().fm_translation_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def n_runs(self) -> int:
        return load_library().fm_translation_num_runs(self._h)

    def loss_grad(self):
        """(loss (runs,), gradient (runs, n_cams, 3), camera losses (runs, n_cams))."""
        r = self.n_runs
        loss = np.empty(r)
        g = np.empty((r, self.n_cams, 3))
        cl = np.empty((r, self.n_cams))
        _check(load_library().fm_translation_loss_grad(self._h, _ptr(loss), _ptr(g), _ptr(cl)))
        return loss, g, cl

    def step(self, n_iters: int = 1):
        _check(load_library().fm_translation_step(self._h, int(n_iters)))

    def merge(self):
        _check(load_library().fm_translation_merge(self._h))

    def set_learning_rate(self, lr: float):
        _check(load_library().fm_translation_set_learning_rate(self._h, float(lr)))

    def centres(self) -> np.ndarray:
        out = np.empty((self.n_runs, self.n_cams, 3))
        _check(load_library().fm_translation_get_centres(self._h, _ptr(out)))
        return out

    def set_centres(self, o):
        o = np.ascontiguousarray(_host(o, np.float64).reshape(self.n_runs, self.n_cams, 3))
        _check(load_library().fm_translation_set_centres(self._h, _ptr(o)))


class RotationOptions(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("adam_eps", ctypes.c_double), ("cg_tol", ctypes.c_double), ("cg_max_iters", ctypes.c_int32),
                ("use_graph", ctypes.c_int32)]


def rotation_options(**kw) -> RotationOptions:
    o = RotationOptions()
    load_library().fm_rotation_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Rotation:
    """Global rotation stage on the GPU (fm_rotation_*): column-wise initialisation by
    conjugate gradients, then Adam on the geodesic objective in the 6D representation."""

    def __init__(self, cam_i, cam_j, R_rel, n_cams: int, options: RotationOptions | None = None, stream=None):
        lib = load_library()
        ci = _host(cam_i, np.int32).reshape(-1)
        cj = _host(cam_j, np.int32).reshape(-1)
        Rr = _host(R_rel, np.float64).reshape(-1, 9)
        self.n_cams, self.n_pairs = int(n_cams), ci.shape[0]
        h = ctypes.c_void_p()
        _check(lib.fm_rotation_create(self.n_cams, self.n_pairs, _ptr(ci), _ptr(cj), _ptr(Rr),
                                      ctypes.byref(options) if options is not None else None,
                                      stream if stream is not None else _current_stream(), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load_library().fm_rotation_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def initialize(self):
        """Column-wise initialisation; returns (conjugate-gradient iterations, relative residual)."""
        it = ctypes.c_int32()
        res = ctypes.c_double()
        _check(load_library().fm_rotation_initialize(self._h, ctypes.byref(it), ctypes.byref(res)))
        return it.value, res.value

    def loss_grad(self):
        loss = ctypes.c_double()
        g = np.empty((self.n_cams, 6))
        _check(load_library().fm_rotation_loss_grad(self._h, ctypes.byref(loss), _ptr(g)))
        return loss.value, g

    def step(self, n_iters: int = 1):
        _check(load_library().fm_rotation_step(self._h, int(n_iters)))

    def set_learning_rate(self, lr: float):
        _check(load_library().fm_rotation_set_learning_rate(self._h, float(lr)))

    def rotations(self) -> np.ndarray:
        out = np.empty((self.n_cams, 3, 3))
        _check(load_library().fm_rotation_get_rotations(self._h, _ptr(out)))
        return out

    def params(self) -> np.ndarray:
        out = np.empty((self.n_cams, 6))
        _check(load_library().fm_rotation_get_params(self._h, _ptr(out)))
        return out

    def set_rotations(self, R):
        R = np.ascontiguousarray(_host(R, np.float64).reshape(self.n_cams, 9))
        _check(load_library().fm_rotation_set_rotations(self._h, _ptr(R)))

    def set_params(self, a6):
        a6 = np.ascontiguousarray(_host(a6, np.float64).reshape(self.n_cams, 6))
        _check(load_library().fm_rotation_set_params(self._h, _ptr(a6)))


def focal_vote(F, candidates, tau: float, f1_known=None, f2_known=None, timed: bool = False, stream=None):
    """Votes v(f) of the candidate focal lengths (fm_focal_vote; Sec. "Intrinsics Estimation").
    F: (B, 3, 3) fundamental matrices in pixels from the image centre; f1_known / f2_known: (B,)
    known focal length of each pair side, 0 where the candidate is used. Returns the votes
    (FP64 array), and with timed=True also the kernels' device time in ms."""
    Fh = np.ascontiguousarray(_host(F, np.float64).reshape(-1, 9))
    ch = np.ascontiguousarray(_host(candidates, np.float64).reshape(-1))
    k1 = None if f1_known is None else np.ascontiguousarray(_host(f1_known, np.float64).reshape(-1))
    k2 = None if f2_known is None else np.ascontiguousarray(_host(f2_known, np.float64).reshape(-1))
    for k in (k1, k2):
        if k is not None and k.shape[0] != Fh.shape[0]:
            raise ValueError("known focal lengths need one value per pair")
    out = np.empty(ch.shape[0], np.float64)
    ms = ctypes.c_float()
    _check(load_library().fm_focal_vote(Fh.shape[0], _ptr(Fh), None if k1 is None else _ptr(k1),
                                        None if k2 is None else _ptr(k2), ch.shape[0], _ptr(ch), float(tau),
                                        _ptr(out), ctypes.byref(ms) if timed else None,
                                        stream if stream is not None else _current_stream()))
    return (out, ms.value) if timed else out


class Mlp:
    """The learned inlier-weight network on the GPU (fm_mlp_*): FP32 masters, BF16 copies."""

    def __init__(self, params):
        lib = load_library()
        self.n_params = lib.fm_mlp_num_params()
        pv = _host(params, np.float32).reshape(-1)
        if pv.shape[0] != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters")
        h = ctypes.c_void_p()
        _check(lib.fm_mlp_create(_ptr(pv), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load_library().fm_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.empty(self.n_params, np.float32)
        _check(load_library().fm_mlp_get_params(self._h, _ptr(out)))
        return out

    def set_params(self, params):
        pv = _host(params, np.float32).reshape(-1)
        _check(load_library().fm_mlp_set_params(self._h, _ptr(pv)))

    def train_step(self, feats, labels, lr: float, want_loss: bool = True, stream=None):
        """One Adam step on CUDA tensors feats (n x 8 bfloat16) and labels (n float32)."""
        loss = ctypes.c_float()
        _check(load_library().fm_mlp_train_step(
            self._h, ctypes.c_void_p(feats.data_ptr()), ctypes.c_void_p(labels.data_ptr()), int(labels.numel()),
            float(lr), ctypes.byref(loss) if want_loss else None,
            stream if stream is not None else _current_stream()))
        return loss.value if want_loss else None

    def gradient(self, feats, labels):
        g = np.empty(self.n_params, np.float32)
        loss = ctypes.c_float()
        _check(load_library().fm_mlp_gradient(self._h, ctypes.c_void_p(feats.data_ptr()),
                                              ctypes.c_void_p(labels.data_ptr()), int(labels.numel()),
                                              _ptr(g), ctypes.byref(loss)))
        return loss.value, g

    def forward(self, feats, out):
        _check(load_library().fm_mlp_forward(self._h, ctypes.c_void_p(feats.data_ptr()), int(out.numel()),
                                             ctypes.c_void_p(out.data_ptr()), _current_stream()))
