"""Seeded synthetic scenes for epipolar pose adjustment.

This module only produces inputs: ground-truth cameras, image pairs, matched keypoint pairs
in normalized image coordinates, outlier labels, match scores and perturbed initial poses.
It holds none of the adjustment's arithmetic (no essential matrices, residuals, weights or
gradients). The oracle and the CUDA path both consume the arrays it returns, so the two
sides see identical inputs.

Scenes stand in for the datasets of the FastMap experiments (Sec. "Experiments"), which are
not available here. Their shapes follow the workloads the paper times: hundreds to
thousands of images and 5k-500k image pairs (Table "Effect of kernel fusion").

Camera model (Sec. "Camera Assumptions"): principal point at the image centre, known focal
length f, no distortion. A keypoint in pixels (u, v) maps to normalized homogeneous
coordinates ((u - W/2)/f, (v - H/2)/f, 1); this module returns the first two components.

Conventions: camera k is world-to-camera, x_cam = R_k X + t_k, with camera centre
c_k = -R_k^T t_k. Pairs are (i, j) with i < j; x1 is the keypoint in image i, x2 the
keypoint in image j.

Generation runs on any torch device (CPU for the oracle-sized scenes, CUDA for the
full-size ones). Keypoint noise of one (image, 3D point) observation comes from a
counter-based hash of (seed, image, point), so a point keeps the same noisy keypoint in
every pair that contains its image.
"""
from __future__ import annotations

import dataclasses
import math

import torch

__all__ = ["Scene", "CONFIGS", "make_scene", "perturb_poses", "rotation_exp", "fundamental_matrices"]

F64 = torch.float64


@dataclasses.dataclass
class Scene:
    name: str
    R_gt: torch.Tensor        # (N,3,3) f64 world-to-camera rotations
    t_gt: torch.Tensor        # (N,3)   f64 world-to-camera translations
    R_init: torch.Tensor      # (N,3,3) f64 perturbed initial rotations
    t_init: torch.Tensor      # (N,3)   f64 perturbed initial translations
    cam_i: torch.Tensor       # (B,) int32, first image of each pair
    cam_j: torch.Tensor       # (B,) int32, second image of each pair (cam_i < cam_j)
    pair_id: torch.Tensor     # (P,) int32, image pair of each point pair (sorted)
    x1: torch.Tensor          # (P,2) f32 normalized keypoint in image cam_i[pair_id]
    x2: torch.Tensor          # (P,2) f32 normalized keypoint in image cam_j[pair_id]
    outlier: torch.Tensor     # (P,) bool, match replaced by a random keypoint
    score: torch.Tensor       # (P,) f32 synthetic matcher confidence in [0,1]
    points: torch.Tensor      # (M,3) f64 scene points
    f: float = 500.0
    width: int = 640
    height: int = 480
    sigma_px: float = 1.0
    iters: int = 200

    @property
    def n_cams(self) -> int:
        return int(self.R_gt.shape[0])

    @property
    def n_pairs(self) -> int:
        return int(self.cam_i.shape[0])

    @property
    def n_pp(self) -> int:
        return int(self.pair_id.shape[0])

    def to(self, device) -> "Scene":
        kw = {}
        for fld in dataclasses.fields(self):
            v = getattr(self, fld.name)
            kw[fld.name] = v.to(device) if isinstance(v, torch.Tensor) else v
        return Scene(**kw)


# Workloads. Sizes follow the five workload descriptions of the adjustment benchmark:
#   ring16    : 16 cameras on a radius-3 ring, 2,000 points, all 120 pairs, 50% of co-visible
#               points kept per pair (~1.2e5 point pairs), 10% outliers, sigma 0.5 px.
#   sphere128 : 128 cameras on a sphere, 50k points, 16 nearest views (~1e3 pairs),
#               log-normal counts (median 2k, cap 20k, ~3e6 point pairs), 15% outliers, 1 px.
#   traj1000  : 1,000 cameras along a smooth random trajectory, 500k points, 20 neighbours
#               (~1e4 pairs), log-normal counts (~5e7 point pairs), 20% outliers, 1 px.
#   traj1000_o30 : traj1000 with 30% outliers.
#   sphere128_o30 : sphere128 with 30% outliers (the learned weights' training shape with twice
#               the outliers; evaluated on seeds outside the training seeds 1000-1199).
#   traj4000  : 4,000 cameras, 2M points, 25 neighbours (~5e4 pairs), Pareto(1.5) counts
#               capped at 50k (~1.5e8 point pairs), 25% outliers, 1.5 px.
#   loop1000  : 1,000 cameras along a random smooth closed trajectory that winds 20 times
#               around a 500k-point cloud while its height sweeps +-70 degrees of elevation and
#               back (every lap closes a loop, neighbouring laps revisit the same views),
#               looking inward; 20 neighbours per camera: 8 along the path and 12 nearest views
#               of other laps (~1.2e4 pairs), log-normal counts (~6e7 point pairs), 20% outliers,
#               1 px.
#   loop1000_o30 : loop1000 with 30% outliers (learned-weight evaluation scene).
#   loop4000  : the same layout at the size of traj4000 (4,000 cameras in 40 laps, 2M points,
#               25 neighbours, Pareto(1.5) counts capped at 50k, 25% outliers, 1.5 px).
CONFIGS = {
    "ring16": dict(kind="ring", n_cams=16, n_pts=2000, sigma_px=0.5, outlier=0.10,
                   keep=0.5, iters=200),
    "sphere128": dict(kind="sphere", n_cams=128, n_pts=50_000, sigma_px=1.0, outlier=0.15,
                      knn=16, counts=("lognormal", 2000.0, 0.9, 20_000), iters=300),
    "sphere128_o30": dict(kind="sphere", n_cams=128, n_pts=50_000, sigma_px=1.0, outlier=0.30,
                          knn=16, counts=("lognormal", 2000.0, 0.9, 20_000), iters=300),
    "traj1000": dict(kind="trajectory", n_cams=1000, n_pts=500_000, sigma_px=1.0,
                     outlier=0.20, knn=20, counts=("lognormal", 3900.0, 0.9, 20_000),
                     spacing=0.25, depth=(3.0, 9.0), iters=300),
    "traj1000_o30": dict(kind="trajectory", n_cams=1000, n_pts=500_000, sigma_px=1.0,
                         outlier=0.30, knn=20, counts=("lognormal", 3900.0, 0.9, 20_000),
                         spacing=0.25, depth=(3.0, 9.0), iters=300),
    "traj4000": dict(kind="trajectory", n_cams=4000, n_pts=2_000_000, sigma_px=1.5,
                     outlier=0.25, knn=25, counts=("pareto", 1.5, 1100.0, 50_000),
                     spacing=0.1, depth=(4.0, 16.0), iters=300),
    "loop1000": dict(kind="loop", n_cams=1000, n_pts=500_000, sigma_px=1.0, outlier=0.20,
                     knn=20, path_nb=4, laps=20, elev_deg=70.0, counts=("lognormal", 3900.0, 0.9, 20_000),
                     iters=300),
    "loop1000_o30": dict(kind="loop", n_cams=1000, n_pts=500_000, sigma_px=1.0, outlier=0.30,
                         knn=20, path_nb=4, laps=20, elev_deg=70.0, counts=("lognormal", 3900.0, 0.9, 20_000),
                         iters=300),
    "loop4000": dict(kind="loop", n_cams=4000, n_pts=2_000_000, sigma_px=1.5, outlier=0.25,
                     knn=25, path_nb=5, laps=40, elev_deg=70.0, counts=("pareto", 1.5, 1100.0, 50_000), iters=300),
}


# ----------------------------------------------------------------------------------------
# counter-based randomness (splitmix64 finalizer, Steele et al. 2014) on int64 tensors
# ----------------------------------------------------------------------------------------
_MASK = (1 << 64) - 1


def _s64(v: int) -> int:
    v &= _MASK
    return v - (1 << 64) if v >= (1 << 63) else v


_GOLDEN = _s64(0x9E3779B97F4A7C15)
_MIX1 = _s64(0xBF58476D1CE4E5B9)
_MIX2 = _s64(0x94D049BB133111EB)


def _lsr(x: torch.Tensor, k: int) -> torch.Tensor:
    return (x >> k) & ((1 << (64 - k)) - 1)


def _mix64(x: torch.Tensor) -> torch.Tensor:
    x = x ^ _lsr(x, 30)
    x = x * _MIX1
    x = x ^ _lsr(x, 27)
    x = x * _MIX2
    return x ^ _lsr(x, 31)


def _hash_uniform(seed: int, a: torch.Tensor, b: torch.Tensor, stream: int) -> torch.Tensor:
    """Uniform (0,1) doubles from the counter (seed, a, b, stream)."""
    x = _mix64(a.to(torch.int64) * _GOLDEN + _s64(seed * 0x2545F4914F6CDD1D + stream))
    x = _mix64(x + b.to(torch.int64) * _MIX2)
    return (_lsr(x, 11).to(F64) + 0.5) * (1.0 / (1 << 53))


def _hash_normal2(seed: int, a: torch.Tensor, b: torch.Tensor, stream: int):
    """Two independent standard normals per counter (Box-Muller)."""
    u1 = _hash_uniform(seed, a, b, 2 * stream)
    u2 = _hash_uniform(seed, a, b, 2 * stream + 1)
    r = torch.sqrt(-2.0 * torch.log(u1))
    return r * torch.cos(2.0 * math.pi * u2), r * torch.sin(2.0 * math.pi * u2)


# ----------------------------------------------------------------------------------------
# rotations
# ----------------------------------------------------------------------------------------
def _hat(w: torch.Tensor) -> torch.Tensor:
    z = torch.zeros_like(w[..., 0])
    return torch.stack([
        torch.stack([z, -w[..., 2], w[..., 1]], -1),
        torch.stack([w[..., 2], z, -w[..., 0]], -1),
        torch.stack([-w[..., 1], w[..., 0], z], -1)], -2)


def rotation_exp(w: torch.Tensor) -> torch.Tensor:
    """Rotation matrices exp([w]_x) for rotation vectors w (..., 3), Rodrigues' formula."""
    w = w.to(F64)
    th = torch.linalg.norm(w, dim=-1, keepdim=True)[..., None]
    K = _hat(w)
    small = th < 1e-12
    ths = torch.where(small, torch.ones_like(th), th)
    a = torch.where(small, torch.ones_like(th), torch.sin(ths) / ths)
    b = torch.where(small, torch.full_like(th, 0.5), (1 - torch.cos(ths)) / ths ** 2)
    eye = torch.eye(3, dtype=F64, device=w.device).expand(K.shape)
    return eye + a * K + b * (K @ K)


def _look_rotation(forward: torch.Tensor, up: torch.Tensor) -> torch.Tensor:
    """World-to-camera rotations for cameras looking along `forward` (x right, y down)."""
    z = forward / torch.linalg.norm(forward, dim=-1, keepdim=True)
    y = -(up - (up * z).sum(-1, keepdim=True) * z)
    y = y / torch.linalg.norm(y, dim=-1, keepdim=True)
    x = torch.cross(y, z, dim=-1)
    return torch.stack([x, y, z], dim=-2)


def _random_unit(n: int, g: torch.Generator, device) -> torch.Tensor:
    v = torch.randn(n, 3, dtype=F64, generator=g, device=device)
    return v / torch.linalg.norm(v, dim=-1, keepdim=True)


# ----------------------------------------------------------------------------------------
# camera layouts
# ----------------------------------------------------------------------------------------
def _cams_ring(n: int, g, device, jitter_deg: float):
    ang = torch.arange(n, dtype=F64, device=device) * (2 * math.pi / n)
    C = torch.stack([3 * torch.cos(ang), 3 * torch.sin(ang), torch.zeros_like(ang)], -1)
    up = torch.tensor([0.0, 0.0, 1.0], dtype=F64, device=device).expand(n, 3)
    R = _look_rotation(-C, up)
    jit = (torch.rand(n, 3, dtype=F64, generator=g, device=device) * 2 - 1) * math.radians(jitter_deg)
    return rotation_exp(jit) @ R, C


def _cams_sphere(n: int, g, device, radius: float, jitter_deg: float):
    k = torch.arange(n, dtype=F64, device=device) + 0.5
    phi = torch.acos(1 - 2 * k / n)
    theta = math.pi * (1 + math.sqrt(5.0)) * k
    d = torch.stack([torch.cos(theta) * torch.sin(phi), torch.sin(theta) * torch.sin(phi),
                     torch.cos(phi)], -1)
    d = d + 0.05 * torch.randn(n, 3, dtype=F64, generator=g, device=device)
    d = d / torch.linalg.norm(d, dim=-1, keepdim=True)
    C = radius * d
    # an up vector that is never parallel to the viewing direction
    up = torch.where((d[:, 2:3].abs() < 0.9), torch.tensor([0.0, 0.0, 1.0], dtype=F64, device=device),
                     torch.tensor([1.0, 0.0, 0.0], dtype=F64, device=device))
    R = _look_rotation(-C, up)
    jit = (torch.rand(n, 3, dtype=F64, generator=g, device=device) * 2 - 1) * math.radians(jitter_deg)
    return rotation_exp(jit) @ R, C


def _cams_loop(n: int, laps: int, g, device, radius: float = 3.0, jitter_deg: float = 10.0,
               elev_deg: float = 35.0):
    """Cameras along a random smooth closed trajectory around the origin, looking inward.

    The path winds `laps` times around the vertical axis; its elevation follows one slow
    cosine over the whole path (so later laps pass over the heights of earlier ones) and its
    radius and elevation carry random low-order Fourier terms that are periodic over the whole
    path, so the curve is smooth and closes on itself.
    """
    s = (torch.arange(n, dtype=F64, device=device) + 0.5) / n          # path parameter in [0, 1)
    theta = 2 * math.pi * laps * s
    phase = 2 * math.pi * float(torch.rand(1, dtype=F64, generator=g, device=device))
    elev = math.radians(elev_deg) * torch.cos(2 * math.pi * s + phase)
    rad = torch.full_like(s, radius)
    for k in range(1, 4):   # wobble: closed (periodic in s), decaying with the order
        a = torch.randn(4, dtype=F64, generator=g, device=device) / k
        arg = 2 * math.pi * (k * (laps + 1)) * s
        rad = rad + radius * 0.06 * (a[0] * torch.cos(arg) + a[1] * torch.sin(arg))
        elev = elev + math.radians(4.0) * (a[2] * torch.cos(arg) + a[3] * torch.sin(arg))
    C = torch.stack([rad * torch.cos(elev) * torch.cos(theta), rad * torch.cos(elev) * torch.sin(theta),
                     rad * torch.sin(elev)], -1)
    up = torch.tensor([0.0, 0.0, 1.0], dtype=F64, device=device).expand(n, 3)
    R = _look_rotation(-C, up)
    jit = (torch.rand(n, 3, dtype=F64, generator=g, device=device) * 2 - 1) * math.radians(jitter_deg)
    return rotation_exp(jit) @ R, C


def _loop_pairs(C: torch.Tensor, path_nb: int, k_far: int, far_steps: int):
    """Pairs of a closed path: every camera with its `path_nb` neighbours on each side along
    the path (wrapping around), and with its `k_far` nearest cameras that are more than
    `far_steps` steps away along the path (the views of other laps: revisits)."""
    n = C.shape[0]
    dev = C.device
    idx = torch.arange(n, device=dev)
    near = (idx[:, None] + torch.arange(1, path_nb + 1, device=dev)[None, :]) % n
    a0 = torch.minimum(idx[:, None].expand_as(near), near).reshape(-1)
    b0 = torch.maximum(idx[:, None].expand_as(near), near).reshape(-1)
    d = torch.cdist(C, C)
    steps = (idx[:, None] - idx[None, :]).abs()
    steps = torch.minimum(steps, n - steps)
    d = torch.where(steps > far_steps, d, torch.full_like(d, float("inf")))
    far = torch.topk(d, k_far, dim=1, largest=False).indices
    a1 = torch.minimum(idx[:, None].expand_as(far), far).reshape(-1)
    b1 = torch.maximum(idx[:, None].expand_as(far), far).reshape(-1)
    key = torch.unique(torch.cat([a0 * n + b0, a1 * n + b1]))
    return key // n, key % n


def _trajectory(n: int, spacing: float, g, device):
    """Smooth random planar-ish trajectory (Catmull-Rom through seeded waypoints).

    Returns positions p(s) and horizontal left normals at n + 1 arc-length samples per
    camera plus a dense table used to place the scene points.
    """
    length = n * spacing
    n_way = max(8, n // 40)
    seg = length / (n_way - 1)
    heading = torch.cumsum(torch.randn(n_way, dtype=F64, generator=g, device=device) * 0.5, 0)
    steps = torch.stack([torch.cos(heading), torch.sin(heading),
                         0.05 * torch.randn(n_way, dtype=F64, generator=g, device=device)], -1) * seg
    way = torch.cumsum(steps, 0)
    way = torch.cat([2 * way[:1] - way[1:2], way, 2 * way[-1:] - way[-2:-1]], 0)
    dense = 64
    tt = torch.arange(dense, dtype=F64, device=device) / dense
    p0, p1, p2, p3 = way[:-3], way[1:-2], way[2:-1], way[3:]
    t = tt[None, :, None]
    curve = 0.5 * ((2 * p1[:, None]) + (-p0 + p2)[:, None] * t
                   + (2 * p0 - 5 * p1 + 4 * p2 - p3)[:, None] * t ** 2
                   + (-p0 + 3 * p1 - 3 * p2 + p3)[:, None] * t ** 3)
    curve = torch.cat([curve.reshape(-1, 3), way[-2:-1]], 0)
    dl = torch.linalg.norm(curve[1:] - curve[:-1], dim=-1)
    arc = torch.cat([torch.zeros(1, dtype=F64, device=device), torch.cumsum(dl, 0)])
    return curve, arc


def _interp_curve(curve, arc, s):
    idx = torch.searchsorted(arc, s).clamp(1, arc.shape[0] - 1)
    a0, a1 = arc[idx - 1], arc[idx]
    w = ((s - a0) / (a1 - a0).clamp_min(1e-12))[:, None]
    pos = curve[idx - 1] * (1 - w) + curve[idx] * w
    tan = curve[idx] - curve[idx - 1]
    tan = tan / torch.linalg.norm(tan, dim=-1, keepdim=True)
    zhat = torch.tensor([0.0, 0.0, 1.0], dtype=F64, device=s.device).expand_as(tan)
    left = torch.cross(zhat, tan, dim=-1)
    left = left / torch.linalg.norm(left, dim=-1, keepdim=True)
    return pos, left


# ----------------------------------------------------------------------------------------
# projection helpers (scene synthesis only)
# ----------------------------------------------------------------------------------------
def _project(R, C, X, f, W, H):
    """Noise-free normalized projections and visibility of points X seen by cameras (R, C).

    R, C are per-row (…,3,3)/(…,3); X is (…,3).
    """
    Xc = torch.einsum("nab,nb->na", R, X - C)
    z = Xc[:, 2]
    zs = torch.where(z > 1e-9, z, torch.ones_like(z))
    u = Xc[:, 0] / zs
    v = Xc[:, 1] / zs
    vis = (z > 0.1) & (u.abs() <= (W / 2) / f) & (v.abs() <= (H / 2) / f)
    return u, v, vis


def _systematic_pick(valid_counts: torch.Tensor, want: torch.Tensor, g, device):
    """For each segment choose `want` distinct ranks in [0, valid_counts) spread evenly."""
    k = torch.minimum(want, valid_counts)
    seg = torch.repeat_interleave(torch.arange(k.shape[0], device=device), k)
    start = torch.cumsum(k, 0) - k
    local = torch.arange(int(k.sum()), device=device) - start[seg]
    u0 = torch.rand(k.shape[0], dtype=F64, generator=g, device=device)
    step = valid_counts[seg].to(F64) / k[seg].to(F64)
    rank = torch.floor((local.to(F64) + u0[seg]) * step).to(torch.int64)
    rank = torch.minimum(rank, valid_counts[seg] - 1)
    return seg, rank, k


def _beta_order_stat(a: int, b: int, n: int, g, device) -> torch.Tensor:
    """Beta(a, b) for integers a, b: the a-th smallest of a + b - 1 uniforms."""
    u = torch.rand(n, a + b - 1, dtype=torch.float32, generator=g, device=device)
    return torch.sort(u, dim=1).values[:, a - 1]


# ----------------------------------------------------------------------------------------
# scene assembly
# ----------------------------------------------------------------------------------------
def _knn_pairs(C: torch.Tensor, k: int) -> tuple[torch.Tensor, torch.Tensor]:
    d = torch.cdist(C, C)
    d.fill_diagonal_(float("inf"))
    nn = torch.topk(d, k, dim=1, largest=False).indices
    i = torch.arange(C.shape[0], device=C.device)[:, None].expand_as(nn)
    a = torch.minimum(i, nn).reshape(-1)
    b = torch.maximum(i, nn).reshape(-1)
    key = torch.unique(a * C.shape[0] + b)
    return (key // C.shape[0]), (key % C.shape[0])


def _draw_counts(spec, n: int, g, device) -> torch.Tensor:
    kind = spec[0]
    if kind == "lognormal":
        _, median, s, cap = spec
        x = median * torch.exp(s * torch.randn(n, dtype=F64, generator=g, device=device))
    elif kind == "pareto":
        _, alpha, xm, cap = spec
        u = torch.rand(n, dtype=F64, generator=g, device=device)
        x = xm * (1 - u) ** (-1.0 / alpha)
    else:
        raise ValueError(kind)
    return torch.clamp(torch.round(x), 1, cap).to(torch.int64)


def make_scene(name: str, seed: int = 0, device="cpu", **overrides) -> Scene:
    """Build the seeded scene `name` (a key of CONFIGS) on `device`."""
    cfg = dict(CONFIGS[name])
    cfg.update(overrides)
    device = torch.device(device)
    g = torch.Generator(device=device)
    g.manual_seed(1_000_003 * seed + 17)
    f, W, H = 500.0, 640, 480
    n = cfg["n_cams"]
    kind = cfg["kind"]

    if kind == "ring":
        R, C = _cams_ring(n, g, device, 10.0)
        X = _ball_points(cfg["n_pts"], g, device)
        cam_i, cam_j = torch.triu_indices(n, n, 1, device=device)
    elif kind == "sphere":
        R, C = _cams_sphere(n, g, device, 3.0, 5.0)
        X = _ball_points(cfg["n_pts"], g, device)
        cam_i, cam_j = _knn_pairs(C, cfg["knn"])
    elif kind == "trajectory":
        curve, arc = _trajectory(n, cfg["spacing"], g, device)
        L = float(arc[-1])
        s_cam = (torch.arange(n, dtype=F64, device=device) + 0.5) * (L / n)
        C, left = _interp_curve(curve, arc, s_cam)
        up = torch.tensor([0.0, 0.0, 1.0], dtype=F64, device=device).expand(n, 3)
        R = _look_rotation(left, up)
        jit = (torch.rand(n, 3, dtype=F64, generator=g, device=device) * 2 - 1) * math.radians(10.0)
        R = rotation_exp(jit) @ R
        s_pt = torch.sort(torch.rand(cfg["n_pts"], dtype=F64, generator=g, device=device) * L).values
        P0, left_p = _interp_curve(curve, arc, s_pt)
        d0, d1 = cfg["depth"]
        dep = d0 + (d1 - d0) * torch.rand(cfg["n_pts"], dtype=F64, generator=g, device=device)
        hgt = (torch.rand(cfg["n_pts"], dtype=F64, generator=g, device=device) * 2 - 1) * (0.4 * d0)
        X = P0 + left_p * dep[:, None]
        X[:, 2] += hgt
        # neighbours along the trajectory: the knn/2 cameras on each side
        half = cfg["knn"] // 2
        ii = torch.arange(n, device=device)[:, None].expand(n, half)
        jj = ii + torch.arange(1, half + 1, device=device)[None, :]
        keep = jj < n
        cam_i, cam_j = ii[keep], jj[keep]
    elif kind == "loop":
        R, C = _cams_loop(n, cfg["laps"], g, device, elev_deg=cfg.get("elev_deg", 35.0))
        X = _ball_points(cfg["n_pts"], g, device)
        cam_i, cam_j = _loop_pairs(C, cfg["path_nb"], cfg["knn"] - 2 * cfg["path_nb"],
                                   n // (4 * cfg["laps"]))
    else:
        raise ValueError(kind)

    cam_i = cam_i.to(torch.int64)
    cam_j = cam_j.to(torch.int64)
    B = cam_i.shape[0]
    want = None if kind == "ring" else _draw_counts(cfg["counts"], B, g, device)
    if kind == "trajectory":
        cand_lo, cand_hi = _trajectory_windows(s_cam, s_pt, cam_i, cam_j, cfg["depth"][1], f, W)
    elif kind == "loop":
        # every camera sees most of the cloud: a random window of about twice the wanted count
        # of (unordered, hence random) points holds enough co-visible candidates
        size = torch.clamp(2 * want + 64, max=X.shape[0])
        u = torch.rand(B, dtype=F64, generator=g, device=device)
        cand_lo = torch.floor(u * (X.shape[0] - size + 1).to(F64)).to(torch.int64)
        cand_hi = cand_lo + size
    else:
        cand_lo = torch.zeros(B, dtype=torch.int64, device=device)
        cand_hi = torch.full((B,), X.shape[0], dtype=torch.int64, device=device)

    pid, pt = _covisible_matches(R, C, X, cam_i, cam_j, cand_lo, cand_hi, want,
                                 cfg.get("keep", 1.0), f, W, H, g, device)
    # drop pairs that received no matches and renumber (every pair must be non-empty)
    used = torch.bincount(pid, minlength=B) > 0
    remap = torch.cumsum(used.to(torch.int64), 0) - 1
    pid = remap[pid]
    cam_i, cam_j = cam_i[used], cam_j[used]

    sigma = cfg["sigma_px"] / f
    ci, cj = cam_i[pid], cam_j[pid]
    u1, v1, _ = _project(R[ci], C[ci], X[pt], f, W, H)
    u2, v2, _ = _project(R[cj], C[cj], X[pt], f, W, H)
    n1a, n1b = _hash_normal2(seed, ci, pt, 0)
    n2a, n2b = _hash_normal2(seed, cj, pt, 0)
    x1 = torch.stack([u1 + sigma * n1a, v1 + sigma * n1b], -1)
    x2 = torch.stack([u2 + sigma * n2a, v2 + sigma * n2b], -1)
    P = pid.shape[0]
    out = torch.rand(P, dtype=F64, generator=g, device=device) < cfg["outlier"]
    rnd = torch.rand(P, 2, dtype=F64, generator=g, device=device)
    rnd = torch.stack([(rnd[:, 0] - 0.5) * (W / f), (rnd[:, 1] - 0.5) * (H / f)], -1)
    x2 = torch.where(out[:, None], rnd, x2)
    score = torch.where(out, _beta_order_stat(2, 3, P, g, device), _beta_order_stat(4, 2, P, g, device))

    t = -torch.einsum("nab,nb->na", R, C)
    R0, t0 = perturb_poses(R, t, cam_i, cam_j, 5.0, 0.1, g, kind)
    return Scene(name=name, R_gt=R, t_gt=t, R_init=R0, t_init=t0,
                 cam_i=cam_i.to(torch.int32), cam_j=cam_j.to(torch.int32),
                 pair_id=pid.to(torch.int32), x1=x1.to(torch.float32), x2=x2.to(torch.float32),
                 outlier=out, score=score.to(torch.float32), points=X,
                 f=f, width=W, height=H, sigma_px=cfg["sigma_px"], iters=cfg["iters"])


def _ball_points(m: int, g, device) -> torch.Tensor:
    d = torch.randn(m, 3, dtype=F64, generator=g, device=device)
    d = d / torch.linalg.norm(d, dim=-1, keepdim=True)
    r = torch.rand(m, dtype=F64, generator=g, device=device) ** (1.0 / 3.0)
    return d * r[:, None]


def _trajectory_windows(s_cam, s_pt, cam_i, cam_j, dmax, f, W):
    half = dmax * (W / 2) / f * 1.4 + 0.5
    lo = torch.minimum(s_cam[cam_i], s_cam[cam_j]) - half
    hi = torch.maximum(s_cam[cam_i], s_cam[cam_j]) + half
    return torch.searchsorted(s_pt, lo), torch.searchsorted(s_pt, hi)


def _covisible_matches(R, C, X, cam_i, cam_j, lo, hi, want, keep, f, W, H, g, device,
                       chunk=40_000_000):
    """Point indices of the matches of every pair, grouped (sorted) by pair.

    Candidates of pair n are points lo[n]..hi[n]-1; those visible in both images are the
    co-visible set. With `want` given, each pair keeps min(want, |co-visible|) of them
    (evenly spread ranks); otherwise each co-visible point is kept with probability `keep`.
    """
    B = cam_i.shape[0]
    out_pid, out_pt = [], []
    n0 = 0
    while n0 < B:
        # take as many pairs as fit in one chunk of candidates
        sizes = hi[n0:] - lo[n0:]
        cum = torch.cumsum(sizes, 0)
        n1 = n0 + max(1, int(torch.searchsorted(cum, torch.tensor(chunk, device=device))))
        n1 = min(n1, B)
        sz = hi[n0:n1] - lo[n0:n1]
        seg = torch.repeat_interleave(torch.arange(n0, n1, device=device), sz)
        start = torch.cumsum(sz, 0) - sz
        pt = lo[seg] + (torch.arange(int(sz.sum()), device=device) - start[seg - n0])
        _, _, vis1 = _project(R[cam_i[seg]], C[cam_i[seg]], X[pt], f, W, H)
        _, _, vis2 = _project(R[cam_j[seg]], C[cam_j[seg]], X[pt], f, W, H)
        vis = vis1 & vis2
        seg, pt = seg[vis], pt[vis]
        if want is None:
            k = torch.rand(seg.shape[0], dtype=F64, generator=g, device=device) < keep
            out_pid.append(seg[k])
            out_pt.append(pt[k])
        else:
            nvis = torch.bincount(seg - n0, minlength=n1 - n0)
            vstart = torch.cumsum(nvis, 0) - nvis
            s2, rank, _ = _systematic_pick(nvis, want[n0:n1], g, device)
            idx = vstart[s2] + rank
            out_pid.append(seg[idx])
            out_pt.append(pt[idx])
        n0 = n1
    return torch.cat(out_pid), torch.cat(out_pt)


def perturb_poses(R, t, cam_i, cam_j, rot_deg: float, trans_frac: float, g, kind: str):
    """Initial poses: each rotation turned by `rot_deg` about a random axis and each camera
    centre moved by a random vector.

    The move is `trans_frac` of the camera's distance from the scene centre for object-centred
    scenes (ring, sphere) and `trans_frac` of the median pair baseline for trajectories (open or
    closed), whose cameras stand much closer to their neighbours than to the scene centre.
    """
    n = R.shape[0]
    device = R.device
    axis = _random_unit(n, g, device)
    R0 = rotation_exp(axis * math.radians(rot_deg)) @ R
    C = -torch.einsum("nba,nb->na", R, t)
    if kind in ("trajectory", "loop"):
        base = torch.median(torch.linalg.norm(C[cam_i] - C[cam_j], dim=-1))
        mag = trans_frac * base * torch.ones(n, 1, dtype=F64, device=device)
    else:
        mag = trans_frac * torch.linalg.norm(C, dim=-1, keepdim=True)
    C0 = C + mag * _random_unit(n, g, device)
    t0 = -torch.einsum("nab,nb->na", R0, C0)
    return R0, t0


def relative_translations(sc: Scene, noise_deg: float = 1.0, outlier_frac: float = 0.05, seed: int = 0):
    """Unit relative translations of the scene's image pairs as a relative-pose step would
    deliver them: t_{i->j} = R_j (c_i - c_j) / |c_i - c_j| from the true poses, turned by a
    random angle of about `noise_deg` degrees, and for a fraction `outlier_frac` of the pairs
    replaced by a uniform random direction. Returns (t_rel (B, 3) float64, outlier mask)."""
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed) * 7919 + 17)
    R = sc.R_gt.detach().cpu().to(F64)
    t = sc.t_gt.detach().cpu().to(F64)
    C = -torch.einsum("nba,nb->na", R, t)
    ci, cj = sc.cam_i.detach().cpu().long(), sc.cam_j.detach().cpu().long()
    d = torch.einsum("nab,nb->na", R[cj], C[ci] - C[cj])
    d = d / torch.linalg.norm(d, dim=-1, keepdim=True)
    B = d.shape[0]
    axis = _random_unit(B, g, torch.device("cpu"))
    ang = math.radians(noise_deg) * torch.randn(B, 1, dtype=F64, generator=g)
    d = torch.einsum("nab,nb->na", rotation_exp(axis * ang), d)
    out = torch.rand(B, dtype=F64, generator=g) < outlier_frac
    d[out] = _random_unit(int(out.sum()), g, torch.device("cpu"))
    d = d / torch.linalg.norm(d, dim=-1, keepdim=True)
    return d.numpy(), out.numpy()


def relative_rotations(sc: Scene, noise_deg: float = 1.0, outlier_frac: float = 0.05, seed: int = 0):
    """Relative rotations R_{i->j} = R_j R_i^T of the scene's image pairs from the true
    rotations, each turned by a random rotation of about `noise_deg` degrees, and for a fraction
    `outlier_frac` of the pairs turned by a uniformly random rotation angle instead.
    Returns (R_rel (B, 3, 3) float64, outlier mask)."""
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed) * 104729 + 29)
    R = sc.R_gt.detach().cpu().to(F64)
    ci, cj = sc.cam_i.detach().cpu().long(), sc.cam_j.detach().cpu().long()
    Rrel = R[cj] @ R[ci].transpose(1, 2)
    B = Rrel.shape[0]
    axis = _random_unit(B, g, torch.device("cpu"))
    ang = math.radians(noise_deg) * torch.randn(B, 1, dtype=F64, generator=g)
    out = torch.rand(B, dtype=F64, generator=g) < outlier_frac
    ang[out, 0] = math.pi * torch.rand(int(out.sum()), dtype=F64, generator=g)
    Rrel = rotation_exp(axis * ang) @ Rrel
    return Rrel.numpy(), out.numpy()


def fundamental_matrices(sc: Scene, noise: float = 1e-3, wrong_frac: float = 0.1, seed: int = 0, f=None):
    """Fundamental matrices of the scene's image pairs as an upstream two-view estimation would
    deliver them (the input of the focal-length vote): F = K_j^-T [t]_x R_ij K_i^-1 from the true
    relative pose (R_ij = R_j R_i^T, t = R_j (c_i - c_j)), K = diag(f, f, 1) in pixels from the
    image centre, with Gaussian noise of standard deviation `noise` added to every entry in
    calibrated coordinates (where the entries share one scale) and a fraction `wrong_frac` of the
    pairs replaced by random matrices. f: per-camera focal lengths (default: the scene's).
    Returns (F (B, 3, 3) float64, wrong-pair mask)."""
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed) * 15485863 + 41)
    R = sc.R_gt.detach().cpu().to(F64)
    t = sc.t_gt.detach().cpu().to(F64)
    C = -torch.einsum("nba,nb->na", R, t)
    ci, cj = sc.cam_i.detach().cpu().long(), sc.cam_j.detach().cpu().long()
    Rij = R[cj] @ R[ci].transpose(1, 2)
    tij = torch.einsum("nab,nb->na", R[cj], C[ci] - C[cj])
    E = _hat(tij) @ Rij
    B = E.shape[0]
    E = E + noise * torch.randn(B, 3, 3, dtype=F64, generator=g)
    wrong = torch.rand(B, dtype=F64, generator=g) < wrong_frac
    E[wrong] = torch.randn(int(wrong.sum()), 3, 3, dtype=F64, generator=g)
    fv = torch.full((sc.n_cams,), float(sc.f), dtype=F64) if f is None else torch.as_tensor(f, dtype=F64)
    one = torch.ones(B, dtype=F64)
    si = torch.stack([fv[ci], fv[ci], one], 1)
    sj = torch.stack([fv[cj], fv[cj], one], 1)
    return (E / (sj[:, :, None] * si[:, None, :])).numpy(), wrong.numpy()
