"""Splitting one epipolar-adjustment problem across processes (one GPU each).

The objective is a sum over image pairs (Eq. epipolar-objective), so the pair-sorted point
pairs split into contiguous ranges of whole image pairs, balanced by point-pair count. Every
process holds a full replica of the poses and of the optimiser state and runs the
loss/gradient pass on its range only, normalised by the total number of point pairs Z of all
ranges; one all-reduce (sum) of the N x 6 gradient and the loss per iteration gives every
process the full gradient, and the replicated optimiser step keeps the replicas identical.
The reweighting passes are local (a point pair's weight depends on its own residual only).

Host control flow only; the per-rank compute comes from a backend, the collective from
torch.distributed. Two data planes:
  * host (`GpuShard`): the gradient comes to the host each iteration and is all-reduced as a
    CPU tensor (gloo);
  * device (`DeviceGpuShard`): the library writes the loss and gradient into one device buffer
    (fm_loss_grad_device), the collective sums that buffer in place on the device (NCCL), and
    the library takes the optimiser step from it (fm_apply_gradient on device memory). All three
    are ordered on the current CUDA stream; nothing waits on the host inside an iteration.
A backend that has `new_buffer`, `loss_grad_into` and `apply_gradient_from` gets the device
plane.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def partition_pairs(pair_counts, world: int):
    """Contiguous ranges [begin, end) of image pairs, one per rank, each rank's range ending at
    the first pair where the running point-pair count reaches (rank+1)/world of the total.
    Ranges may be empty when there are fewer pairs than ranks."""
    counts = np.asarray(pair_counts, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    cum = np.cumsum(counts)
    total = int(cum[-1]) if len(cum) else 0
    bounds = [0]
    for r in range(1, world):
        target = total * r / world
        b = int(np.searchsorted(cum, target, side="left")) + 1 if total else 0
        bounds.append(min(max(b, bounds[-1]), len(counts)))
    bounds.append(len(counts))
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def shard_point_pairs(pair_id, begin: int, end: int):
    """Index range of the point pairs of image pairs [begin, end) in a pair-sorted array."""
    pid = np.asarray(pair_id)
    lo = int(np.searchsorted(pid, begin, side="left"))
    hi = int(np.searchsorted(pid, end, side="left"))
    return lo, hi


class GpuShard:
    """Backend over a binding.Problem built from one shard (with options.z_total = Z)."""

    def __init__(self, problem):
        self.p = problem

    def loss_grad(self):
        return self.p.loss_grad()

    def apply_gradient(self, grad):
        self.p.apply_gradient(grad)

    def reweight(self, tau):
        return self.p.irls_weights(tau)

    def set_learning_rate(self, lr_rot, lr_c):
        self.p.set_learning_rate(lr_rot, lr_c)


class DeviceGpuShard(GpuShard):
    """Backend with the device data plane: gradient and loss stay in device memory."""

    def new_buffer(self):
        """[n_cams * 6 gradient entries, loss] as one float64 tensor on the problem's device."""
        return torch.zeros(self.p.n_cams * 6 + 1, dtype=torch.float64, device="cuda")

    def loss_grad_into(self, buf):
        self.p.loss_grad_device(buf[-1:], buf[:-1])

    def apply_gradient_from(self, buf):
        self.p.apply_gradient(buf[:-1].view(-1, 6))


class ShardedAdjustment:
    """The IRLS loop over a sharded problem: local reweighting, per-iteration all-reduce of
    the gradient and the loss, replicated optimiser step."""

    def __init__(self, backend, group=None):
        self.b = backend
        self.group = group
        self.device_plane = all(hasattr(backend, a) for a in ("new_buffer", "loss_grad_into", "apply_gradient_from"))
        self.buf = backend.new_buffer() if self.device_plane else None

    def _all_reduce(self, buf):
        if dist.is_available() and dist.is_initialized():
            dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=self.group)

    def iteration(self):
        """One iteration; returns the total loss (a float on the host plane, a one-element
        tensor on the device plane, read without waiting only when the caller converts it)."""
        if self.device_plane:
            self.b.loss_grad_into(self.buf)
            self._all_reduce(self.buf)
            self.b.apply_gradient_from(self.buf)
            return self.buf[-1:]
        loss, grad = self.b.loss_grad()
        buf = torch.from_numpy(np.concatenate([np.asarray(grad, np.float64).ravel(), [loss]]))
        self._all_reduce(buf)
        total = buf.numpy()
        self.b.apply_gradient(total[:-1].reshape(-1, 6))
        return float(total[-1])

    def round(self, tau: float, iters: int, lr_rot: float, lr_c: float) -> float:
        self.b.reweight(tau)
        self.b.set_learning_rate(lr_rot, lr_c)
        loss = float("nan")
        for _ in range(iters):
            loss = self.iteration()
        return float(loss[0]) if self.device_plane and iters > 0 else float(loss)

    def run(self, schedule) -> float:
        loss = float("nan")
        for r in range(schedule.rounds):
            s = schedule.decay ** r
            loss = self.round(schedule.tau(r), schedule.iters_per_round, schedule.lr_rot * s, schedule.lr_c * s)
        return loss
