"""Sharding across processes, tested without a GPU: the partition, and gloo ranks (world
sizes 2 and 3) that each compute their shard with the oracle, all-reduce, and take the
replicated optimiser step; the result must equal the single-process oracle on the whole
problem. Both data planes of the sharded loop run: the host plane (gradient returned to the
caller) and the device plane's control flow (gradient and loss written into one buffer that is
all-reduced in place and read back by the optimiser step), here with CPU tensors and gloo in
place of device memory and NCCL."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2605_18052_gb300.shard import ShardedAdjustment, partition_pairs, shard_point_pairs


def test_partition_balances_whole_pairs():
    counts = np.array([5, 1, 1, 10, 3, 3, 2, 8, 1, 6])
    for world in (1, 2, 3, 4, 10, 13):
        parts = partition_pairs(counts, world)
        assert parts[0][0] == 0 and parts[-1][1] == len(counts)
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
        sizes = [counts[b:e].sum() for b, e in parts]
        assert sum(sizes) == counts.sum()
        if world <= len(counts):
            # no rank holds more than its share plus one image pair
            assert max(sizes) <= counts.sum() / world + counts.max()


def test_shard_point_pairs_ranges():
    pid = np.array([0, 0, 1, 2, 2, 2, 4])
    assert shard_point_pairs(pid, 0, 2) == (0, 3)
    assert shard_point_pairs(pid, 2, 5) == (3, 7)
    assert shard_point_pairs(pid, 3, 4) == (6, 6)


class _OracleShard:
    """Backend running the oracle on one shard, normalised by the total Z."""

    def __init__(self, prob, n_total, R, c, delta=1e-6):
        import oracle as O
        self.O = O
        self.prob, self.frac = prob, prob.n_pp / n_total
        self.R, self.c = R.copy(), c.copy()
        self.m = np.zeros((R.shape[0], 6))
        self.v = np.zeros((R.shape[0], 6))
        self.step = 0
        self.w = np.ones(prob.n_pp)
        self.delta = delta
        self.lr = (1e-2, 1e-2)

    def loss_grad(self):
        loss, g = self.O.loss_grad(self.prob, self.R, self.c, self.w)
        return loss * self.frac, g * self.frac

    def apply_gradient(self, grad):
        self.step += 1
        self.O.adam_step(self.R, self.c, grad, self.m, self.v, self.step, self.lr[0], self.lr[1])

    def reweight(self, tau):
        self.w = self.O.irls_weights(self.O.residuals(self.prob, self.R, self.c), tau, self.delta)[0]

    def set_learning_rate(self, lr_rot, lr_c):
        self.lr = (lr_rot, lr_c)


class _OracleBufferShard(_OracleShard):
    """The same oracle shard behind the device plane's interface (one buffer per iteration)."""

    def new_buffer(self):
        return torch.zeros(self.R.shape[0] * 6 + 1, dtype=torch.float64)

    def loss_grad_into(self, buf):
        loss, g = self.loss_grad()
        buf[:-1] = torch.from_numpy(g.ravel())
        buf[-1] = loss

    def apply_gradient_from(self, buf):
        self.apply_gradient(buf[:-1].numpy().reshape(-1, 6).copy())


def _problem():
    import oracle as O
    import scenegen
    sc = scenegen.make_scene("ring16", seed=21)
    prob = O.Problem.from_scene(sc)
    R0 = sc.R_init.numpy()
    c0 = O.centres_from_poses(R0, sc.t_init.numpy())
    return prob, R0, c0


def _rank(rank, world, port, out, plane="host"):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    prob, R0, c0 = _problem()
    counts = np.bincount(prob.pair_id, minlength=prob.n_pairs)
    b, e = partition_pairs(counts, world)[rank]
    lo, hi = shard_point_pairs(prob.pair_id, b, e)
    sub = O.Problem(prob.n_cams, prob.cam_i, prob.cam_j, prob.pair_id[lo:hi], prob.x1[lo:hi], prob.x2[lo:hi])
    be = (_OracleBufferShard if plane == "device" else _OracleShard)(sub, prob.n_pp, R0, c0)
    adj = ShardedAdjustment(be)
    assert adj.device_plane == (plane == "device")
    # one sharded gradient vs the whole problem
    loss, g = be.loss_grad()
    buf = torch.from_numpy(np.concatenate([g.ravel(), [loss]]))
    dist.all_reduce(buf)
    # two rounds of the loop
    adj.round(0.5, 5, 1e-2, 3e-2)
    last = adj.round(0.4, 5, 9e-3, 2.7e-2)
    out[rank] = (buf.numpy().copy(), be.R.copy(), be.c.copy(), last)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,plane", [(2, "host"), (3, "host"), (2, "device")])
def test_gloo_ranks_match_single_process(world, plane):
    import oracle as O
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    mp.start_processes(_rank, args=(world, port, out, plane), nprocs=world, join=True, start_method="spawn")
    prob, R0, c0 = _problem()
    l_full, g_full = O.loss_grad(prob, R0, c0, np.ones(prob.n_pp))
    for r in range(world):
        buf = out[r][0]
        np.testing.assert_allclose(buf[:-1].reshape(-1, 6), g_full, rtol=1e-10, atol=1e-13 * np.abs(g_full).max())
        assert buf[-1] == pytest.approx(l_full, rel=1e-12)
    # replicas stayed identical
    for r in range(1, world):
        np.testing.assert_array_equal(out[0][1], out[r][1])
        np.testing.assert_array_equal(out[0][2], out[r][2])
    # and equal the single-process loop (same rounds)
    R, c = R0.copy(), c0.copy()
    m, v = np.zeros((prob.n_cams, 6)), np.zeros((prob.n_cams, 6))
    step = 0
    for tau, lr_r, lr_c in ((0.5, 1e-2, 3e-2), (0.4, 9e-3, 2.7e-2)):
        w = O.irls_weights(O.residuals(prob, R, c), tau, 1e-6)[0]
        for _ in range(5):
            _, g = O.loss_grad(prob, R, c, w)
            step += 1
            O.adam_step(R, c, g, m, v, step, lr_r, lr_c)
    np.testing.assert_allclose(out[0][1], R, atol=1e-12)
    np.testing.assert_allclose(out[0][2], c, atol=1e-12)
