"""Data-parallel exchange of the NBM step on CPU ranks (gloo, world size 2).

Sec. 3 of the paper reduces multi-GPU NBM to data-parallel training: points are
distributed over processors and the locally computed gradient updates are
aggregated.  Each rank here takes half of a batch through the FP64 oracle; a
count-weighted all-reduce of the gradients and losses must give the full-batch
gradient and loss, so that a replicated Adam step stays identical on every
rank.  Also checks bench.py's max-over-ranks timing helper.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import pyoracle as O
from tests import inputs


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pr = O.make_problem(geometry=O.GEOM_SPHERE, n_hidden=2, width=16, h=2.0 / 32,
                            mu_minus=1.0, mu_plus=10.0)
        th = inputs.glorot_params(16, 2, seed=3, bias_scale=0.1).astype(np.float64)
        pts = inputs.mixed_points(300, 100, seed=12)
        parts = np.array_split(pts, world)
        mine = parts[rank]
        loss, g = O.loss_grad(pr, th, mine, n_threads=1)
        n_mine = len(mine)
        gt = torch.from_numpy(g * n_mine)
        lt = torch.tensor([loss * n_mine, float(n_mine)], dtype=torch.float64)
        dist.all_reduce(gt)
        dist.all_reduce(lt)
        g_dp = (gt / lt[1]).numpy()
        loss_dp = float(lt[0] / lt[1])
        # replicated Adam on the aggregated gradient
        m = np.zeros_like(th)
        v = np.zeros_like(th)
        th_new = th.copy()
        O.adam_step(th_new, m, v, g_dp, 1)
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.concatenate([[loss_dp], g_dp, th_new]))
        import bench
        t = bench._max_over_ranks(world, float(rank + 1))
        np.save(os.path.join(out_dir, f"max{rank}.npy"), np.array([t]))
    finally:
        dist.destroy_process_group()


def test_gradient_aggregation_over_two_gloo_ranks(tmp_path):
    world = 2
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world,
                       start_method="spawn")
    r0 = np.load(tmp_path / "rank0.npy")
    r1 = np.load(tmp_path / "rank1.npy")
    assert np.array_equal(r0, r1)  # identical replicated state on both ranks
    pr = O.make_problem(geometry=O.GEOM_SPHERE, n_hidden=2, width=16, h=2.0 / 32, mu_minus=1.0,
                        mu_plus=10.0)
    th = inputs.glorot_params(16, 2, seed=3, bias_scale=0.1).astype(np.float64)
    pts = inputs.mixed_points(300, 100, seed=12)
    loss, g = O.loss_grad(pr, th, pts)
    P = len(g)
    assert abs(r0[0] - loss) <= 1e-13 * loss
    assert np.allclose(r0[1:1 + P], g, rtol=1e-12, atol=1e-16)
    assert np.load(tmp_path / "max0.npy")[0] == 2.0 and np.load(tmp_path / "max1.npy")[0] == 2.0


class _OracleShardProblem:
    """Stands in for a libnbm Problem on CPU ranks: the shard's loss and gradient
    come from the FP64 oracle on the points the whole batch would put there,
    scaled by 1/n_total, and Adam is the oracle's update."""

    def __init__(self):
        self.o = O.make_problem(geometry=O.GEOM_FLOWER, n_hidden=2, width=16, h=2.0 / 32,
                                mu_minus=1.0, mu_plus=100.0)

    def batch(self, seed, step, n_total):
        return O.sample_points(self.o, seed, step, n_total, int(np.floor(0.3 * n_total + 0.5)))

    def loss_grad_shard(self, params, n_total, first, n, seed=1, step=1, pts=None, grad=None,
                        loss=None):
        x = self.batch(seed, step, n_total)[first:first + n] if pts is None else pts.numpy()
        L, g = O.loss_grad(self.o, params.numpy(), x, n_threads=1)
        grad.copy_(torch.from_numpy(g * n / n_total))
        loss.fill_(L * n / n_total)
        return loss, grad

    def adam_step(self, params, m, v, grad, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                  loss=None):
        th, mm, vv = params.numpy(), m.numpy(), v.numpy()
        O.adam_step(th, mm, vv, grad.numpy().copy(), step + 1, lr, beta1, beta2, eps)
        return step + 1


def _trainer_rank(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2210_14907_gb300.data_parallel import DataParallelTrainer, torch_all_reduce
        th = torch.from_numpy(inputs.glorot_params(16, 2, seed=3, bias_scale=0.1)
                              .astype(np.float64))
        m, v = torch.zeros_like(th), torch.zeros_like(th)
        tr = DataParallelTrainer(_OracleShardProblem(), th, m, v, 301, rank=rank, world=world,
                                 all_reduce=torch_all_reduce(), seed=4)
        losses = [float(tr.step().item()) for _ in range(3)]
        np.save(os.path.join(out_dir, f"tr{rank}.npy"),
                np.concatenate([losses, th.numpy(), m.numpy(), v.numpy()]))
    finally:
        dist.destroy_process_group()


def test_data_parallel_trainer_over_two_gloo_ranks(tmp_path):
    """The trainer's orchestration (uneven shards of a 301-point batch with band
    points, all-reduce of gradient and loss, replicated Adam) on two CPU ranks
    equals three whole-batch oracle steps."""
    world = 2
    mp.start_processes(_trainer_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    r0 = np.load(tmp_path / "tr0.npy")
    r1 = np.load(tmp_path / "tr1.npy")
    assert np.array_equal(r0, r1)
    fake = _OracleShardProblem()
    th = inputs.glorot_params(16, 2, seed=3, bias_scale=0.1).astype(np.float64)
    m, v = np.zeros_like(th), np.zeros_like(th)
    losses = []
    for t in range(1, 4):
        L, g = O.loss_grad(fake.o, th, fake.batch(4, t, 301))
        losses.append(L)
        O.adam_step(th, m, v, g, t)
    assert np.allclose(r0[:3], losses, rtol=1e-12, atol=0)
    P = len(th)
    assert np.allclose(r0[3:3 + P], th, rtol=0, atol=1e-12)
    assert np.allclose(r0[3 + P:3 + 2 * P], m, rtol=1e-10, atol=1e-18)
    assert np.allclose(r0[3 + 2 * P:], v, rtol=1e-10, atol=1e-24)


def test_shard_range_partitions_the_batch():
    from paper_2210_14907_gb300.data_parallel import shard_range
    for n_total in (1, 2, 7, 301, 262144, 1048577):
        for world in (1, 2, 3, 4, 8):
            if n_total < world:
                with pytest.raises(ValueError):
                    shard_range(n_total, world, 0)
                continue
            spans = [shard_range(n_total, world, r) for r in range(world)]
            assert spans[0][0] == 0
            for (f0, n0), (f1, _) in zip(spans, spans[1:]):
                assert f0 + n0 == f1
            assert spans[-1][0] + spans[-1][1] == n_total
            assert max(n for _, n in spans) - min(n for _, n in spans) <= 1
