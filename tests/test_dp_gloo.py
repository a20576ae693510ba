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
